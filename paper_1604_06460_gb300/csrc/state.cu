// State initialisation kernels: basis states and the seeded Gaussian state.
#include <cmath>

#include "qe_arith.cuh"
#include "qe_internal.h"

namespace qe {

void fail(int status, const std::string& msg) { throw Error{status, msg}; }

void check_cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear sticky-free errors
        fail(e == cudaErrorMemoryAllocation ? QE_ERR_OOM : QE_ERR_CUDA,
             std::string(what) + ": " + cudaGetErrorString(e));
    }
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        QE_CUDA(cudaGetDevice(&dev));
        QE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    return sms;
}

void* ensure_scratch(qe_state* s, size_t bytes) {
    if (s->scratch_bytes < bytes) {
        if (s->scratch) {
            QE_CUDA(cudaStreamSynchronize(s->stream));
            QE_CUDA(cudaFree(s->scratch));
            s->scratch = nullptr;
            s->scratch_bytes = 0;
        }
        size_t b = bytes < (1u << 20) ? (1u << 20) : bytes;
        QE_CUDA(cudaMalloc(&s->scratch, b));
        s->scratch_bytes = b;
    }
    return s->scratch;
}

void* ensure_oz_workspace(qe_state* s, size_t bytes) {
    if (s->oz_ws_bytes < bytes) {
        if (s->oz_ws) {
            QE_CUDA(cudaStreamSynchronize(s->stream));
            QE_CUDA(cudaFree(s->oz_ws));
            s->oz_ws = nullptr;
            s->oz_ws_bytes = 0;
        }
        QE_CUDA(cudaMalloc(&s->oz_ws, bytes));
        s->oz_ws_bytes = bytes;
    }
    return s->oz_ws;
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit products with multipliers 0xD2511F53 / 0xCD9E8D57 and a Weyl
// key schedule with increments 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

template <class S>
__device__ __forceinline__ S make_amp(double re, double im);
template <>
__device__ __forceinline__ double2 make_amp<double2>(double re, double im) { return make_double2(re, im); }
template <>
__device__ __forceinline__ float2 make_amp<float2>(double re, double im) {
    return make_float2((float)re, (float)im);
}

// Amplitude i: Box-Muller on two 53-bit uniforms drawn by Philox with
// counter (lo32(i), hi32(i), 0, 0) and key (lo32(seed), hi32(seed)).
template <class S>
__global__ void k_init_gaussian(S* __restrict__ x, uint64_t count, uint64_t seed) {
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint4 w = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, 0u), key);
        uint64_t a = ((uint64_t)w.y << 32) | w.x;
        uint64_t b = ((uint64_t)w.w << 32) | w.z;
        double u1 = (double)((a >> 11) + 1) * 0x1.0p-53;
        double u2 = (double)(b >> 11) * 0x1.0p-53;
        double r = sqrt(-2.0 * log(u1));
        double th = 2.0 * 3.14159265358979323846 * u2;
        x[i] = make_amp<S>(r * cos(th), r * sin(th));
    }
}

template <class S>
__global__ void k_set_one(S* __restrict__ x, uint64_t index) {
    x[index] = make_amp<S>(1.0, 0.0);
}

template <class S>
__global__ void k_scale(S* __restrict__ x, uint64_t count, double f);
template <>
__global__ void k_scale<double2>(double2* __restrict__ x, uint64_t count, double f) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        double2 v = x[i];
        x[i] = make_double2(v.x * f, v.y * f);
    }
}
template <>
__global__ void k_scale<float2>(float2* __restrict__ x, uint64_t count, double f) {
    const float ff = (float)f;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        float2 v = x[i];
        x[i] = make_float2(v.x * ff, v.y * ff);
    }
}

static unsigned grid_for(uint64_t count, int threads) {
    uint64_t want = (count + threads - 1) / threads;
    uint64_t cap = (uint64_t)num_sms() * 16;
    return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

void launch_init_basis(qe_state* s, uint64_t index) {
    QE_CUDA(cudaMemsetAsync(s->d, 0, dim(s) * amp_bytes(s), s->stream));
    s->stats.bytes += (double)dim(s) * amp_bytes(s);
    Launch L(s, "init_basis", 0.0, false);
    if (s->dtype == QE_C128)
        k_set_one<double2><<<1, 1, 0, s->stream>>>((double2*)s->d, index);
    else
        k_set_one<float2><<<1, 1, 0, s->stream>>>((float2*)s->d, index);
    QE_CUDA(cudaGetLastError());
}

void launch_init_random(qe_state* s, uint64_t seed) {
    uint64_t N = dim(s);
    {
        Launch L(s, "init_gaussian", (double)N * amp_bytes(s));
        if (s->dtype == QE_C128)
            k_init_gaussian<double2><<<grid_for(N, 256), 256, 0, s->stream>>>((double2*)s->d, N, seed);
        else
            k_init_gaussian<float2><<<grid_for(N, 256), 256, 0, s->stream>>>((float2*)s->d, N, seed);
        QE_CUDA(cudaGetLastError());
    }
    double nrm = reduce_norm2(s);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) fail(QE_ERR_CUDA, "random state has zero norm");
    launch_scale(s, 1.0 / std::sqrt(nrm));
}

void launch_scale(qe_state* s, double f) {
    uint64_t N = dim(s);
    Launch L(s, "scale", 2.0 * N * amp_bytes(s));
    if (s->dtype == QE_C128)
        k_scale<double2><<<grid_for(N, 256), 256, 0, s->stream>>>((double2*)s->d, N, f);
    else
        k_scale<float2><<<grid_for(N, 256), 256, 0, s->stream>>>((float2*)s->d, N, f);
    QE_CUDA(cudaGetLastError());
}

}  // namespace qe

namespace qe {

static cudaEvent_t pool_event(qe_state* s) {
    if (!s->event_pool.empty()) {
        cudaEvent_t e = s->event_pool.back();
        s->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    QE_CUDA(cudaEventCreate(&e));
    return e;
}

Launch::Launch(qe_state* s, const char* tag, double bytes, bool full_pass) : s_(s) {
    s->stats.launches += 1;
    if (full_pass) s->stats.passes += 1;
    s->stats.bytes += bytes;
    if (s->profile) {
        ProfRec r{tag, pool_event(s), pool_event(s), bytes};
        QE_CUDA(cudaEventRecord(r.start, s->stream));
        s->prof.push_back(r);
        idx_ = (int)s->prof.size() - 1;
    }
}

Launch::~Launch() {
    if (idx_ >= 0) cudaEventRecord(s_->prof[idx_].stop, s_->stream);
}

void profile_clear(qe_state* s) {
    for (auto& r : s->prof) {
        s->event_pool.push_back(r.start);
        s->event_pool.push_back(r.stop);
    }
    s->prof.clear();
}

}  // namespace qe
