// Marginal probabilities without any device allocation.
//
// Some callers cannot call cudaMalloc at all: code that runs while a CUDA
// graph is being captured by someone else, processes whose device memory is
// entirely owned by another allocator or arena, or embedded/real-time hosts
// that forbid allocation after start-up.  qe_probs_noalloc serves them: it
// computes the same marginal probabilities as qe_probs from a raw state
// pointer, and keeps its block partial sums in a fixed, file-scope device
// array instead of allocated scratch.  The caller passes the state and the
// output buffer; nothing is allocated on the device or through any library.
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/qe.h"
#include "qe_arith.cuh"

namespace {

// Scratch for block partials: 65536 (sum, compensation) pairs = 1 MiB.  Every
// GPU that loads this library holds it until the process exits.
constexpr int kNoAllocPartials = 65536;
static __device__ __align__(256) double2 g_noalloc_partials[kNoAllocPartials];

constexpr int kThreads = 256;

struct Args {
    const void* x;
    int c128;
    uint64_t per_bin;
    uint64_t chunks;
    uint64_t chunk_len;
    int m;
    uint8_t q[32];
    uint8_t q_sorted[32];
};

__device__ __forceinline__ void two_sum_add(float& s, float& e, float ph, float pl) {
    float t = __fadd_rn(s, ph);
    float bb = __fsub_rn(t, s);
    float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(ph, bb));
    s = t;
    e = __fadd_rn(e, __fadd_rn(err, pl));
}

// Each block sums |alpha|^2 over its chunk of one bin and writes one partial.
__global__ void __launch_bounds__(kThreads) k_noalloc_partial(const __grid_constant__ Args a,
                                                              double2* __restrict__ partial) {
    __shared__ double sh[kThreads / 32];
    const uint64_t bin = blockIdx.x / a.chunks, ch = blockIdx.x % a.chunks;
    uint64_t dep = 0;
    for (int j = 0; j < a.m; ++j) dep |= ((bin >> j) & 1ull) << a.q[j];
    const uint64_t t0 = ch * a.chunk_len;
    const uint64_t t1 = min(a.per_bin, t0 + a.chunk_len);
    float s = 0.f, e = 0.f;
    for (uint64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        const uint64_t x = qe::insert_zero_bits(t, a.q_sorted, a.m) | dep;
        float h, l;
        if (a.c128) {
            const double2 v = static_cast<const double2*>(a.x)[x];
            const qe::df re = qe::d2df(v.x), im = qe::d2df(v.y);
            qe::df_first(h, l, re, re);
            qe::df_acc(h, l, im, im);
        } else {
            const float2 v = static_cast<const float2*>(a.x)[x];
            qe::df_first(h, l, qe::df{v.x, 0.f}, qe::df{v.x, 0.f});
            qe::df_acc(h, l, qe::df{v.y, 0.f}, qe::df{v.y, 0.f});
        }
        two_sum_add(s, e, h, l);
    }
    // per-thread partial -> FP64, then a fixed-order block sum
    double d = qe::df2d(s, e);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0, comp = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            const double t = sum + sh[w];
            comp += (fabs(sum) >= fabs(sh[w])) ? (sum - t) + sh[w] : (sh[w] - t) + sum;
            sum = t;
        }
        partial[blockIdx.x] = make_double2(sum, comp);
    }
}

// One thread per bin: Neumaier sum of its chunks' partials in chunk order.
__global__ void k_noalloc_sum(const double2* __restrict__ partial, uint64_t bins, uint64_t chunks,
                              double* __restrict__ out) {
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < bins;
         b += (uint64_t)gridDim.x * blockDim.x) {
        double sum = 0.0, comp = 0.0;
        for (uint64_t i = 0; i < chunks; ++i) {
            const double2 p = partial[b * chunks + i];
            for (double v : {p.x, p.y}) {
                const double t = sum + v;
                comp += (fabs(sum) >= fabs(v)) ? (sum - t) + v : (v - t) + sum;
                sum = t;
            }
        }
        out[b] = sum + comp;
    }
}

}  // namespace

extern "C" int qe_probs_noalloc(const void* state, int n, int dtype, int m, const int* qubits,
                                double* out, void* stream) {
    if (!state || !out || !qubits) return QE_ERR_ARG;
    if (n < 1 || n > 34) return QE_ERR_ARG;
    if (dtype != QE_C64 && dtype != QE_C128) return QE_ERR_ARG;
    if (m < 1 || m > 16 || m > n) return QE_ERR_ARG;
    Args a{};
    uint64_t used = 0;
    int tmp[32];
    for (int j = 0; j < m; ++j) {
        if (qubits[j] < 0 || qubits[j] >= n || ((used >> qubits[j]) & 1ull)) return QE_ERR_ARG;
        used |= 1ull << qubits[j];
        a.q[j] = (uint8_t)qubits[j];
        tmp[j] = qubits[j];
    }
    for (int i = 1; i < m; ++i)
        for (int j = i; j > 0 && tmp[j - 1] > tmp[j]; --j) { int t = tmp[j]; tmp[j] = tmp[j - 1]; tmp[j - 1] = t; }
    for (int j = 0; j < m; ++j) a.q_sorted[j] = (uint8_t)tmp[j];
    const uint64_t bins = 1ull << m;
    a.x = state;
    a.c128 = dtype == QE_C128;
    a.m = m;
    a.per_bin = 1ull << (n - m);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return QE_ERR_CUDA;
    }
    // the array's address on the current device, looked up on every call (a
    // lookup once the module is loaded; it allocates nothing), so that an
    // address from a context that was reset is never reused
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
        cudaGetLastError();
        return QE_ERR_CUDA;
    }
    double2* partial = static_cast<double2*>(p);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t chunks = (uint64_t)(sms > 0 ? sms : 1) * 8 / bins;
    if (chunks < 1) chunks = 1;
    if (chunks > (a.per_bin >> 14)) chunks = (a.per_bin >> 14) ? (a.per_bin >> 14) : 1;
    if (bins * chunks > (uint64_t)kNoAllocPartials) chunks = kNoAllocPartials / bins;
    if (chunks < 1 || bins * chunks > (uint64_t)kNoAllocPartials) return QE_ERR_ARG;
    a.chunks = chunks;
    a.chunk_len = (a.per_bin + chunks - 1) / chunks;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_noalloc_partial<<<(unsigned)(bins * chunks), kThreads, 0, st>>>(a, partial);
    unsigned g2 = (unsigned)((bins + 255) / 256);
    k_noalloc_sum<<<g2, 256, 0, st>>>(partial, bins, chunks, out);
    return cudaGetLastError() == cudaSuccess ? QE_OK : QE_ERR_CUDA;
}
