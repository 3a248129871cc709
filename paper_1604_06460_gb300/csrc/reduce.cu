// Direct read-out of the state (Sec. III-D): expectation values of Pauli
// sums, marginal probabilities and the norm, computed in one pass each
// instead of by repeated sampling.
//
// Accumulation: each thread keeps a compensated sum (s, e) per quantity on
// the FP32 pipes (TwoProd for |alpha|^2 and products of amplitudes, TwoSum for
// additions, so the per-thread partial carries about 44 significant bits);
// the block combines its threads' partials with double-float additions and
// writes one FP64 pair (sum, Neumaier compensation) per block; a final
// single-block kernel adds the block partials in FP64 with Neumaier's
// compensation in a fixed order, so results are deterministic.
// The native-FP64 policy accumulates in FP64 directly.
#include <algorithm>
#include <type_traits>

#include "qe_arith.cuh"
#include "qe_internal.h"

namespace qe {

namespace {

constexpr int kRThreads = 256;

// ------------------------------------------------ compensated accumulators
struct Acc {
    float s, e;
};
__device__ __forceinline__ void acc_add(Acc& a, float ph, float pl) {
    float t = fadd(a.s, ph);
    float bb = fsub(t, a.s);
    float err = fadd(fsub(a.s, fsub(t, bb)), fsub(ph, bb));
    a.s = t;
    a.e = fadd(a.e, fadd(err, pl));
}
__device__ __forceinline__ Acc acc_merge(Acc a, Acc b) {
    df r = df_add(df{a.s, a.e}, df{b.s, b.e});
    return Acc{r.h, r.l};
}

// |v|^2 and Re(conj(w) v i^ny) as unevaluated (hi, lo) float pairs.
__device__ __forceinline__ void abs2(const float2& v, float& h, float& l) {
    df_first(h, l, df{v.x, 0.f}, df{v.x, 0.f});
    df_acc(h, l, df{v.y, 0.f}, df{v.y, 0.f});
}
__device__ __forceinline__ void abs2(const DF::V& v, float& h, float& l) {
    df_first(h, l, v.re, v.re);
    df_acc(h, l, v.im, v.im);
}
// Re(conj(w) * v * i^ny):  conj(w) v = (w.re v.re + w.im v.im) + i (w.re v.im - w.im v.re)
__device__ __forceinline__ void corr(const float2& w, const float2& v, int ny, float& h, float& l) {
    df wr{w.x, 0.f}, wi{w.y, 0.f}, vr{v.x, 0.f}, vi{v.y, 0.f};
    if ((ny & 1) == 0) {
        df_first(h, l, wr, vr);
        df_acc(h, l, wi, vi);
    } else {
        df_first(h, l, wr, vi);
        df_acc_neg(h, l, wi, vr);
    }
    if (ny == 1 || ny == 2) { h = -h; l = -l; }
}
__device__ __forceinline__ void corr(const DF::V& w, const DF::V& v, int ny, float& h, float& l) {
    if ((ny & 1) == 0) {
        df_first(h, l, w.re, v.re);
        df_acc(h, l, w.im, v.im);
    } else {
        df_first(h, l, w.re, v.im);
        df_acc_neg(h, l, w.im, v.re);
    }
    if (ny == 1 || ny == 2) { h = -h; l = -l; }
}

__device__ __forceinline__ Acc block_reduce(Acc a, Acc* sh) {
    for (int o = 16; o > 0; o >>= 1) {
        Acc b{__shfl_down_sync(0xffffffffu, a.s, o), __shfl_down_sync(0xffffffffu, a.e, o)};
        a = acc_merge(a, b);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = a;
    __syncthreads();
    if (w == 0) {
        a = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : Acc{0.f, 0.f};
        for (int o = 16; o > 0; o >>= 1) {
            Acc b{__shfl_down_sync(0xffffffffu, a.s, o), __shfl_down_sync(0xffffffffu, a.e, o)};
            a = acc_merge(a, b);
        }
    }
    return a;   // valid in thread 0
}

__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
    double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

// Policy views of an amplitude for the reducers.
__device__ __forceinline__ float2 rview(float2 v) { return v; }
__device__ __forceinline__ DF::V rview(double2 v) { return DF::load(v); }

// ---------------------------------------------------------------- probs
// Block b handles bin r = b / chunks and the chunk b % chunks of the
// 2^(n-m) amplitudes whose bits at the qubits spell r.
template <class S>
struct ProbArgs {
    const S* x;
    uint64_t per_bin;     // 2^(n-m)
    uint64_t chunks;      // blocks per bin
    uint64_t chunk_len;
    int m;
    uint8_t q[32];
    uint8_t q_sorted[32];
    double2* partial;     // [bins * chunks]
};

template <class S>
__global__ void __launch_bounds__(kRThreads) k_probs_partial(const __grid_constant__ ProbArgs<S> a) {
    __shared__ Acc sh[32];
    const uint64_t bin = blockIdx.x / a.chunks, ch = blockIdx.x % a.chunks;
    uint64_t dep = 0;
    for (int j = 0; j < a.m; ++j) dep |= ((bin >> j) & 1ull) << a.q[j];
    const uint64_t t0 = ch * a.chunk_len;
    const uint64_t t1 = min(a.per_bin, t0 + a.chunk_len);
    Acc acc{0.f, 0.f};
    for (uint64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        const uint64_t x = insert_zero_bits(t, a.q_sorted, a.m) | dep;
        float h, l;
        abs2(rview(a.x[x]), h, l);
        acc_add(acc, h, l);
    }
    acc = block_reduce(acc, sh);
    if (threadIdx.x == 0) {
        df r = df_norm(acc.s, acc.e);
        a.partial[blockIdx.x] = make_double2(df2d(r.h, r.l), 0.0);
    }
}

// One thread per output: Neumaier sum of `count` partials (stride 1).
__global__ void k_sum_partials(const double2* __restrict__ partial, uint64_t nout, uint64_t count,
                               const double* __restrict__ weight, double* __restrict__ out) {
    for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < nout;
         o += (uint64_t)gridDim.x * blockDim.x) {
        double s = 0.0, c = 0.0;
        for (uint64_t i = 0; i < count; ++i) {
            double2 p = partial[o * count + i];
            neumaier(s, c, p.x);
            neumaier(s, c, p.y);
        }
        out[o] = (s + c) * (weight ? weight[o] : 1.0);
    }
}

// ---------------------------------------------------------- expectation
// Up to NT Pauli terms per launch.  For term t and amplitude index x:
//   xm == 0: |alpha_x|^2 (-1)^popc(x & zm)
//   xm != 0: over x with the lowest bit of xm clear,
//            2 Re(conj(alpha_{x^xm}) alpha_x i^ny) (-1)^popc(x & zm)
constexpr int kNT = 8;
template <class S>
struct ExpArgs {
    const S* x;
    uint64_t count;            // 2^n
    int nt;
    uint64_t xm[kNT], zm[kNT];
    int ny[kNT];
    double w[kNT];
    double2* partial;          // one per block
};

template <class S>
__global__ void __launch_bounds__(kRThreads) k_expect_partial(const __grid_constant__ ExpArgs<S> a) {
    __shared__ Acc sh[32];
    Acc acc[kNT];
#pragma unroll
    for (int t = 0; t < kNT; ++t) acc[t] = Acc{0.f, 0.f};
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < a.count;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const auto v = rview(a.x[x]);
        float ph = 0.f, pl = 0.f;
        bool have_p = false;
#pragma unroll
        for (int t = 0; t < kNT; ++t) {
            if (t >= a.nt) break;
            const uint64_t xm = a.xm[t];
            const bool neg = __popcll(x & a.zm[t]) & 1;
            float h, l;
            if (xm == 0) {
                if (!have_p) { abs2(v, ph, pl); have_p = true; }
                h = ph; l = pl;
            } else {
                if (x & (xm & (~xm + 1ull))) continue;   // lowest bit of xm must be 0
                corr(rview(a.x[x ^ xm]), v, a.ny[t], h, l);
                h *= 2.f; l *= 2.f;
            }
            if (neg) { h = -h; l = -l; }
            acc_add(acc[t], h, l);
        }
    }
    double s = 0.0, c = 0.0;
#pragma unroll
    for (int t = 0; t < kNT; ++t) {
        if (t >= a.nt) break;
        Acc r = block_reduce(acc[t], sh);
        if (threadIdx.x == 0) {
            df d = df_norm(r.s, r.e);
            neumaier(s, c, df2d(d.h, d.l) * a.w[t]);
        }
    }
    if (threadIdx.x == 0) a.partial[blockIdx.x] = make_double2(s, c);
}

// Native FP64 variants (baseline policy).
__global__ void __launch_bounds__(kRThreads) k_probs_partial_f64(const __grid_constant__ ProbArgs<double2> a) {
    __shared__ double shs[32], shc[32];
    const uint64_t bin = blockIdx.x / a.chunks, ch = blockIdx.x % a.chunks;
    uint64_t dep = 0;
    for (int j = 0; j < a.m; ++j) dep |= ((bin >> j) & 1ull) << a.q[j];
    const uint64_t t0 = ch * a.chunk_len;
    const uint64_t t1 = min(a.per_bin, t0 + a.chunk_len);
    double s = 0.0, c = 0.0;
    for (uint64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        const double2 v = a.x[insert_zero_bits(t, a.q_sorted, a.m) | dep];
        neumaier(s, c, v.x * v.x + v.y * v.y);
    }
    s += c;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) shs[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tc = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) neumaier(ts, tc, shs[w]);
        a.partial[blockIdx.x] = make_double2(ts, tc);
    }
    (void)shc;
}

template <class S>
void probs_impl(qe_state* s, int m, const int* qubits, double* host_out) {
    static thread_local ProbArgs<S> a;
    a.x = reinterpret_cast<const S*>(s->d);
    a.m = m;
    int tmp[32];
    for (int j = 0; j < m; ++j) {
        a.q[j] = (uint8_t)qubits[j];
        tmp[j] = qubits[j];
    }
    std::sort(tmp, tmp + m);
    for (int j = 0; j < m; ++j) a.q_sorted[j] = (uint8_t)tmp[j];
    const uint64_t bins = 1ull << m;
    a.per_bin = 1ull << (s->n - m);
    // about 8 blocks per SM in total, at least 2^14 amplitudes per block
    uint64_t want_blocks = (uint64_t)num_sms() * 8;
    uint64_t chunks = std::max<uint64_t>(1, want_blocks / bins);
    chunks = std::min<uint64_t>(chunks, std::max<uint64_t>(1, a.per_bin >> 14));
    a.chunks = chunks;
    a.chunk_len = (a.per_bin + chunks - 1) / chunks;
    const uint64_t nblocks = bins * chunks;
    char* scr = (char*)ensure_scratch(s, nblocks * sizeof(double2) + bins * sizeof(double));
    a.partial = (double2*)scr;
    double* dout = (double*)(scr + nblocks * sizeof(double2));
    if (nblocks > 0x7FFFFFFFull) fail(QE_ERR_UNSUPPORTED, "too many probability blocks");
    {
        Launch L(s, "probs_partial", (double)dim(s) * amp_bytes(s));
        if (std::is_same<S, double2>::value && s->c128_native)
            k_probs_partial_f64<<<(unsigned)nblocks, kRThreads, 0, s->stream>>>(
                *reinterpret_cast<ProbArgs<double2>*>(&a));
        else
            k_probs_partial<S><<<(unsigned)nblocks, kRThreads, 0, s->stream>>>(a);
        QE_CUDA(cudaGetLastError());
    }
    {
        Launch L(s, "sum_partials", 0.0, false);
        unsigned g2 = (unsigned)std::min<uint64_t>((bins + 255) / 256, 4096);
        k_sum_partials<<<g2, 256, 0, s->stream>>>(a.partial, bins, chunks, nullptr, dout);
        QE_CUDA(cudaGetLastError());
    }
    QE_CUDA(cudaMemcpyAsync(host_out, dout, bins * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QE_CUDA(cudaStreamSynchronize(s->stream));
}

template <class S>
double expect_impl(qe_state* s, int nterms, const uint64_t* xm, const uint64_t* zm, const double* cf) {
    static thread_local ExpArgs<S> a;
    a.x = reinterpret_cast<const S*>(s->d);
    a.count = dim(s);
    const int launches = (nterms + kNT - 1) / kNT;
    unsigned grid = (unsigned)std::min<uint64_t>((a.count + kRThreads - 1) / kRThreads,
                                                 (uint64_t)num_sms() * 8);
    char* scr = (char*)ensure_scratch(s, (size_t)launches * grid * sizeof(double2) + 64);
    double2* partial = (double2*)scr;
    double* dout = (double*)(scr + (size_t)launches * grid * sizeof(double2));
    for (int L = 0; L < launches; ++L) {
        a.nt = std::min(kNT, nterms - L * kNT);
        for (int t = 0; t < a.nt; ++t) {
            const int g = L * kNT + t;
            a.xm[t] = xm[g];
            a.zm[t] = zm[g];
            a.ny[t] = __builtin_popcountll(xm[g] & zm[g]) & 3;
            a.w[t] = cf[g];
        }
        a.partial = partial + (size_t)L * grid;
        Launch Lz(s, "expect_partial", (double)dim(s) * amp_bytes(s));
        k_expect_partial<S><<<grid, kRThreads, 0, s->stream>>>(a);
        QE_CUDA(cudaGetLastError());
    }
    {
        Launch Lz(s, "sum_partials", 0.0, false);
        k_sum_partials<<<1, 1, 0, s->stream>>>(partial, 1, (uint64_t)launches * grid, nullptr, dout);
        QE_CUDA(cudaGetLastError());
    }
    double out = 0.0;
    QE_CUDA(cudaMemcpyAsync(&out, dout, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QE_CUDA(cudaStreamSynchronize(s->stream));
    return out;
}

}  // namespace

double reduce_norm2(qe_state* s) {
    double out = 0.0;
    if (s->dtype == QE_C128) probs_impl<double2>(s, 0, nullptr, &out);
    else probs_impl<float2>(s, 0, nullptr, &out);
    return out;
}

void reduce_probs(qe_state* s, int m, const int* qubits, double* out) {
    if (s->dtype == QE_C128) probs_impl<double2>(s, m, qubits, out);
    else probs_impl<float2>(s, m, qubits, out);
}

double reduce_expectation(qe_state* s, int nterms, const uint64_t* xm, const uint64_t* zm,
                          const double* cf) {
    if (nterms == 0) return 0.0;
    if (s->dtype == QE_C128) return expect_impl<double2>(s, nterms, xm, zm, cf);
    return expect_impl<float2>(s, nterms, xm, zm, cf);
}

}  // namespace qe
