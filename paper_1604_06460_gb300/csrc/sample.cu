// Measurement (Sec. II): measuring qubits yields the value r of their bits
// with probability P(r), the sum of |alpha_x|^2 over the basis states x whose
// bits spell r, and leaves the state collapsed onto that value.  An emulator
// can draw many samples from the full distribution at once (Sec. III-D) and
// can apply the collapse directly.
//
// Sampling inverts the cumulative distribution with uniforms the caller
// passes in (so that samples are reproducible): shot s returns the smallest
// r whose cumulative probability exceeds u_s times the total, or, when
// rounding leaves none, the largest r with P(r) > 0.
//   - all qubits: the state is cut into blocks of 2^12 amplitudes; one pass
//     sums |alpha|^2 per block (FP64), one CTA scans the block sums, and a
//     warp per shot finds the block by binary search and the amplitude
//     inside it by a warp scan of lane sums and a scan of one lane's run;
//   - m <= 16 qubits: the 2^m marginal probabilities (the probability
//     reduction), the same scan, and a binary search per shot.
// All sums are FP64 in a fixed order, so a sample depends only on the state
// and the uniforms.
//
// Collapse: one reduction of the outcome's probability p (FP64), then one
// pass that zeroes the other amplitudes and scales the outcome's by 1/sqrt(p).
#include <algorithm>
#include <cmath>
#include <vector>

#include "qe_arith.cuh"
#include "qe_internal.h"

namespace qe {

namespace {

constexpr int kBlockBits = 12;   // amplitudes per block of the full distribution
constexpr int kMassThreads = 256;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ double prob_of(double2 v) { return __fma_rn(v.x, v.x, __dmul_rn(v.y, v.y)); }
__device__ __forceinline__ double prob_of(float2 v) {
    const double re = v.x, im = v.y;
    return __fma_rn(re, re, __dmul_rn(im, im));
}

// mass[k] = sum of |alpha|^2 over block k: thread t takes elements t, t + 256,
// ... of the block, then a fixed reduction tree.
template <class S>
__global__ void __launch_bounds__(kMassThreads) k_block_mass(const S* __restrict__ x, uint64_t nblocks, int B,
                                                             double* __restrict__ mass) {
    __shared__ double sh[kMassThreads / 32];
    const uint32_t E = 1u << B;
    for (uint64_t k = blockIdx.x; k < nblocks; k += gridDim.x) {
        const S* blk = x + (k << B);
        double acc = 0.0;
        for (uint32_t i = threadIdx.x; i < E; i += blockDim.x) acc += prob_of(blk[i]);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kMassThreads / 32; ++w) t += sh[w];
            mass[k] = t;
        }
        __syncthreads();
    }
}

// Inclusive prefix sums of K values by one CTA: thread t owns a contiguous
// chunk, the chunk totals are scanned in order by thread 0.
__global__ void __launch_bounds__(kScanThreads) k_scan(const double* __restrict__ w, uint64_t K,
                                                       double* __restrict__ incl) {
    __shared__ double off[kScanThreads];
    const uint64_t C = (K + kScanThreads - 1) / kScanThreads;
    const uint64_t b = threadIdx.x * C, e = min(K, b + C);
    double s = 0.0;
    for (uint64_t i = b; i < e; ++i) s += w[i];
    off[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = 0.0;
        for (int t = 0; t < kScanThreads; ++t) {
            const double v = off[t];
            off[t] = run;
            run += v;
        }
    }
    __syncthreads();
    double run = off[threadIdx.x];
    for (uint64_t i = b; i < e; ++i) {
        run += w[i];
        incl[i] = run;
    }
}

// Smallest k < K with incl[k] > target, or K if none.
__device__ __forceinline__ uint64_t first_above(const double* incl, uint64_t K, double target) {
    uint64_t lo = 0, hi = K;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (incl[mid] > target) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Largest k < K with w[k] > 0 (0 if none).
__device__ __forceinline__ uint64_t last_positive(const double* w, uint64_t K) {
    for (uint64_t k = K; k > 0; --k)
        if (w[k - 1] > 0.0) return k - 1;
    return 0;
}

// One thread per shot over K bins (the marginal distribution).
__global__ void k_shots_bins(const double* __restrict__ w, const double* __restrict__ incl, uint64_t K,
                             const double* __restrict__ u, int nshots, uint64_t* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nshots) return;
    const double target = u[s] * incl[K - 1];
    const uint64_t k = first_above(incl, K, target);
    out[s] = (k < K) ? k : last_positive(w, K);
}

// One warp per shot over the full distribution: block by binary search, then
// lane runs of C = 2^B / 32 contiguous amplitudes, scanned in order.
template <class S>
__global__ void __launch_bounds__(256) k_shots_full(const S* __restrict__ x, int B, uint64_t nblocks,
                                                    const double* __restrict__ mass,
                                                    const double* __restrict__ incl,
                                                    const double* __restrict__ u, int nshots,
                                                    uint64_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nshots) return;
    const double total = incl[nblocks - 1];
    const double target = u[s] * total;
    uint64_t k = first_above(incl, nblocks, target);
    const bool fallback = k >= nblocks;
    if (fallback) k = last_positive(mass, nblocks);
    const double rem = target - (k > 0 ? incl[k - 1] : 0.0);
    const uint32_t C = (1u << B) / 32u;
    const S* run = x + (k << B) + (uint64_t)lane * C;
    double ls = 0.0;
    uint32_t lastnz = 0xFFFFFFFFu;
    for (uint32_t i = 0; i < C; ++i) {
        const double p = prob_of(run[i]);
        ls += p;
        if (p > 0.0) lastnz = i;
    }
    // inclusive scan of the lane sums
    double inc = ls;
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    const double exc = inc - ls;
    uint64_t result = ~0ull;
    if (!fallback) {
        const uint32_t hit = __ballot_sync(0xffffffffu, inc > rem);
        if (hit) {
            const int l = __ffs(hit) - 1;
            if (lane == l) {
                double acc = exc;
                for (uint32_t i = 0; i < C; ++i) {
                    acc += prob_of(run[i]);
                    if (acc > rem) {
                        result = (k << B) + (uint64_t)lane * C + i;
                        break;
                    }
                }
            }
            // the lane's own rescan can miss by rounding: then its last nonzero
            const uint32_t found = __ballot_sync(0xffffffffu, result != ~0ull);
            if (!found && lane == l && lastnz != 0xFFFFFFFFu) result = (k << B) + (uint64_t)lane * C + lastnz;
        }
    }
    // no crossing in this block (rounding, or the target at the total): the
    // block's last amplitude of nonzero probability
    const uint32_t have = __ballot_sync(0xffffffffu, result != ~0ull);
    if (!have) {
        const uint32_t nz = __ballot_sync(0xffffffffu, lastnz != 0xFFFFFFFFu);
        const int l = nz ? 31 - __clz(nz) : 0;
        if (lane == l) result = (k << B) + (uint64_t)lane * C + (lastnz != 0xFFFFFFFFu ? lastnz : 0u);
    }
    const uint32_t who = __ballot_sync(0xffffffffu, result != ~0ull);
    if (lane == __ffs(who) - 1) out[s] = result;
}

// Probability of the outcome: the 2^(n - m) amplitudes whose measured bits
// spell it, FP64 partial sums per block.
template <class S>
struct MaskedArgs {
    const S* x;
    uint64_t count;     // 2^(n - m)
    uint64_t value;     // the outcome deposited on the measured qubits
    int m;
    uint8_t sorted[64];
    double* partial;
};

template <class S>
__global__ void __launch_bounds__(kMassThreads) k_masked_mass(const __grid_constant__ MaskedArgs<S> a) {
    __shared__ double sh[kMassThreads / 32];
    double acc = 0.0;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < a.count;
         t += (uint64_t)gridDim.x * blockDim.x)
        acc += prob_of(a.x[insert_zero_bits(t, a.sorted, a.m) | a.value]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kMassThreads / 32; ++w) t += sh[w];
        a.partial[blockIdx.x] = t;
    }
}

// One thread: Neumaier sum of the block partials in order.
__global__ void k_sum_ordered(const double* __restrict__ partial, int count, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0, c = 0.0;
    for (int i = 0; i < count; ++i) {
        const double v = partial[i];
        const double t = s + v;
        if (fabs(s) >= fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    out[0] = s + c;
}

__device__ __forceinline__ double2 scaled(double2 v, double f) { return make_double2(v.x * f, v.y * f); }
__device__ __forceinline__ float2 scaled(float2 v, double f) {
    const float g = (float)f;
    return make_float2(v.x * g, v.y * g);
}

template <class S>
__global__ void __launch_bounds__(256) k_collapse(S* __restrict__ x, uint64_t dim, uint64_t mask, uint64_t value,
                                                  double inv) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < dim; i += (uint64_t)gridDim.x * blockDim.x)
        x[i] = ((i & mask) == value) ? scaled(x[i], inv) : S{};
}

template <class S>
void sample_impl(qe_state* s, int m, const int* qubits, int nshots, const double* u_host, uint64_t* out_host) {
    const bool full = (m == 0);
    const int B = std::min(kBlockBits, s->n);
    const uint64_t K = full ? (dim(s) >> B) : (1ull << m);
    const uint64_t nparts = full ? 0 : probs_partials_needed(s, m);
    // scratch: [weights K][inclusive sums K][uniforms][outcomes][probability partials]
    const size_t w_off = 0, i_off = w_off + K * 8, u_off = i_off + K * 8;
    const size_t o_off = u_off + (size_t)nshots * 8, p_off = o_off + (size_t)nshots * 8;
    char* scr = (char*)ensure_scratch(s, p_off + nparts * sizeof(double2) + 256);
    double* w = (double*)(scr + w_off);
    double* incl = (double*)(scr + i_off);
    double* u = (double*)(scr + u_off);
    uint64_t* out = (uint64_t*)(scr + o_off);
    QE_CUDA(cudaMemcpyAsync(u, u_host, (size_t)nshots * 8, cudaMemcpyHostToDevice, s->stream));
    const S* x = reinterpret_cast<const S*>(s->d);
    if (full) {
        Launch L(s, "sample_block_mass", (double)dim(s) * amp_bytes(s));
        const unsigned grid = (unsigned)std::min<uint64_t>(K, (uint64_t)num_sms() * 8);
        k_block_mass<S><<<grid, kMassThreads, 0, s->stream>>>(x, K, B, w);
        QE_CUDA(cudaGetLastError());
    } else {
        reduce_probs_device(s, m, qubits, (double2*)(scr + p_off), w);
    }
    {
        Launch L(s, "sample_scan", 0.0, false);
        k_scan<<<1, kScanThreads, 0, s->stream>>>(w, K, incl);
        QE_CUDA(cudaGetLastError());
    }
    {
        Launch L(s, "sample_shots", 0.0, false);
        if (full) {
            const unsigned grid = (unsigned)(((uint64_t)nshots * 32 + 255) / 256);
            k_shots_full<S><<<grid, 256, 0, s->stream>>>(x, B, K, w, incl, u, nshots, out);
        } else {
            k_shots_bins<<<(nshots + 255) / 256, 256, 0, s->stream>>>(w, incl, K, u, nshots, out);
        }
        QE_CUDA(cudaGetLastError());
    }
    QE_CUDA(cudaMemcpyAsync(out_host, out, (size_t)nshots * 8, cudaMemcpyDeviceToHost, s->stream));
    QE_CUDA(cudaStreamSynchronize(s->stream));
}

template <class S>
double collapse_impl(qe_state* s, int m, const int* qubits, uint64_t outcome) {
    static thread_local MaskedArgs<S> a;
    a.x = reinterpret_cast<const S*>(s->d);
    a.m = m;
    uint64_t mask = 0, value = 0;
    int srt[64];
    for (int j = 0; j < m; ++j) {
        mask |= 1ull << qubits[j];
        if ((outcome >> j) & 1ull) value |= 1ull << qubits[j];
        srt[j] = qubits[j];
    }
    std::sort(srt, srt + m);
    for (int j = 0; j < m; ++j) a.sorted[j] = (uint8_t)srt[j];
    a.value = value;
    a.count = 1ull << (s->n - m);
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((a.count + kMassThreads - 1) / kMassThreads,
                                                                   (uint64_t)num_sms() * 8));
    char* scr = (char*)ensure_scratch(s, (size_t)grid * 8 + 256);
    a.partial = (double*)(scr + 256);
    double* dp = (double*)scr;
    {
        Launch L(s, "collapse_mass", (double)a.count * amp_bytes(s), false);
        k_masked_mass<S><<<grid, kMassThreads, 0, s->stream>>>(a);
        QE_CUDA(cudaGetLastError());
        k_sum_ordered<<<1, 32, 0, s->stream>>>(a.partial, grid, dp);
        QE_CUDA(cudaGetLastError());
    }
    double p = 0.0;
    QE_CUDA(cudaMemcpyAsync(&p, dp, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QE_CUDA(cudaStreamSynchronize(s->stream));
    if (!(p > 0.0)) fail(QE_ERR_ARG, "the outcome has probability zero");
    {
        Launch L(s, "collapse", 2.0 * dim(s) * amp_bytes(s));
        const unsigned g = (unsigned)std::min<uint64_t>((dim(s) + 255) / 256, (uint64_t)num_sms() * 8);
        k_collapse<S><<<g, 256, 0, s->stream>>>(reinterpret_cast<S*>(s->d), dim(s), mask, value, 1.0 / std::sqrt(p));
        QE_CUDA(cudaGetLastError());
    }
    return p;
}

}  // namespace

void sample_shots(qe_state* s, int m, const int* qubits, int nshots, const double* u, uint64_t* out) {
    if (nshots == 0) return;
    int all[16];
    if (m == 0 && s->n <= 16) {   // small states: all qubits as one marginal of 2^n bins
        for (int j = 0; j < s->n; ++j) all[j] = j;
        m = s->n;
        qubits = all;
    }
    if (s->dtype == QE_C128) sample_impl<double2>(s, m, qubits, nshots, u, out);
    else sample_impl<float2>(s, m, qubits, nshots, u, out);
}

double collapse(qe_state* s, int m, const int* qubits, uint64_t outcome) {
    if (s->dtype == QE_C128) return collapse_impl<double2>(s, m, qubits, outcome);
    return collapse_impl<float2>(s, m, qubits, outcome);
}

}  // namespace qe
