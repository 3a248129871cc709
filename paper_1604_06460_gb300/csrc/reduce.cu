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
// In the FP64 mode (complex128) the products and per-thread sums of the
// probability and pair-indexed expectation kernels are native FP64 (53-bit
// significands) instead, with the same FP64 compensated combination of the
// block partials.  Expectation values of complex128 states whose terms fit
// the register rounds are computed in exact fixed point instead, in either
// mode (k_expect_fx).
#include <algorithm>
#include <cstdlib>
#include <type_traits>
#include <vector>

#include "qe_arith.cuh"
#include "qe_internal.h"
#include "qe_oz.cuh"

namespace qe {

namespace {

constexpr int kRThreads = 256;

// Expectation kernel choice (a test and measurement switch, read per call):
// QE_EXPECT_TILE=1 keeps every expectation on the pair-indexed tile kernel,
// =2 takes the register-round kernel whenever the terms fit it; otherwise it
// is taken when it needs no more launches.
int expect_kernel_switch() {
    const char* e = std::getenv("QE_EXPECT_TILE");
    return (e && (e[0] == '1' || e[0] == '2')) ? e[0] - '0' : 0;
}

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
// FP32 inputs: exact products by TwoProd (no low parts to cross).
__device__ __forceinline__ void two_prod_sum(float a, float b, float c, float d, float& h, float& l) {
    // a*b + c*d with both products exact and one TwoSum
    const float p = fmul(a, b), pe = __fmaf_rn(a, b, -p);
    const float q = fmul(c, d), qe = __fmaf_rn(c, d, -q);
    const float s = fadd(p, q), bb = fsub(s, p);
    const float e = fadd(fsub(p, fsub(s, bb)), fsub(q, bb));
    h = s;
    l = fadd(e, fadd(pe, qe));
}
__device__ __forceinline__ void abs2(const float2& v, float& h, float& l) {
    two_prod_sum(v.x, v.x, v.y, v.y, h, l);
}
__device__ __forceinline__ void abs2(const DF::V& v, float& h, float& l) {
    df_first(h, l, v.re, v.re);
    df_acc(h, l, v.im, v.im);
}
// Re(conj(w) * v * i^ny):  conj(w) v = (w.re v.re + w.im v.im) + i (w.re v.im - w.im v.re)
__device__ __forceinline__ void corr(const float2& w, const float2& v, int ny, float& h, float& l) {
    if ((ny & 1) == 0) two_prod_sum(w.x, v.x, w.y, v.y, h, l);
    else two_prod_sum(w.x, v.y, -w.y, v.x, h, l);
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

// -v, and acc += Re (im = false) or Im (im = true) of conj(w) v, accumulated
// with exact products and TwoSum (no intermediate rounding of the pair).
__device__ __forceinline__ float2 vneg(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ DF::V vneg(const DF::V& v) {
    return DF::V{df{-v.re.h, -v.re.l}, df{-v.im.h, -v.im.l}};
}
__device__ __forceinline__ void corr_acc(Acc& a, const float2& w, const float2& v, bool im) {
    float h, l;
    if (!im) two_prod_sum(w.x, v.x, w.y, v.y, h, l);
    else two_prod_sum(w.x, v.y, -w.y, v.x, h, l);
    acc_add(a, h, l);
}
__device__ __forceinline__ void corr_acc(Acc& a, const DF::V& w, const DF::V& v, bool im) {
    if (!im) {
        df_acc(a.s, a.e, w.re, v.re);
        df_acc(a.s, a.e, w.im, v.im);
    } else {
        df_acc(a.s, a.e, w.re, v.im);
        df_acc_neg(a.s, a.e, w.im, v.re);
    }
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

// Asynchronous global -> shared copy of one amplitude (8 or 16 bytes).
template <int N>
__device__ __forceinline__ void async_copy(void* dst, const void* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if (N == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src));
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src));
}

// Policy views of an amplitude for the reducers.
__device__ __forceinline__ float2 rview(float2 v) { return v; }
__device__ __forceinline__ DF::V rview(double2 v) { return DF::load(v); }

// Native FP64 reductions (the FP64 mode of complex128 states): one FP64
// accumulator per quantity, products by fused multiply-add.
struct AccD {
    double s;
};
__device__ __forceinline__ double abs2d(const double2& v) { return __fma_rn(v.x, v.x, __dmul_rn(v.y, v.y)); }
__device__ __forceinline__ double block_reduce_d(double a, double* sh) {
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = a;
    __syncthreads();
    if (w == 0) {
        a = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    }
    return a;   // valid in thread 0
}

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

// One block per output (grid-stride over outputs): Neumaier sums of the
// `count` partials of an output, thread t taking partials t, t + 256, ...;
// the 256 compensated sums are then combined pairwise in a fixed tree, so the
// result does not depend on timing.
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) k_sum_partials(const double2* __restrict__ partial, uint64_t nout,
                                                              uint64_t count, const double* __restrict__ weight,
                                                              double* __restrict__ out) {
    __shared__ double ss[kSumThreads], cs[kSumThreads];
    for (uint64_t o = blockIdx.x; o < nout; o += gridDim.x) {
        double s = 0.0, c = 0.0;
        for (uint64_t i = threadIdx.x; i < count; i += kSumThreads) {
            const double2 p = partial[o * count + i];
            neumaier(s, c, p.x);
            neumaier(s, c, p.y);
        }
        ss[threadIdx.x] = s;
        cs[threadIdx.x] = c;
        __syncthreads();
        for (int h = kSumThreads / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) {
                double a = ss[threadIdx.x], ac = cs[threadIdx.x];
                neumaier(a, ac, ss[threadIdx.x + h]);
                ss[threadIdx.x] = a;
                cs[threadIdx.x] = ac + cs[threadIdx.x + h];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) out[o] = (ss[0] + cs[0]) * (weight ? weight[o] : 1.0);
        __syncthreads();
    }
}

// ---------------------------------------------------------- expectation
// Terms are evaluated on shared-memory tiles.  A launch covers one tile
// layout: the chunk bits [0, L) plus a set of higher qubits (hq); every term
// it evaluates has its X/Y qubits inside the layout, so the partner
// amplitude alpha_{x ^ xm} is in the same tile.  An index is x = base + l,
// base the tile's offset (zero at the layout's bits) and l the tile-local
// index, so every parity splits as popc(x & z) = popc(l & z_loc) +
// popc(base & z_out): the second part is one bit per tile, computed once by
// the first warp.  Z-only terms of equal weight share one integer count of
// odd parities per amplitude:
//     sum_t w (-1)^popc(x & z_t) = w (N_g - 2 #{t : popc(x & z_t) odd});
// masks with no bit in the layout contribute a per-tile constant.  Terms with
// X/Y parts accumulate Re or Im of conj(alpha_{x^xm}) alpha_x, signed by
// (-1)^popc(x & zm), over the x whose lowest xm bit is clear; the factor 2 and
// the sign of i^ny sit in the coefficient.
constexpr int kZW = 4;     // Z-only weight groups per launch
constexpr int kZT = 64;    // Z-only masks per launch
constexpr int kXT = 12;    // terms with X/Y parts per launch
template <class S>
struct ExpArgs {
    const S* x;
    uint64_t ntiles;
    int L, T, kh;
    uint8_t hq[16];
    int nzg;                   // weight groups
    int zg_loc_end[kZW];       // group g: masks [begin, zg_loc_end) touch the layout,
    int zg_end[kZW];           //          [zg_loc_end, zg_end) lie outside it
    double zw[kZW];
    int nz;
    uint32_t zl[kZT];          // mask bits inside the layout, at tile-local positions
    uint64_t zo[kZT];          // mask bits outside the layout (global positions)
    int nxt;
    uint32_t xloc[kXT];        // X/Y mask at tile-local positions
    uint32_t xzl[kXT];         // Z mask inside the layout (tile-local positions)
    uint64_t xzo[kXT];         // Z mask outside the layout
    uint32_t xbelow[kXT];      // bits below the lowest X/Y bit (tile-local)
    int ximag[kXT];            // 1: Im(conj(alpha_{x^xm}) alpha_x), 0: Re
    int xsigned[kXT];          // the term has a Z part (a sign per amplitude)
    double xw[kXT];            // 2 * coefficient * (+-1 from i^ny)
    double2* partial;          // one per block
};

// Amplitudes per thread in one tile (the tile has at most 2^Tmax amplitudes).
template <class S>
constexpr int kPer = (sizeof(S) >= 16 ? (1 << 11) : (1 << 12)) / kRThreads;

__device__ __forceinline__ void acc_zero(Acc& a) { a = Acc{0.f, 0.f}; }
__device__ __forceinline__ void acc_zero(AccD& a) { a.s = 0.0; }

// NAT: native FP64 (complex128 in the FP64 mode); otherwise double-float
// views (complex128) or FP32 (complex64) with compensated float sums.
template <class S, bool NAT>
__global__ void __launch_bounds__(kRThreads) k_expect_tile(const __grid_constant__ ExpArgs<S> a) {
    using V = std::conditional_t<NAT, S, decltype(rview(S{}))>;
    using A = std::conditional_t<NAT, AccD, Acc>;
    constexpr int PER = kPer<S>;
    static_assert(sizeof(V) == sizeof(S), "tiles are converted in place");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // two tiles: the raw amplitudes of the next tile stream in (cp.async)
    // while the current one is evaluated, then are converted in place
    V* const tiles = reinterpret_cast<V*>(smem_raw);
    __shared__ Acc sh[32];
    __shared__ double shd[32];
    __shared__ uint64_t offA[64], offB[64];
    __shared__ uint32_t s_zl[kZT];       // zl with the tile's outside parity in bit 31
    __shared__ int s_zout[kZW];          // per group: odd outside-only masks of this tile
    __shared__ uint32_t s_xflip;         // bit k: outside parity of X/Y term k's Z mask
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < 64) {
        uint64_t oa = 0, ob = 0;
        for (int j = 0; j < 6 && j < a.kh; ++j)
            if ((tid >> j) & 1) oa |= 1ull << a.hq[j];
        for (int j = 6; j < a.kh; ++j)
            if ((tid >> (j - 6)) & 1) ob |= 1ull << a.hq[j];
        offA[tid] = oa;
        offB[tid] = ob;
    }
    __syncthreads();
    A zacc[kZW], zacc2[kZW], xacc[kXT];
#pragma unroll
    for (int g = 0; g < kZW; ++g) {
        acc_zero(zacc[g]);
        acc_zero(zacc2[g]);
    }
#pragma unroll
    for (int t = 0; t < kXT; ++t) acc_zero(xacc[t]);
    const uint32_t Tn = 1u << a.T, lowmask = (1u << a.L) - 1u;
    auto load = [&](uint64_t t, V* buf) {   // this thread's elements, raw
        const uint64_t b = insert_zero_bits(t << a.L, a.hq, a.kh);
        for (uint32_t l = tid; l < Tn; l += blockDim.x) {
            const uint32_t h = l >> a.L;
            async_copy<sizeof(S)>(buf + l, a.x + (b + (l & lowmask) + offA[h & 63] + offB[h >> 6]));
        }
        asm volatile("cp.async.commit_group;");
    };
    int cur = 0;
    if (blockIdx.x < a.ntiles) load(blockIdx.x, tiles);
    for (uint64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const uint64_t base = insert_zero_bits(t << a.L, a.hq, a.kh);
        V* const tile = tiles + (size_t)cur * Tn;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        if constexpr (sizeof(S) == 16 && !NAT)   // complex128: split into double-float in place
            for (uint32_t l = tid; l < Tn; l += blockDim.x) tile[l] = rview(*reinterpret_cast<const S*>(tile + l));
        __syncthreads();
        if (t + gridDim.x < a.ntiles) load(t + gridDim.x, tiles + (size_t)(cur ^ 1) * Tn);
        cur ^= 1;
        if (warp == 0) {
            // outside parities of this tile: Z-only masks, then X/Y terms
            uint32_t b0 = 0, b1 = 0;
            {
                const int k0 = lane, k1 = lane + 32;
                const uint32_t p0 = (k0 < a.nz) ? (uint32_t)(__popcll(base & a.zo[k0]) & 1) : 0u;
                const uint32_t p1 = (k1 < a.nz) ? (uint32_t)(__popcll(base & a.zo[k1]) & 1) : 0u;
                if (k0 < a.nz) s_zl[k0] = a.zl[k0] | (p0 << 31);
                if (k1 < a.nz) s_zl[k1] = a.zl[k1] | (p1 << 31);
                b0 = __ballot_sync(0xffffffffu, p0);
                b1 = __ballot_sync(0xffffffffu, p1);
            }
            const uint32_t px = (lane < a.nxt) ? (uint32_t)(__popcll(base & a.xzo[lane]) & 1) : 0u;
            const uint32_t xb = __ballot_sync(0xffffffffu, px);
            if (lane == 0) {
                s_xflip = xb;
                const uint64_t bits = ((uint64_t)b1 << 32) | b0;
                int begin = 0;
                for (int g = 0; g < a.nzg; ++g) {
                    const int lo = a.zg_loc_end[g], hi = a.zg_end[g];
                    const uint64_t m = (hi > lo) ? ((hi - lo >= 64 ? ~0ull : ((1ull << (hi - lo)) - 1ull)) << lo) : 0ull;
                    s_zout[g] = __popcll(bits & m);
                    begin = hi;
                }
                (void)begin;
            }
        }
        __syncthreads();
        if (a.nzg > 0) {
            constexpr int C = PER < 8 ? PER : 8;    // amplitudes per chunk
#pragma unroll 1
            for (int j0 = 0; j0 < PER; j0 += C) {
                float ph[C], pl[C];
                double pd[C];
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const uint32_t l = tid + (uint32_t)(j0 + j) * kRThreads;
                    if constexpr (NAT) {
                        pd[j] = (l < Tn) ? abs2d(tile[l]) : 0.0;
                    } else {
                        if (l < Tn) abs2(tile[l], ph[j], pl[j]);
                        else ph[j] = pl[j] = 0.f;
                    }
                }
                int begin = 0;
#pragma unroll
                for (int g = 0; g < kZW; ++g) {
                    if (g >= a.nzg) break;
                    int odd[C];
#pragma unroll
                    for (int j = 0; j < C; ++j) odd[j] = s_zout[g];
                    for (int k = begin; k < a.zg_loc_end[g]; ++k) {
                        const uint32_t zk = s_zl[k];
#pragma unroll
                        for (int j = 0; j < C; ++j)
                            odd[j] += __popc(((uint32_t)tid + (uint32_t)(j0 + j) * kRThreads + 0x80000000u) & zk) & 1;
                    }
                    const int ng = a.zg_end[g] - begin;
                    begin = a.zg_end[g];
#pragma unroll
                    for (int j = 0; j < C; ++j) {
                        if constexpr (NAT) {
                            A& z = (j & 1) ? zacc2[g] : zacc[g];
                            z.s = __fma_rn(pd[j], (double)(ng - 2 * odd[j]), z.s);
                        } else {
                            const float f = (float)(ng - 2 * odd[j]);
                            const float p = fmul(ph[j], f);
                            acc_add((j & 1) ? zacc2[g] : zacc[g], p, __fmaf_rn(pl[j], f, __fmaf_rn(ph[j], f, -p)));
                        }
                    }
                }
            }
        }
        // terms with X/Y parts: one thread per pair (l, l ^ xm) with the
        // lowest xm bit of l clear; the term loop is innermost so that
        // consecutive updates go to different accumulators
        const uint32_t xflip = s_xflip;
#pragma unroll 1
        for (int j = 0; j < PER / 2; ++j) {
            const uint32_t i = tid + (uint32_t)j * kRThreads;
            if (i >= Tn / 2) break;
#pragma unroll
            for (int k = 0; k < kXT; ++k) {
                if (k >= a.nxt) break;
                const uint32_t xl = a.xloc[k], below = a.xbelow[k];
                const uint32_t l = ((i & ~below) << 1) | (i & below);
                const bool flip = a.xsigned[k] && ((__popc(l & a.xzl[k]) ^ (xflip >> k)) & 1u);
                if constexpr (NAT) {
                    // Re or Im of conj(w) v as w.x p + w.y q, the operands
                    // chosen and signed with integer selects, so that the FP64
                    // pipe runs exactly two fused multiply-adds per pair
                    const double2 w = tile[l ^ xl], v = tile[l];
                    const bool im = a.ximag[k] != 0;
                    const unsigned long long sgn = flip ? 0x8000000000000000ull : 0ull;
                    const unsigned long long vx = __double_as_longlong(v.x), vy = __double_as_longlong(v.y);
                    const double p = __longlong_as_double((im ? vy : vx) ^ sgn);
                    const double q = __longlong_as_double((im ? (vx ^ 0x8000000000000000ull) : vy) ^ sgn);
                    xacc[k].s = __fma_rn(w.x, p, __fma_rn(w.y, q, xacc[k].s));
                } else {
                    V w = tile[l ^ xl];
                    const V v = tile[l];
                    if (flip) w = vneg(w);
                    corr_acc(xacc[k], w, v, a.ximag[k] != 0);
                }
            }
        }
        __syncthreads();
    }
    double s = 0.0, c = 0.0;
#pragma unroll
    for (int g = 0; g < kZW; ++g) {
        if (g >= a.nzg) break;
        if constexpr (NAT) {
            const double r = block_reduce_d(zacc[g].s + zacc2[g].s, shd);
            if (tid == 0) neumaier(s, c, r * a.zw[g]);
        } else {
            Acc r = block_reduce(acc_merge(zacc[g], zacc2[g]), sh);
            if (tid == 0) {
                df d = df_norm(r.s, r.e);
                neumaier(s, c, df2d(d.h, d.l) * a.zw[g]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kXT; ++k) {
        if (k >= a.nxt) break;
        if constexpr (NAT) {
            const double r = block_reduce_d(xacc[k].s, shd);
            if (tid == 0) neumaier(s, c, r * a.xw[k]);
        } else {
            Acc r = block_reduce(xacc[k], sh);
            if (tid == 0) {
                df d = df_norm(r.s, r.e);
                neumaier(s, c, df2d(d.h, d.l) * a.xw[k]);
            }
        }
    }
    if (tid == 0) a.partial[blockIdx.x] = make_double2(s, c);
}

// ------------------------------------- expectation by register rounds
// Tiles of 2^12 amplitudes (the chunk bits [0, L) plus 12 - L high qubits),
// 512 threads, eight amplitudes a thread at a time.  The tile's local bits
// form four triples {0,1,2}, {3,4,5}, {6,7,8}, {9,10,11}; in round r a thread
// holds the eight amplitudes that differ only in triple r (its other nine
// local bits come from the thread index), so a term whose X/Y bits lie in
// triple r pairs two of those registers: no index arithmetic and one shared
// load per amplitude and round.  Z-only masks are counted in round 0 from
// per-mask parity bytes (bit j: the parity of amplitude j), summed bytewise.
// All X/Y terms of a launch share one weight, so one accumulator serves them.
// Shared tiles are XOR-swizzled so that every round's loads are free of bank
// conflicts; three tile buffers keep two tiles in flight (cp.async).
constexpr int kT2 = 12, kThr2 = 512, kXT2 = 24, kNB2 = 3;

template <class S>
struct RoundArgs {
    const S* x;
    uint64_t ntiles;
    int L, kh;
    uint8_t hq[8];            // local bit L + j <-> qubit hq[j]
    uint8_t hq_sorted[8];     // the same qubits ascending (tile base)
    int nzg, nz;
    int zg_end[kZW];          // group g: Z masks [zg_end[g - 1], zg_end[g])
    double zw[kZW];
    uint32_t zl[kZT];         // tile-local bits of Z mask m
    uint64_t zo[kZT];         // its bits outside the tile
    uint8_t zpz[kZT];         // bit j: parity of j & (its bits in triple 0)
    int rb[5];                // round r: X/Y terms [rb[r], rb[r + 1])
    int nxt;
    uint32_t xw[kXT2];        // bits 0-2: X bits in the round's triple; 3-10: bit j = parity of j & the
                              // term's Z bits in the triple; 11: Im part; 12: negated (i^ny); 13: has a
                              // Z part (a sign per pair)
    uint32_t xzl[kXT2];       // the term's Z bits at tile-local positions
    uint64_t xzo[kXT2];       // and outside the tile
    double wx;                // 2 x the common coefficient of the X/Y terms
    double2* partial;
    // fixed-point kernel: per weight group, the Z masks (bit m) inside the
    // tile, wholly outside it, and with bits on both sides
    uint64_t zin[kZW], zout[kZW], zmix[kZW];
    uint8_t xtb[4][9];        // round r: its terms with X/Y bits x (in the triple) are [xtb[r][x], xtb[r][x + 1])
    uint8_t xplain[4][8];     // round r: how many X strings without Z bits have the pattern x (not in the lists)
    int rmask;                // bit r: round r has X/Y terms
    uint32_t* status;         // raised when a copy wait ran out
    long long spin_limit;
    int stall_test;           // failure-path test: block 0's first tile is announced but never copied
};

template <int EB>
__device__ __forceinline__ uint32_t swz(uint32_t l) {
    if constexpr (EB == 16) return l ^ ((l >> 3) & 7u);
    else return l ^ ((l >> 4) & 7u) ^ ((l >> 3) & 8u);
}

// tile-local index of a thread's amplitude 0 in round r (triple r zero)
__device__ __forceinline__ uint32_t round_base(uint32_t tid, int r) {
    const int s = 3 * r;
    return (tid & ((1u << s) - 1u)) | ((tid >> s) << (s + 3));
}

// acc += (-1)^neg Re (IM = false) or Im (IM = true) of conj(w) v (float
// pairs); SIGNED = false: no per-pair sign (neg is ignored)
template <bool IM, bool SIGNED, class V>
__device__ __forceinline__ void pair_acc(Acc& acc, const V& w, const V& v, uint32_t neg) {
    if constexpr (SIGNED) corr_acc(acc, neg ? vneg(w) : w, v, IM);
    else corr_acc(acc, w, v, IM);
}

// the four pairs (j, j ^ XT) with the lowest bit of XT clear in j
template <int XT, bool IM, bool SIGNED, class V, class A>
__device__ __forceinline__ void round_pairs(const V (&v)[8], uint32_t zp, uint32_t f, A& acc) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j & (XT & -XT)) continue;
        pair_acc<IM, SIGNED>(acc, v[j ^ XT], v[j], f ^ ((zp >> j) & 1u));
    }
}

// One term: XT and Im select the code path (uniform across the block); each
// pair is signed with selects.
template <int XT, class V, class A>
__device__ __forceinline__ void round_term(const V (&v)[8], uint32_t zp, uint32_t f, bool im, A& xacc) {
    if (im) round_pairs<XT, true, true>(v, zp, f, xacc);
    else round_pairs<XT, false, true>(v, zp, f, xacc);
}

// complex64 (complex128 states take k_expect_fx)
template <class S>
__global__ void __launch_bounds__(kThr2, 1) k_expect_rounds(const __grid_constant__ RoundArgs<S> a) {
    static_assert(sizeof(S) == 8, "complex64 tiles");
    using V = S;
    using A = Acc;
    using W = float;
    constexpr int EB = (int)sizeof(S);
    constexpr uint32_t Tn = 1u << kT2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* const tiles = reinterpret_cast<V*>(smem_raw);
    __shared__ Acc sh[32];
    __shared__ uint64_t offA[64];
    __shared__ uint64_t spread[256];          // byte j of spread[p] = bit j of p
    __shared__ W s_cnt[kZW][kZT + 1];         // group g, o odd masks: (masks of g) - 2 o
    __shared__ uint64_t s_zbits;              // bit m: outside parity of Z mask m (this tile)
    __shared__ uint32_t s_xbits;              // bit k: outside parity of term k's Z bits
    const uint32_t tid = threadIdx.x;
    if (tid < 64) {
        uint64_t o = 0;
        for (int j = 0; j < a.kh; ++j)
            if ((tid >> j) & 1u) o |= 1ull << a.hq[j];
        offA[tid] = o;
    }
    if (tid < 256) {
        uint64_t sp = 0;
        for (int j = 0; j < 8; ++j) sp |= (uint64_t)((tid >> j) & 1u) << (8 * j);
        spread[tid] = sp;
    }
    for (uint32_t i = tid; i < (uint32_t)(kZW * (kZT + 1)); i += blockDim.x) {
        const int g = (int)i / (kZT + 1), o = (int)i % (kZT + 1);
        const int ng = g < a.nzg ? a.zg_end[g] - (g ? a.zg_end[g - 1] : 0) : 0;
        s_cnt[g][o] = (W)(ng - 2 * o);
    }
    // parities of the thread's part of each mask (fixed for the launch)
    uint64_t tz = 0;
    {
        const uint32_t lt0 = round_base(tid, 0);
        for (int m = 0; m < a.nz; ++m) tz |= (uint64_t)(__popc(lt0 & a.zl[m]) & 1) << m;
    }
    uint32_t tx = 0;
    for (int r = 0; r < 4; ++r) {
        const uint32_t lt = round_base(tid, r);
        for (int k = a.rb[r]; k < a.rb[r + 1]; ++k) tx |= (uint32_t)(__popc(lt & a.xzl[k]) & 1) << k;
    }
    A zacc[kZW], xacc;
#pragma unroll
    for (int g = 0; g < kZW; ++g) acc_zero(zacc[g]);
    acc_zero(xacc);
    __syncthreads();
    const uint32_t lowmask = (1u << a.L) - 1u;
    auto load = [&](uint64_t t, V* buf) {
        const uint64_t b = insert_zero_bits(t << a.L, a.hq_sorted, a.kh);
#pragma unroll
        for (int i = 0; i < (int)(Tn / kThr2); ++i) {
            const uint32_t l = tid + (uint32_t)i * kThr2;
            async_copy<EB>(buf + swz<EB>(l), a.x + (b + (l & lowmask) + offA[l >> a.L]));
        }
    };
    const uint64_t step = gridDim.x;
#pragma unroll
    for (int s = 0; s < kNB2 - 1; ++s) {
        const uint64_t t = blockIdx.x + (uint64_t)s * step;
        if (t < a.ntiles) load(t, tiles + (size_t)s * Tn);
        asm volatile("cp.async.commit_group;");
    }
    int it = 0;
    for (uint64_t t = blockIdx.x; t < a.ntiles; t += step, ++it) {
        V* const tile = tiles + (size_t)(it % kNB2) * Tn;
        asm volatile("cp.async.wait_group %0;" ::"n"(kNB2 - 2) : "memory");
        if (tid < 32) {   // outside parities of this tile
            const uint64_t base = insert_zero_bits(t << a.L, a.hq_sorted, a.kh);
            const int lane = (int)tid;
            const uint32_t p0 = (lane < a.nz) ? (uint32_t)(__popcll(base & a.zo[lane]) & 1) : 0u;
            const uint32_t p1 = (lane + 32 < a.nz) ? (uint32_t)(__popcll(base & a.zo[lane + 32]) & 1) : 0u;
            const uint32_t px = (lane < a.nxt) ? (uint32_t)(__popcll(base & a.xzo[lane]) & 1) : 0u;
            const uint32_t b0 = __ballot_sync(0xffffffffu, p0), b1 = __ballot_sync(0xffffffffu, p1);
            const uint32_t xb = __ballot_sync(0xffffffffu, px);
            if (lane == 0) {
                s_zbits = ((uint64_t)b1 << 32) | b0;
                s_xbits = xb;
            }
        }
        __syncthreads();
        {
            const uint64_t tn = t + (uint64_t)(kNB2 - 1) * step;
            if (tn < a.ntiles) load(tn, tiles + (size_t)((it + kNB2 - 1) % kNB2) * Tn);
            asm volatile("cp.async.commit_group;");
        }
        const uint64_t zbits = tz ^ s_zbits;
        const uint32_t xflip = tx ^ s_xbits;
#pragma unroll 1
        for (int r = 0; r < 4; ++r) {
            const bool zr = (r == 0) && (a.nzg > 0);
            const int k0 = a.rb[r], k1 = a.rb[r + 1];
            if (k0 == k1 && !zr) continue;
            const uint32_t lt = round_base(tid, r);
            V v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = tile[swz<EB>(lt | ((uint32_t)j << (3 * r)))];
            if (zr) {
                uint64_t cnt[kZW];
                int m = 0;
#pragma unroll
                for (int g = 0; g < kZW; ++g) {
                    cnt[g] = 0;
                    if (g >= a.nzg) continue;
                    for (; m < a.zg_end[g]; ++m) {
                        const uint32_t pat = a.zpz[m] ^ ((uint32_t)((zbits >> m) & 1ull) * 0xFFu);
                        cnt[g] += spread[pat];
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float ph, pl;
                    abs2(v[j], ph, pl);
#pragma unroll
                    for (int g = 0; g < kZW; ++g) {
                        if (g >= a.nzg) break;
                        const float f = s_cnt[g][(cnt[g] >> (8 * j)) & 0xFFu];
                        const float p = fmul(ph, f);
                        acc_add(zacc[g], p, __fmaf_rn(pl, f, __fmaf_rn(ph, f, -p)));
                    }
                }
            }
            for (int k = k0; k < k1; ++k) {
                const uint32_t w = a.xw[k];
                const uint32_t f = ((xflip >> k) & 1u) ^ ((w >> 12) & 1u);
                const uint32_t zp = (w >> 3) & 0xFFu;
                const bool im = ((w >> 11) & 1u) != 0;
                switch (w & 7u) {
                    case 1: round_term<1>(v, zp, f, im, xacc); break;
                    case 2: round_term<2>(v, zp, f, im, xacc); break;
                    case 3: round_term<3>(v, zp, f, im, xacc); break;
                    case 4: round_term<4>(v, zp, f, im, xacc); break;
                    case 5: round_term<5>(v, zp, f, im, xacc); break;
                    case 6: round_term<6>(v, zp, f, im, xacc); break;
                    default: round_term<7>(v, zp, f, im, xacc); break;
                }
            }
        }
        __syncthreads();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    double s = 0.0, c = 0.0;
#pragma unroll
    for (int g = 0; g < kZW; ++g) {
        if (g >= a.nzg) break;
        Acc r = block_reduce(zacc[g], sh);
        if (tid == 0) {
            df d = df_norm(r.s, r.e);
            neumaier(s, c, df2d(d.h, d.l) * a.zw[g]);
        }
    }
    if (a.nxt > 0) {
        Acc r = block_reduce(xacc, sh);
        if (tid == 0) {
            df d = df_norm(r.s, r.e);
            neumaier(s, c, df2d(d.h, d.l) * a.wx);
        }
    }
    if (tid == 0) a.partial[blockIdx.x] = make_double2(s, c);
}

// ------------------------ expectation by register rounds in fixed point
// complex128 (both arithmetic modes): the round schedule of k_expect_rounds
// on integers.  Each tile arrives by bulk copies (one per contiguous run of
// the layout, or 16 KB pieces) on an mbarrier, three buffers deep, unswizzled:
// round 0's loads, whose eight amplitudes per thread are adjacent, go in a
// rotated order (amplitude j ^ (tid & 7) first), and the loads of rounds 1-3
// are conflict-free as they stand.
//
// Fixed point.  With E the largest biased exponent of the tile's components,
// component v becomes the integer q = v 2^(1076 - E) rounded to the nearest
// (|q| < 2^54; the largest component keeps its 53 significant bits, the
// others lose at most a quarter unit of the 53-bit grid 2^(E - 1075);
// rounding, not truncation, so the errors do not bias |v|^2 downwards).  A
// tile whose largest component is below 2^-959 is taken as zero (the products of
// such values underflow FP64 as well).  q is held as two limbs q = h 2^28 + l,
// |h| < 2^26, |l| < 2^28, so the product of two components is three
// 32 x 32 -> 64-bit integer multiply-adds: h h' at unit 2^56 and h l' + l h'
// at unit 2^28 are summed exactly in int64 accumulators (two independent
// chains each, positive and negative terms apart); the dropped l l' is below
// 2^-52 of the largest product.  A launch has at most 24 X/Y terms, so a
// thread's tile sums stay below 2^62.6.  At the end of a tile they are folded
// into one int64 at unit 2^56 (rounding to the nearest unit), summed exactly
// over four lanes, and one lane in four adds the tile's value, scaled by
// 2^(2 E - 2152), to its FP64 sum.  Z-only masks weigh |q|^2 (at unit 2^56,
// rounded the same way) by the integer count of even minus odd parities:
// masks inside the tile are counted once per launch, masks wholly outside it
// once per tile by a population count, and only masks with bits on both
// sides per amplitude.  The products thus run on the integer pipes, whose
// multiply-add rate is many times the FP64 pipe's.
struct Fx {
    int xh, xl, yh, yl;   // Re q = xh 2^28 + xl, Im q = yh 2^28 + yl
};
constexpr uint32_t kFxFlush = 64;   // tiles whose largest biased exponent is below this: zero

__device__ __forceinline__ uint32_t fx_exp(double v) { return ((uint32_t)__double2hiint(v) >> 20) & 0x7FFu; }

// the limbs of q = v 2^(1076 - emx) rounded to the nearest integer (ties
// away from zero), emx >= the exponent of v (and emx >= 64, so zero and
// subnormal v give d = 63 and q = 0)
__device__ __forceinline__ void fx_limbs(double v, uint32_t emx, int& h, int& l) {
    const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
    const uint64_t m4 = ((((uint64_t)((hi & 0xFFFFFu) | 0x100000u)) << 32) | lo) << 2;   // 4 m, below 2^55
    const uint32_t d = min(emx - ((hi >> 20) & 0x7FFu), 63u);
    const uint64_t q2 = ((m4 >> d) + 1u) >> 1;
    const int s = (int)hi >> 31;
    h = ((int)(q2 >> 28) ^ s) - s;
    l = ((int)((uint32_t)q2 & 0xFFFFFFFu) ^ s) - s;
}

// X/Y accumulators: two chains at unit 2^56 (H) and two at unit 2^28 (M)
struct FxAcc {
    long long h0, h1, m0, m1;
};

// acc += (-1)^neg Re (IM = false) or Im (IM = true) of conj(w) v
template <bool IM, bool SIGNED>
__device__ __forceinline__ void pair_fx(FxAcc& a, Fx w, const Fx& v, uint32_t neg) {
    if constexpr (SIGNED) {
        const int m = -(int)neg;
        w.xh = (w.xh ^ m) - m;
        w.xl = (w.xl ^ m) - m;
        w.yh = (w.yh ^ m) - m;
        w.yl = (w.yl ^ m) - m;
    }
    // C products (not inline PTX): each compiles to one 32 x 32 + 64 multiply-add
    if constexpr (!IM) {   // w.x v.x + w.y v.y
        a.h0 += (long long)w.xh * v.xh;
        a.h1 += (long long)w.yh * v.yh;
        a.m0 += (long long)w.xh * v.xl;
        a.m0 += (long long)w.xl * v.xh;
        a.m1 += (long long)w.yh * v.yl;
        a.m1 += (long long)w.yl * v.yh;
    } else {               // w.x v.y - w.y v.x
        a.h0 += (long long)w.xh * v.yh;
        a.h1 -= (long long)w.yh * v.xh;
        a.m0 += (long long)w.xh * v.yl;
        a.m0 += (long long)w.xl * v.yh;
        a.m1 -= (long long)w.yh * v.xl;
        a.m1 -= (long long)w.yl * v.xh;
    }
}

template <int XT, bool IM, bool SIGNED>
__device__ __forceinline__ void round_pairs_fx(const Fx (&v)[8], uint32_t zp, uint32_t f, FxAcc& a) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j & (XT & -XT)) continue;
        pair_fx<IM, SIGNED>(a, v[j ^ XT], v[j], f ^ ((zp >> j) & 1u));
    }
}

// one term: pairs signed by the Z parity (zp = 0 without a Z part) and the
// thread's sign f, unless no pair of the warp is negated
template <int XT>
__device__ __forceinline__ void round_term_fx(const Fx (&v)[8], uint32_t zp, uint32_t f, bool im, bool signed_term,
                                              FxAcc& acc) {
    if (signed_term || __any_sync(0xffffffffu, f != 0u)) {
        const uint32_t z = signed_term ? zp : 0u;
        if (im) round_pairs_fx<XT, true, true>(v, z, f, acc);
        else round_pairs_fx<XT, false, true>(v, z, f, acc);
    } else {
        if (im) round_pairs_fx<XT, true, false>(v, 0u, 0u, acc);
        else round_pairs_fx<XT, false, false>(v, 0u, 0u, acc);
    }
}

// the terms of round r whose X/Y bits in the triple are XT (sorted so on the
// host: one code block per pattern, no indirect branch)
template <int XT>
__device__ __forceinline__ void round_xt(const RoundArgs<double2>& a, int r, uint32_t rot, uint32_t xflip,
                                         const Fx (&v)[8], FxAcc& acc) {
#pragma unroll 1
    for (int k = a.xtb[r][XT]; k < a.xtb[r][XT + 1]; ++k) {
        const uint32_t w = a.xw[k];
        uint32_t f = ((xflip >> k) & 1u) ^ ((w >> 12) & 1u);
        const uint32_t zp = (w >> 3) & 0xFFu;
        const bool im = ((w >> 11) & 1u) != 0, sg = ((w >> 13) & 1u) != 0;
        if (r == 0) {
            // register i holds amplitude i ^ rot.  A pair (i, i ^ XT), i
            // without XT's lowest bit, is the amplitude pair (j, j ^ XT) with
            // j = i ^ rot, or with the roles of its two members swapped when
            // rot has that bit (Im changes sign); its Z parity is that of i,
            // flipped by the parity of rot (of rot ^ XT when swapped) with
            // the term's Z bits
            const uint32_t swp = (rot & (uint32_t)(XT & -XT)) != 0u;
            f ^= im ? swp : 0u;
            if (sg) f ^= ((zp >> rot) ^ (swp ? (zp >> XT) : 0u)) & 1u;
        }
        round_term_fx<XT>(v, zp, f, im, sg, acc);
    }
}

// X strings without Z bits (in any round order: the pairs are symmetric
// under the rotation of round 0): Re conj(w) v, one sign
template <int XT>
__device__ __forceinline__ void round_plain(const RoundArgs<double2>& a, int r, const Fx (&v)[8], FxAcc& acc) {
#pragma unroll 1
    for (int c = a.xplain[r][XT]; c > 0; --c) round_pairs_fx<XT, false, false>(v, 0u, 0u, acc);
}

// 2^(x - 1023) for a biased exponent x >= 1 (infinity above 2046)
__device__ __forceinline__ double fx_pow2(uint32_t x) { return __hiloint2double((int)(min(x, 2047u) << 20), 0); }

__global__ void __launch_bounds__(kThr2, 1) k_expect_fx(const __grid_constant__ RoundArgs<double2> a) {
    constexpr uint32_t Tn = 1u << kT2;
    constexpr uint64_t kOnes = 0x0101010101010101ull;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* const tiles = reinterpret_cast<double2*>(smem_raw);
    __shared__ __align__(8) uint64_t full[kNB2];
    __shared__ double shd[32];
    __shared__ uint64_t offA[64];
    __shared__ uint64_t spread[256];          // byte j of spread[p] = bit j of p
    // per tile, two slots (a warp may start the next tile while others finish this one)
    __shared__ uint64_t s_zbits[2];           // bit m: outside parity of Z mask m
    __shared__ uint32_t s_xbits[2];           // bit k: outside parity of term k's Z bits
    __shared__ __align__(16) uint32_t s_wmax[2][kThr2 / 32];   // largest exponent of each warp's amplitudes
    __shared__ uint32_t abort_flag;
    __shared__ uint64_t s_cnt_in[kZW][kThr2];   // per thread: odd parities of the masks inside the tile
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    if (tid < 64) {
        uint64_t o = 0;
        for (int j = 0; j < a.kh; ++j)
            if ((tid >> j) & 1u) o |= 1ull << a.hq[j];
        offA[tid] = o;
    }
    if (tid < 256) {
        uint64_t sp = 0;
        for (int j = 0; j < 8; ++j) sp |= (uint64_t)((tid >> j) & 1u) << (8 * j);
        spread[tid] = sp;
    }
    if (tid == 0) {
        for (int b = 0; b < kNB2; ++b) oz::mbar_init_count(&full[b], 1);
        abort_flag = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // parities of the thread's part of each mask (fixed for the launch)
    const uint32_t l0 = round_base(tid, 0);
    uint64_t tz = 0;
    for (int m = 0; m < a.nz; ++m) tz |= (uint64_t)(__popc(l0 & a.zl[m]) & 1) << m;
    uint32_t tx = 0;
    for (int r = 0; r < 4; ++r) {
        const uint32_t lt = round_base(tid, r);
        for (int k = a.rb[r]; k < a.rb[r + 1]; ++k) tx |= (uint32_t)(__popc(lt & a.xzl[k]) & 1) << k;
    }
    __syncthreads();
    // the counts of the masks inside the tile (odd parities per amplitude, one byte each)
    for (int g = 0; g < a.nzg; ++g) {
        uint64_t ci = 0;
        for (uint64_t bits = a.zin[g]; bits; bits &= bits - 1) {
            const int m = __ffsll((long long)bits) - 1;
            ci += spread[a.zpz[m] ^ ((uint32_t)((tz >> m) & 1ull) * 0xFFu)];
        }
        s_cnt_in[g][tid] = ci;
    }
    FxAcc acc{0, 0, 0, 0};
    double xs = 0.0, zs = 0.0;   // X/Y sum (common weight applied at the end); weighted Z sum
    const bool later_rounds = (a.rmask & 0xE) != 0;
    // tile copies: piece p of a tile by thread p (512 / npieces); the bytes
    // of a buffer's next tile are announced by thread 0 before the barrier
    // that precedes the copies, which follow a generic-proxy fence of every
    // thread (the buffer's previous contents were read and written by them)
    const uint32_t npieces = max(4u, 1u << a.kh), pamps = Tn / npieces;
    const uint32_t istride = kThr2 / npieces;
    const bool issuer = tid % istride == 0u;
    const uint32_t lp = (tid / istride) * pamps;   // the piece's first tile-local amplitude
    const uint32_t lowmask = (1u << a.L) - 1u;
    const uint64_t step = gridDim.x;
    auto issue = [&](uint64_t t, int b) {
        const uint64_t base = insert_zero_bits(t << a.L, a.hq_sorted, a.kh);
        oz::bulk_g2s(oz::smem_u32(tiles + (size_t)b * Tn + lp), a.x + (base + (lp & lowmask) + offA[lp >> a.L]),
                     pamps * 16u, &full[b]);
    };
    if (tid == 0)
        for (int b = 0; b < kNB2 - 1; ++b)
            if (blockIdx.x + (uint64_t)b * step < a.ntiles) oz::mbar_expect_tx(&full[b], Tn * 16u);
    __syncthreads();
    if (issuer)
        for (int b = 0; b < kNB2 - 1; ++b) {
            const uint64_t t = blockIdx.x + (uint64_t)b * step;
            if (t < a.ntiles && !(a.stall_test && blockIdx.x == 0 && b == 0)) issue(t, b);
        }
    int it = 0;
    bool ok = true;
    for (uint64_t t = blockIdx.x; t < a.ntiles; t += step, ++it) {
        const int b = it % kNB2;
        const double2* const tile = tiles + (size_t)b * Tn;
        const uint64_t tn = t + (uint64_t)(kNB2 - 1) * step;   // copied after this tile's first barrier
        if (tid < 32) {
            if (tid == 0 && tn < a.ntiles) oz::mbar_expect_tx(&full[(it + kNB2 - 1) % kNB2], Tn * 16u);
            // outside parities of this tile
            const uint64_t base = insert_zero_bits(t << a.L, a.hq_sorted, a.kh);
            const uint32_t p0 = ((int)lane < a.nz) ? (uint32_t)(__popcll(base & a.zo[lane]) & 1) : 0u;
            const uint32_t p1 = ((int)lane + 32 < a.nz) ? (uint32_t)(__popcll(base & a.zo[lane + 32]) & 1) : 0u;
            const uint32_t px = ((int)lane < a.nxt) ? (uint32_t)(__popcll(base & a.xzo[lane]) & 1) : 0u;
            const uint32_t b0 = __ballot_sync(0xffffffffu, p0), b1 = __ballot_sync(0xffffffffu, p1);
            const uint32_t xb = __ballot_sync(0xffffffffu, px);
            if (lane == 0) {
                s_zbits[it & 1] = ((uint64_t)b1 << 32) | b0;
                s_xbits[it & 1] = xb;
            }
        }
        const bool arrived = oz::wait_or_abort(oz::smem_u32(&full[b]), (uint32_t)(it / kNB2) & 1u, a.spin_limit,
                                               &abort_flag);
        // the thread's round-0 amplitudes (rotated order): the tile's largest exponent
        const uint32_t rot = tid & 7u;
        double2 d[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) d[j] = tile[l0 | ((uint32_t)j ^ rot)];
        uint32_t em = 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) em = max(em, max(fx_exp(d[j].x), fx_exp(d[j].y)));
        em = __reduce_max_sync(0xffffffffu, em);
        if (lane == 0) s_wmax[it & 1][tid >> 5] = em;
        if (__syncthreads_or(!arrived)) {
            ok = false;
            break;
        }
        // every thread is past the previous tile: its buffer takes tile tn
        if (issuer && tn < a.ntiles) issue(tn, (it + kNB2 - 1) % kNB2);
        uint32_t emax = 0u;
#pragma unroll
        for (int w = 0; w < kThr2 / 32; w += 4) {
            const uint4 q = *reinterpret_cast<const uint4*>(&s_wmax[it & 1][w]);
            emax = max(emax, max(max(q.x, q.y), max(q.z, q.w)));
        }
        const bool flush = emax < kFxFlush;
        const uint32_t emx = flush ? 4095u : emax;
        Fx v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            fx_limbs(d[j].x, emx, v[j].xh, v[j].xl);
            fx_limbs(d[j].y, emx, v[j].yh, v[j].yl);
        }
        if (later_rounds) {
            int4* const ti = reinterpret_cast<int4*>(tiles + (size_t)b * Tn);
#pragma unroll
            for (int j = 0; j < 8; ++j) ti[l0 | ((uint32_t)j ^ rot)] = make_int4(v[j].xh, v[j].xl, v[j].yh, v[j].yl);
        }
        // v[i] holds amplitude l0 | (i ^ rot): round 0 works in that order
        // (below: the count bytes permuted alike, and the terms' signs)
        if (later_rounds) __syncthreads();
        const double f2 = flush ? 0.0 : fx_pow2(emax - 53u);   // 2^(E - 1076)
        const uint64_t zbits = tz ^ s_zbits[it & 1];
        const uint32_t xflip = tx ^ s_xbits[it & 1];
        if (a.nzg > 0) {
            const double f1 = fx_pow2(emax + 5u);   // 2^(E - 1018): unit 2^58 of the folded sums
#pragma unroll 1
            for (int g = 0; g < a.nzg; ++g) {
                uint64_t cg = s_cnt_in[g][tid] + (uint64_t)__popcll(zbits & a.zout[g]) * kOnes;
                for (uint64_t bits = a.zmix[g]; bits; bits &= bits - 1) {
                    const int m = __ffsll((long long)bits) - 1;
                    cg += spread[a.zpz[m] ^ ((uint32_t)((zbits >> m) & 1ull) * 0xFFu)];
                }
                // byte i <- byte i ^ rot
                uint32_t lo = (uint32_t)cg, hi = (uint32_t)(cg >> 32);
                if (rot & 4u) {
                    const uint32_t t2 = lo;
                    lo = hi;
                    hi = t2;
                }
                if (rot & 2u) {
                    lo = __byte_perm(lo, 0u, 0x1032u);
                    hi = __byte_perm(hi, 0u, 0x1032u);
                }
                if (rot & 1u) {
                    lo = __byte_perm(lo, 0u, 0x2301u);
                    hi = __byte_perm(hi, 0u, 0x2301u);
                }
                const int ngm = a.zg_end[g] - (g ? a.zg_end[g - 1] : 0);   // masks of group g
                long long zt = 0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    // |q|^2 at unit 2^56: h^2 terms plus the cross terms 2 h l / 2^28
                    const long long ph = (long long)v[j].xh * v[j].xh + (long long)v[j].yh * v[j].yh;
                    const long long pm = (long long)v[j].xh * v[j].xl + (long long)v[j].yh * v[j].yl;
                    const uint32_t byte = ((j < 4 ? lo : hi) >> (8 * (j & 3))) & 0xFFu;
                    zt += (long long)(ngm - 2 * (int)byte) * (ph + ((pm + (1ll << 26)) >> 27));
                }
                long long z = (zt + 2) >> 2;
                z += __shfl_xor_sync(0xffffffffu, z, 1);
                z += __shfl_xor_sync(0xffffffffu, z, 2);
                if ((lane & 3u) == 0u) zs = __fma_rn(__dmul_rn(__dmul_rn((double)z, f1), a.zw[g]), f2, zs);
            }
        }
#pragma unroll 1
        for (int r = 0; r < 4; ++r) {
            if (!((a.rmask >> r) & 1)) continue;
            if (r > 0) {
                const uint32_t lt = round_base(tid, r);
                const int4* const ti = reinterpret_cast<const int4*>(tile);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int4 q = ti[lt | ((uint32_t)j << (3 * r))];
                    v[j] = Fx{q.x, q.y, q.z, q.w};
                }
            }
            round_plain<1>(a, r, v, acc);
            round_plain<2>(a, r, v, acc);
            round_plain<3>(a, r, v, acc);
            round_plain<4>(a, r, v, acc);
            round_plain<5>(a, r, v, acc);
            round_plain<6>(a, r, v, acc);
            round_plain<7>(a, r, v, acc);
            round_xt<1>(a, r, rot, xflip, v, acc);
            round_xt<2>(a, r, rot, xflip, v, acc);
            round_xt<3>(a, r, rot, xflip, v, acc);
            round_xt<4>(a, r, rot, xflip, v, acc);
            round_xt<5>(a, r, rot, xflip, v, acc);
            round_xt<6>(a, r, rot, xflip, v, acc);
            round_xt<7>(a, r, rot, xflip, v, acc);
        }
        if (a.rmask != 0) {
            long long x = acc.h0 + acc.h1 + ((acc.m0 + acc.m1 + (1ll << 27)) >> 28);   // |m0 + m1| < 2^62.6
            acc = FxAcc{0, 0, 0, 0};
            x += __shfl_xor_sync(0xffffffffu, x, 1);
            x += __shfl_xor_sync(0xffffffffu, x, 2);
            if ((lane & 3u) == 0u) xs = __fma_rn(__dmul_rn((double)x, fx_pow2(emax + 3u)), f2, xs);   // unit 2^56
        }
        // the buffer is refilled by bulk copies (async proxy) after the next
        // tile's first barrier
        asm volatile("fence.proxy.async.shared::cta;");
    }
    if (!ok) {
        // copies still in flight land before the CTA exits (bounded waits)
        if (tid == 0) {
            atomicExch(a.status, 1u);
            for (int k = 0; k < kNB2 - 1; ++k) {
                const int i2 = it + k;
                if (blockIdx.x + (uint64_t)i2 * step < a.ntiles)
                    tc::mbar_wait(oz::smem_u32(&full[i2 % kNB2]), (uint32_t)(i2 / kNB2) & 1u, a.spin_limit);
            }
        }
        return;
    }
    double s = 0.0, c = 0.0;
    if (a.nzg > 0) {
        const double r = block_reduce_d(zs, shd);
        if (tid == 0) neumaier(s, c, r);
    }
    if (a.rmask != 0) {
        const double r = block_reduce_d(xs, shd);
        if (tid == 0) neumaier(s, c, r * a.wx);
    }
    if (tid == 0) a.partial[blockIdx.x] = make_double2(s, c);
}

// Native FP64 variants (baseline policy).
__global__ void __launch_bounds__(kRThreads) k_probs_partial_f64(const __grid_constant__ ProbArgs<double2> a) {
    __shared__ double shs[32];
    const uint64_t bin = blockIdx.x / a.chunks, ch = blockIdx.x % a.chunks;
    uint64_t dep = 0;
    for (int j = 0; j < a.m; ++j) dep |= ((bin >> j) & 1ull) << a.q[j];
    const uint64_t t0 = ch * a.chunk_len;
    const uint64_t t1 = min(a.per_bin, t0 + a.chunk_len);
    // two FP64 accumulators a thread (products by fused multiply-add); the
    // block's warp sums are combined with Neumaier's compensation
    double s = 0.0, c = 0.0;
    uint64_t t = t0 + threadIdx.x;
    for (; t + blockDim.x < t1; t += 2 * (uint64_t)blockDim.x) {
        const double2 v = a.x[insert_zero_bits(t, a.q_sorted, a.m) | dep];
        const double2 u = a.x[insert_zero_bits(t + blockDim.x, a.q_sorted, a.m) | dep];
        s = __fma_rn(v.x, v.x, __fma_rn(v.y, v.y, s));
        c = __fma_rn(u.x, u.x, __fma_rn(u.y, u.y, c));
    }
    if (t < t1) {
        const double2 v = a.x[insert_zero_bits(t, a.q_sorted, a.m) | dep];
        s = __fma_rn(v.x, v.x, __fma_rn(v.y, v.y, s));
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
}

// Marginals of qubits that all lie below qubit 8: thread t of a 256-thread
// block reads the amplitudes whose low 8 bits are t, so its bin is fixed and
// the block reads a contiguous range (the bin-major kernels read each bin
// with a stride); the block then sums its threads per bin.  Partials at
// [bin * nblocks + block].  FP64 mode: FP64 products and sums (two
// accumulators a thread); otherwise float-pair sums as in k_probs_partial.
constexpr int kLowBits = 8;
template <class S, bool NAT>
__global__ void __launch_bounds__(1 << kLowBits) k_probs_low(const __grid_constant__ ProbArgs<S> a) {
    constexpr uint32_t T = 1u << kLowBits;
    __shared__ double ss[T], sc[T];
    const uint32_t t = threadIdx.x;
    uint32_t bin = 0;
    for (int j = 0; j < a.m; ++j) bin |= ((t >> a.q[j]) & 1u) << j;
    const uint64_t base = blockIdx.x * a.chunk_len + t;   // chunk_len: amplitudes a block, a multiple of 4 T
    double s = 0.0, c = 0.0;
    if constexpr (NAT) {
        double s2 = 0.0, s3 = 0.0, s4 = 0.0;
        for (uint64_t k = 0; k < a.chunk_len; k += 4 * T) {
            const double2 v0 = reinterpret_cast<const double2*>(a.x)[base + k];
            const double2 v1 = reinterpret_cast<const double2*>(a.x)[base + k + T];
            const double2 v2 = reinterpret_cast<const double2*>(a.x)[base + k + 2 * T];
            const double2 v3 = reinterpret_cast<const double2*>(a.x)[base + k + 3 * T];
            s = __fma_rn(v0.x, v0.x, __fma_rn(v0.y, v0.y, s));
            s2 = __fma_rn(v1.x, v1.x, __fma_rn(v1.y, v1.y, s2));
            s3 = __fma_rn(v2.x, v2.x, __fma_rn(v2.y, v2.y, s3));
            s4 = __fma_rn(v3.x, v3.x, __fma_rn(v3.y, v3.y, s4));
        }
        neumaier(s, c, s2);
        neumaier(s, c, s3);
        neumaier(s, c, s4);
    } else {
        Acc acc{0.f, 0.f};
        for (uint64_t k = 0; k < a.chunk_len; k += 4 * T) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                float h, l;
                abs2(rview(a.x[base + k + (uint64_t)u * T]), h, l);
                acc_add(acc, h, l);
            }
        }
        const df r = df_norm(acc.s, acc.e);
        s = df2d(r.h, r.l);
    }
    ss[t] = s;
    sc[t] = c;
    __syncthreads();
    if (t < (1u << a.m)) {
        // the threads of bin t, in index order
        double bs = 0.0, bc = 0.0;
        for (uint32_t u = 0; u < T; ++u) {
            uint32_t b = 0;
            for (int j = 0; j < a.m; ++j) b |= ((u >> a.q[j]) & 1u) << j;
            if (b != t) continue;
            neumaier(bs, bc, ss[u]);
            bc += sc[u];
        }
        a.partial[(uint64_t)t * gridDim.x + blockIdx.x] = make_double2(bs, bc);
    }
}

// Blocks of the low-qubit marginal kernel: about 8 per SM, at least 2^14
// amplitudes each (a power of two).
uint64_t probs_low_blocks(const qe_state* s) {
    if (s->n < 14) return 0;
    uint64_t per = 1ull << 14;
    while (((1ull << s->n) / per) > (uint64_t)num_sms() * 8) per <<= 1;
    return (1ull << s->n) / per;
}

// Blocks of the probability reduction for m register qubits: about 8 blocks
// per SM in total, at least 2^14 amplitudes per block.
uint64_t probs_chunks(const qe_state* s, int m) {
    const uint64_t bins = 1ull << m;
    const uint64_t want_blocks = (uint64_t)num_sms() * 8;
    uint64_t chunks = std::max<uint64_t>(1, want_blocks / bins);
    return std::min<uint64_t>(chunks, std::max<uint64_t>(1, (1ull << (s->n - m)) >> 14));
}

template <class S>
void probs_device(qe_state* s, int m, const int* qubits, double2* partial, double* dout);

uint64_t probs_partials(const qe_state* s, int m) {
    return (1ull << m) * std::max(probs_chunks(s, m), probs_low_blocks(s));
}

template <class S>
void probs_impl(qe_state* s, int m, const int* qubits, double* host_out) {
    const uint64_t bins = 1ull << m;
    const uint64_t nblocks = probs_partials(s, m);
    char* scr = (char*)ensure_scratch(s, nblocks * sizeof(double2) + bins * sizeof(double));
    double* dout = (double*)(scr + nblocks * sizeof(double2));
    probs_device<S>(s, m, qubits, (double2*)scr, dout);
    QE_CUDA(cudaMemcpyAsync(host_out, dout, bins * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QE_CUDA(cudaStreamSynchronize(s->stream));
}

// The 2^m marginal probabilities into device memory dout (partial: room for
// 2^m * probs_chunks(s, m) block partials); enqueued only.
template <class S>
void probs_device(qe_state* s, int m, const int* qubits, double2* partial, double* dout) {
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
    bool low = m >= 1 && probs_low_blocks(s) > 0;
    for (int j = 0; j < m; ++j) low &= qubits[j] < kLowBits;
    if (low) {
        const uint64_t nb = probs_low_blocks(s);
        a.chunk_len = (1ull << s->n) / nb;
        a.partial = partial;
        {
            Launch L(s, "probs_low", (double)dim(s) * amp_bytes(s));
            if (std::is_same<S, double2>::value && c128_f64(s))
                k_probs_low<S, true><<<(unsigned)nb, 1 << kLowBits, 0, s->stream>>>(a);
            else
                k_probs_low<S, false><<<(unsigned)nb, 1 << kLowBits, 0, s->stream>>>(a);
            QE_CUDA(cudaGetLastError());
        }
        Launch L(s, "sum_partials", 0.0, false);
        const unsigned g2 = (unsigned)std::min<uint64_t>(bins, 4096);
        k_sum_partials<<<g2, kSumThreads, 0, s->stream>>>(a.partial, bins, nb, nullptr, dout);
        QE_CUDA(cudaGetLastError());
        return;
    }
    a.per_bin = 1ull << (s->n - m);
    const uint64_t chunks = probs_chunks(s, m);
    a.chunks = chunks;
    a.chunk_len = (a.per_bin + chunks - 1) / chunks;
    const uint64_t nblocks = bins * chunks;
    a.partial = partial;
    if (nblocks > 0x7FFFFFFFull) fail(QE_ERR_UNSUPPORTED, "too many probability blocks");
    {
        Launch L(s, "probs_partial", (double)dim(s) * amp_bytes(s));
        if (std::is_same<S, double2>::value && c128_f64(s))
            k_probs_partial_f64<<<(unsigned)nblocks, kRThreads, 0, s->stream>>>(
                *reinterpret_cast<ProbArgs<double2>*>(&a));
        else
            k_probs_partial<S><<<(unsigned)nblocks, kRThreads, 0, s->stream>>>(a);
        QE_CUDA(cudaGetLastError());
    }
    {
        Launch L(s, "sum_partials", 0.0, false);
        const unsigned g2 = (unsigned)std::min<uint64_t>(bins, 4096);
        k_sum_partials<<<g2, kSumThreads, 0, s->stream>>>(a.partial, bins, chunks, nullptr, dout);
        QE_CUDA(cudaGetLastError());
    }
}

// Terms whose X/Y qubits do not fit one tile layout: grid-stride over x with
// the partner amplitude read from global memory.
template <class S>
struct WideArgs {
    const S* x;
    uint64_t count;
    int nt;
    uint64_t xm[kXT], zm[kXT];
    int ny[kXT];
    double w[kXT];
    double2* partial;
};

template <class S, bool NAT>
__global__ void __launch_bounds__(kRThreads) k_expect_wide(const __grid_constant__ WideArgs<S> a) {
    using A = std::conditional_t<NAT, AccD, Acc>;
    __shared__ Acc sh[32];
    __shared__ double shd[32];
    A acc[kXT];
#pragma unroll
    for (int t = 0; t < kXT; ++t) acc_zero(acc[t]);
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < a.count;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const S raw = a.x[x];
#pragma unroll
        for (int t = 0; t < kXT; ++t) {
            if (t >= a.nt) break;
            const uint64_t xm = a.xm[t];
            if (x & (xm & (~xm + 1ull))) continue;
            const bool neg = (__popcll(x & a.zm[t]) & 1) != 0;
            if constexpr (NAT) {
                // Re(conj(w) v i^ny), as in corr()
                const S w = a.x[x ^ xm];
                const int ny = a.ny[t];
                double h = ((ny & 1) == 0) ? __fma_rn(w.x, raw.x, __dmul_rn(w.y, raw.y))
                                           : __fma_rn(w.x, raw.y, -__dmul_rn(w.y, raw.x));
                if ((ny == 1 || ny == 2) != neg) h = -h;
                acc[t].s = __fma_rn(2.0, h, acc[t].s);
            } else {
                float h, l;
                corr(rview(a.x[x ^ xm]), rview(raw), a.ny[t], h, l);
                if (neg) { h = -h; l = -l; }
                acc_add(acc[t], 2.f * h, 2.f * l);
            }
        }
    }
    double s = 0.0, c = 0.0;
#pragma unroll
    for (int t = 0; t < kXT; ++t) {
        if (t >= a.nt) break;
        if constexpr (NAT) {
            const double r = block_reduce_d(acc[t].s, shd);
            if (threadIdx.x == 0) neumaier(s, c, r * a.w[t]);
        } else {
            Acc r = block_reduce(acc[t], sh);
            if (threadIdx.x == 0) {
                df d = df_norm(r.s, r.e);
                neumaier(s, c, df2d(d.h, d.l) * a.w[t]);
            }
        }
    }
    if (threadIdx.x == 0) a.partial[blockIdx.x] = make_double2(s, c);
}

// Launches of the register-round kernel: layout 0 (qubits [0, 12)) and
// layouts of six high qubits above the chunk bits [0, 6), two triples each;
// one launch per layout and common X/Y weight (at most kXT2 terms), the Z-only
// groups on layout 0.  False when a term does not fit: X/Y bits below qubit
// 12 outside one triple, three or more high X/Y bits, or both kinds at once.
struct RoundLaunch {
    std::vector<int> hq;                                  // high qubits, local order (empty: layout 0)
    std::vector<std::pair<int, int>> x;                   // (term, round), ascending rounds
    std::vector<std::pair<int, std::vector<int>>> z;      // (weight group, Z masks)
    double wx = 0.0;
};

bool plan_rounds(int n, int nterms, const uint64_t* xm, const double* cf,
                 const std::vector<std::pair<int, std::vector<int>>>& zchunks, std::vector<RoundLaunch>& out) {
    out.clear();
    if (n < kT2) return false;
    const uint64_t lowq = (1ull << kT2) - 1ull;
    std::vector<std::pair<int, int>> low;
    std::vector<int> high;
    for (int t = 0; t < nterms; ++t) {
        if (xm[t] == 0) continue;
        if ((xm[t] & ~lowq) == 0) {
            int r = -1;
            for (int q = 0; q < 4; ++q)
                if ((xm[t] & ~(7ull << (3 * q))) == 0) r = q;
            if (r < 0) return false;
            low.push_back({t, r});
        } else if ((xm[t] & lowq) == 0 && __builtin_popcountll(xm[t]) <= 3) {
            high.push_back(t);
        } else {
            return false;
        }
    }
    // high qubits grouped into triples, each term inside one
    std::vector<uint64_t> trip;
    std::vector<int> trip_of(high.size());
    for (size_t i = 0; i < high.size(); ++i) {
        const uint64_t q = xm[high[i]];
        int f = -1;
        for (size_t j = 0; j < trip.size() && f < 0; ++j)
            if ((trip[j] & q) == q) f = (int)j;
        for (size_t j = 0; j < trip.size() && f < 0; ++j)
            if (__builtin_popcountll(trip[j] | q) <= 3) f = (int)j;
        if (f < 0) {
            trip.push_back(0ull);
            f = (int)trip.size() - 1;
        }
        trip[f] |= q;
        trip_of[i] = f;
    }
    struct Lay {
        std::vector<int> hq;
        std::vector<std::pair<int, int>> x;
    };
    // pair disjoint triples into layouts (triples that share a qubit may not
    // sit in one layout)
    std::vector<Lay> lays(1);
    lays[0].x = low;
    std::vector<int> lay_of(trip.size(), -1), round_of(trip.size(), 2);
    for (size_t j = 0; j < trip.size(); ++j) {
        if (lay_of[j] >= 0) continue;
        int mate = -1;
        for (size_t k = j + 1; k < trip.size() && mate < 0; ++k)
            if (lay_of[k] < 0 && (trip[k] & trip[j]) == 0) mate = (int)k;
        Lay ly;
        int pad = 6;   // fill short triples with qubits of [6, 12), never high-term qubits
        for (int h = 0; h < 2; ++h) {
            const uint64_t tq = h == 0 ? trip[j] : (mate >= 0 ? trip[mate] : 0ull);
            int c = 0;
            for (int q = 0; q < n; ++q)
                if ((tq >> q) & 1ull) {
                    ly.hq.push_back(q);
                    ++c;
                }
            for (; c < 3; ++c) ly.hq.push_back(pad++);
        }
        lay_of[j] = (int)lays.size();
        if (mate >= 0) {
            lay_of[mate] = (int)lays.size();
            round_of[mate] = 3;
        }
        lays.push_back(ly);
    }
    for (size_t i = 0; i < high.size(); ++i) lays[lay_of[trip_of[i]]].x.push_back({high[i], round_of[trip_of[i]]});
    size_t zi = 0;
    for (size_t li = 0; li < lays.size(); ++li) {
        std::vector<double> ws;
        for (const auto& tr : lays[li].x)
            if (std::find(ws.begin(), ws.end(), 2.0 * cf[tr.first]) == ws.end()) ws.push_back(2.0 * cf[tr.first]);
        std::vector<RoundLaunch> mine;
        for (double w : ws) {
            std::vector<std::pair<int, int>> xs;
            for (const auto& tr : lays[li].x)
                if (2.0 * cf[tr.first] == w) xs.push_back(tr);
            std::stable_sort(xs.begin(), xs.end(),
                             [](const std::pair<int, int>& p, const std::pair<int, int>& q) { return p.second < q.second; });
            for (size_t i = 0; i < xs.size(); i += kXT2) {
                RoundLaunch R;
                R.hq = lays[li].hq;
                R.wx = w;
                R.x.assign(xs.begin() + i, xs.begin() + std::min(xs.size(), i + kXT2));
                mine.push_back(R);
            }
        }
        if (li == 0) {
            size_t k = 0;
            while (zi < zchunks.size()) {
                if (k == mine.size()) mine.push_back(RoundLaunch{});
                RoundLaunch& R = mine[k++];
                int masks = 0;
                while (zi < zchunks.size() && (int)R.z.size() < kZW &&
                       masks + (int)zchunks[zi].second.size() <= kZT) {
                    masks += (int)zchunks[zi].second.size();
                    R.z.push_back(zchunks[zi++]);
                }
            }
        }
        for (auto& R : mine) out.push_back(std::move(R));
    }
    return true;
}

template <class S, bool NAT>
double expect_rounds(qe_state* s, const std::vector<RoundLaunch>& rl, const uint64_t* xm, const uint64_t* zm,
                     const std::vector<double>& wv) {
    // complex128 (either arithmetic mode): the fixed-point kernel
    constexpr bool kFx = sizeof(S) == 16;
    const auto kern = [] {
        if constexpr (kFx) return k_expect_fx;
        else return k_expect_rounds<S>;
    }();
    const int n = s->n;
    const size_t smem = (size_t)kNB2 * (sizeof(S) << kT2);
    QE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    QE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThr2, smem));
    const uint64_t ntiles = 1ull << (n - kT2);
    const unsigned grid = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)num_sms() * std::max(occ, 1));
    char* scr = (char*)ensure_scratch(s, rl.size() * grid * sizeof(double2) + 64);
    double2* partial = (double2*)scr;
    double* dout = (double*)(scr + rl.size() * grid * sizeof(double2));
    uint32_t* status = reinterpret_cast<uint32_t*>(dout + 1);   // fixed-point kernel: a copy wait ran out
    if (kFx) QE_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s->stream));
    auto pattern = [](uint32_t bits3) {   // bit j: parity of j & bits3
        uint32_t p = 0;
        for (uint32_t j = 0; j < 8; ++j) p |= (uint32_t)(__builtin_popcount(j & bits3) & 1) << j;
        return p;
    };
    static thread_local RoundArgs<S> a;
    for (size_t i = 0; i < rl.size(); ++i) {
        const RoundLaunch& R = rl[i];
        a = RoundArgs<S>{};
        a.x = reinterpret_cast<const S*>(s->d);
        a.ntiles = ntiles;
        a.kh = (int)R.hq.size();
        a.L = kT2 - a.kh;
        std::vector<int> so(R.hq);
        std::sort(so.begin(), so.end());
        for (int j = 0; j < a.kh; ++j) {
            a.hq[j] = (uint8_t)R.hq[j];
            a.hq_sorted[j] = (uint8_t)so[j];
        }
        uint64_t inside = (1ull << a.L) - 1ull;
        for (int q : R.hq) inside |= 1ull << q;
        auto to_local = [&](uint64_t m) {
            uint32_t loc = (uint32_t)(m & ((1ull << a.L) - 1ull));
            for (int h = 0; h < a.kh; ++h)
                if ((m >> R.hq[h]) & 1ull) loc |= 1u << (a.L + h);
            return loc;
        };
        a.nzg = (int)R.z.size();
        int k = 0;
        for (int g = 0; g < a.nzg; ++g) {
            a.zw[g] = wv[R.z[g].first];
            for (int t : R.z[g].second) {
                a.zl[k] = to_local(zm[t]);
                a.zo[k] = zm[t] & ~inside;
                a.zpz[k] = (uint8_t)pattern(a.zl[k] & 7u);
                uint64_t& cls = a.zl[k] == 0 ? a.zout[g] : a.zo[k] == 0 ? a.zin[g] : a.zmix[g];
                cls |= 1ull << k;
                ++k;
            }
            a.zg_end[g] = k;
        }
        a.nz = k;
        a.nxt = (int)R.x.size();
        int per[4] = {0, 0, 0, 0};
        for (const auto& tr : R.x) ++per[tr.second];
        a.rb[0] = 0;
        for (int r = 0; r < 4; ++r) a.rb[r + 1] = a.rb[r] + per[r];
        auto xt_of = [&](const std::pair<int, int>& tr) { return (to_local(xm[tr.first]) >> (3 * tr.second)) & 7u; };
        // X strings without Z bits: counted per round and pattern (fixed-point kernel)
        std::vector<std::pair<int, int>> xs;
        a.rmask = 0;
        for (const auto& tr : R.x) {
            const uint32_t xl = to_local(xm[tr.first]);
            if ((xl >> (3 * tr.second) & 7u) == 0 || (xl & ~(7u << (3 * tr.second))) != 0)
                fail(QE_ERR_STATE, "expectation term outside its round");
            a.rmask |= 1 << tr.second;
            if (kFx && zm[tr.first] == 0) ++a.xplain[tr.second][xt_of(tr)];
            else xs.push_back(tr);
        }
        if (kFx) {
            a.nxt = (int)xs.size();
            for (int r = 0; r < 4; ++r) per[r] = 0;
            for (const auto& tr : xs) ++per[tr.second];
            for (int r = 0; r < 4; ++r) a.rb[r + 1] = a.rb[r] + per[r];
        }
        // within a round, by the pattern of X/Y bits in its triple
        std::stable_sort(xs.begin(), xs.end(), [&](const std::pair<int, int>& p, const std::pair<int, int>& q) {
            return p.second != q.second ? p.second < q.second : xt_of(p) < xt_of(q);
        });
        for (int r = 0; r < 4; ++r) {
            for (int x = 0; x <= 8; ++x) a.xtb[r][x] = (uint8_t)a.rb[r];
            for (int j = a.rb[r]; j < a.rb[r + 1]; ++j)
                for (int x = (int)xt_of(xs[j]) + 1; x <= 8; ++x) a.xtb[r][x] = (uint8_t)(j + 1);
        }
        for (int j = 0; j < a.nxt; ++j) {
            const int t = xs[j].first, r = xs[j].second;
            const uint32_t xl = to_local(xm[t]), zl = to_local(zm[t]);
            const uint32_t xt = (xl >> (3 * r)) & 7u;
            const int ny = __builtin_popcountll(xm[t] & zm[t]) & 3;
            a.xw[j] = xt | (pattern((zl >> (3 * r)) & 7u) << 3) | ((uint32_t)(ny & 1) << 11) |
                      ((uint32_t)(ny == 1 || ny == 2) << 12) | ((uint32_t)(zm[t] != 0) << 13);
            a.xzl[j] = zl;
            a.xzo[j] = zm[t] & ~inside;
        }
        a.wx = R.wx;
        a.partial = partial + i * grid;
        a.status = status;
        a.spin_limit = 1ll << 20;   // polls of up to 1 us each
        // Failure-path test (QE_TEST_STALL_EXPECT=1, fixed-point kernel): block
        // 0 announces its first tile's bytes but copies none, so its wait runs
        // out after a short limit, the block drains its other copies and
        // leaves, and the host reports QE_ERR_TIMEOUT with the context intact.
        const char* stall = std::getenv("QE_TEST_STALL_EXPECT");
        a.stall_test = (kFx && stall != nullptr && stall[0] == '1') ? 1 : 0;
        if (a.stall_test) a.spin_limit = 1ll << 12;
        Launch L(s, kFx ? "expect_fx" : "expect_rounds", (double)dim(s) * amp_bytes(s));
        kern<<<grid, kThr2, smem, s->stream>>>(a);
        QE_CUDA(cudaGetLastError());
    }
    {
        Launch L(s, "sum_partials", 0.0, false);
        k_sum_partials<<<1, kSumThreads, 0, s->stream>>>(partial, 1, (uint64_t)rl.size() * grid, nullptr, dout);
        QE_CUDA(cudaGetLastError());
    }
    struct {
        double v;
        uint32_t st;
    } out{0.0, 0u};
    QE_CUDA(cudaMemcpyAsync(&out, dout, kFx ? 12 : sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QE_CUDA(cudaStreamSynchronize(s->stream));
    if (out.st != 0) fail(QE_ERR_TIMEOUT, "an expectation tile copy wait ran out");
    return out.v;
}

template <class S, bool NAT>
double expect_impl(qe_state* s, int nterms, const uint64_t* xm, const uint64_t* zm, const double* cf) {
    const int n = s->n;
    const int Tmax = std::min(n, sizeof(S) >= 16 ? 11 : 12);
    // chunk bits of the high layouts: 2^6-amplitude runs (1 KB for
    // complex128) keep DRAM efficient when the high qubits are far apart
    // (measured: 512-byte runs took 2.3x longer at n = 30)
    const int Lh = std::min(6, Tmax);
    const uint64_t nmask = (n >= 64) ? ~0ull : ((1ull << n) - 1ull);
    // --- layouts: 0 = contiguous tiles of 2^Tmax; others = chunk + high set
    struct Layout {
        int L = 0;
        std::vector<int> high;   // sorted qubits >= L
        std::vector<int> xterms;
    };
    std::vector<Layout> lay(1);
    lay[0].L = Tmax;
    std::vector<int> zterms, wide;
    for (int t = 0; t < nterms; ++t) {
        if (xm[t] == 0) { zterms.push_back(t); continue; }
        if ((xm[t] >> Tmax) == 0) { lay[0].xterms.push_back(t); continue; }
        const uint64_t hb = xm[t] & nmask & ~((1ull << Lh) - 1ull);
        if (__builtin_popcountll(hb) > Tmax - Lh) { wide.push_back(t); continue; }
        bool placed = false;
        for (size_t j = 1; j < lay.size() && !placed; ++j) {
            uint64_t cur = 0;
            for (int q : lay[j].high) cur |= 1ull << q;
            if (__builtin_popcountll(cur | hb) <= Tmax - Lh) {
                for (int q = 0; q < n; ++q)
                    if (((hb >> q) & 1ull) && !((cur >> q) & 1ull)) lay[j].high.push_back(q);
                std::sort(lay[j].high.begin(), lay[j].high.end());
                lay[j].xterms.push_back(t);
                placed = true;
            }
        }
        if (!placed) {
            Layout L;
            L.L = Lh;
            for (int q = 0; q < n; ++q)
                if ((hb >> q) & 1ull) L.high.push_back(q);
            L.xterms.push_back(t);
            lay.push_back(L);
        }
    }
    // Z-only terms grouped by weight
    std::vector<double> wv;
    std::vector<std::vector<int>> wg;
    for (int t : zterms) {
        size_t g = std::find(wv.begin(), wv.end(), cf[t]) - wv.begin();
        if (g == wv.size()) { wv.push_back(cf[t]); wg.emplace_back(); }
        wg[g].push_back(t);
    }
    // --- launches
    std::vector<std::pair<int, std::vector<int>>> zchunks;   // (group, masks) pieces of <= kZT
    for (size_t g = 0; g < wg.size(); ++g)
        for (size_t i = 0; i < wg[g].size(); i += kZT)
            zchunks.push_back({(int)g, std::vector<int>(wg[g].begin() + i,
                                                        wg[g].begin() + std::min(wg[g].size(), i + kZT))});
    static thread_local ExpArgs<S> a;
    a.x = reinterpret_cast<const S*>(s->d);
    const size_t smem = 2 * (sizeof(decltype(rview(S{}))) << Tmax);   // two tiles
    QE_CUDA(cudaFuncSetAttribute(k_expect_tile<S, NAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    QE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_expect_tile<S, NAT>, kRThreads, smem));
    // count launches first to size the scratch
    struct Plan { int layout; std::vector<std::pair<int, std::vector<int>>> z; std::vector<int> x; };
    std::vector<Plan> plans;
    {
        // layout 0 carries the Z groups; every layout splits its X terms by kXT
        size_t zi = 0;
        for (size_t j = 0; j < lay.size(); ++j) {
            size_t xi = 0;
            const auto& xs = lay[j].xterms;
            do {
                Plan p;
                p.layout = (int)j;
                if (j == 0) {
                    int masks = 0;
                    while (zi < zchunks.size() && (int)p.z.size() < kZW &&
                           masks + (int)zchunks[zi].second.size() <= kZT) {
                        masks += (int)zchunks[zi].second.size();
                        p.z.push_back(zchunks[zi++]);
                    }
                }
                for (; xi < xs.size() && (int)p.x.size() < kXT; ++xi) p.x.push_back(xs[xi]);
                if (!p.z.empty() || !p.x.empty()) plans.push_back(p);
            } while (xi < xs.size() || (j == 0 && zi < zchunks.size()));
        }
    }
    const int nwide = (int)((wide.size() + kXT - 1) / kXT);
    if (plans.empty() && nwide == 0) return 0.0;
    // the register-round kernel when every term fits it: always for
    // complex128 (fixed point; the tile kernel's FP64 products are bound by
    // the FP64 pipe), for complex64 when it needs no more launches (its
    // per-pair cost is instruction issue, which it cuts by a third)
    if (const int sw = expect_kernel_switch(); sw != 1) {
        constexpr bool kFx = sizeof(S) == 16;
        std::vector<RoundLaunch> rl;
        if (plan_rounds(n, nterms, xm, cf, zchunks, rl) && !rl.empty() &&
            (sw == 2 || kFx || rl.size() <= plans.size() + (size_t)nwide))
            return expect_rounds<S, NAT>(s, rl, xm, zm, wv);
    }
    uint64_t max_grid = (uint64_t)num_sms() * 8;
    std::vector<unsigned> grids(plans.size());
    for (size_t i = 0; i < plans.size(); ++i) {
        const Layout& L = lay[plans[i].layout];
        const int T = L.L + (int)L.high.size();
        const uint64_t ntiles = 1ull << (n - T);
        grids[i] = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)num_sms() * std::max(occ, 1));
        max_grid = std::max<uint64_t>(max_grid, grids[i]);
    }
    const size_t nlaunch = plans.size() + (size_t)nwide;
    char* scr = (char*)ensure_scratch(s, nlaunch * max_grid * sizeof(double2) + 64);
    double2* partial = (double2*)scr;
    double* dout = (double*)(scr + nlaunch * max_grid * sizeof(double2));
    for (int w = 0; w < nwide; ++w) {
        static thread_local WideArgs<S> b;
        b.x = reinterpret_cast<const S*>(s->d);
        b.count = dim(s);
        b.nt = std::min(kXT, (int)wide.size() - w * kXT);
        for (int j = 0; j < b.nt; ++j) {
            const int t = wide[w * kXT + j];
            b.xm[j] = xm[t];
            b.zm[j] = zm[t];
            b.ny[j] = __builtin_popcountll(xm[t] & zm[t]) & 3;
            b.w[j] = cf[t];
        }
        b.partial = partial + (plans.size() + w) * max_grid;
        QE_CUDA(cudaMemsetAsync(b.partial, 0, max_grid * sizeof(double2), s->stream));
        const unsigned g = (unsigned)std::min<uint64_t>((dim(s) + kRThreads - 1) / kRThreads, max_grid);
        Launch Lw(s, "expect_wide", (double)dim(s) * amp_bytes(s));
        k_expect_wide<S, NAT><<<g, kRThreads, 0, s->stream>>>(b);
        QE_CUDA(cudaGetLastError());
    }
    for (size_t i = 0; i < plans.size(); ++i) {
        const Plan& p = plans[i];
        const Layout& L = lay[p.layout];
        a.L = L.L;
        a.kh = (int)L.high.size();
        a.T = a.L + a.kh;
        if (a.kh > 12) fail(QE_ERR_UNSUPPORTED, "expectation layout too wide");
        for (int j = 0; j < a.kh; ++j) a.hq[j] = (uint8_t)L.high[j];
        a.ntiles = 1ull << (n - a.T);
        a.nzg = (int)p.z.size();
        // layout bits: [0, L) and the high qubits
        uint64_t inside = (a.L >= 64) ? ~0ull : ((1ull << a.L) - 1ull);
        for (int j = 0; j < a.kh; ++j) inside |= 1ull << L.high[j];
        auto to_local = [&](uint64_t m) {
            uint32_t loc = (uint32_t)(m & ((1ull << a.L) - 1ull));
            for (int h = 0; h < a.kh; ++h)
                if ((m >> L.high[h]) & 1ull) loc |= 1u << (a.L + h);
            return loc;
        };
        int k = 0;
        for (int g = 0; g < a.nzg; ++g) {
            a.zw[g] = wv[p.z[g].first];
            for (int pass = 0; pass < 2; ++pass) {          // masks touching the layout first
                for (int t : p.z[g].second) {
                    const bool touches = (zm[t] & inside) != 0;
                    if (touches != (pass == 0)) continue;
                    a.zl[k] = to_local(zm[t]);
                    a.zo[k] = zm[t] & ~inside;
                    ++k;
                }
                if (pass == 0) a.zg_loc_end[g] = k;
            }
            a.zg_end[g] = k;
        }
        a.nz = k;
        a.nxt = (int)p.x.size();
        for (int j = 0; j < a.nxt; ++j) {
            const int t = p.x[j];
            if (xm[t] & ~inside) fail(QE_ERR_STATE, "expectation term outside its layout");
            a.xloc[j] = to_local(xm[t]);
            a.xzl[j] = to_local(zm[t]);
            a.xzo[j] = zm[t] & ~inside;
            // Re(conj(w) v i^ny): ny = 0: +Re, 1: -Im, 2: -Re, 3: +Im
            const int ny = __builtin_popcountll(xm[t] & zm[t]) & 3;
            a.xbelow[j] = (a.xloc[j] & (~a.xloc[j] + 1u)) - 1u;
            a.xsigned[j] = zm[t] != 0;
            a.ximag[j] = ny & 1;
            a.xw[j] = 2.0 * cf[t] * ((ny == 1 || ny == 2) ? -1.0 : 1.0);
        }
        a.partial = partial + i * max_grid;
        // unused partial slots of this launch read as zero
        QE_CUDA(cudaMemsetAsync(a.partial, 0, max_grid * sizeof(double2), s->stream));
        Launch Lz(s, "expect_tile", (double)dim(s) * amp_bytes(s));
        k_expect_tile<S, NAT><<<grids[i], kRThreads, smem, s->stream>>>(a);
        QE_CUDA(cudaGetLastError());
    }
    {
        Launch Lz(s, "sum_partials", 0.0, false);
        k_sum_partials<<<1, kSumThreads, 0, s->stream>>>(partial, 1, (uint64_t)nlaunch * max_grid, nullptr, dout);
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

uint64_t probs_partials_needed(const qe_state* s, int m) { return probs_partials(s, m); }

void reduce_probs_device(qe_state* s, int m, const int* qubits, double2* partial, double* dout) {
    if (s->dtype == QE_C128) probs_device<double2>(s, m, qubits, partial, dout);
    else probs_device<float2>(s, m, qubits, partial, dout);
}

void reduce_probs(qe_state* s, int m, const int* qubits, double* out) {
    if (s->dtype == QE_C128) probs_impl<double2>(s, m, qubits, out);
    else probs_impl<float2>(s, m, qubits, out);
}

double reduce_expectation(qe_state* s, int nterms, const uint64_t* xm, const uint64_t* zm,
                          const double* cf) {
    if (nterms == 0) return 0.0;
    if (s->dtype == QE_C128) {
        if (c128_f64(s)) return expect_impl<double2, true>(s, nterms, xm, zm, cf);
        return expect_impl<double2, false>(s, nterms, xm, zm, cf);
    }
    return expect_impl<float2, false>(s, nterms, xm, zm, cf);
}

}  // namespace qe
