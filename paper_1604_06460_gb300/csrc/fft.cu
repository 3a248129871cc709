// Emulated QFT (Sec. III-B): the QFT of a register [lo, lo+m) equals, for
// every assignment of the other qubits, the length-2^m discrete Fourier
// transform with kernel exp(+2 pi i k l / 2^m) and scale 2^{-m/2}.  The
// emulator computes it as an in-place FFT instead of m(m+1)/2 gates.
//
// Decomposition: radix-2^r passes from the top register bits down
// (decimation in frequency).  A pass loads tiles that hold whole groups of
// 2^r elements strided along its r bits into shared memory, runs r radix-2
// DIF stages there, multiplies every element by the inter-pass twiddle
// exp(s 2 pi i j2 k1 / 2^(b0+r)) (j2: the register bits below the pass, k1:
// the pass's output digit), and writes the tile back in place.  After the
// last pass the register holds the transform in bit-reversed order; a
// separate in-place tiled pass reverses it.  A register that fits in one
// tile is transformed in a single pass with the reversal done in shared
// memory.  Twiddles come from two tables of FP64-generated roots (fine and
// coarse, 2^ceil(m/2) + 2^floor(m/2) entries) stored in the policy's type.
#include <algorithm>
#include <cmath>
#include <map>
#include <type_traits>

#include "qe_arith.cuh"
#include "qe_internal.h"

namespace qe {

namespace {

constexpr int kFftThreads = 256;

template <class P>
__global__ void k_twiddles(typename P::M* fine, typename P::M* coarse, int m, int h, int sign) {
    const uint64_t nf = 1ull << h, nc = 1ull << (m - h);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nf + nc;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t e = i < nf ? i : ((i - nf) << h);
        // exp(sign * 2 pi i e / 2^m): the angle in units of pi is exact
        const double x = scalbn((double)e, 1 - m);
        double sn, cs;
        sincospi(x, &sn, &cs);
        typename P::M w = P::from_d(cs, sign > 0 ? sn : -sn);
        if (i < nf) fine[i] = w;
        else coarse[i - nf] = w;
    }
}

template <class P>
struct FftArgs {
    typename P::S* x;
    const typename P::M* fine;
    const typename P::M* coarse;
    uint64_t ntiles;
    int L, T, kh;
    uint8_t hq[16];
    int P0;       // tile-local position of the lowest pass bit
    int r;        // bits in this pass
    int b0;       // lowest register bit of this pass (register-relative)
    int lo, m, h; // register placement, size, fine-table bits
    int twiddle;  // multiply by the inter-pass twiddle
    int natural;  // single pass: undo the bit reversal inside the tile
    int scale_on;
    int gmax;     // radix-2 stages per register group (1..4)
    typename P::M scale;
};

template <class P>
__device__ __forceinline__ typename P::M root(const FftArgs<P>& a, uint64_t e) {
    return P::cmul(a.coarse[e >> a.h], a.fine[e & ((1ull << a.h) - 1ull)]);
}

// Asynchronous global -> shared copy of one amplitude (cp.async, 16 or 8 bytes).
template <class S>
__device__ __forceinline__ void async_copy(void* dst, const S* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if (sizeof(S) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Shared-memory slot of tile element i: one pad slot per 16 elements, so that
// the 16-element stride of the lowest register group maps lanes to distinct
// banks.
__device__ __forceinline__ uint32_t pad16(uint32_t i) { return i + (i >> 4); }

// G radix-2 DIF stages s_hi, s_hi-1, ..., s_hi-G+1 of the tile's groups, in
// registers.  Element j (G bits) of a thread's set sits at local index
// base | (j << (P0 + s_lo)); its in-group index is gp = (local >> P0) & (R-1)
// and stage s multiplies the difference by roots[2^s - 1 + (gp mod 2^s)].
template <class P, int G>
__device__ __forceinline__ void stage_group(typename P::V* tile, const typename P::M* roots, int Tn, int P0,
                                            int s_hi) {
    using V = typename P::V;
    constexpr int E = 1 << G;
    const int s_lo = s_hi - G + 1;
    const int sh = P0 + s_lo;
    const uint32_t below = (1u << sh) - 1u;
    const int nbase = Tn >> G;
    for (int b = threadIdx.x; b < nbase; b += blockDim.x) {
        const uint32_t base = (((uint32_t)b & ~below) << G) | ((uint32_t)b & below);
        V v[E];
#pragma unroll
        for (int j = 0; j < E; ++j) v[j] = tile[pad16(base | ((uint32_t)j << sh))];
        const uint32_t gp0 = base >> P0;   // the thread's fixed in-group bits (group bits zero)
#pragma unroll
        for (int t = G - 1; t >= 0; --t) {
            const int s = s_lo + t;
            const uint32_t smask = (1u << s) - 1u;
#pragma unroll
            for (int j = 0; j < E; ++j) {
                if (j & (1 << t)) continue;
                const int j2 = j | (1 << t);
                const uint32_t p = (gp0 | ((uint32_t)j << s_lo)) & smask;
                const typename P::M w = roots[(1u << s) - 1u + p];
                const V u = v[j], x = v[j2];
                v[j] = P::add(u, x);
                v[j2] = P::cmul(w, P::sub(u, x));
            }
        }
#pragma unroll
        for (int j = 0; j < E; ++j) tile[pad16(base | ((uint32_t)j << sh))] = v[j];
    }
}

template <class P>
__global__ void __launch_bounds__(kFftThreads) k_fft_pass(const __grid_constant__ FftArgs<P> a) {
    using V = typename P::V;
    using M = typename P::M;
    using S = typename P::S;
    static_assert(sizeof(V) == sizeof(S), "tile slots hold the raw amplitude before conversion");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Tn = 1 << a.T;
    const int slots = Tn + Tn / 16;
    // two tiles: the next one is copied asynchronously while the current one is transformed
    V* buf[2] = {reinterpret_cast<V*>(smem_raw), reinterpret_cast<V*>(smem_raw) + slots};
    M* roots = reinterpret_cast<M*>(buf[1] + slots);
    __shared__ uint64_t offA[64], offB[64];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int R = 1 << a.r;
    // per-stage tables: roots[2^s - 1 + p] = exp(sign 2 pi i p / 2^(s+1)), p < 2^s,
    // so that lanes with consecutive p read consecutive entries
    for (int e = tid; e < R - 1; e += nth) {
        const int s = 31 - __clz(e + 1);
        const uint64_t p = (uint64_t)(e + 1 - (1 << s));
        roots[e] = root(a, p << (a.m - s - 1));
    }
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
    const uint32_t lowmask = (1u << a.L) - 1u;
    const uint64_t j2mask = (1ull << a.b0) - 1ull;
    const uint64_t emask = (1ull << (a.b0 + a.r)) - 1ull;
    auto issue = [&](uint64_t t, V* dst) {
        const uint64_t base = insert_zero_bits(t << a.L, a.hq, a.kh);
        for (int i = tid; i < Tn; i += nth) {
            const uint32_t hi = (uint32_t)i >> a.L;
            async_copy<S>(dst + pad16(i), a.x + base + (i & lowmask) + offA[hi & 63] + offB[hi >> 6]);
        }
    };
    uint64_t t = blockIdx.x;
    if (t < a.ntiles) issue(t, buf[0]);
    async_commit();
    for (int it = 0; t < a.ntiles; t += gridDim.x, ++it) {
        V* tile = buf[it & 1];
        const uint64_t tn = t + gridDim.x;
        if (tn < a.ntiles) issue(tn, buf[(it + 1) & 1]);
        async_commit();
        async_wait_prev();
        __syncthreads();
        if (sizeof(S) == 16 && !std::is_same<V, S>::value) {
            // raw amplitudes -> the policy's working type, in place
            for (int i = tid; i < Tn; i += nth) {
                const S raw = *reinterpret_cast<const S*>(tile + pad16(i));
                tile[pad16(i)] = P::load(raw);
            }
            __syncthreads();
        }
        const uint64_t base = insert_zero_bits(t << a.L, a.hq, a.kh);
        // radix-2 DIF stages from the top pass bit down, a few at a time in
        // registers: a thread owns the 2^g elements that differ in the g bits
        // of the group, so each group costs one shared-memory round trip
        for (int s_hi = a.r - 1; s_hi >= 0; s_hi -= a.gmax) {
            const int g = s_hi + 1 < a.gmax ? s_hi + 1 : a.gmax;
            switch (g) {
                case 4: stage_group<P, 4>(tile, roots, Tn, a.P0, s_hi); break;
                case 3: stage_group<P, 3>(tile, roots, Tn, a.P0, s_hi); break;
                case 2: stage_group<P, 2>(tile, roots, Tn, a.P0, s_hi); break;
                default: stage_group<P, 1>(tile, roots, Tn, a.P0, s_hi); break;
            }
            __syncthreads();
        }
        for (int i = tid; i < Tn; i += nth) {
            const uint32_t hi = (uint32_t)i >> a.L;
            const uint64_t G = base + (i & lowmask) + offA[hi & 63] + offB[hi >> 6];
            const uint32_t gp = ((uint32_t)i >> a.P0) & (uint32_t)(R - 1);
            const uint32_t rev = (a.r > 0) ? (__brev(gp) >> (32 - a.r)) : 0u;
            V v;
            if (a.natural) {
                // position gp receives the element whose in-group index is rev(gp)
                const uint32_t src = ((uint32_t)i & ~((uint32_t)(R - 1) << a.P0)) | (rev << a.P0);
                v = tile[pad16(src)];
            } else {
                v = tile[pad16(i)];
            }
            if (a.twiddle) {
                const uint64_t j2 = (G >> a.lo) & j2mask;
                const uint64_t e = ((j2 * (uint64_t)rev) & emask) << (a.m - a.b0 - a.r);
                v = P::cmul(root(a, e), v);
            }
            if (a.scale_on) v = P::cmul(a.scale, v);
            a.x[G] = P::store(v);
        }
        __syncthreads();
    }
    async_wait_prev();
}

// --------------------------------------------------------------- bitrev
// In-place reversal of the order of the register value's D-bit digits (D = 1:
// the bit reversal).  Work item = (outer bits, middle value Mv <= rev(Mv));
// tiles X(Mv) and Y(rev Mv) hold elements [b][a][w] (b: top c register bits,
// a: bottom c register bits, c a multiple of D, w: the lo qubits below the
// register) and are exchanged transposed and digit-reversed.
template <class P>
struct RevArgs {
    typename P::S* x;
    uint64_t items;
    int lo, m, c, D;
};

// v (bits bits, a multiple of D) with the order of its D-bit digits reversed.
__device__ __forceinline__ uint64_t digit_rev(uint64_t v, int bits, int D) {
    if (D == 1) return bits > 0 ? (__brevll(v) >> (64 - bits)) : 0ull;
    uint64_t r = 0;
    const uint64_t dm = (1ull << D) - 1ull;
    for (int i = 0; i < bits; i += D) r = (r << D) | ((v >> i) & dm);
    return r;
}

template <class P>
__global__ void __launch_bounds__(256) k_bitrev(const __grid_constant__ RevArgs<P> a) {
    using S = typename P::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = 1 << a.c, W = 1 << a.lo;
    const int row = C * W + 1;   // odd stride in elements: conflict-free 16-byte accesses
    S* X = reinterpret_cast<S*>(smem_raw);
    S* Y = X + C * row;
    const int mid_bits = a.m - 2 * a.c;
    const uint64_t nmid = 1ull << mid_bits;
    for (uint64_t item = blockIdx.x; item < a.items; item += gridDim.x) {
        const uint64_t mv = item & (nmid - 1ull);
        const uint64_t outer = item >> mid_bits;
        const uint64_t mr = digit_rev(mv, mid_bits, a.D);
        if (mv > mr) continue;
        const bool self = (mv == mr);
        const uint64_t obase = outer << (a.lo + a.m);
        const uint64_t bx = obase | (mv << (a.lo + a.c));
        const uint64_t by = obase | (mr << (a.lo + a.c));
        const int shb = a.lo + a.m - a.c;
        const int n = C * C * W;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int b = i / (C * W), aw = i % (C * W);
            const uint64_t off = ((uint64_t)b << shb) | (uint64_t)aw;
            X[b * row + aw] = a.x[bx + off];
            if (!self) Y[b * row + aw] = a.x[by + off];
        }
        __syncthreads();
        const S* srcX = self ? X : Y;   // destination tile X(mv) receives from Y
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int b2 = i / (C * W), aw = i % (C * W);
            const int a2 = aw / W, w = aw % W;
            const int rb = (int)digit_rev((uint64_t)a2, a.c, a.D);   // source b
            const int ra = (int)digit_rev((uint64_t)b2, a.c, a.D);   // source a
            const uint64_t off = ((uint64_t)b2 << shb) | (uint64_t)aw;
            a.x[bx + off] = srcX[rb * row + ra * W + w];
            if (!self) a.x[by + off] = X[rb * row + ra * W + w];
        }
        __syncthreads();
    }
}

struct TableKey {
    int m, sign, policy;
    bool operator<(const TableKey& o) const {
        return m != o.m ? m < o.m : sign != o.sign ? sign < o.sign : policy < o.policy;
    }
};
struct Table {
    void* fine = nullptr;
    void* coarse = nullptr;
};
std::map<std::pair<int, TableKey>, Table> g_tables;   // (device, key) -> table

template <class P>
Table get_tables(qe_state* s, int m, int sign, int pol) {
    int dev = 0;
    QE_CUDA(cudaGetDevice(&dev));
    auto key = std::make_pair(dev, TableKey{m, sign, pol});
    auto it = g_tables.find(key);
    if (it != g_tables.end()) return it->second;
    const int h = (m + 1) / 2;
    Table t;
    QE_CUDA(cudaMalloc(&t.fine, sizeof(typename P::M) << h));
    QE_CUDA(cudaMalloc(&t.coarse, sizeof(typename P::M) << (m - h)));
    uint64_t total = (1ull << h) + (1ull << (m - h));
    unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, 4096);
    Launch L(s, "fft_twiddles", 0.0, false);
    k_twiddles<P><<<grid, 256, 0, s->stream>>>((typename P::M*)t.fine, (typename P::M*)t.coarse, m, h, sign);
    QE_CUDA(cudaGetLastError());
    g_tables[key] = t;
    return t;
}

struct Geom {
    int T = 0, L = 0, kh = 0;
    uint8_t hq[16] = {0};
};
// Tile of at most 2^Tt elements containing the register bits [g0, g0+r).
Geom pass_geom(int n, int g0, int r, int Tt) {
    Tt = std::min(Tt, n);
    for (int L = Tt; L >= 0; --L) {
        int kh = 0;
        for (int q = g0; q < g0 + r; ++q) kh += q >= L;
        if (L + kh <= Tt) {
            Geom g;
            g.L = L;
            g.kh = kh;
            g.T = L + kh;
            int j = 0;
            for (int q = g0; q < g0 + r; ++q)
                if (q >= L) g.hq[j++] = (uint8_t)q;
            return g;
        }
    }
    fail(QE_ERR_ARG, "no FFT tile geometry");
}

template <class P>
void fft_impl(qe_state* s, int lo, int m, int inverse, int pol) {
    const int sign = inverse ? -1 : 1;
    Table tb = get_tables<P>(s, m, sign, pol);
    const int Tmax = (sizeof(typename P::V) >= 16) ? 11 : 12;
    const int Lmin = 3;   // runs of >= 8 amplitudes (measured best: fewer passes outweigh shorter runs)
    const int rb_max = Tmax - std::min(lo, Lmin);
    std::vector<std::pair<int, int>> passes;   // (b0, r), top first
    if (m <= rb_max) {
        passes.push_back({0, m});
    } else {
        const int ru_max = Tmax - Lmin;
        const int rest = m - rb_max;
        const int nup = (rest + ru_max - 1) / ru_max;
        int top = m;
        for (int p = 0; p < nup; ++p) {
            int r = rest / nup + (p < rest % nup ? 1 : 0);
            passes.push_back({top - r, r});
            top -= r;
        }
        passes.push_back({0, top});
    }
    static thread_local FftArgs<P> a;
    a.x = reinterpret_cast<typename P::S*>(s->d);
    a.fine = (const typename P::M*)tb.fine;
    a.coarse = (const typename P::M*)tb.coarse;
    a.lo = lo;
    a.m = m;
    a.h = (m + 1) / 2;
    const double scale = std::pow(2.0, -0.5 * m);
    a.scale = P::mat(scale, 0.0);
    const bool single = passes.size() == 1;
    for (size_t p = 0; p < passes.size(); ++p) {
        const int b0 = passes[p].first, r = passes[p].second;
        Geom g = pass_geom(s->n, lo + b0, r, Tmax);
        a.L = g.L;
        a.T = g.T;
        a.kh = g.kh;
        for (int j = 0; j < 16; ++j) a.hq[j] = g.hq[j];
        a.P0 = std::min(lo + b0, g.L);
        a.r = r;
        a.b0 = b0;
        a.ntiles = 1ull << (s->n - g.T);
        a.twiddle = b0 > 0;
        a.natural = single;
        a.scale_on = (p + 1 == passes.size());
        size_t smem = 2 * sizeof(typename P::V) * (((size_t)1 << g.T) + ((size_t)1 << g.T) / 16) +
                      sizeof(typename P::M) * ((size_t)1 << r);
        // three radix-2 stages per register group and 256 threads measured
        // fastest on GB300 for both complex64 and complex128 tiles
        a.gmax = 3;
        const int threads = std::max(64, std::min(256, (1 << g.T) >> a.gmax));
        auto fn = k_fft_pass<P>;
        QE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int occ = 0;
        QE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem));
        uint64_t grid = std::min<uint64_t>(a.ntiles, (uint64_t)num_sms() * std::max(occ, 1));
        Launch L(s, "fft_pass", 2.0 * dim(s) * amp_bytes(s));
        fn<<<(unsigned)grid, threads, smem, s->stream>>>(a);
        QE_CUDA(cudaGetLastError());
    }
    if (!single) launch_bitrev(s, lo, m);
}

template <class S>
__global__ void __launch_bounds__(256) k_bitrev_chunks(S* __restrict__ x, uint64_t count, int lo, int m, int D) {
    const uint64_t rmask = ((1ull << m) - 1ull) << lo;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = (i & rmask) >> lo;
        const uint64_t kr = digit_rev(k, m, D);
        if (k < kr) {
            const uint64_t j = (i & ~rmask) | (kr << lo);
            S t = x[i];
            x[i] = x[j];
            x[j] = t;
        }
    }
}

template <class P>
void bitrev_impl(qe_state* s, int lo, int m, int D = 1) {
    if (m <= D) return;
    using S = typename P::S;
    Launch L(s, D == 1 ? "bitrev" : "digitrev", 2.0 * dim(s) * amp_bytes(s));
    // end blocks of c bits (a multiple of D, 2c <= m) in tiles of 2^(2c + lo) <= 2^11
    const int c = D * std::min(m / (2 * D), std::max(0, (11 - lo) / 2) / D);
    if (lo >= 5 || c == 0) {
        // chunks of >= 32 contiguous amplitudes move as units: coalesced pair swaps
        const uint64_t count = dim(s);
        unsigned grid = (unsigned)std::min<uint64_t>((count + 255) / 256, (uint64_t)num_sms() * 8);
        k_bitrev_chunks<S><<<grid, 256, 0, s->stream>>>(reinterpret_cast<S*>(s->d), count, lo, m, D);
    } else {
        static thread_local RevArgs<P> a;
        a.x = reinterpret_cast<S*>(s->d);
        a.lo = lo;
        a.m = m;
        a.D = D;
        a.c = c;
        a.items = (1ull << (s->n - lo - m)) << (m - 2 * a.c);
        const int C = 1 << a.c, W = 1 << lo;
        size_t smem = sizeof(S) * 2 * (size_t)C * (C * W + 1);
        auto fn = k_bitrev<P>;
        QE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int occ = 0;
        QE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, smem));
        uint64_t grid = std::min<uint64_t>(a.items, (uint64_t)num_sms() * std::max(occ, 1));
        fn<<<(unsigned)grid, 256, smem, s->stream>>>(a);
    }
    QE_CUDA(cudaGetLastError());
}

// ------------------------------------------------ tensor-core digit passes
// The QFT of a register of m = G d bits as G dense d-qubit blocks on the
// tensor cores (the 2^d-point DFT, the same matrix for every group of the
// other qubits) with diagonal twiddles between them (Cooley-Tukey, digits
// from the top): with k = k0 2^(m-d) + k' and l = l0 + 2^d l',
//   y_l = sum_k' w_(2^(m-d))^(k' l') [ w_(2^m)^(k' l0) sum_k0 x_(k0, k') w_(2^d)^(k0 l0) ],
// so a pass applies the DFT to the top digit (output l0 left in its qubits),
// a twiddle pass multiplies by w_(2^m)^(k' l0), and the rest is the QFT of
// the lower m - d bits; at the end the digits sit in reversed order and one
// digit-reversal pass restores the natural order.  Scale 2^(-d/2) per block.
template <class P>
struct TwArgs {
    typename P::S* x;
    const typename P::M* fine;
    const typename P::M* coarse;
    const typename P::M* direct;   // w_(2^(top + d))^j for all j, when the order is at most 2^20 (else null)
    uint64_t count;
    int lo, m, h;
    int top;      // the digit just transformed: register bits [top, top + d)
    int d;
    int shift;    // the twiddle exponent's scale to the 2^m table: 2^shift
};

// x *= w_(2^(top + d))^(k' l0), k' = register bits [0, top), l0 = bits [top, top + d)
template <class P>
__global__ void __launch_bounds__(256) k_digit_twiddle(const __grid_constant__ TwArgs<P> a) {
    const uint64_t rmask = (1ull << a.m) - 1ull;
    const uint64_t hmask = (1ull << a.h) - 1ull;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = (i >> a.lo) & rmask;
        const uint64_t kp = r & ((1ull << a.top) - 1ull);
        const uint64_t l0 = (r >> a.top) & ((1ull << a.d) - 1ull);
        if (kp == 0 || l0 == 0) continue;
        // exponent over 2^(top + d): one table entry when the order is small
        // enough for a direct table, else the product of the two 2^m tables
        const uint64_t e0 = (kp * l0) & ((1ull << (a.top + a.d)) - 1ull);
        typename P::M w;
        if (a.direct) {
            w = a.direct[e0];
        } else {
            const uint64_t e = e0 << a.shift;
            w = P::cmul(a.coarse[e >> a.h], a.fine[e & hmask]);
        }
        a.x[i] = P::store(P::cmul(w, P::load(a.x[i])));
    }
}

// Digit size for the tensor-core QFT of an m-bit register: the largest of
// 5, 4, 3 dividing m (0: none).
int qft_digit(int m) {
    for (int d : {5, 4, 3})
        if (m % d == 0) return d;
    return 0;
}

// Direct table of the 2^k roots of unity w_(2^k)^j (FP64-generated, stored in
// the policy's type), cached per (device, k, sign, policy) like the two-level
// tables; k <= 20 (16 MB for complex128, resident in L2).
template <class P>
__global__ void k_roots_direct(typename P::M* t, int k, int sign) {
    const uint64_t N = 1ull << k;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < N; j += (uint64_t)gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(scalbn((double)j, 1 - k), &sn, &cs);
        t[j] = P::from_d(cs, sign > 0 ? sn : -sn);
    }
}
std::map<std::pair<int, TableKey>, void*> g_direct;   // (device, (k, sign, policy)) -> table

template <class P>
const typename P::M* get_direct(qe_state* s, int k, int sign, int pol) {
    int dev = 0;
    QE_CUDA(cudaGetDevice(&dev));
    auto key = std::make_pair(dev, TableKey{k, sign, pol});
    auto it = g_direct.find(key);
    if (it != g_direct.end()) return (const typename P::M*)it->second;
    void* t = nullptr;
    QE_CUDA(cudaMalloc(&t, sizeof(typename P::M) << k));
    Launch L(s, "fft_twiddles", 0.0, false);
    const unsigned grid = (unsigned)std::min<uint64_t>(((1ull << k) + 255) / 256, 4096);
    k_roots_direct<P><<<grid, 256, 0, s->stream>>>((typename P::M*)t, k, sign);
    QE_CUDA(cudaGetLastError());
    g_direct[key] = t;
    return (const typename P::M*)t;
}

template <class P>
void qft_tc_impl(qe_state* s, int lo, int m, int inverse, int pol, int d) {
    const int sign = inverse ? -1 : 1;
    Table tb = get_tables<P>(s, m, sign, pol);
    const int D = 1 << d;
    std::vector<cd> F((size_t)D * D);
    const double sc = 1.0 / std::sqrt((double)D);
    for (int l = 0; l < D; ++l)
        for (int k = 0; k < D; ++k) {
            const double t = sign * 2.0 * ((double)((k * l) % D) / D);   // angle in units of pi
            F[(size_t)l * D + k] = cd(sc * std::cos(M_PI * t), sc * std::sin(M_PI * t));
        }
    // exact values at the quarter turns (cos/sin of multiples of pi/2)
    for (auto& v : F) {
        if (std::fabs(v.real()) < 1e-17) v = cd(0.0, v.imag());
        if (std::fabs(v.imag()) < 1e-17) v = cd(v.real(), 0.0);
    }
    static thread_local TwArgs<P> a;
    a.x = reinterpret_cast<typename P::S*>(s->d);
    a.fine = (const typename P::M*)tb.fine;
    a.coarse = (const typename P::M*)tb.coarse;
    a.count = dim(s);
    a.lo = lo;
    a.m = m;
    a.h = (m + 1) / 2;
    a.d = d;
    const int G = m / d;
    for (int t = 0; t < G; ++t) {
        const int top = m - d * (t + 1);
        int q[5];
        for (int j = 0; j < d; ++j) q[j] = lo + top + j;
        launch_gate_dense(s, d, q, F.data());
        if (top == 0) break;
        a.top = top;
        a.shift = m - (top + d);
        a.direct = (top + d <= 20) ? get_direct<P>(s, top + d, sign, pol) : nullptr;
        const unsigned grid = (unsigned)std::min<uint64_t>((a.count + 255) / 256, (uint64_t)num_sms() * 8);
        Launch L(s, "fft_twiddle", 2.0 * dim(s) * amp_bytes(s));
        k_digit_twiddle<P><<<grid, 256, 0, s->stream>>>(a);
        QE_CUDA(cudaGetLastError());
    }
    bitrev_impl<F64>(s, lo, m, d);
}

}  // namespace

// Tensor-core digit passes in the FP64 mode where a dense block of 3-5
// qubits runs on the tensor cores (n >= 12) and a digit size divides m;
// otherwise the radix-2 shared-memory FFT.
void launch_qft_fft(qe_state* s, int lo, int m, int inverse) {
    const int d = qft_digit(m);
    // (in the double-float mode the shared-memory FFT is the faster: its
    // twiddle joins cost as much FP64 work as the digit passes save)
    const bool tc = s->dtype == QE_C128 && s->arith == QE_ARITH_FP64 && s->c128_tc && s->tensor_cores &&
                    !s->force_tile && s->n >= 12 && d >= c128_tc_kmin(s) && m > 1;
    if (tc) {
        qft_tc_impl<F64>(s, lo, m, inverse, 1, d);
        return;
    }
    if (s->dtype == QE_C64) fft_impl<F32>(s, lo, m, inverse, 0);
    else if (s->arith == QE_ARITH_FP64) fft_impl<F64>(s, lo, m, inverse, 1);
    else fft_impl<DF>(s, lo, m, inverse, 2);
}

void launch_bitrev(qe_state* s, int lo, int m) {
    if (s->dtype == QE_C64) bitrev_impl<F32>(s, lo, m);
    else bitrev_impl<F64>(s, lo, m);   // pure data movement: storage type only
}

}  // namespace qe
