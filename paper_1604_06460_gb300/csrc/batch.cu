// Batch of parameterised circuits in one persistent launch (CUDA graph).
//
// Each circuit is the hardware-efficient ansatz: `layers` times (RY(theta),
// RZ(phi) on every qubit, then CZ on (q, q+1) for q = 0..n-2), started from
// |0...0>, and returns the energy of the transverse-field Ising Hamiltonian
// sum_i Z_i Z_{i+1} + h sum_i X_i (open chain), the expectation evaluated
// directly (Sec. III-D).  The RY/RZ pair of a qubit is fused on the host into
// one 2x2 matrix; the CZ ladder of a layer is one diagonal phase
// (-1)^popcount(x & x>>1).
//
// Work decomposition (one work queue, claimed in order with an atomic head):
//   - a circuit with n <= T qubits is one item: its whole state lives in one
//     CTA's shared memory, HBM is never touched;
//   - a circuit with n > T qubits keeps its state in HBM and is processed in
//     2*layers + 1 passes over tiles of 2^T amplitudes: per layer a "low"
//     pass (contiguous tiles, gates on qubits < T) and a "high" pass (tiles
//     of 2^(2T-n)-amplitude chunks, gates on qubits >= T, then the CZ phase);
//     the last high pass also accumulates the ZZ terms and the X terms of the
//     high qubits; a final read-only low pass adds the X terms of the low
//     qubits.  Each pass is split into items of a few tiles.
// An item may start only when every item of the circuit's earlier passes has
// finished: CTAs wait on a per-circuit completion counter.  Large circuits
// are queued in waves of at most 64 MiB of state (half the L2 cache),
// pass-major inside a wave, with the small circuits spread between the
// passes; the dependencies of any claimed item were claimed earlier by
// running CTAs; waits are bounded and report a timeout.
#include <algorithm>
#include <cmath>
#include <vector>

#include "qe_arith.cuh"
#include "qe_batch.h"
#include "qe_internal.h"

namespace qe {

namespace {

struct Item {
    int circuit;
    int kind;          // 0 small, 1 low layer pass, 2 high layer pass, 3 energy low pass
    int layer;
    uint32_t tile0, tile1;
    uint32_t dep;      // completed items of this circuit required before starting
    int slot;          // energy partial slot (or -1)
    int last_energy;   // 1: high pass of the last layer (accumulates energy)
};

struct Circ {
    int n;
    int nitems;        // items of this circuit
    int slot0, nslots; // energy partial slots
    uint64_t state_off; // amplitude offset of its HBM state (large circuits)
    uint64_t u_off;     // offset of its matrices (layers * n * 4 entries)
};

template <class P>
struct BatchArgs {
    typename P::S* states;
    const typename P::M* U;
    const Item* items;
    const Circ* circ;
    int nitems;
    int T;
    int layers;
    double hx;
    unsigned* head;
    unsigned* counters;
    unsigned* status;      // nonzero: a wait timed out
    double2* partials;     // (zz sum, x sum) per energy slot
    double* energies;
    long long spin_limit;
    int gmax;              // single-qubit gates per register group
};

template <class P>
__device__ __forceinline__ typename P::V outv(const typename P::A& a);
template <>
__device__ __forceinline__ F32::V outv<F32>(const F32::A& a) { return make_float2(a.re, a.im); }
template <>
__device__ __forceinline__ F64::V outv<F64>(const F64::A& a) { return make_double2(a.re, a.im); }
template <>
__device__ __forceinline__ DF::V outv<DF>(const DF::A& a) {
    return DF::V{df_norm(a.rs, a.re_), df_norm(a.is, a.ie)};
}

// |v|^2 and Re(conj(w) v) as double-float pairs.
__device__ __forceinline__ void sq(const float2& v, float& h, float& l) {
    df_first(h, l, df{v.x, 0.f}, df{v.x, 0.f});
    df_acc(h, l, df{v.y, 0.f}, df{v.y, 0.f});
}
__device__ __forceinline__ void sq(const DF::V& v, float& h, float& l) {
    df_first(h, l, v.re, v.re);
    df_acc(h, l, v.im, v.im);
}
__device__ __forceinline__ void sq(const double2& v, float& h, float& l) { sq(DF::load(v), h, l); }
__device__ __forceinline__ void re_dot(const float2& w, const float2& v, float& h, float& l) {
    df_first(h, l, df{w.x, 0.f}, df{v.x, 0.f});
    df_acc(h, l, df{w.y, 0.f}, df{v.y, 0.f});
}
__device__ __forceinline__ void re_dot(const DF::V& w, const DF::V& v, float& h, float& l) {
    df_first(h, l, w.re, v.re);
    df_acc(h, l, w.im, v.im);
}
__device__ __forceinline__ void re_dot(const double2& w, const double2& v, float& h, float& l) {
    re_dot(DF::load(w), DF::load(v), h, l);
}
__device__ __forceinline__ void acc2(float& s, float& e, float ph, float pl) {
    float t = fadd(s, ph);
    float bb = fsub(t, s);
    float err = fadd(fsub(s, fsub(t, bb)), fsub(ph, bb));
    s = t;
    e = fadd(e, fadd(err, pl));
}

template <class P>
__device__ __forceinline__ typename P::V zero_v();
template <>
__device__ __forceinline__ float2 zero_v<F32>() { return make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ double2 zero_v<F64>() { return make_double2(0.0, 0.0); }
template <>
__device__ __forceinline__ DF::V zero_v<DF>() { return DF::V{df{0.f, 0.f}, df{0.f, 0.f}}; }
template <class P>
__device__ __forceinline__ typename P::V one_v();
template <>
__device__ __forceinline__ float2 one_v<F32>() { return make_float2(1.f, 0.f); }
template <>
__device__ __forceinline__ double2 one_v<F64>() { return make_double2(1.0, 0.0); }
template <>
__device__ __forceinline__ DF::V one_v<DF>() { return DF::V{df{1.f, 0.f}, df{0.f, 0.f}}; }
template <class P>
__device__ __forceinline__ typename P::V neg_v(const typename P::V& v);
template <>
__device__ __forceinline__ float2 neg_v<F32>(const float2& v) { return make_float2(-v.x, -v.y); }
template <>
__device__ __forceinline__ double2 neg_v<F64>(const double2& v) { return make_double2(-v.x, -v.y); }
template <>
__device__ __forceinline__ DF::V neg_v<DF>(const DF::V& v) {
    return DF::V{df{-v.re.h, -v.re.l}, df{-v.im.h, -v.im.l}};
}

// Shared-memory slot of tile element i (one pad slot per 16 elements keeps
// the 16-element strides of register groups on distinct banks).
__device__ __forceinline__ uint32_t pad16(uint32_t i) { return i + (i >> 4); }

// Apply the G single-qubit matrices of tile-local bits b0 .. b0+G-1
// (U + 4*t for bit b0+t) in registers: a thread owns the 2^G elements that
// differ in those bits, so G gates cost one shared-memory round trip.
template <class P, int G>
__device__ void tile_gates_reg(typename P::V* tile, int T, int b0, const typename P::M* U) {
    using V = typename P::V;
    constexpr int E = 1 << G;
    typename P::M u[G][4];
#pragma unroll
    for (int t = 0; t < G; ++t)
#pragma unroll
        for (int k = 0; k < 4; ++k) u[t][k] = U[4 * t + k];
    const uint32_t below = (1u << b0) - 1u;
    const int nbase = 1 << (T - G);
    for (int b = threadIdx.x; b < nbase; b += blockDim.x) {
        const uint32_t base = (((uint32_t)b & ~below) << G) | ((uint32_t)b & below);
        V v[E];
#pragma unroll
        for (int j = 0; j < E; ++j) v[j] = tile[pad16(base | ((uint32_t)j << b0))];
#pragma unroll
        for (int t = 0; t < G; ++t)
#pragma unroll
            for (int j = 0; j < E; ++j) {
                if (j & (1 << t)) continue;
                const int j2 = j | (1 << t);
                typename P::A a0, a1;
                P::mac_first(a0, u[t][0], v[j]);
                P::mac(a0, u[t][1], v[j2]);
                P::mac_first(a1, u[t][2], v[j]);
                P::mac(a1, u[t][3], v[j2]);
                v[j] = outv<P>(a0);
                v[j2] = outv<P>(a1);
            }
#pragma unroll
        for (int j = 0; j < E; ++j) tile[pad16(base | ((uint32_t)j << b0))] = v[j];
    }
    __syncthreads();
}

// Gates on the tile-local bits [b0, b0 + cnt), whose matrices are U + 4*i.
template <class P>
__device__ void tile_gates(typename P::V* tile, int T, int b0, int cnt, const typename P::M* U, int gmax_arg) {
    // register budget: 16 complex64 or 8 double-float values per thread
    // double-float groups hold at most 2 gates: wider groups are not even
    // instantiated for it (their registers would spill)
    constexpr bool wide = sizeof(typename P::V) < 16;
    const int gmax = wide ? gmax_arg : (gmax_arg < 2 ? gmax_arg : 2);
    while (cnt > 0) {
        const int g = cnt >= gmax ? gmax : cnt;
        if constexpr (wide) {
            switch (g) {
                case 4: tile_gates_reg<P, 4>(tile, T, b0, U); break;
                case 3: tile_gates_reg<P, 3>(tile, T, b0, U); break;
                case 2: tile_gates_reg<P, 2>(tile, T, b0, U); break;
                default: tile_gates_reg<P, 1>(tile, T, b0, U); break;
            }
        } else {
            if (g == 2) tile_gates_reg<P, 2>(tile, T, b0, U);
            else tile_gates_reg<P, 1>(tile, T, b0, U);
        }
        b0 += g;
        cnt -= g;
        U += 4 * g;
    }
}

// Block-wide double-float sum of (s, e) pairs; result valid in thread 0.
__device__ double block_sum(float s, float e, double* sh) {
    double d = df2d(s, e);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = d;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
    return tot;
}
// ... of FP64 values; result valid in thread 0
__device__ double block_sum_d(double d, double* sh) {
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = d;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
    return tot;
}

// Energy sums of one CTA: float pairs (s, e) with exact products for the
// FP32 and double-float policies, plain FP64 fused multiply-adds for FP64.
template <class P>
struct EAcc {
    float zs = 0.f, ze = 0.f, xs = 0.f, xe = 0.f;
    // z += |v|^2 f (f a small integer), x += Re(conj(w) v)
    __device__ __forceinline__ void add_z(const typename P::V& v, float f) {
        float h, l;
        sq(v, h, l);
        const float p = fmul(h, f);
        const float pe = __fmaf_rn(h, f, -p);
        acc2(zs, ze, p, __fmaf_rn(l, f, pe));
    }
    __device__ __forceinline__ void add_x(const typename P::V& w, const typename P::V& v) {
        float h, l;
        re_dot(w, v, h, l);
        acc2(xs, xe, h, l);
    }
    __device__ double z_total(double* sh) { return block_sum(zs, ze, sh); }
    __device__ double x_total(double* sh) { return block_sum(xs, xe, sh); }
};
template <>
struct EAcc<F64> {
    double z = 0.0, x = 0.0;
    __device__ __forceinline__ void add_z(const double2& v, float f) {
        z = __fma_rn(__fma_rn(v.x, v.x, __dmul_rn(v.y, v.y)), (double)f, z);
    }
    __device__ __forceinline__ void add_x(const double2& w, const double2& v) {
        x = __fma_rn(w.x, v.x, __fma_rn(w.y, v.y, x));
    }
    __device__ double z_total(double* sh) { return block_sum_d(z, sh); }
    __device__ double x_total(double* sh) { return block_sum_d(x, sh); }
};


template <class P>
__global__ void __launch_bounds__(512) k_batch(const __grid_constant__ BatchArgs<P> a) {
    using V = typename P::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tile = reinterpret_cast<V*>(smem_raw);
    __shared__ double shred[32];
    __shared__ int s_item;
    __shared__ int s_ok;
    const int T = a.T;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.head, 1u);
        __syncthreads();
        const int idx = s_item;
        __syncthreads();
        if (idx >= a.nitems) return;
        const Item it = a.items[idx];
        const Circ cc = a.circ[it.circuit];
        const int n = cc.n;
        // wait for the circuit's earlier passes (bounded)
        if (threadIdx.x == 0) {
            int ok = 1;
            if (it.dep > 0) {
                long long spins = 0;
                while (*((volatile unsigned*)&a.counters[it.circuit]) < it.dep) {
                    // give up after the limit, or at once if another wait already failed
                    if (++spins > a.spin_limit || *((volatile unsigned*)a.status) != 0u) {
                        ok = 0;
                        atomicExch(a.status, 1u);
                        break;
                    }
                    __nanosleep(256);
                }
                __threadfence();
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) continue;
        const typename P::M* U = a.U + cc.u_off;
        EAcc<P> acc;
        if (it.kind == 0) {
            // ------------------------------------------------ small circuit
            const uint32_t N = 1u << n;
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x)
                tile[pad16(i)] = (i == 0) ? one_v<P>() : zero_v<P>();
            __syncthreads();
            for (int l = 0; l < a.layers; ++l) {
                tile_gates<P>(tile, n, 0, n, U + (size_t)l * n * 4, a.gmax);
                for (uint32_t i = threadIdx.x; i < N; i += blockDim.x)
                    if (__popc(i & (i >> 1)) & 1) tile[pad16(i)] = neg_v<P>(tile[pad16(i)]);
                __syncthreads();
            }
            const uint32_t zmask = (n > 1) ? ((1u << (n - 1)) - 1u) : 0u;
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
                acc.add_z(tile[pad16(i)], (float)((n - 1) - 2 * __popc((i ^ (i >> 1)) & zmask)));
                for (int q = 0; q < n; ++q)
                    if (!((i >> q) & 1u)) acc.add_x(tile[pad16(i | (1u << q))], tile[pad16(i)]);
            }
            const double z = acc.z_total(shred);
            const double x = acc.x_total(shred);
            if (threadIdx.x == 0) a.energies[it.circuit] = z + 2.0 * a.hx * x;
            __syncthreads();
            continue;
        }
        // ---------------------------------------------------- large circuit
        typename P::S* st = a.states + cc.state_off;
        const int L = 2 * T - n;                 // chunk bits of the high layout
        const uint32_t lowmask = (1u << L) - 1u;
        const uint64_t zmask = (n > 1) ? ((1ull << (n - 1)) - 1ull) : 0ull;
        for (uint32_t t = it.tile0; t < it.tile1; ++t) {
            const bool high = it.kind == 2;
            auto gidx = [&](uint32_t l) -> uint64_t {
                if (!high) return ((uint64_t)t << T) | l;
                return (uint64_t)(l & lowmask) | ((uint64_t)t << L) | ((uint64_t)(l >> L) << T);
            };
            const uint32_t TN = 1u << T;
            if (it.kind == 1 && it.layer == 0) {
                for (uint32_t l = threadIdx.x; l < TN; l += blockDim.x)
                    tile[pad16(l)] = (t == 0 && l == 0) ? one_v<P>() : zero_v<P>();
            } else {
                for (uint32_t l = threadIdx.x; l < TN; l += blockDim.x) tile[pad16(l)] = P::load(st[gidx(l)]);
            }
            __syncthreads();
            if (it.kind == 1) {
                tile_gates<P>(tile, T, 0, T, U + (size_t)it.layer * n * 4, a.gmax);
            } else if (it.kind == 2) {
                tile_gates<P>(tile, T, L, n - T, U + ((size_t)it.layer * n + T) * 4, a.gmax);
                for (uint32_t l = threadIdx.x; l < TN; l += blockDim.x) {
                    const uint64_t x = gidx(l);
                    if (__popcll(x & (x >> 1)) & 1) tile[pad16(l)] = neg_v<P>(tile[pad16(l)]);
                }
                __syncthreads();
            }
            if (it.kind == 2 && it.last_energy) {
                for (uint32_t l = threadIdx.x; l < TN; l += blockDim.x) {
                    const uint64_t x = gidx(l);
                    acc.add_z(tile[pad16(l)], (float)((n - 1) - 2 * __popcll((x ^ (x >> 1)) & zmask)));
                    for (int q = T; q < n; ++q) {
                        const int b = L + (q - T);
                        if (!((l >> b) & 1u)) acc.add_x(tile[pad16(l | (1u << b))], tile[pad16(l)]);
                    }
                }
            }
            if (it.kind == 3) {
                for (uint32_t l = threadIdx.x; l < TN; l += blockDim.x)
                    for (int q = 0; q < T; ++q)
                        if (!((l >> q) & 1u)) acc.add_x(tile[pad16(l | (1u << q))], tile[pad16(l)]);
            } else {
                for (uint32_t l = threadIdx.x; l < TN; l += blockDim.x) st[gidx(l)] = P::store(tile[pad16(l)]);
            }
            __syncthreads();
        }
        if (it.slot >= 0) {
            const double z = acc.z_total(shred);
            const double x = acc.x_total(shred);
            if (threadIdx.x == 0) a.partials[it.slot] = make_double2(z, x);
        }
        // publish completion; the CTA that completes the circuit sums its energy
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned done = atomicAdd(&a.counters[it.circuit], 1u) + 1u;
            if (done == (unsigned)cc.nitems) {
                __threadfence();
                double zsum = 0.0, xsum = 0.0;
                for (int k = 0; k < cc.nslots; ++k) {
                    // written by other CTAs before their counter increments:
                    // read through L2 (bypassing this SM's L1)
                    const double2 p = __ldcg(&a.partials[cc.slot0 + k]);
                    zsum += p.x;
                    xsum += p.y;
                }
                a.energies[it.circuit] = zsum + 2.0 * a.hx * xsum;
            }
        }
        __syncthreads();
    }
}

}  // namespace

}  // namespace qe

namespace qe {

namespace {

template <class P>
void upload_matrices(qe_batch* b, std::vector<uint64_t>& u_off) {
    std::vector<typename P::M> h;
    u_off.resize(b->count);
    size_t ai = 0;
    for (int c = 0; c < b->count; ++c) {
        const int n = b->n[c];
        u_off[c] = h.size();
        for (int l = 0; l < b->layers; ++l)
            for (int q = 0; q < n; ++q) {
                const double th = b->angles[ai++], ph = b->angles[ai++];
                // RZ(ph) * RY(th)
                const double c2 = std::cos(0.5 * th), s2 = std::sin(0.5 * th);
                const cd em = std::polar(1.0, -0.5 * ph), ep = std::polar(1.0, 0.5 * ph);
                const cd m[4] = {em * c2, -em * s2, ep * s2, ep * c2};
                for (int k = 0; k < 4; ++k) h.push_back(P::mat(m[k].real(), m[k].imag()));
            }
    }
    if (b->U) cudaFree(b->U);
    QE_CUDA(cudaMalloc(&b->U, h.size() * sizeof(typename P::M)));
    QE_CUDA(cudaMemcpy(b->U, h.data(), h.size() * sizeof(typename P::M), cudaMemcpyHostToDevice));
}

// States of the large circuits of one wave: together at most this many bytes
// (half the 129 MB L2 cache).
constexpr uint64_t kWaveBytes = 64ull << 20;

template <class P>
void build_plan(qe_batch* b) {
    const int T = b->plan.T;
    std::vector<uint64_t> u_off;
    upload_matrices<P>(b, u_off);
    std::vector<Circ> circ(b->count);
    std::vector<Item> items;
    uint64_t state_off = 0;
    int slots = 0;
    std::vector<int> large;
    for (int c = 0; c < b->count; ++c) {
        Circ& cc = circ[c];
        cc.n = b->n[c];
        cc.u_off = u_off[c];
        cc.state_off = 0;
        if (cc.n <= T) {
            cc.nitems = 1;
            cc.slot0 = 0;
            cc.nslots = 0;
        } else {
            cc.state_off = state_off;
            state_off += 1ull << cc.n;
            large.push_back(c);
        }
    }
    // large circuits largest first
    std::stable_sort(large.begin(), large.end(), [&](int x, int y) { return circ[x].n > circ[y].n; });
    const int P_ = 2 * b->layers + 1;
    std::vector<std::vector<int>> per_pass_count(b->count, std::vector<int>(P_, 0));
    for (int c : large) {
        Circ& cc = circ[c];
        const uint32_t tiles = 1u << (cc.n - T);
        const uint32_t per = (uint32_t)std::max(1, b->plan.tiles_per_item);
        const int nper = (int)((tiles + per - 1) / per);
        cc.nitems = P_ * nper;
        cc.slot0 = slots;
        cc.nslots = 2 * nper;   // last high pass + energy low pass
        slots += cc.nslots;
    }
    auto push_pass = [&](int c, int p) {
        const Circ& cc = circ[c];
        const uint32_t tiles = 1u << (cc.n - T);
        const uint32_t per = (uint32_t)std::max(1, b->plan.tiles_per_item);
        const int nper = (int)((tiles + per - 1) / per);
        for (int j = 0; j < nper; ++j) {
            Item it{};
            it.circuit = c;
            it.kind = (p == P_ - 1) ? 3 : (p % 2 == 0 ? 1 : 2);
            it.layer = p / 2;
            it.tile0 = j * per;
            it.tile1 = std::min(tiles, (uint32_t)(j + 1) * per);
            it.dep = (uint32_t)(p * nper);
            it.last_energy = (p == P_ - 2) ? 1 : 0;
            it.slot = (p == P_ - 2) ? cc.slot0 + j : (p == P_ - 1) ? cc.slot0 + nper + j : -1;
            items.push_back(it);
        }
    };
    auto push_small = [&](int c) {
        Item it{};
        it.circuit = c;
        it.kind = 0;
        it.slot = -1;
        items.push_back(it);
    };
    // small circuits (largest first): one item each, without dependencies
    std::vector<int> small;
    for (int c = 0; c < b->count; ++c)
        if (circ[c].n <= T) small.push_back(c);
    std::stable_sort(small.begin(), small.end(), [&](int x, int y) { return circ[x].n > circ[y].n; });
    // Large circuits go in waves whose states together fit in the L2 cache,
    // pass-major inside a wave, so that a circuit's passes find its state in
    // L2 instead of HBM; the small circuits' items are spread evenly between
    // the passes, where they occupy CTAs that would otherwise wait for a
    // pass to finish.  Every item's dependencies (its circuit's earlier
    // passes) come earlier in this order, so the claimed items never wait on
    // unclaimed ones.
    std::vector<std::vector<int>> waves;
    uint64_t in_wave = 0;
    for (int c : large) {
        const uint64_t bytes = (1ull << circ[c].n) * sizeof(typename P::S);
        if (waves.empty() || in_wave + bytes > kWaveBytes) {
            waves.emplace_back();
            in_wave = 0;
        }
        waves.back().push_back(c);
        in_wave += bytes;
    }
    const size_t gaps = waves.size() * (size_t)P_;
    size_t si = 0, gap = 0;
    for (const auto& w : waves)
        for (int p = 0; p < P_; ++p) {
            for (int c : w) push_pass(c, p);
            const size_t upto = small.size() * (++gap) / gaps;
            for (; si < upto; ++si) push_small(small[si]);
        }
    for (; si < small.size(); ++si) push_small(small[si]);
    b->nitems = (int)items.size();
    // device buffers
    const size_t need_states = state_off * sizeof(typename P::S);
    if (b->state_bytes < need_states) {
        if (b->states) cudaFree(b->states);
        b->states = nullptr;
        QE_CUDA(cudaMalloc(&b->states, std::max<size_t>(need_states, 256)));
        b->state_bytes = need_states;
    }
    if (b->items) cudaFree(b->items);
    if (b->circ) cudaFree(b->circ);
    if (b->partials) cudaFree(b->partials);
    b->items = b->circ = nullptr;
    b->partials = nullptr;
    QE_CUDA(cudaMalloc(&b->items, items.size() * sizeof(Item)));
    QE_CUDA(cudaMemcpy(b->items, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice));
    QE_CUDA(cudaMalloc(&b->circ, circ.size() * sizeof(Circ)));
    QE_CUDA(cudaMemcpy(b->circ, circ.data(), circ.size() * sizeof(Circ), cudaMemcpyHostToDevice));
    QE_CUDA(cudaMalloc(&b->partials, std::max(1, slots) * sizeof(double2)));
    // algorithmic HBM bytes of one run: the first pass of a large circuit only
    // writes its state, the energy pass only reads it, the others do both:
    // 1 + 2 (P - 2) + 1 = 2 (P - 1) state sizes
    double bytes = 0.0;
    for (int c : large) bytes += 2.0 * (P_ - 1) * (double)((1ull << circ[c].n) * sizeof(typename P::S));
    b->hbm_bytes = bytes;
}

template <class P>
void capture(qe_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    static thread_local BatchArgs<P> a;
    a.states = reinterpret_cast<typename P::S*>(b->states);
    a.U = reinterpret_cast<const typename P::M*>(b->U);
    a.items = reinterpret_cast<const Item*>(b->items);
    a.circ = reinterpret_cast<const Circ*>(b->circ);
    a.nitems = b->nitems;
    a.T = b->plan.T;
    a.layers = b->layers;
    a.hx = b->hx;
    a.head = b->sync;
    a.status = b->sync + 1;
    a.counters = b->sync + 2;
    a.partials = b->partials;
    a.energies = b->energies;
    a.spin_limit = 1ll << 24;   // ~4 s of 256 ns sleeps
    // gates per register group, measured best on GB300: 2 (double-float), 4 (FP32)
    a.gmax = sizeof(typename P::V) >= 16 ? 2 : 4;
    const size_t smem = (sizeof(typename P::V) << b->plan.T) + (sizeof(typename P::V) << b->plan.T) / 16;
    auto fn = k_batch<P>;
    QE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    QE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, b->plan.threads, smem));
    if (occ < 1) fail(QE_ERR_UNSUPPORTED, "batch tile does not fit on an SM");
    const unsigned grid = (unsigned)std::min<long long>((long long)num_sms() * occ, b->nitems);
    cudaStream_t cs;
    QE_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    QE_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(b->sync, 0, (2 + b->count) * sizeof(unsigned), cs);
    fn<<<grid, b->plan.threads, smem, cs>>>(a);
    cudaMemcpyAsync(b->host_energies, b->energies, b->count * sizeof(double), cudaMemcpyDeviceToHost, cs);
    cudaMemcpyAsync(b->host_status, b->sync + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, cs);
    cudaError_t e = cudaStreamEndCapture(cs, &b->graph);
    cudaStreamDestroy(cs);
    QE_CUDA(e);
    QE_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
}

void prepare(qe_batch* b) {
    if (b->dtype == QE_C64) {
        build_plan<F32>(b);
        capture<F32>(b);
    } else if (b->arith == QE_ARITH_FP64) {
        build_plan<F64>(b);
        capture<F64>(b);
    } else {
        build_plan<DF>(b);
        capture<DF>(b);
    }
}

}  // namespace

void batch_create(qe_batch* b) {
    QE_CUDA(cudaMalloc(&b->sync, (2 + b->count) * sizeof(unsigned)));
    QE_CUDA(cudaMalloc(&b->energies, b->count * sizeof(double)));
    QE_CUDA(cudaMallocHost(&b->host_energies, b->count * sizeof(double)));
    QE_CUDA(cudaMallocHost(&b->host_status, sizeof(unsigned)));
    prepare(b);
}

void batch_run(qe_batch* b, double* out) {
    *b->host_status = 0;
    QE_CUDA(cudaGraphLaunch(b->exec, b->stream));
    QE_CUDA(cudaStreamSynchronize(b->stream));
    b->launches += 1;
    if (*b->host_status != 0) fail(QE_ERR_TIMEOUT, "a batch work item waited too long for its dependencies");
    if (out) std::copy(b->host_energies, b->host_energies + b->count, out);
}

void batch_set_arith(qe_batch* b, int arith) {
    b->arith = arith;
    prepare(b);
}

void batch_set_plan(qe_batch* b, int T, int tiles_per_item, int threads) {
    const int maxT = b->dtype == QE_C64 ? 13 : 12;
    int nmax = 0;
    for (int v : b->n) nmax = std::max(nmax, v);
    if (T < 4 || T > maxT || 2 * T - 1 < nmax) fail(QE_ERR_ARG, "tile bits out of range for this batch");
    if (tiles_per_item < 1 || (threads != 128 && threads != 256 && threads != 512)) fail(QE_ERR_ARG, "bad plan");
    b->plan.T = T;
    b->plan.tiles_per_item = tiles_per_item;
    b->plan.threads = threads;
    prepare(b);
}

void batch_destroy(qe_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void* p : {b->states, b->U, b->items, b->circ, (void*)b->sync, (void*)b->partials, (void*)b->energies})
        if (p) cudaFree(p);
    if (b->host_energies) cudaFreeHost(b->host_energies);
    if (b->host_status) cudaFreeHost(b->host_status);
}

}  // namespace qe
