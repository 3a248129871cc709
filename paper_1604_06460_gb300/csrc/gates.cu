// Gate kernels (Sec. II): a sparse 2^n x 2^n gate acts as a small dense
// matrix on every group of 2^k amplitudes that agree outside its qubits.
//
// Dense gates run through shared-memory tiles: a tile is 2^T amplitudes made
// of 2^kh contiguous chunks of 2^L amplitudes (L >= 5, so each chunk is at
// least 256 contiguous bytes), one chunk per combination of the gate qubits
// at or above L.  Gate qubits below L fall inside each chunk.  Each tile is
// read once and written once, so a pass moves 2 * 2^n * bytes_per_amplitude.
//
// Structured gates (Sec. II: skip multiplications by ones and zeros) only
// touch the amplitudes they change: controlled gates the 2^-nc fraction
// whose controls are set, a single-entry diagonal (e.g. CR(theta),
// Sec. III-B) one amplitude per group, permutations move bits exactly.
#include <algorithm>
#include <vector>

#include "qe_arith.cuh"
#include "qe_internal.h"

namespace qe {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxFixed = 40;

struct Geom {
    int T = 0, L = 0, kh = 0;
    uint8_t hq[8] = {0};
};

// Choose the chunk size L and the high gate qubits of a tile of 2^T amplitudes.
Geom make_geom(int n, int k, const int* qubits, int T_target) {
    int sorted[8];
    for (int j = 0; j < k; ++j) sorted[j] = qubits[j];
    std::sort(sorted, sorted + k);
    int Tt = std::min(T_target, n);
    Geom g;
    for (int L = Tt; L >= 0; --L) {
        int kh = 0;
        for (int j = 0; j < k; ++j) kh += sorted[j] >= L;
        if (L + kh <= Tt) {
            g.L = L;
            g.kh = kh;
            g.T = L + kh;
            int h = 0;
            for (int j = 0; j < k; ++j)
                if (sorted[j] >= L) g.hq[h++] = (uint8_t)sorted[j];
            return g;
        }
    }
    fail(QE_ERR_ARG, "no tile geometry");
}

// Tile-local bit position of global qubit q.
int local_pos(const Geom& g, int q) {
    if (q < g.L) return q;
    for (int j = 0; j < g.kh; ++j)
        if (g.hq[j] == q) return g.L + j;
    fail(QE_ERR_ARG, "qubit not in tile");
}

template <class P>
typename P::M to_m(cd v) { return P::mat(v.real(), v.imag()); }

unsigned persistent_grid(const void* fn, int threads, size_t smem, uint64_t work) {
    int occ = 0;
    QE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem));
    if (occ < 1) occ = 1;
    uint64_t cap = (uint64_t)num_sms() * occ;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(work, cap));
}

// --------------------------------------------------------------- dense
template <class P, int K>
struct DenseArgs {
    typename P::S* x;
    uint64_t ntiles;
    int L, T, kh;
    uint8_t hq[8];
    uint8_t pos[8];
    typename P::M U[(1 << K) * (1 << K)];
};

template <class P, int K>
__global__ void __launch_bounds__(kThreads) k_gate_dense(const __grid_constant__ DenseArgs<P, K> a) {
    constexpr int D = 1 << K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename P::M* Us = reinterpret_cast<typename P::M*>(smem_raw);
    typename P::V* tile = reinterpret_cast<typename P::V*>(Us + D * D);
    __shared__ uint64_t hoff[32];
    __shared__ uint32_t dep[D];
    const int tid = threadIdx.x;
    // column-major copy: lanes of a warp that need different rows r of the
    // same column c read consecutive words (no bank conflicts)
    for (int i = tid; i < D * D; i += blockDim.x) Us[(i % D) * D + i / D] = a.U[i];
    if (tid < (1 << a.kh)) {
        uint64_t o = 0;
        for (int j = 0; j < a.kh; ++j)
            if ((tid >> j) & 1) o |= 1ull << a.hq[j];
        hoff[tid] = o;
    }
    if (tid < D) {
        uint32_t o = 0;
        for (int j = 0; j < K; ++j)
            if ((tid >> j) & 1) o |= 1u << a.pos[j];
        dep[tid] = o;
    }
    __syncthreads();
    const uint32_t gmask = dep[D - 1];
    const int Tn = 1 << a.T;
    const uint32_t lowmask = (1u << a.L) - 1u;
    for (uint64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const uint64_t base = insert_zero_bits(t << a.L, a.hq, a.kh);
        for (int i = tid; i < Tn; i += blockDim.x)
            tile[i] = P::load(a.x[base + (i & lowmask) + hoff[i >> a.L]]);
        __syncthreads();
        for (int i = tid; i < Tn; i += blockDim.x) {
            uint32_t r = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) r |= (((uint32_t)i >> a.pos[j]) & 1u) << j;
            const uint32_t b = (uint32_t)i & ~gmask;
            typename P::A acc;
            P::mac_first(acc, Us[r], tile[b]);
#pragma unroll
            for (int c = 1; c < D; ++c) P::mac(acc, Us[c * D + r], tile[b | dep[c]]);
            a.x[base + (i & lowmask) + hoff[i >> a.L]] = P::out(acc);
        }
        __syncthreads();
    }
}

template <class P, int K>
void dense_impl(qe_state* s, const int* qubits, const cd* U) {
    constexpr int D = 1 << K;
    // the argument block lives in constant parameter space; keep it off the stack
    static thread_local DenseArgs<P, K> a;
    Geom g = make_geom(s->n, K, qubits, 10);
    a.x = reinterpret_cast<typename P::S*>(s->d);
    a.ntiles = 1ull << (s->n - g.T);
    a.L = g.L;
    a.T = g.T;
    a.kh = g.kh;
    for (int j = 0; j < 8; ++j) a.hq[j] = g.hq[j];
    for (int j = 0; j < K; ++j) a.pos[j] = (uint8_t)local_pos(g, qubits[j]);
    for (int i = 0; i < D * D; ++i) a.U[i] = to_m<P>(U[i]);
    size_t smem = sizeof(typename P::M) * D * D + sizeof(typename P::V) * ((size_t)1 << g.T);
    auto fn = k_gate_dense<P, K>;
    QE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    unsigned grid = persistent_grid((const void*)fn, kThreads, smem, a.ntiles);
    static const char* names[] = {"", "gate_dense_k1", "gate_dense_k2", "gate_dense_k3",
                                  "gate_dense_k4", "gate_dense_k5"};
    Launch L(s, names[K], 2.0 * dim(s) * amp_bytes(s));
    fn<<<grid, kThreads, smem, s->stream>>>(a);
    QE_CUDA(cudaGetLastError());
}

template <class P, int K>
void direct_impl(qe_state* s, const int* qubits, const cd* U);

template <class P>
void dense_k(qe_state* s, int k, const int* qubits, const cd* U) {
    // 1..3 qubits: direct kernel (dense_tile forces the shared-memory tile path)
    const bool tile = s->force_tile;
    switch (k) {
        case 1: tile ? dense_impl<P, 1>(s, qubits, U) : direct_impl<P, 1>(s, qubits, U); break;
        case 2: tile ? dense_impl<P, 2>(s, qubits, U) : direct_impl<P, 2>(s, qubits, U); break;
        case 3: tile ? dense_impl<P, 3>(s, qubits, U) : direct_impl<P, 3>(s, qubits, U); break;
        case 4: dense_impl<P, 4>(s, qubits, U); break;
        case 5: dense_impl<P, 5>(s, qubits, U); break;
        default: fail(QE_ERR_ARG, "dense gate needs 1 <= k <= 5");
    }
}

// --------------------------------------------------------------- direct
// Small dense gates (k <= 3) without shared memory: each thread owns whole
// groups of 2^k amplitudes, loads them straight from global memory and
// multiplies by the matrix held in the kernel parameters (a uniform,
// broadcast constant-bank operand).  Consecutive threads own groups that are
// consecutive in the non-gate index bits, so every load and store instruction
// of a warp covers contiguous sectors.  G groups per iteration keep 2^k * G
// independent loads in flight per thread.
template <class P, int K>
struct DirectArgs {
    typename P::S* x;
    uint64_t ngroups;
    uint8_t sorted[8];
    uint64_t dep[1 << K];
    typename P::M U[(1 << K) * (1 << K)];
};

template <class P, int K, int G>
__global__ void __launch_bounds__(kThreads) k_gate_direct(const __grid_constant__ DirectArgs<P, K> a) {
    constexpr int D = 1 << K;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g0 < a.ngroups; g0 += stride * G) {
        uint64_t base[G];
        typename P::V v[G][D];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const uint64_t g = g0 + j * stride;
            base[j] = insert_zero_bits(g < a.ngroups ? g : 0, a.sorted, K);
#pragma unroll
            for (int c = 0; c < D; ++c)
                if (g < a.ngroups) v[j][c] = P::load(a.x[base[j] + a.dep[c]]);
        }
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (g0 + j * stride >= a.ngroups) break;
#pragma unroll
            for (int r = 0; r < D; ++r) {
                typename P::A acc;
                P::mac_first(acc, a.U[r * D], v[j][0]);
#pragma unroll
                for (int c = 1; c < D; ++c) P::mac(acc, a.U[r * D + c], v[j][c]);
                a.x[base[j] + a.dep[r]] = P::out(acc);
            }
        }
    }
}

template <class P, int K>
void direct_impl(qe_state* s, const int* qubits, const cd* U) {
    constexpr int D = 1 << K;
    static thread_local DirectArgs<P, K> a;
    a.x = reinterpret_cast<typename P::S*>(s->d);
    a.ngroups = dim(s) >> K;
    int srt[8];
    for (int j = 0; j < K; ++j) srt[j] = qubits[j];
    std::sort(srt, srt + K);
    for (int j = 0; j < K; ++j) a.sorted[j] = (uint8_t)srt[j];
    for (int c = 0; c < D; ++c) {
        uint64_t o = 0;
        for (int j = 0; j < K; ++j)
            if ((c >> j) & 1) o |= 1ull << qubits[j];
        a.dep[c] = o;
    }
    for (int i = 0; i < D * D; ++i) a.U[i] = to_m<P>(U[i]);
    constexpr int G = (K <= 2 && sizeof(typename P::V) < 16) ? 2 : 1;
    auto fn = k_gate_direct<P, K, G>;
    unsigned grid = persistent_grid((const void*)fn, kThreads, 0, (a.ngroups + kThreads * G - 1) / (kThreads * G));
    static const char* names[] = {"", "gate_direct_k1", "gate_direct_k2", "gate_direct_k3"};
    Launch L(s, names[K], 2.0 * dim(s) * amp_bytes(s));
    fn<<<grid, kThreads, 0, s->stream>>>(a);
    QE_CUDA(cudaGetLastError());
}

// --------------------------------------------------------------- diagonal
template <class P>
struct DiagArgs {
    typename P::S* x;
    uint64_t count;
    int k;
    uint8_t q[8];
    typename P::M d[32];
};

template <class P>
__global__ void __launch_bounds__(kThreads) k_gate_diag(const __grid_constant__ DiagArgs<P> a) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t r = 0;
        for (int j = 0; j < a.k; ++j) r |= (uint32_t)((i >> a.q[j]) & 1u) << j;
        typename P::A acc;
        P::mac_first(acc, a.d[r], P::load(a.x[i]));
        a.x[i] = P::out(acc);
    }
}

// --------------------------------------------- controlled / phase / permute
// Shared indexing: thread item t enumerates the bases x = insert zeros at
// fixed[] (sorted) | cmask; group element c is x | dep(c) over the targets.
template <class P>
struct CtrlArgs {
    typename P::S* x;
    uint64_t count;      // number of groups
    uint64_t cmask;      // value ORed into every base
    int nfixed;
    uint8_t fixed[kMaxFixed];
    int k;               // targets
    uint64_t tdep[4];    // offsets of the 2^k group members
    int perm[4];         // permute: out[r] = in[perm[r]]
    typename P::M U[16]; // controlled: 2^k x 2^k matrix
};

template <class P>
__global__ void __launch_bounds__(kThreads) k_controlled(const __grid_constant__ CtrlArgs<P> a) {
    const int D = 1 << a.k;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < a.count;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t base = insert_zero_bits(t, a.fixed, a.nfixed) | a.cmask;
        typename P::V v[4];
        for (int c = 0; c < D; ++c) v[c] = P::load(a.x[base + a.tdep[c]]);
        for (int r = 0; r < D; ++r) {
            typename P::A acc;
            P::mac_first(acc, a.U[r * D], v[0]);
            for (int c = 1; c < D; ++c) P::mac(acc, a.U[r * D + c], v[c]);
            a.x[base + a.tdep[r]] = P::out(acc);
        }
    }
}

template <class P>
__global__ void __launch_bounds__(kThreads) k_permute(const __grid_constant__ CtrlArgs<P> a) {
    const int D = 1 << a.k;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < a.count;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t base = insert_zero_bits(t, a.fixed, a.nfixed) | a.cmask;
        typename P::S v[4];
        for (int c = 0; c < D; ++c) v[c] = a.x[base + a.tdep[c]];
        for (int r = 0; r < D; ++r)
            if (a.perm[r] != r) a.x[base + a.tdep[r]] = v[a.perm[r]];
    }
}

unsigned flat_grid(uint64_t count) {
    uint64_t want = (count + kThreads - 1) / kThreads;
    uint64_t cap = (uint64_t)num_sms() * 8;
    return (unsigned)std::max<uint64_t>(1, std::min(want, cap));
}

template <class P>
void fill_ctrl(CtrlArgs<P>& a, qe_state* s, uint64_t cmask, uint64_t zmask, int k, const int* targets) {
    a.x = reinterpret_cast<typename P::S*>(s->d);
    a.cmask = cmask;
    uint64_t fixed = cmask | zmask;
    for (int j = 0; j < k; ++j) fixed |= 1ull << targets[j];
    int nf = 0;
    for (int q = 0; q < s->n; ++q)
        if ((fixed >> q) & 1) {
            if (nf >= kMaxFixed) fail(QE_ERR_ARG, "too many fixed qubits");
            a.fixed[nf++] = (uint8_t)q;
        }
    a.nfixed = nf;
    a.count = 1ull << (s->n - nf);
    a.k = k;
    for (int c = 0; c < (1 << k); ++c) {
        uint64_t o = 0;
        for (int j = 0; j < k; ++j)
            if ((c >> j) & 1) o |= 1ull << targets[j];
        a.tdep[c] = o;
    }
}

template <class P>
void controlled_impl(qe_state* s, uint64_t cmask, uint64_t zmask, int k, const int* targets,
                     const cd* U) {
    static thread_local CtrlArgs<P> a;
    fill_ctrl(a, s, cmask, zmask, k, targets);
    const int D = 1 << k;
    for (int i = 0; i < D * D; ++i) a.U[i] = to_m<P>(U[i]);
    Launch L(s, k == 0 ? "gate_phase" : "gate_controlled", 2.0 * (double)a.count * D * amp_bytes(s));
    k_controlled<P><<<flat_grid(a.count), kThreads, 0, s->stream>>>(a);
    QE_CUDA(cudaGetLastError());
}

template <class P>
void permute_impl(qe_state* s, uint64_t cmask, int k, const int* targets, const int* perm) {
    static thread_local CtrlArgs<P> a;
    fill_ctrl(a, s, cmask, 0, k, targets);
    const int D = 1 << k;
    int moved = 0;
    for (int r = 0; r < D; ++r) {
        a.perm[r] = perm[r];
        moved += perm[r] != r;
    }
    Launch L(s, "gate_permute", 2.0 * (double)a.count * moved * amp_bytes(s));
    k_permute<P><<<flat_grid(a.count), kThreads, 0, s->stream>>>(a);
    QE_CUDA(cudaGetLastError());
}

template <class P>
void diag_impl(qe_state* s, int k, const int* qubits, const cd* d) {
    static thread_local DiagArgs<P> a;
    a.x = reinterpret_cast<typename P::S*>(s->d);
    a.count = dim(s);
    a.k = k;
    for (int j = 0; j < k; ++j) a.q[j] = (uint8_t)qubits[j];
    for (int r = 0; r < (1 << k); ++r) a.d[r] = to_m<P>(d[r]);
    Launch L(s, "gate_diag", 2.0 * dim(s) * amp_bytes(s));
    k_gate_diag<P><<<flat_grid(a.count), kThreads, 0, s->stream>>>(a);
    QE_CUDA(cudaGetLastError());
}

}  // namespace

#define QE_DISPATCH(s, FN, ...)                                  \
    do {                                                         \
        if ((s)->dtype == QE_C64) FN<F32>(__VA_ARGS__);          \
        else if ((s)->arith == QE_ARITH_FP64) FN<F64>(__VA_ARGS__); \
        else FN<DF>(__VA_ARGS__);                                \
    } while (0)

void launch_gate_dense(qe_state* s, int k, const int* qubits, const cd* U) {
    const bool tc64 = s->dtype == QE_C64;
    const bool tc128 = s->dtype == QE_C128 && s->c128_tc;
    // complex64 blocks of 4-5 qubits and complex128 blocks of 3-5 qubits
    // run on the tensor cores (3-qubit blocks are ALU-bound in double-float
    // and in native FP64 arithmetic)
    const int kmin = tc64 ? 4 : c128_tc_kmin(s);
    if ((tc64 || tc128) && s->tensor_cores && !s->force_tile && s->n >= 12 && k >= kmin) {
        auto run = [&](const int* q5, const cd* U5) {
            if (tc64) launch_gate_tc5(s, q5, U5);
            else launch_gate_tc5_c128(s, q5, U5);
        };
        if (k == 5) {
            run(qubits, U);
            return;
        }
        // widen the block by 5 - k idle qubits (the lowest ones not in the
        // block): U5 = 1 (x) U, the idle qubits as the high matrix bits
        int q5[5];
        for (int j = 0; j < k; ++j) q5[j] = qubits[j];
        int w = k;
        for (int c = 0; c < s->n && w < 5; ++c) {
            bool used = false;
            for (int j = 0; j < k; ++j) used |= qubits[j] == c;
            if (!used) q5[w++] = c;
        }
        const int d = 1 << k;
        std::vector<cd> U5(32 * 32, cd(0.0));
        for (int hb = 0; hb < (32 >> k); ++hb)
            for (int r = 0; r < d; ++r)
                for (int c = 0; c < d; ++c) U5[(r | (hb << k)) * 32 + (c | (hb << k))] = U[r * d + c];
        run(q5, U5.data());
        return;
    }
    QE_DISPATCH(s, dense_k, s, k, qubits, U);
}

void launch_gate_diag(qe_state* s, int k, const int* qubits, const cd* d) {
    QE_DISPATCH(s, diag_impl, s, k, qubits, d);
}

void launch_phase_pattern(qe_state* s, uint64_t mask, uint64_t value, cd phase) {
    // the amplitudes with (x & mask) == value: the one-bits of the pattern
    // act as controls, its zero-bits are pinned to 0, no target remains
    QE_DISPATCH(s, controlled_impl, s, value & mask, mask & ~value, 0, (const int*)nullptr, &phase);
}

void launch_controlled(qe_state* s, uint64_t cmask, int k, const int* targets, const cd* U) {
    if (k < 0 || k > 2) fail(QE_ERR_ARG, "controlled gate needs 0 <= k <= 2 targets");
    QE_DISPATCH(s, controlled_impl, s, cmask, (uint64_t)0, k, targets, U);
}

void launch_permute(qe_state* s, uint64_t cmask, int k, const int* targets, const int* perm) {
    if (k < 1 || k > 2) fail(QE_ERR_ARG, "permutation needs 1 <= k <= 2 targets");
    QE_DISPATCH(s, permute_impl, s, cmask, k, targets, perm);
}

}  // namespace qe
