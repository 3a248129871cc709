// Emulated multiplication and division (Sec. III-A): instead of simulating
// the Toffoli network of a reversible multiplier or divider, the emulator
// evaluates the classical function on every basis state and moves each
// amplitude to its image.  Three registers a, b, c of N qubits (bit j of a
// value <-> qa[j], qb[j], qc[j]):
//   multiplication  c -> (c + a b) mod 2^N      (the paper's (a, b, 0) -> (a, b, ab)),
//   division        the restoring division: for i = N-1 .. 0,
//                   c_i ^= [b != 0 and a >= b 2^i], then a -= b 2^i if c_i = 1
//                   (the paper's (a, b, 0) -> (a mod b, b, a / b)).
// Both maps are permutations of the basis states; amplitudes are moved bit
// for bit, no arithmetic touches them.
//
// Each map is closed on "planes": the multiplication permutes the 2^N values
// of c for fixed a, b and the other qubits; the division permutes the 2^(2N)
// values of (a, c) for fixed b and the other qubits.  A plane that fits one
// CTA's shared memory is loaded, then every output slot is written from the
// slot of its preimage (one read and one write of every amplitude).  Larger
// planes go through a scratch buffer in batches: a gather of the preimages
// into the buffer, then a copy back.
#include <algorithm>
#include <cstring>

#include "qe_arith.cuh"
#include "qe_internal.h"

namespace qe {

namespace {

constexpr int kArithThreads = 512;

struct RegArg {
    int lo;            // qubit of bit 0
    int contiguous;    // qubits lo .. lo + N - 1 in order
    uint8_t q[16];
};

__device__ __forceinline__ uint32_t reg_get(const RegArg& r, int N, uint64_t x) {
    if (r.contiguous) return (uint32_t)(x >> r.lo) & ((1u << N) - 1u);
    uint32_t v = 0;
    for (int j = 0; j < N; ++j) v |= (uint32_t)((x >> r.q[j]) & 1u) << j;
    return v;
}
__device__ __forceinline__ uint64_t reg_put(const RegArg& r, int N, uint32_t v) {
    if (r.contiguous) return (uint64_t)v << r.lo;
    uint64_t x = 0;
    for (int j = 0; j < N; ++j) x |= (uint64_t)((v >> j) & 1u) << r.q[j];
    return x;
}

enum { kMul = 0, kDiv = 1 };

template <class S>
struct ArithArgs {
    S* x;
    S* scratch;
    uint64_t plane0, nplanes;   // planes [plane0, plane0 + nplanes) of this launch
    int N, P, op;               // register width, plane bits (N or 2N), operation
    RegArg a, b, c;
    int nsorted;
    uint8_t plane_sorted[32];   // the plane's qubits ascending (to enumerate plane bases)
};

// Offset of plane-local value y: the c register holds its low N bits, and for
// the division the a register its high N bits.
template <class S>
__device__ __forceinline__ uint64_t plane_offset(const ArithArgs<S>& a, uint32_t y) {
    const uint32_t mask = (1u << a.N) - 1u;
    if (a.op == kMul) return reg_put(a.c, a.N, y);
    return reg_put(a.c, a.N, y & mask) | reg_put(a.a, a.N, y >> a.N);
}

// Plane-local value of the preimage of output y, in the plane whose other
// qubits are those of base (the inverse map).
template <class S>
__device__ __forceinline__ uint32_t preimage(const ArithArgs<S>& a, uint64_t base, uint32_t y) {
    const uint32_t mask = (1u << a.N) - 1u;
    const uint32_t bv = reg_get(a.b, a.N, base);
    if (a.op == kMul) {
        const uint32_t av = reg_get(a.a, a.N, base);
        return (y - av * bv) & mask;        // c - a b mod 2^N (products wrap mod 2^32 alike)
    }
    // the restoring steps undone in reverse order (i = 0 .. N-1): if c_i,
    // a += b 2^i; then c_i ^= [b != 0 and a >= b 2^i]
    uint32_t cv = y & mask;
    uint64_t av = y >> a.N;
    for (int i = 0; i < a.N; ++i) {
        const uint64_t bi = (uint64_t)bv << i;
        if ((cv >> i) & 1u) av = (av + bi) & mask;
        const uint32_t t = (bv != 0u && av >= bi) ? 1u : 0u;
        cv ^= t << i;
    }
    return cv | ((uint32_t)av << a.N);
}

// Whole planes in shared memory: one read and one write per amplitude.
template <class S>
__global__ void __launch_bounds__(kArithThreads) k_arith_plane(const __grid_constant__ ArithArgs<S> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* buf = reinterpret_cast<S*>(smem_raw);
    const uint32_t E = 1u << a.P;
    for (uint64_t p = blockIdx.x; p < a.nplanes; p += gridDim.x) {
        const uint64_t base = insert_zero_bits(a.plane0 + p, a.plane_sorted, a.nsorted);
        for (uint32_t i = threadIdx.x; i < E; i += blockDim.x) buf[i] = a.x[base | plane_offset(a, i)];
        __syncthreads();
        for (uint32_t y = threadIdx.x; y < E; y += blockDim.x)
            a.x[base | plane_offset(a, y)] = buf[preimage(a, base, y)];
        __syncthreads();
    }
}

// Larger planes, a batch at a time: gather the preimages into scratch ...
template <class S>
__global__ void __launch_bounds__(256) k_arith_gather(const __grid_constant__ ArithArgs<S> a) {
    const uint64_t total = a.nplanes << a.P;
    const uint32_t emask = (1u << a.P) - 1u;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t base = insert_zero_bits(a.plane0 + (e >> a.P), a.plane_sorted, a.nsorted);
        const uint32_t y = (uint32_t)e & emask;
        a.scratch[e] = a.x[base | plane_offset(a, preimage(a, base, y))];
    }
}

// ... then copy the batch back to its planes.
template <class S>
__global__ void __launch_bounds__(256) k_arith_copy_back(const __grid_constant__ ArithArgs<S> a) {
    const uint64_t total = a.nplanes << a.P;
    const uint32_t emask = (1u << a.P) - 1u;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t base = insert_zero_bits(a.plane0 + (e >> a.P), a.plane_sorted, a.nsorted);
        a.x[base | plane_offset(a, (uint32_t)e & emask)] = a.scratch[e];
    }
}

RegArg make_reg(int N, const int* q) {
    RegArg r{};
    r.lo = q[0];
    r.contiguous = 1;
    for (int j = 0; j < N; ++j) {
        r.q[j] = (uint8_t)q[j];
        if (q[j] != q[0] + j) r.contiguous = 0;
    }
    return r;
}

template <class S>
void arith_impl(qe_state* s, int op, int N, const int* qa, const int* qb, const int* qc) {
    static thread_local ArithArgs<S> a;
    std::memset(&a, 0, sizeof(a));
    a.x = reinterpret_cast<S*>(s->d);
    a.N = N;
    a.op = op;
    a.P = op == kMul ? N : 2 * N;
    a.a = make_reg(N, qa);
    a.b = make_reg(N, qb);
    a.c = make_reg(N, qc);
    int pq[32], np = 0;
    for (int j = 0; j < N; ++j) pq[np++] = qc[j];
    if (op == kDiv)
        for (int j = 0; j < N; ++j) pq[np++] = qa[j];
    std::sort(pq, pq + np);
    a.nsorted = np;
    for (int j = 0; j < np; ++j) a.plane_sorted[j] = (uint8_t)pq[j];
    const uint64_t planes = 1ull << (s->n - a.P);
    const size_t plane_bytes = sizeof(S) << a.P;
    const char* tag = op == kMul ? "mul_emulated" : "div_emulated";
    if (plane_bytes <= 64 * 1024) {
        a.plane0 = 0;
        a.nplanes = planes;
        const size_t smem = plane_bytes;
        auto fn = k_arith_plane<S>;
        QE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int occ = 0;
        QE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kArithThreads, smem));
        const uint64_t grid = std::min<uint64_t>(planes, (uint64_t)num_sms() * std::max(occ, 1));
        Launch L(s, tag, 2.0 * dim(s) * amp_bytes(s));
        fn<<<(unsigned)grid, kArithThreads, smem, s->stream>>>(a);
        QE_CUDA(cudaGetLastError());
        return;
    }
    // batches of whole planes through a scratch buffer of at most 1 GiB
    const uint64_t per_batch = std::max<uint64_t>(1, std::min<uint64_t>(planes, (1ull << 30) / plane_bytes));
    a.scratch = reinterpret_cast<S*>(ensure_scratch(s, per_batch * plane_bytes));
    for (uint64_t p0 = 0; p0 < planes; p0 += per_batch) {
        a.plane0 = p0;
        a.nplanes = std::min<uint64_t>(per_batch, planes - p0);
        const uint64_t total = a.nplanes << a.P;
        const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, (uint64_t)num_sms() * 16);
        {
            Launch L(s, tag, 2.0 * (double)total * amp_bytes(s), false);
            k_arith_gather<S><<<grid, 256, 0, s->stream>>>(a);
            QE_CUDA(cudaGetLastError());
        }
        {
            Launch L(s, "arith_copy_back", 2.0 * (double)total * amp_bytes(s), false);
            k_arith_copy_back<S><<<grid, 256, 0, s->stream>>>(a);
            QE_CUDA(cudaGetLastError());
        }
    }
    s->stats.passes += 2;   // two full passes in total over the batches
}

}  // namespace

void launch_mul(qe_state* s, int N, const int* qa, const int* qb, const int* qc) {
    if (s->dtype == QE_C128) arith_impl<double2>(s, kMul, N, qa, qb, qc);
    else arith_impl<float2>(s, kMul, N, qa, qb, qc);
}

void launch_div(qe_state* s, int N, const int* qa, const int* qb, const int* qc) {
    if (s->dtype == QE_C128) arith_impl<double2>(s, kDiv, N, qa, qb, qc);
    else arith_impl<float2>(s, kDiv, N, qa, qb, qc);
}

}  // namespace qe
