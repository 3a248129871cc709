// Fused 5-qubit gates on complex64 states with the 5th-generation tensor
// cores (tcgen05.mma, accumulators in tensor memory).
//
// A 5-qubit block U (32x32 complex) acts on each group of 32 amplitudes.  In
// real arithmetic a group is a 64-vector v = [Re x ; Im x] and the block is
// W = [[Re U, -Im U], [Im U, Re U]] (64x64), so a tile of 128 groups is one
// real matrix product  Out(128x64) = In(128x64) * W^T.  FP32 inputs are split
// into TF32 high and low parts (x = hi + lo, hi = x rounded to 10 mantissa
// bits, lo = x - hi); the product keeps the three significant terms
//   In_hi W_hi + In_hi W_lo + In_lo W_hi
// accumulated in FP32 (the dropped lo*lo term is ~2^-22 relative).
//
// Per tile (128 groups = 4096 amplitudes, 12 tile-local index bits: the 5
// gate qubits and 7 others, chunks of >= 2^L contiguous amplitudes):
//   1. thread t loads 4 column quads of group row t % 128 (a warp reads 32
//      consecutive rows), splits each value and stores In_hi / In_lo as
//      16-byte chunks of the K-major 128-byte-swizzled operand layout (no
//      bank conflicts: 8 consecutive rows hit 8 different chunks);
//   2. one thread issues 24 tcgen05.mma (M=128, N=64, K=8, kind::tf32) into a
//      64-column tensor-memory accumulator and commits them to an mbarrier;
//   3. all threads wait on the mbarrier (bounded), read the accumulator with
//      tcgen05.ld and store the outputs straight from registers (TMEM lane =
//      group row, so a warp's stores cover consecutive rows).
// W_hi / W_lo (64x64 each) are loaded once per CTA.  Waits that exceed their
// limit set a status word and end the kernel after freeing tensor memory.
#include <algorithm>
#include <cstring>

#include "qe_arith.cuh"
#include "qe_internal.h"
#include "qe_tc.cuh"

namespace qe {

namespace {

using tc::smem_u32;
using tc::mbar_wait;

constexpr int kTcThreads = 256;
constexpr int kRows = 128;           // groups per tile (MMA M)
constexpr int kK = 64;               // real K (32 complex)
constexpr int kN = 64;               // real N
constexpr uint32_t kTmemCols = 64;

struct TcArgs {
    float2* x;
    uint64_t ntiles;
    int L, kh;
    uint8_t hq[8];
    uint8_t gpos[5];          // tile-local bit positions of the matrix bits
    uint32_t* status;
    long long spin_limit;
    const float* W;           // [2][kN * kK]: hi, lo parts of W, row n, column k
};

// Round an FP32 value to TF32 (10 explicit mantissa bits, nearest, ties
// away from zero) with integer instructions.
__device__ __forceinline__ float tf32_hi(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Byte offset of element (row r, k) in a K-major, 128-byte-swizzled operand
// of `rows` rows and 64 K-elements of 4 bytes: two K atoms of 32 elements,
// each rows x 128 bytes; within an atom the 16-byte chunk index is XORed with
// the row index modulo 8.
__device__ __forceinline__ uint32_t sw128_offset(int r, int k, int rows) {
    const int atom = k >> 5, kk = k & 31;
    const uint32_t chunk = (uint32_t)((kk >> 2) ^ (r & 7));
    return (uint32_t)atom * (uint32_t)rows * 128u + (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u +
           chunk * 16u + (uint32_t)(kk & 3) * 4u;
}

constexpr uint32_t kIdesc = tc::idesc(2u, kN, kRows);   // tf32 x tf32 -> f32, M = 128, N = 64

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__global__ void __launch_bounds__(kTcThreads) k_gate_tc5(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned regions: A_hi, A_lo (128 x 64 x 4 B each), W_hi, W_lo (64 x 64 x 4 B)
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* sA_hi = base;
    unsigned char* sA_lo = sA_hi + kRows * kK * 4;
    unsigned char* sW_hi = sA_lo + kRows * kK * 4;
    unsigned char* sW_lo = sW_hi + kN * kK * 4;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ uint64_t hoff[32];
    __shared__ uint32_t cpos[32];
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // W into its swizzled operand layout
    for (int i = tid; i < kN * kK; i += blockDim.x) {
        const int n = i / kK, k = i % kK;
        *reinterpret_cast<float*>(sW_hi + sw128_offset(n, k, kN)) = a.W[i];
        *reinterpret_cast<float*>(sW_lo + sw128_offset(n, k, kN)) = a.W[kN * kK + i];
    }
    if (tid < (1 << a.kh)) {
        uint64_t o = 0;
        for (int j = 0; j < a.kh; ++j)
            if ((tid >> j) & 1) o |= 1ull << a.hq[j];
        hoff[tid] = o;
    }
    if (tid < 32) {
        uint32_t o = 0;
        for (int j = 0; j < 5; ++j)
            if ((tid >> j) & 1) o |= 1u << a.gpos[j];
        cpos[tid] = o;
    }
    if (tid == 0) {
        s_abort = 0;
        tc::mbar_init(&mbar);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t gmask = cpos[31];
    const uint32_t lowmask = (1u << a.L) - 1u;
    // Load side: lane <-> group row (rows r = tid % 128, consecutive across a
    // warp), each thread owns the column quads q = tid / 128 + 2 j, j < 4, so
    // it writes whole 16-byte chunks of the swizzled operand.
    const int lr = tid & (kRows - 1);
    const int qbase = tid >> 7;
    // Epilogue side: TMEM lane quarter of this warp, and which 16 columns of
    // the real (0..31) and imaginary (32..63) halves it reads
    const uint32_t equarter = (uint32_t)(warp & 3) * 32u;
    const uint32_t ehalf = (uint32_t)(warp >> 2) * 16u;
    const int er = (int)equarter + lane;
    auto rowbits = [&](int r) {
        uint32_t l = 0;
        int j = 0;
        for (int b = 0; b < 12; ++b)
            if (!((gmask >> b) & 1u)) l |= (((uint32_t)r >> (j++)) & 1u) << b;
        return l;
    };
    const uint32_t lrow_load = rowbits(lr);
    const uint32_t lrow_out = rowbits(er);
    auto goff = [&](uint32_t l) -> uint64_t { return (l & lowmask) + hoff[l >> a.L]; };
    float2 cur[16], nxt[16];
    auto load_tile = [&](uint64_t t, float2* dst) {
        const uint64_t gb = insert_zero_bits(t << a.L, a.hq, a.kh);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = 4 * (qbase + 2 * j) + u;
                dst[4 * j + u] = a.x[gb + goff(lrow_load | cpos[c])];
            }
    };
    uint32_t phase = 0;
    uint64_t t = blockIdx.x;
    if (t < a.ntiles) load_tile(t, cur);
    for (; t < a.ntiles; t += gridDim.x) {
        const uint64_t gbase = insert_zero_bits(t << a.L, a.hq, a.kh);
        // 1. split into TF32 hi/lo; 16-byte chunks of 4 consecutive K values
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = qbase + 2 * j;
            float4 rh, ih, rl, il;
            float* prh = &rh.x; float* pih = &ih.x; float* prl = &rl.x; float* pil = &il.x;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 v = cur[4 * j + u];
                prh[u] = tf32_hi(v.x);
                pih[u] = tf32_hi(v.y);
                prl[u] = __fsub_rn(v.x, prh[u]);
                pil[u] = __fsub_rn(v.y, pih[u]);
            }
            *reinterpret_cast<float4*>(sA_hi + sw128_offset(lr, 4 * q, kRows)) = rh;
            *reinterpret_cast<float4*>(sA_hi + sw128_offset(lr, 32 + 4 * q, kRows)) = ih;
            *reinterpret_cast<float4*>(sA_lo + sw128_offset(lr, 4 * q, kRows)) = rl;
            *reinterpret_cast<float4*>(sA_lo + sw128_offset(lr, 32 + 4 * q, kRows)) = il;
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        // 2. one thread issues the 24 MMAs and commits them to the mbarrier
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t ah = smem_u32(sA_hi), al = smem_u32(sA_lo);
            const uint32_t wh = smem_u32(sW_hi), wl = smem_u32(sW_lo);
            uint32_t acc = 0;
            for (int ks = 0; ks < kK / 8; ++ks) {
                const uint32_t aoff = (uint32_t)(ks >> 2) * kRows * 128u + (uint32_t)(ks & 3) * 32u;
                const uint32_t boff = (uint32_t)(ks >> 2) * kN * 128u + (uint32_t)(ks & 3) * 32u;
                mma_tf32(tmem, tc::sdesc_sw128(ah + aoff), tc::sdesc_sw128(wh + boff), acc);
                acc = 1;
                mma_tf32(tmem, tc::sdesc_sw128(ah + aoff), tc::sdesc_sw128(wl + boff), 1);
                mma_tf32(tmem, tc::sdesc_sw128(al + aoff), tc::sdesc_sw128(wh + boff), 1);
            }
            tc::mma_commit(&mbar);
        }
        // prefetch the next tile while the tensor cores work
        const uint64_t tn = t + gridDim.x;
        if (tn < a.ntiles) load_tile(tn, nxt);
        // 3. wait for the accumulator (bounded), then write the outputs
        //    straight from the tensor-memory registers
        if (!mbar_wait(smem_u32(&mbar), phase, a.spin_limit)) {
            atomicExch(a.status, 1u);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        uint32_t re[16], im[16];
        {
            const uint32_t taddr = tmem + (equarter << 16) + ehalf;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]), "=r"(re[6]),
                  "=r"(re[7]), "=r"(re[8]), "=r"(re[9]), "=r"(re[10]), "=r"(re[11]), "=r"(re[12]), "=r"(re[13]),
                  "=r"(re[14]), "=r"(re[15])
                : "r"(taddr));
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]), "=r"(im[6]),
                  "=r"(im[7]), "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]), "=r"(im[12]), "=r"(im[13]),
                  "=r"(im[14]), "=r"(im[15])
                : "r"(taddr + 32u));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const uint32_t l = lrow_out | cpos[ehalf + c];
            a.x[gbase + goff(l)] = make_float2(__uint_as_float(re[c]), __uint_as_float(im[c]));
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) cur[i] = nxt[i];
    }
    // free tensor memory (all MMAs of this CTA have completed or timed out)
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

}  // namespace

// Apply a 5-qubit block to a complex64 state with the tensor cores.
void launch_gate_tc5(qe_state* s, const int* qubits, const cd* U) {
    if (s->dtype != QE_C64) fail(QE_ERR_UNSUPPORTED, "tensor-core gates are complex64 only");
    if (s->n < 12) fail(QE_ERR_UNSUPPORTED, "tensor-core gates need n >= 12");
    TcArgs a;
    const tc::Geometry g = tc::tile_geometry(qubits);
    a.x = reinterpret_cast<float2*>(s->d);
    a.L = g.L;
    a.kh = g.kh;
    std::memcpy(a.hq, g.hq, sizeof(a.hq));
    std::memcpy(a.gpos, g.gpos, sizeof(a.gpos));
    a.ntiles = 1ull << (s->n - 12);
    // W = [[Re U, -Im U], [Im U, Re U]], row n (output), column k (input)
    static thread_local float W[2 * kN * kK];
    for (int n = 0; n < kN; ++n)
        for (int k = 0; k < kK; ++k) {
            const cd u = U[(n & 31) * 32 + (k & 31)];
            double w;
            if (n < 32) w = (k < 32) ? u.real() : -u.imag();
            else w = (k < 32) ? u.imag() : u.real();
            const float f = (float)w;
            // TF32 high part: round to 10 mantissa bits (nearest, ties away)
            uint32_t bits;
            std::memcpy(&bits, &f, 4);
            bits = (bits + 0x1000u) & 0xFFFFE000u;
            float hi;
            std::memcpy(&hi, &bits, 4);
            W[n * kK + k] = hi;
            W[kN * kK + n * kK + k] = f - hi;
        }
    complete_pending(s);   // the previous tensor-core launch, before the scratch is reused
    char* scr = (char*)ensure_scratch(s, 256 + sizeof(W));
    uint32_t* status = (uint32_t*)scr;
    QE_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s->stream));
    QE_CUDA(cudaMemcpyAsync(scr + 256, W, sizeof(W), cudaMemcpyHostToDevice, s->stream));
    a.status = status;
    a.W = (const float*)(scr + 256);
    a.spin_limit = 1ll << 26;
    const size_t smem = 1024 + (size_t)2 * kRows * kK * 4 + (size_t)2 * kN * kK * 4;
    QE_CUDA(cudaFuncSetAttribute(k_gate_tc5, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    QE_CUDA(cudaFuncSetAttribute(k_gate_tc5, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int occ = 0;
    QE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gate_tc5, kTcThreads, smem));
    const uint64_t grid = std::min<uint64_t>(a.ntiles, (uint64_t)num_sms() * std::max(occ, 1));
    {
        Launch Lc(s, "gate_tc_k5", 2.0 * dim(s) * amp_bytes(s));
        k_gate_tc5<<<(unsigned)grid, kTcThreads, smem, s->stream>>>(a);
        QE_CUDA(cudaGetLastError());
    }
    // checked before the next tensor-core launch or at the end of the flush,
    // so that the host plans the next block while this one runs
    QE_CUDA(cudaMemcpyAsync(status_word_host(s), status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream));
    s->status_pending = true;
}

}  // namespace qe
