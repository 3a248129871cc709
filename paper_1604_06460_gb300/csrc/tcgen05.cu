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
//   1. all threads load the tile, split each value and store In_hi / In_lo
//      into shared memory in the K-major 128-byte-swizzled operand layout;
//   2. one thread issues 24 tcgen05.mma (M=128, N=64, K=8, kind::tf32) into a
//      64-column tensor-memory accumulator and commits them to an mbarrier;
//   3. all threads wait on the mbarrier (bounded), read the accumulator with
//      tcgen05.ld, stage the results in shared memory and store the tile.
// W_hi / W_lo (64x64 each) are loaded once per CTA.  Waits that exceed their
// limit set a status word and end the kernel after freeing tensor memory.
#include <algorithm>
#include <cstring>

#include "qe_arith.cuh"
#include "qe_internal.h"

namespace qe {

namespace {

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

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

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

// Shared-memory matrix descriptor: start >> 4, leading offset (unused for
// swizzled K-major) 16 bytes, stride between 8-row groups 1024 bytes,
// descriptor version 1, layout SWIZZLE_128B (2).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: D f32, A/B tf32, both K-major, N = 64, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, long long limit) {
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase));
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(kTcThreads) k_gate_tc5(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned regions: A_hi, A_lo (128 x 64 x 4 B each), W_hi, W_lo (64 x 64 x 4 B)
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* sA_hi = base;
    unsigned char* sA_lo = sA_hi + kRows * kK * 4;
    unsigned char* sW_hi = sA_lo + kRows * kK * 4;
    unsigned char* sW_lo = sW_hi + kN * kK * 4;
    float2* stage = reinterpret_cast<float2*>(sA_hi);   // reused after the MMAs complete
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ uint64_t hoff[32];
    __shared__ uint32_t cpos[32];
    __shared__ uint8_t s_row[4096], s_col[4096];   // tile-local index -> (group row, matrix column)
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
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
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
    // row of a tile-local index: its 7 non-gate bits in order; column: its gate bits
    for (uint32_t l = tid; l < 4096u; l += blockDim.x) {
        uint32_t r = 0, c = 0;
        int j = 0;
        for (int b = 0; b < 12; ++b)
            if (!((gmask >> b) & 1u)) r |= ((l >> b) & 1u) << (j++);
        for (int q = 0; q < 5; ++q) c |= ((l >> a.gpos[q]) & 1u) << q;
        s_row[l] = (uint8_t)r;
        s_col[l] = (uint8_t)c;
    }
    __syncthreads();
    // each thread moves 16 amplitudes of a tile: l = tid + 256 * i
    constexpr int kPer = 4096 / kTcThreads;
    float2 cur[kPer], nxt[kPer];
    auto load_tile = [&](uint64_t t, float2* dst) {
        const uint64_t gb = insert_zero_bits(t << a.L, a.hq, a.kh);
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const uint32_t l = (uint32_t)tid + (uint32_t)kTcThreads * i;
            dst[i] = a.x[gb + (l & lowmask) + hoff[l >> a.L]];
        }
    };
    uint32_t phase = 0;
    uint64_t t = blockIdx.x;
    if (t < a.ntiles) load_tile(t, cur);
    for (; t < a.ntiles; t += gridDim.x) {
        const uint64_t gbase = insert_zero_bits(t << a.L, a.hq, a.kh);
        // 1. split into TF32 hi/lo and store the operand, swizzled
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const uint32_t l = (uint32_t)tid + (uint32_t)kTcThreads * i;
            const float2 v = cur[i];
            const int r = s_row[l], c = s_col[l];
            const float rh = tf32_hi(v.x), ih = tf32_hi(v.y);
            *reinterpret_cast<float*>(sA_hi + sw128_offset(r, c, kRows)) = rh;
            *reinterpret_cast<float*>(sA_hi + sw128_offset(r, 32 + c, kRows)) = ih;
            *reinterpret_cast<float*>(sA_lo + sw128_offset(r, c, kRows)) = __fsub_rn(v.x, rh);
            *reinterpret_cast<float*>(sA_lo + sw128_offset(r, 32 + c, kRows)) = __fsub_rn(v.y, ih);
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
                mma_tf32(tmem, sdesc(ah + aoff), sdesc(wh + boff), acc);
                acc = 1;
                mma_tf32(tmem, sdesc(ah + aoff), sdesc(wl + boff), 1);
                mma_tf32(tmem, sdesc(al + aoff), sdesc(wh + boff), 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar)));
        }
        // prefetch the next tile while the tensor cores work
        const uint64_t tn = t + gridDim.x;
        if (tn < a.ntiles) load_tile(tn, nxt);
        // 3. wait for the accumulator (bounded), read it, stage and store
        if (!mbar_wait(smem_u32(&mbar), phase, a.spin_limit)) {
            atomicExch(a.status, 1u);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        uint32_t v[32];
        {
            const uint32_t quarter = (uint32_t)(warp & 3) * 32u;
            const uint32_t col = (warp < 4) ? 0u : 32u;
            const uint32_t taddr = tmem + (quarter << 16) + col;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                  "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                  "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
        }
        // row r = TMEM lane; output element c of row r sits at the tile-local
        // index with row bits r and gate bits c; the staging buffer pads one
        // element per 32 so that a warp's 32 rows hit different banks
        {
            const uint32_t r = (uint32_t)(warp & 3) * 32u + (uint32_t)lane;
            uint32_t lrow = 0;
            int j = 0;
            for (int b = 0; b < 12; ++b)
                if (!((gmask >> b) & 1u)) lrow |= ((r >> (j++)) & 1u) << b;
            float* st = reinterpret_cast<float*>(stage);
            const int comp = (warp < 4) ? 0 : 1;
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const uint32_t l = lrow | cpos[c];
                st[2 * (l + (l >> 5)) + comp] = __uint_as_float(v[c]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const uint32_t l = (uint32_t)tid + (uint32_t)kTcThreads * i;
            a.x[gbase + (l & lowmask) + hoff[l >> a.L]] = stage[l + (l >> 5)];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kPer; ++i) cur[i] = nxt[i];
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
    // tile geometry: 12 local bits, the 5 gate qubits among them
    int srt[5];
    for (int j = 0; j < 5; ++j) srt[j] = qubits[j];
    std::sort(srt, srt + 5);
    int L = -1, kh = 0;
    for (int l = 12; l >= 0; --l) {
        int h = 0;
        for (int j = 0; j < 5; ++j) h += srt[j] >= l;
        if (l + h <= 12) { L = l; kh = h; break; }
    }
    if (L < 0) fail(QE_ERR_ARG, "no tensor-core tile geometry");
    a.x = reinterpret_cast<float2*>(s->d);
    a.L = L;
    a.kh = kh;
    int h = 0;
    for (int j = 0; j < 5; ++j)
        if (srt[j] >= L) a.hq[h++] = (uint8_t)srt[j];
    for (int j = 0; j < 5; ++j) {
        int q = qubits[j], pos = q;
        if (q >= L)
            for (int i = 0; i < kh; ++i)
                if (a.hq[i] == q) pos = L + i;
        a.gpos[j] = (uint8_t)pos;
    }
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
    char* scr = (char*)ensure_scratch(s, 256 + sizeof(W));
    uint32_t* status = (uint32_t*)scr;
    QE_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), s->stream));
    QE_CUDA(cudaMemcpyAsync(scr + 256, W, sizeof(W), cudaMemcpyHostToDevice, s->stream));
    a.status = status;
    a.W = (const float*)(scr + 256);
    a.spin_limit = 1ll << 26;
    const size_t smem = 1024 + (size_t)2 * kRows * kK * 4 + (size_t)2 * kN * kK * 4;
    QE_CUDA(cudaFuncSetAttribute(k_gate_tc5, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    QE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gate_tc5, kTcThreads, smem));
    const uint64_t grid = std::min<uint64_t>(a.ntiles, (uint64_t)num_sms() * std::max(occ, 1));
    {
        Launch Lc(s, "gate_tc_k5", 2.0 * dim(s) * amp_bytes(s));
        k_gate_tc5<<<(unsigned)grid, kTcThreads, smem, s->stream>>>(a);
        QE_CUDA(cudaGetLastError());
    }
    uint32_t host_status = 0;
    QE_CUDA(cudaMemcpyAsync(&host_status, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream));
    QE_CUDA(cudaStreamSynchronize(s->stream));
    if (host_status) fail(QE_ERR_TIMEOUT, "tensor-core gate: an mbarrier wait exceeded its limit");
}

}  // namespace qe
