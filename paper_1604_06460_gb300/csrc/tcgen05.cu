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
// Tiles of 128 groups (4096 amplitudes, 12 tile-local index bits: the 5
// gate qubits and 7 others, chunks of >= 2^L contiguous amplitudes) flow
// through a warp-specialised pipeline, one persistent CTA per SM:
//   - sixteen splitting warps: thread t owns 2 column quads of group row
//     t % 128 (a warp covers 32 consecutive rows); it loads the next tile's 8
//     amplitudes into registers while it splits the current ones into TF32
//     hi / lo and stores them as 16-byte chunks of the K-major 128-byte
//     swizzled operand (8 consecutive rows hit 8 different chunks);
//   - one thread issues the 24 tcgen05.mma (M=128, N=64, K=8, kind::tf32) of a
//     tile into one of two 64-column tensor-memory accumulators and commits
//     them to that buffer's mbarrier;
//   - eight epilogue warps read the accumulator with tcgen05.ld (TMEM lane =
//     group row), release it, and store the outputs straight from registers.
// Operand tiles and accumulators are double-buffered, so the splitting of
// tile t+1, the MMAs of tile t and the stores of tile t-1 overlap.  W_hi /
// W_lo (64x64 each) are loaded once per CTA.  Every wait is bounded and
// raises a shared abort flag on a timeout; the status word reports it and
// tensor memory is freed after the MMAs have drained.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "qe_arith.cuh"
#include "qe_internal.h"
#include "qe_tc.cuh"

namespace qe {

namespace {

using tc::smem_u32;
using tc::mbar_wait;

constexpr int kEpiWarps = 8;         // warps [0, 8): epilogue, two per TMEM lane quarter
constexpr int kSplitWarps = 16;      // warps [8, 24): loads and splitting
constexpr int kMmaWarp = kEpiWarps + kSplitWarps;
constexpr int kTcThreads = 32 * (kMmaWarp + 1);   // 800: at most 7 warps per SM sub-partition
constexpr int kRows = 128;           // groups per tile (MMA M)
constexpr int kK = 64;               // real K (32 complex)
constexpr int kN = 64;               // real N
constexpr uint32_t kTmemCols = 128;  // two 64-column accumulators
constexpr int kSuspendNs = 1000;

struct TcArgs {
    float2* x;
    uint64_t ntiles;
    int L, kh;
    uint8_t hq[8];
    uint8_t gpos[5];          // tile-local bit positions of the matrix bits
    uint32_t* status;
    long long spin_limit;
    const float* W;           // [2][kN * kK]: hi, lo parts of W, row n, column k
    int stall_test;           // failure-path test: the first tile's operand is never announced
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

// Wait (every lane of the warp) for phase `phase` of an mbarrier, each poll
// suspending for up to kSuspendNs; false on every lane when a lane's wait
// ran out (it then raises the shared abort flag) or the flag was raised.
__device__ __forceinline__ bool wait_warp(uint64_t* mbar, uint32_t phase, long long limit, int* abort_flag) {
    bool ok = false;
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(phase), "n"(kSuspendNs)
            : "memory");
        if (done) { ok = true; break; }
        if ((i & 7) == 7 && *reinterpret_cast<volatile int*>(abort_flag)) break;
        if (i + 1 == limit) *reinterpret_cast<volatile int*>(abort_flag) = 1;
    }
    return !__any_sync(0xFFFFFFFFu, !ok);
}

__device__ __forceinline__ void mbar_init_count(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

__global__ void __maxnreg__(72) k_gate_tc5(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned regions: W_hi, W_lo (64 x 64 x 4 B), then per operand
    // buffer A_hi, A_lo (128 x 64 x 4 B each)
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* sW_hi = base;
    unsigned char* sW_lo = sW_hi + kN * kK * 4;
    unsigned char* sA0 = sW_lo + kN * kK * 4;
    constexpr uint32_t kABuf = 2u * kRows * kK * 4;   // one operand buffer (hi + lo)
    // mbarriers per buffer b: operand stored (splitters), MMAs done (commit:
    // operand and accumulator b may be reused / read), accumulator read
    // (epilogue); and the final drain
    __shared__ __align__(8) uint64_t mbAFull[2], mbDone[2], mbAccFree[2], mbDrain;
    __shared__ uint32_t tmem_base;
    __shared__ uint64_t hoff[32];
    __shared__ uint32_t cpos[32];
    __shared__ uint64_t coloff[32];   // element offset of complex column c within a group
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
        for (int b = 0; b < 2; ++b) {
            mbar_init_count(&mbAFull[b], 32 * kSplitWarps);
            mbar_init_count(&mbDone[b], 1);
            mbar_init_count(&mbAccFree[b], 32 * kEpiWarps);
        }
        mbar_init_count(&mbDrain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t lowmask = (1u << a.L) - 1u;
    // the offset of a tile-local index is additive over disjoint bit sets:
    // (row bits | column bits) -> row offset + column offset
    if (tid < 32) coloff[tid] = (cpos[tid] & lowmask) + hoff[cpos[tid] >> a.L];
    __syncthreads();
    const uint32_t tmem = tmem_base;
    const uint32_t gmask = cpos[31];
    auto rowbits = [&](int r) {
        uint32_t l = 0;
        int j = 0;
        for (int b = 0; b < 12; ++b)
            if (!((gmask >> b) & 1u)) l |= (((uint32_t)r >> (j++)) & 1u) << b;
        return l;
    };
    auto goff = [&](uint32_t l) -> uint64_t { return (l & lowmask) + hoff[l >> a.L]; };
    auto fail_status = [&]() { atomicExch(a.status, 1u); };

    if (warp == kMmaWarp) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            bool ok = true;
            int i = 0;
            for (uint64_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++i) {
                const int b = i & 1;
                const uint32_t ph = (uint32_t)(i >> 1) & 1u;
                auto wait1 = [&](uint64_t* m, uint32_t p) {
                    for (long long k = 0; k < a.spin_limit; ++k) {
                        uint32_t done;
                        asm volatile(
                            "{\n\t.reg .pred q;\n\t"
                            "mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, %3;\n\t"
                            "selp.b32 %0, 1, 0, q;\n\t}\n"
                            : "=r"(done)
                            : "r"(smem_u32(m)), "r"(p), "n"(kSuspendNs)
                            : "memory");
                        if (done) return true;
                        if ((k & 7) == 7 && *reinterpret_cast<volatile int*>(&s_abort)) return false;
                    }
                    *reinterpret_cast<volatile int*>(&s_abort) = 1;
                    return false;
                };
                if (!wait1(&mbAFull[b], ph) || (i >= 2 && !wait1(&mbAccFree[b], ph ^ 1u))) {
                    fail_status();
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t ah = smem_u32(sA0) + (uint32_t)b * kABuf, al = ah + kRows * kK * 4;
                const uint32_t wh = smem_u32(sW_hi), wl = smem_u32(sW_lo);
                const uint32_t acc_t = tmem + (uint32_t)b * 64u;
                for (int ks = 0; ks < kK / 8; ++ks) {
                    const uint32_t aoff = (uint32_t)(ks >> 2) * kRows * 128u + (uint32_t)(ks & 3) * 32u;
                    const uint32_t boff = (uint32_t)(ks >> 2) * kN * 128u + (uint32_t)(ks & 3) * 32u;
                    mma_tf32(acc_t, tc::sdesc_sw128(ah + aoff), tc::sdesc_sw128(wh + boff), ks > 0 ? 1u : 0u);
                    mma_tf32(acc_t, tc::sdesc_sw128(ah + aoff), tc::sdesc_sw128(wl + boff), 1u);
                    mma_tf32(acc_t, tc::sdesc_sw128(al + aoff), tc::sdesc_sw128(wh + boff), 1u);
                }
                tc::mma_commit(&mbDone[b]);
            }
            // every MMA issued has completed before tensor memory is freed
            tc::mma_commit(&mbDrain);
            if (!tc::mbar_wait(smem_u32(&mbDrain), 0u, a.spin_limit)) fail_status();
        }
        __syncwarp();
    } else if (warp >= kEpiWarps) {
        // ------------------------------------------------ loads and splitting
        // thread <-> group row lr (a warp covers 32 consecutive rows) and the
        // column quads q = qbase + 4 j, j < 2: whole 16-byte operand chunks
        const int st = tid - 32 * kEpiWarps;
        const int lr = st & (kRows - 1);
        const int qbase = st >> 7;
        const uint64_t rowoff = goff(rowbits(lr));
        float2 cur[8], nxt[8];
        auto load_tile = [&](uint64_t t, float2* dst) {
            const float2* g = a.x + insert_zero_bits(t << a.L, a.hq, a.kh) + rowoff;
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int u = 0; u < 4; ++u) dst[4 * j + u] = g[coloff[4 * (qbase + 4 * j) + u]];
        };
        uint64_t t = blockIdx.x;
        if (t < a.ntiles) load_tile(t, cur);
        for (int i = 0; t < a.ntiles; t += gridDim.x, ++i) {
            const int b = i & 1;
            // the next tile's loads are in flight while this one is split; the
            // tile after it is prefetched into L2 (its 2^kh contiguous runs of
            // 2^L amplitudes, >= 1 KB, one bulk prefetch each)
            const uint64_t tn = t + gridDim.x, tn2 = tn + gridDim.x;
            if (tn < a.ntiles) load_tile(tn, nxt);
            if (tn2 < a.ntiles && st < (1 << a.kh)) {
                const float2* g2 = a.x + insert_zero_bits(tn2 << a.L, a.hq, a.kh) + hoff[st];
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g2), "r"(8u << a.L) : "memory");
            }
            // the MMAs two tiles back have read this operand buffer
            if (i >= 2 && !wait_warp(&mbDone[b], (uint32_t)((i - 2) >> 1) & 1u, a.spin_limit, &s_abort)) {
                fail_status();
                break;
            }
            unsigned char* sA_hi = sA0 + (uint32_t)b * kABuf;
            unsigned char* sA_lo = sA_hi + kRows * kK * 4;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int q = qbase + 4 * j;
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
            if (!(a.stall_test && i == 0)) mbar_arrive(&mbAFull[b]);
#pragma unroll
            for (int k = 0; k < 8; ++k) cur[k] = nxt[k];
        }
    } else {
        // ---------------------------------------------------------- epilogue
        // TMEM lane quarter of this warp, and which 16 columns of the real
        // (0..31) and imaginary (32..63) halves it reads
        const uint32_t equarter = (uint32_t)(warp & 3) * 32u;
        const uint32_t ehalf = (uint32_t)(warp >> 2) * 16u;
        const uint64_t rowoff_out = goff(rowbits((int)equarter + lane));
        int i = 0;
        for (uint64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++i) {
            const int b = i & 1;
            if (!wait_warp(&mbDone[b], (uint32_t)(i >> 1) & 1u, a.spin_limit, &s_abort)) {
                fail_status();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            float2* const gout = a.x + insert_zero_bits(t << a.L, a.hq, a.kh) + rowoff_out;
            // two rounds of 8 columns; the accumulator is released once the
            // second round is in registers
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t re[8], im[8];
                const uint32_t taddr = tmem + (equarter << 16) + (uint32_t)b * 64u + ehalf + 8u * h;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                    : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]), "=r"(re[6]),
                      "=r"(re[7])
                    : "r"(taddr));
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                    : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]), "=r"(im[6]),
                      "=r"(im[7])
                    : "r"(taddr + 32u));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (h == 1) {
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    mbar_arrive(&mbAccFree[b]);
                }
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    gout[coloff[ehalf + 8 * h + c]] = make_float2(__uint_as_float(re[c]), __uint_as_float(im[c]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == kMmaWarp) {
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
    a.spin_limit = 1ll << 21;   // polls of up to kSuspendNs each
    // Failure-path test (QE_TEST_STALL_TC64=1): the splitters withhold the
    // first tile's operand arrival, so the MMA thread's wait runs out after a
    // short limit and every role leaves through the shared abort flag.
    const char* stall = std::getenv("QE_TEST_STALL_TC64");
    a.stall_test = (stall != nullptr && stall[0] == '1') ? 1 : 0;
    if (a.stall_test) a.spin_limit = 1ll << 12;
    const size_t smem = 1024 + (size_t)2 * kN * kK * 4 + (size_t)2 * 2 * kRows * kK * 4;
    QE_CUDA(cudaFuncSetAttribute(k_gate_tc5, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    QE_CUDA(cudaFuncSetAttribute(k_gate_tc5, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    const uint64_t grid = std::min<uint64_t>(a.ntiles, (uint64_t)num_sms());
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
