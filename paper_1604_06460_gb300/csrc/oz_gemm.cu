// Complex matrix products on the tensor cores for the emulated phase
// estimation (Sec. III-C: the powers U^(2^j) by repeated squaring).
//
// C = A B for complex128 matrices is one real product
//     [Re C | Im C] = [Re A | Im A] [[Re B, Im B], [-Im B, Re B]],
// computed from exact integer-digit products on the FP16 tensor pipe with the
// 7-digit (56-bit) splitting of the complex128 gate kernel (qe_oz.cuh), one
// K-chunk of 64 real terms at a time, the chunks' integers summed exactly in
// 128 bits and rounded once to FP64 at the end.
//
// Operands.  Two splitting kernels write the digits of A's rows (one scale
// per row over its 2K real values) and of the rows of the right operand's
// transpose, Bt, whose rows are the real output columns (one scale per
// complex output column, shared by its real and imaginary rows), as fp16
// digits in blocks of one operand tile and K-stage (A: 128 rows, Bt: 32 rows,
// x 32 values of K) per digit, each block already in the 64-byte-swizzled
// K-major layout the MMAs read, so that one bulk copy moves it into shared
// memory.  Bt rows are ordered per tile of 16 complex output columns: their
// 16 real-part rows, then their 16 imaginary-part rows.  Rows of A beyond M
// (up to a multiple of 128) are zero.
//
// Product kernel: one CTA per output tile of 128 rows x 16 complex columns,
// warp-specialised like the gate kernel.  One thread copies each K-stage's
// (32 values) seven A and seven Bt digit blocks (56 + 14 KB, two stage
// buffers, 64-byte swizzle) with the bulk-copy engine (cp.async.bulk,
// completion counted in bytes on the buffer's mbarrier), so the copy of a
// stage overlaps the MMAs of the previous one; one thread issues the 34 digit
// pairs with i + j <= 9 as 8 MMAs per K-step (the Bt digit slices stacked
// along N, as the gate kernel stacks W's) into one of two tensor-memory
// accumulator sets (8 accumulators x 32 columns each; a set sums one chunk of
// 64 values, two stages, exactly); sixteen recombining warps turn a finished
// set into each output's integer Y of the chunk (as in the gate kernel) and
// add it to a 128-bit sum.  The two sets let the recombination of chunk c
// overlap the loads and MMAs of chunk c + 1.
//
// Accuracy.  Each input is rounded once to 56 bits of its row's (column's)
// scale; within a chunk the digit products and Y are exact up to the dropped
// pairs (i + j > 9: below 2^(E+F-57.6) per chunk of 64 terms); the 128-bit
// sums are exact and the result is rounded once (within 1.5 units in the last
// place) and scaled by 2^(E+F-56).  Rows (columns) whose largest magnitude is
// below 2^-920 are flushed to zero.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "qe_internal.h"
#include "qe_oz.cuh"

namespace qe {

namespace {

using namespace oz;

constexpr int kD = 7;
constexpr int kTM = 128;                    // output rows per tile (MMA M)
constexpr int kTN = 32;                     // Bt rows per tile (16 complex output columns)
constexpr int kKC = 64;                     // real K per accumulator set (exact FP32 sums)
constexpr int kKS = 32;                     // real K per operand stage: one 64-byte fp16 row
constexpr uint32_t kASlice = kTM * 64;      // bytes of one digit plane of the A tile (one stage)
constexpr uint32_t kBSlice = kTN * 64;      // bytes of one digit plane of the Bt tile (one stage)
constexpr uint32_t kSetCols = 256;          // 8 accumulators x 32 columns
constexpr int kRecWarps = 16;               // 4 per tensor-memory lane quarter, 8 columns each
constexpr int kMmaWarp = kRecWarps, kLoadWarp = kRecWarps + 1;
constexpr int kThreads = 32 * (kLoadWarp + 1);   // 576
constexpr int kRecThreads = 32 * kRecWarps;
constexpr uint32_t kStageBytes = kD * (kASlice + kBSlice);   // bulk-copied per stage (70 KB)
constexpr int kFlushExp = 100;              // biased exponent below which a row is flushed
constexpr size_t kSmem = 1024 + 2 * (size_t)kStageBytes;      // two stage buffers
static_assert(kSmem <= 227 * 1024, "shared memory per CTA");

// ------------------------------------------------------------- splitting
// Byte offset of the 16-byte chunk `ch` (8 fp16 along K) of row r in a
// K-major operand with 64-byte rows, 64-byte swizzle (the chunk index XOR
// bits 1-2 of the row within its 8-row, 512-byte group).
__device__ __forceinline__ uint32_t sw64_chunk(int r, int ch) {
    return (uint32_t)(r >> 3) * 512u + (uint32_t)(r & 7) * 64u + (uint32_t)((ch ^ ((r >> 1) & 3)) * 16);
}

// Shared-memory matrix descriptor for a K-major operand in the 64-byte swizzle
// layout: start >> 4, leading offset (unused) 16 bytes, stride between 8-row
// groups 512 bytes, descriptor version 1, layout SWIZZLE_64B (4).
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(512u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Digit blocks: digit i of operand-tile t (of nt) and K-stage c (of nc, 32
// values each) is the block ((i nt + t) nc + c) of `block` bytes; inside it,
// values k, k + 1 (k even) of the tile's row r sit at
// sw64_chunk(r, (k mod 32) / 8) + 2 (k mod 8) bytes.
__device__ __forceinline__ size_t block_word(int i, int64_t t, int64_t nt, int64_t c, int64_t nc, uint32_t block,
                                             int r, int64_t k) {
    const uint32_t kk = (uint32_t)(k & 31);
    const size_t base = (((size_t)i * nt + t) * nc + c) * block;
    return (base + sw64_chunk(r, (int)(kk >> 3)) + 2u * (kk & 7u)) >> 2;
}

// The seven digits of two consecutive values (packed fp16 pairs) into their
// blocks (operand row r of tile t, values k, k + 1).
__device__ __forceinline__ void put_pair(uint32_t* dig, int64_t t, int64_t nt, int64_t nc, uint32_t block, int r,
                                         int64_t k, double a, double b, uint32_t base_s) {
    uint32_t w[kD];
    digit_pairs<kD>(split_z<kD>(a, base_s), split_z<kD>(b, base_s), w);
#pragma unroll
    for (int i = 0; i < kD; ++i) dig[block_word(i, t, nt, k >> 5, nc, block, r, k)] = w[i];
}

__device__ __forceinline__ uint32_t biased_exp(double v) { return ((uint32_t)__double2hiint(v) << 1) >> 21; }

__device__ uint32_t block_max(uint32_t v, uint32_t* sh) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, sh[w]);
    return m;
}

__device__ __forceinline__ int64_t insert_one(int64_t r, int bit) {
    if (bit < 0) return r;
    const int64_t low = r & ((1ll << bit) - 1);
    return ((r >> bit) << (bit + 1)) | (1ll << bit) | low;
}

// One CTA per (padded) row of A: the row is [Re a | Im a] (2K reals).
__global__ void __launch_bounds__(256) k_split_a(const double2* __restrict__ src, int64_t M, int64_t K, int64_t lda,
                                                 int rowbit, uint32_t* __restrict__ dig, int* __restrict__ escale,
                                                 int64_t Mp) {
    __shared__ uint32_t sh[32];
    const int64_t r = blockIdx.x;
    const int64_t pairs = K;   // pairs of consecutive reals of the 2K
    const int64_t nt = Mp / kTM, nc = 2 * K / kKS, t = r / kTM;
    const int rl = (int)(r % kTM);
    if (r >= M) {
        for (int64_t p = threadIdx.x; p < pairs; p += blockDim.x)
            for (int i = 0; i < kD; ++i) dig[block_word(i, t, nt, (2 * p) >> 5, nc, kASlice, rl, 2 * p)] = 0u;
        if (threadIdx.x == 0) escale[r] = 0;
        return;
    }
    const double2* row = src + insert_one(r, rowbit) * lda;
    uint32_t em = 0;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
        const double2 v = row[k];
        em = max(em, max(biased_exp(v.x), biased_exp(v.y)));
    }
    em = block_max(em, sh);
    const uint32_t base_s = em < (uint32_t)kFlushExp ? 0x10000u : em;
    for (int64_t p = threadIdx.x; p < pairs; p += blockDim.x) {
        const int64_t k = 2 * p;   // reals k, k + 1 of [Re | Im]
        const double2 u = row[k % K], w = row[(k + 1) % K];
        const bool im = k >= K;
        put_pair(dig, t, nt, nc, kASlice, rl, k, im ? u.y : u.x, im ? w.y : w.x, base_s);
    }
    if (threadIdx.x == 0) escale[r] = (int)em - 1021;
}

// One CTA per tile of 16 complex columns c of B (K x N, row-major): the Bt
// rows of column c are [Re B[:,c] ; -Im B[:,c]] (real part of C) and
// [Im B[:,c] ; Re B[:,c]] (imaginary part).  Digits are written through a
// shared-memory transpose of 32-row blocks of B.
__global__ void __launch_bounds__(256) k_split_b(const double2* __restrict__ src, int64_t K, int64_t ldb,
                                                 uint32_t* __restrict__ dig, int* __restrict__ fscale, int64_t Nr) {
    __shared__ double2 blk[32][17];
    __shared__ uint32_t colmax[16][17];
    __shared__ uint32_t base[16];
    const int tid = threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x * 16;
    const int ci = tid & 15, kr = tid >> 4;
    uint32_t em = 0;
    for (int64_t k = kr; k < K; k += 16) {
        const double2 v = src[k * ldb + c0 + ci];
        em = max(em, max(biased_exp(v.x), biased_exp(v.y)));
    }
    colmax[ci][kr] = em;
    __syncthreads();
    if (tid < 16) {
        uint32_t m = 0;
        for (int j = 0; j < 16; ++j) m = max(m, colmax[tid][j]);
        base[tid] = m < (uint32_t)kFlushExp ? 0x10000u : m;
        fscale[32 * blockIdx.x + tid] = (int)m - 1021;
        fscale[32 * blockIdx.x + 16 + tid] = (int)m - 1021;
    }
    __syncthreads();
    const int64_t nt = Nr / kTN, nc = 2 * K / kKS;
    const int q = tid & 15;    // pair within a 32-value segment
    for (int64_t k0 = 0; k0 < K; k0 += 32) {
        for (int e = tid; e < 32 * 16; e += 256) blk[e >> 4][e & 15] = src[(k0 + (e >> 4)) * ldb + c0 + (e & 15)];
        __syncthreads();
        // segments g = (row rho of the tile, half hf of the K range)
        for (int g = tid >> 4; g < 64; g += 16) {
            const int rho = g & 31, hf = g >> 5, cl = rho & 15, part = rho >> 4;
            const double2 u = blk[2 * q][cl], w = blk[2 * q + 1][cl];
            double a, b;
            if (part == 0) {
                a = hf ? -u.y : u.x;
                b = hf ? -w.y : w.x;
            } else {
                a = hf ? u.x : u.y;
                b = hf ? w.x : w.y;
            }
            const int64_t pos = (hf ? K : 0) + k0 + 2 * q;
            put_pair(dig, blockIdx.x, nt, nc, kBSlice, rho, pos, a, b, base[cl]);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- product
struct GemmOzArgs {
    const uint16_t* adig;   // digit blocks of A (kD x Mp/128 x Kr/64 blocks of 16 KB)
    const uint16_t* bdig;   // digit blocks of Bt (kD x Nr/32 x Kr/64 blocks of 4 KB)
    const int* ea;          // [Mp]
    const int* fb;          // [Nr]
    double2* C;             // row-major, C[r * ldc + c]
    int64_t M, Mp, Nr, Kr, ldc;
    uint32_t* status;
    long long spin_limit;
};

enum GBar { kReady0, kReady1, kOpFree0, kOpFree1, kFull0, kFull1, kFree0, kFree1, kDrain, kGBars };

__device__ __forceinline__ double i128_to_double(long long hi, unsigned long long lo) {
    if ((hi == 0 && (long long)lo >= 0) || (hi == -1 && (long long)lo < 0)) return __ll2double_rn((long long)lo);
    return __fma_rn((double)hi, 18446744073709551616.0, __ull2double_rn(lo));
}

__global__ void __launch_bounds__(kThreads, 1) k_oz_zgemm(const __grid_constant__ GemmOzArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    // stage buffer b (0, 1): 7 digit planes of the A tile, then the 7 of the
    // Bt tile stacked (row j * 32 + r of the stacked operand)
    auto stageA = [&](int b) { return base + (size_t)b * kStageBytes; };
    auto stageB = [&](int b) { return base + (size_t)b * kStageBytes + kD * kASlice; };
    __shared__ __align__(8) uint64_t bars[kGBars];
    __shared__ uint32_t tmem_base, abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = (int64_t)blockIdx.y * kTM, brow0 = (int64_t)blockIdx.x * kTN;
    const int nchunks = (int)(a.Kr / kKC), nstages = (int)(a.Kr / kKS);
    if (tid == 0) {
        const uint32_t counts[kGBars] = {1, 1, 1, 1, 1, 1, kRecThreads, kRecThreads, 1};
        for (int b = 0; b < kGBars; ++b) mbar_init_count(&bars[b], counts[b]);
        abort_flag = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * kSetCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    auto wait = [&](GBar b, uint32_t ph) {
        const bool ok = wait_or_abort(smem_u32(&bars[b]), ph, a.spin_limit, &abort_flag);
        if (__any_sync(0xFFFFFFFFu, !ok)) {
            if (!ok) atomicExch(a.status, 1u);
            return false;
        }
        return true;
    };
    if (warp == kMmaWarp) {
        // ---------------------------------------------------- MMA issuer
        // stage s (32 values of K) from buffer s & 1 into set (s >> 1) & 1;
        // a set holds one chunk of 64 values (two stages), then is recombined
        if (lane == 0) {
            constexpr MmaTable<kD> tab;
            bool ok = true;
            for (int st = 0; st < nstages && ok; ++st) {
                const int buf = st & 1, c = st >> 1, set = c & 1;
                ok = wait_or_abort(smem_u32(&bars[buf ? kReady1 : kReady0]), (uint32_t)(st >> 1) & 1u, a.spin_limit,
                                   &abort_flag);
                if (ok && (st & 1) == 0 && c >= 2)
                    ok = wait_or_abort(smem_u32(&bars[set ? kFree1 : kFree0]), (uint32_t)((c >> 1) - 1) & 1u,
                                       a.spin_limit, &abort_flag);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t dset = tmem + (uint32_t)set * kSetCols;
                const uint64_t da0 = sdesc_sw64(smem_u32(stageA(buf))), db0 = sdesc_sw64(smem_u32(stageB(buf)));
#pragma unroll
                for (int ks = 0; ks < kKS / 16; ++ks) {
#pragma unroll
                    for (int m = 0; m <= kD; ++m) {
                        const int i = tab.i[m], j0 = tab.j0[m], j1 = tab.j1[m];
                        const uint32_t nn = (uint32_t)(j1 - j0 + 1) * kTN;
                        const uint64_t da = da0 + (((uint32_t)(i - 1) * kASlice + 32u * ks) >> 4);
                        const uint64_t db = db0 + (((uint32_t)(j0 - 1) * kBSlice + 32u * ks) >> 4);
                        mma_f16(dset + (uint32_t)(i + j0 - 2) * kTN, da, db, tc::idesc(0u, nn, kTM),
                                ((st & 1) || ks > 0 || m > 1) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&bars[buf ? kOpFree1 : kOpFree0]);
                if (st & 1) tc::mma_commit(&bars[set ? kFull1 : kFull0]);
            }
            if (!ok) atomicExch(a.status, 1u);
            tc::mma_commit(&bars[kDrain]);
            if (!tc::mbar_wait(smem_u32(&bars[kDrain]), 0u, a.spin_limit)) atomicExch(a.status, 1u);
        }
        __syncwarp();
    } else if (warp == kLoadWarp) {
        // ------------------------------------------------------- loads
        // one thread: stage s into buffer s & 1 once that buffer's previous
        // stage (s - 2) has been consumed by its MMAs: the byte count on the
        // buffer's ready barrier and 14 bulk copies
        if (lane == 0) {
            const int64_t ntA = a.Mp / kTM, ntB = a.Nr / kTN;
            const char* ga = reinterpret_cast<const char*>(a.adig);
            const char* gb = reinterpret_cast<const char*>(a.bdig);
            for (int st = 0; st < nstages; ++st) {
                const int buf = st & 1;
                if (st >= 2 && !wait_or_abort(smem_u32(&bars[buf ? kOpFree1 : kOpFree0]), (uint32_t)((st >> 1) - 1) & 1u,
                                              a.spin_limit, &abort_flag)) {
                    atomicExch(a.status, 1u);
                    break;
                }
                uint64_t* rb = &bars[buf ? kReady1 : kReady0];
                mbar_expect_tx(rb, kStageBytes);
#pragma unroll 1
                for (int i = 0; i < kD; ++i) {
                    bulk_g2s(smem_u32(stageA(buf)) + (uint32_t)i * kASlice,
                             ga + (((size_t)i * ntA + blockIdx.y) * nstages + st) * kASlice, kASlice, rb);
                    bulk_g2s(smem_u32(stageB(buf)) + (uint32_t)i * kBSlice,
                             gb + (((size_t)i * ntB + blockIdx.x) * nstages + st) * kBSlice, kBSlice, rb);
                }
            }
        }
        __syncwarp();
    } else {
        // --------------------------------------------- recombination
        // thread <-> (row 32 q + lane, Bt columns [8 u, 8 u + 8) of the tile)
        const int q = warp & 3, u = warp >> 2;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        long long hi[8];
        unsigned long long lo[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            hi[j] = 0;
            lo[j] = 0ull;
        }
        bool ok = true;
        for (int c = 0; c < nchunks && ok; ++c) {
            const int set = c & 1;
            if (!wait(set ? kFull1 : kFull0, (uint32_t)(c >> 1) & 1u)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t tset = lane_base + (uint32_t)set * kSetCols + 8u * u;
#pragma unroll
            for (int h = 0; h < 2; ++h) {   // columns 8u + 4h .. + 3
                uint32_t cc[kD + 1][4];
#pragma unroll
                for (int d = 0; d <= kD; ++d)
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                                 : "=r"(cc[d][0]), "=r"(cc[d][1]), "=r"(cc[d][2]), "=r"(cc[d][3])
                                 : "r"(tset + (uint32_t)(d * kTN + 4 * h)));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (h == 1) {
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    mbar_arrive(&bars[set ? kFree1 : kFree0]);
                }
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    uint32_t c1[kD + 1];
#pragma unroll
                    for (int d = 0; d <= kD; ++d) c1[d] = cc[d][x];
                    const long long Y = combine_y<kD>(c1);
                    const int j = 4 * h + x;
                    const unsigned long long nlo = lo[j] + (unsigned long long)Y;
                    hi[j] += (Y >> 63) + (nlo < lo[j] ? 1 : 0);
                    lo[j] = nlo;
                }
            }
        }
        const int64_t r = row0 + 32 * q + lane;
        if (ok && r < a.M) {
            const int er = a.ea[r];
            double* out = reinterpret_cast<double*>(a.C);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int b = 8 * u + j;                       // Bt row of the tile
                const int64_t cc = (int64_t)blockIdx.x * 16 + (b & 15);
                const double y = i128_to_double(hi[j], lo[j]);
                out[2 * (r * a.ldc + cc) + (b >> 4)] = scalbn(y, er + a.fb[brow0 + b] - 56);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kSetCols));
    }
}

struct Workspace {
    uint16_t* adig;
    uint16_t* bdig;
    int* ea;
    int* fb;
    uint32_t* status;
};

Workspace workspace(qe_state* s, int64_t Mp, int64_t Nr, int64_t Kr) {
    const size_t abytes = (size_t)kD * Mp * Kr * 2, bbytes = (size_t)kD * Nr * Kr * 2;
    const size_t need = abytes + bbytes + (size_t)(Mp + Nr) * 4 + 256;
    char* p = (char*)ensure_oz_workspace(s, need);
    Workspace w;
    w.adig = (uint16_t*)p;
    w.bdig = (uint16_t*)(p + abytes);
    w.ea = (int*)(p + abytes + bbytes);
    w.fb = w.ea + Mp;
    w.status = (uint32_t*)(p + ((abytes + bbytes + (size_t)(Mp + Nr) * 4 + 255) & ~(size_t)255));
    return w;
}

}  // namespace

bool oz_gemm_available(int64_t M, int64_t K, int64_t N) {
    const char* e = std::getenv("QE_GEMM_F64");
    if (e && e[0] == '1') return false;
    return M >= 1 && K >= 32 && K % 32 == 0 && N >= 16 && N % 16 == 0;
}

// C (M x N complex, row-major, ldc) = A (M x K, rows through the optional
// inserted row bit) B (K x N, row-major, ldb); enqueued on s's stream.
void oz_zgemm(qe_state* s, double2* C, int64_t ldc, const double2* A, int64_t M, int64_t K, int64_t lda, int a_rowbit,
              const double2* B, int64_t N, int64_t ldb) {
    if (!oz_gemm_available(M, K, N)) fail(QE_ERR_UNSUPPORTED, "matrix shape not supported by the tensor-core product");
    const int64_t Mp = (M + kTM - 1) / kTM * kTM, Kr = 2 * K, Nr = 2 * N;
    const Workspace w = workspace(s, Mp, Nr, Kr);
    if (Mp / kTM > 65535) fail(QE_ERR_UNSUPPORTED, "matrix product too tall for one launch");
    {
        Launch L(s, "oz_split_a", (double)M * K * 16.0, false);
        k_split_a<<<(unsigned)Mp, 256, 0, s->stream>>>(A, M, K, lda, a_rowbit, reinterpret_cast<uint32_t*>(w.adig), w.ea,
                                                       Mp);
        QE_CUDA(cudaGetLastError());
    }
    {
        Launch L(s, "oz_split_b", (double)K * N * 16.0, false);
        k_split_b<<<(unsigned)(N / 16), 256, 0, s->stream>>>(B, K, ldb, reinterpret_cast<uint32_t*>(w.bdig), w.fb, Nr);
        QE_CUDA(cudaGetLastError());
    }
    GemmOzArgs g;
    g.adig = w.adig;
    g.bdig = w.bdig;
    g.ea = w.ea;
    g.fb = w.fb;
    g.C = C;
    g.M = M;
    g.Mp = Mp;
    g.Nr = Nr;
    g.Kr = Kr;
    g.ldc = ldc;
    g.status = w.status;
    g.spin_limit = 1ll << 21;   // polls of up to 1 us each
    QE_CUDA(cudaMemsetAsync(w.status, 0, sizeof(uint32_t), s->stream));
    QE_CUDA(cudaFuncSetAttribute(k_oz_zgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    {
        Launch L(s, "oz_zgemm", (double)(M * K + K * N + M * N) * 16.0, false);
        k_oz_zgemm<<<dim3((unsigned)(Nr / kTN), (unsigned)(Mp / kTM)), kThreads, kSmem, s->stream>>>(g);
        QE_CUDA(cudaGetLastError());
    }
    uint32_t st = 0;
    QE_CUDA(cudaMemcpyAsync(&st, w.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream));
    QE_CUDA(cudaStreamSynchronize(s->stream));
    if (st != 0) fail(QE_ERR_TIMEOUT, "a tensor-core matrix product wait ran out");
}

}  // namespace qe
