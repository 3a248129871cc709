// Pieces of the exact integer-digit products on the FP16 tensor pipe shared
// by the complex128 gate kernel and the complex GEMM: the 128-byte-swizzled
// K-major operand layout, the fp16 MMA, cp.async and mbarrier hand-offs with
// bounded waits, the splitting of doubles into balanced base-256 digits and
// the exact recombination of the digit-product accumulators (the splitting
// idea of Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012).
#pragma once
#include <cstdint>

#include "qe_tc.cuh"

namespace qe {
namespace oz {

using tc::smem_u32;

// Byte offset of the 16-byte chunk `ch` (8 fp16 along K) of row r in a
// K-major operand with 128-byte rows, 128-byte swizzle.
__device__ __forceinline__ uint32_t sw128_chunk(int r, int ch) {
    return (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u + (uint32_t)((ch ^ (r & 7)) * 16);
}

// D[128 x N] (+)= A[128 x 16] B[N x 16]^T, fp16 inputs, f32 accumulators.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src));
}

// Arrive on the mbarrier once every cp.async issued so far by this thread
// has landed (the arrival is counted in the barrier's expected count).
__device__ __forceinline__ void cp_async_arrive(uint64_t* mbar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_init_count(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
// Wait for phase `phase` of an mbarrier, each poll suspending the thread for
// up to kSuspendNs (it resumes when the phase completes), so waiting warps
// take no issue slots.  False when the shared abort flag is raised (checked
// every 8 polls) or after `limit` polls, in which case this thread raises it.
constexpr int kSuspendNs = 1000;
__device__ __forceinline__ bool wait_or_abort(uint32_t mbar, uint32_t phase, long long limit, uint32_t* abort_flag) {
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase), "n"(kSuspendNs)
            : "memory");
        if (done) return true;
        if ((i & 7) == 7 && *reinterpret_cast<volatile uint32_t*>(abort_flag)) return false;
    }
    *reinterpret_cast<volatile uint32_t*>(abort_flag) = 1u;
    return false;
}

// Bulk prefetch of `bytes` (a multiple of 16) at a 16-byte aligned global
// address into L2.
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}


// The balanced-offset integer Z of v (as two words) for a row whose largest
// biased exponent is em: X = round(|v| 2^(8D - E_r)) = round(M53 2^(e - em + 8D - 54))
// and Z = X + 0x80...80 (D - 1 bytes of 0x80, which makes the lower digits
// balanced).  With q = (M53 << c) >> (base_s - e), c = 3 for D = 7 (M53 << 3
// fits 56 bits) and c = 0 for D = 6, X = (q + 1) >> 1; the shift base is
// base_s = em + 53 + c - 8D (em for D = 7, em + 5 for D = 6), and the shift is
// done as clamped 32-bit shifts (64 or more, which includes zero and subnormal
// v with e = 0, gives q = 0).  Also returns the high word of v (its sign).
struct Zw {
    uint32_t zl, zh, hi;
};
template <int D>
__device__ __forceinline__ Zw split_z(double v, uint32_t base_s) {
    static_assert(D == 6 || D == 7, "6 or 7 digits");
    const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
    const uint32_t s = base_s - ((hi << 1) >> 21);
    const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
    // (H, L): M53 << c as two words
    const uint32_t H = (D == 7) ? __funnelshift_l(lo, mh, 3) : mh;
    const uint32_t L = (D == 7) ? (lo << 3) : lo;
    uint32_t t, qh, ql;
    asm("shf.r.clamp.b32 %0, %1, %2, %3;" : "=r"(t) : "r"(L), "r"(H), "r"(s));    // low word of (H:L) >> min(s, 32)
    asm("shr.b32 %0, %1, %2;" : "=r"(qh) : "r"(H), "r"(s));                         // 0 for s >= 32
    const uint32_t s2 = (uint32_t)max((int)s - 32, 0);
    asm("shr.b32 %0, %1, %2;" : "=r"(ql) : "r"(t), "r"(s2));                         // s >= 32: H >> (s - 32)
    // + 1 rounds, + 2 * 0x80...80 balances (both before the halving)
    constexpr uint64_t kOff = (D == 7) ? 0x1010101010101ull : 0x10101010101ull;
    const uint64_t Z = ((((uint64_t)qh << 32) | ql) + kOff) >> 1;
    return Zw{(uint32_t)Z, (uint32_t)(Z >> 32), hi};
}

// add.rn.f16x2
__device__ __forceinline__ uint32_t hadd2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// The D signed digits of two values a, b as packed fp16 pairs (a in the low
// half).  The bytes of the two Z are first interleaved (a0 b0 a1 b1 ...); one
// byte permute against the constant with bytes 0x64 | sign << 7 then makes
// each pair of bytes the fp16 numbers sign * (1024 + byte), and one f16x2
// addition of -sign * 1152 (-sign * 1024 for the leading digit) gives
// sign * (byte - 128) (sign * byte) exactly.  The leading digit is byte D - 1
// of Z; digits 1 .. D - 1 are bytes D - 2 .. 0 (zh holds bytes 4 and up, zl
// bytes 0..3).
template <int D>
__device__ __forceinline__ void digit_pairs(const Zw& A, const Zw& B, uint32_t w[D]) {
    const uint32_t sg = __byte_perm(A.hi, B.hi, 0x7030u) & 0x80008000u;   // the signs at bits 15 and 31
    const uint32_t hs = 0x64006400u | sg;                         // bytes 1, 3: 0x64 | sign
    const uint32_t c0 = 0x64006400u | (sg ^ 0x80008000u);         // -sign * 1024
    const uint32_t c1 = 0x64806480u | (sg ^ 0x80008000u);         // -sign * 1152
    const uint32_t ph = __byte_perm(A.zh, B.zh, 0x5140u);         // a0 b0 a1 b1 of zh
    const uint32_t p01 = __byte_perm(A.zl, B.zl, 0x5140u);        // a0 b0 a1 b1 of zl
    const uint32_t p23 = __byte_perm(A.zl, B.zl, 0x7362u);        // a2 b2 a3 b3 of zl
    if (D == 7) {
        const uint32_t ph2 = __byte_perm(A.zh, B.zh, 0x7362u);    // a2 b2 a3 b3 of zh
        w[0] = hadd2(__byte_perm(ph2, hs, 0x7150u), c0);          // Z byte 6
        w[1] = hadd2(__byte_perm(ph, hs, 0x7352u), c1);           // Z byte 5
        w[2] = hadd2(__byte_perm(ph, hs, 0x7150u), c1);           // Z byte 4
    } else {
        w[0] = hadd2(__byte_perm(ph, hs, 0x7352u), c0);           // Z byte 5
        w[1] = hadd2(__byte_perm(ph, hs, 0x7150u), c1);           // Z byte 4
    }
    w[D - 4] = hadd2(__byte_perm(p23, hs, 0x7352u), c1);          // Z byte 3
    w[D - 3] = hadd2(__byte_perm(p23, hs, 0x7150u), c1);          // Z byte 2
    w[D - 2] = hadd2(__byte_perm(p01, hs, 0x7352u), c1);          // Z byte 1
    w[D - 1] = hadd2(__byte_perm(p01, hs, 0x7150u), c1);          // Z byte 0
}

// The integer Y of one output from its D + 1 accumulators C_2 .. C_{D+2}
// (raw FP32 bits).
template <int D>
__device__ __forceinline__ long long combine_y(const uint32_t c[D + 1]) {
    const float M = 12582912.0f;   // 1.5 * 2^23; bits 0x4B400000
    const uint32_t u2 = __float_as_uint(__fadd_rn(__uint_as_float(c[0]), M));
    const uint32_t u3 = __float_as_uint(__fadd_rn(__uint_as_float(c[1]), M));
    const uint32_t u4 = __float_as_uint(__fadd_rn(__uint_as_float(c[2]), M));
    const uint32_t u5 = __float_as_uint(__fadd_rn(__uint_as_float(c[3]), M));
    const int c6 = __float2int_rn(__uint_as_float(c[4]));
    // round(C_7 + C_8 / 256 [+ C_9 / 65536]): each FP32 step rounds below a
    // quarter unit (|C_7 + ...| < 2^23)
    float low = __fmaf_rn(__uint_as_float(c[6]), 0.00390625f, __uint_as_float(c[5]));
    if (D == 7) low = __fmaf_rn(__uint_as_float(c[D]), 1.52587890625e-5f, low);
    const int c78 = __float2int_rn(low);
    // u4 2^24 + u5 2^16 carry the offsets 0x4B400000 (2^24 + 2^16) = 0x4B8B40 2^32,
    // taken off H: H = C_2 256 + C_3 - 0x4B8B40 (mod 2^32), and Y is exact mod 2^64
    const int H = (int)(u2 * 256u + u3 - (257u * 0x4B400000u + 0x4B8B40u));
    // C products (each one 32 x 32 + 64 multiply-add; the PTX mad.wide form
    // measured two instructions)
    long long Y = (long long)(int)u5 * (1 << 16) + (long long)(c6 * 256 + c78);   // |C_6 256 + c78| < 2^31
    Y += (long long)(int)u4 * (1 << 24);
    return Y + ((long long)H << 32);
}

// Y as a double, its exponent shifted by eadj = (E_r + F_n - 56) << 20.
__device__ __forceinline__ double finish_y(long long Y, int eadj) {
    const double y = __ll2double_rn(Y);
    const int hi = __double2hiint(y);
    return __hiloint2double(hi == 0 ? 0 : hi + eadj, __double2loint(y));
}

// (i, j0, j1) of the MMAs of one K-step and half, in issue order: (1,1) and
// (2,1..D) start the sums C_2 .. C_{D+2}, then (1,2..D) and (i,1..D+2-i) for
// i = 3..D add to them.
template <int D>
struct MmaTable {
    int i[D + 1], j0[D + 1], j1[D + 1];
    constexpr MmaTable() : i(), j0(), j1() {
        i[0] = 1; j0[0] = 1; j1[0] = 1;
        i[1] = 2; j0[1] = 1; j1[1] = D;
        i[2] = 1; j0[2] = 2; j1[2] = D;
        for (int m = 3; m <= D; ++m) {
            i[m] = m;
            j0[m] = 1;
            j1[m] = D + 2 - m;
        }
    }
};

// IEEE binary16 bits of an integer of magnitude below 2048 (exact).
inline uint16_t fp16_bits(int d) {
    if (d == 0) return 0;
    const uint16_t sign = d < 0 ? 0x8000u : 0u;
    unsigned m = (unsigned)(d < 0 ? -d : d);
    int e = 0;
    while ((m >> (e + 1)) != 0) ++e;                     // m in [2^e, 2^(e+1))
    const unsigned frac = (m << (10 - e)) & 0x3FFu;
    return (uint16_t)(sign | ((unsigned)(e + 15) << 10) | frac);
}

// The executing thread's arrival on the mbarrier, announcing `bytes` of
// asynchronous copies that complete on it.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}
// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to this CTA's shared memory, completion counted on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}
// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from this CTA's shared memory to global memory, in the thread's current
// bulk group (bulk_commit, then bulk_wait_all before the memory is reused).
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

}  // namespace oz
}  // namespace qe
