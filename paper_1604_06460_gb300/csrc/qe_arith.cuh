// Device arithmetic for the state-vector kernels.
//
// GB300 executes FP64 at about 1/64 of its FP32 rate (and converts between
// the two on the same slow pipe), so complex128 states are computed in
// "double-float" arithmetic: every double is split into a pair of floats
// (hi, lo) with integer instructions only, products and sums use the
// error-free transformations TwoProd (Dekker 1971, via fused multiply-add)
// and TwoSum (Knuth, TAOCP vol. 2), and results are joined back into doubles.
// Each conversion keeps 47 significant bits; a k-qubit update loses a few
// units of 2^-46 relative to the group's norm, which meets an FP64-grade
// error budget of 1e-12 absolute over thousands of gates.
//
// Three policies share one interface:
//   F32  - complex64 state, FP32 arithmetic;
//   DF   - complex128 state, double-float arithmetic on the FP32 pipes;
//   F64  - complex128 state, native FP64 (kept as the measured baseline).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qe {

// ------------------------------------------------------------------ floats
struct df { float h, l; };   // value = h + l

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

// Split a double into (hi, lo) floats using integer instructions only.
// hi carries the leading 24 significant bits (truncated), lo the next 23
// (rounded); values below 2^-80 in magnitude lose lo, below 2^-126 become 0.
__device__ __forceinline__ df d2df(double d) {
    uint32_t lo = (uint32_t)__double2loint(d), hi = (uint32_t)__double2hiint(d);
    uint32_t e = (hi >> 20) & 0x7FFu;
    uint32_t sign = hi & 0x80000000u;
    // (hi << 3) | (lo >> 29): exponent low bits + top 23 mantissa bits
    uint32_t body = __funnelshift_l(lo, hi, 3);
    // float exponent = e - 896; for e in [897, 1150] its 8 bits equal the
    // low byte of e with bit 7 flipped (896 = 3*256 + 128)
    uint32_t hb = ((body & 0x7FFFFFFFu) ^ 0x40000000u) | sign;
    uint32_t N = ((lo & 0x1FFFFFFFu) + 32u) >> 6;                 // 23-bit residual, rounded
    float f = __fsub_rn(__uint_as_float(0x4B000000u + N), 8388608.0f);  // == N exactly
    float scale = __uint_as_float(((e - 942u) << 23) | sign);        // +-2^(e-1069)
    df r;
    r.h = (e >= 897u) ? __uint_as_float(hb) : 0.0f;
    r.l = (e >= 943u) ? __fmul_rn(f, scale) : 0.0f;
    return r;
}

// Exact widening of a normal float to double with integer instructions;
// zero and subnormal floats become (signed) zero.
__device__ __forceinline__ double f2d_exact(float f) {
    uint32_t b = __float_as_uint(f);
    uint32_t sign = b & 0x80000000u;
    uint32_t H = sign | (((b & 0x7FFFFFFFu) >> 3) + (896u << 20));
    uint32_t L = b << 29;
    bool zero = ((b >> 23) & 0xFFu) == 0u;
    return __hiloint2double((int)(zero ? sign : H), (int)(zero ? 0u : L));
}

// Join (hi, lo) into the nearest double: one FP64 addition of exact parts.
__device__ __forceinline__ double df2d(float h, float l) {
    return __dadd_rn(f2d_exact(h), f2d_exact(l));
}

// s + e (an unevaluated sum being accumulated) += a * b, a and b double-float.
__device__ __forceinline__ void df_acc(float& s, float& e, df a, df b) {
    float ph = fmul(a.h, b.h);
    float pl = __fmaf_rn(a.h, b.h, -ph);
    pl = __fmaf_rn(a.h, b.l, pl);
    pl = __fmaf_rn(a.l, b.h, pl);
    float t = fadd(s, ph);
    float bb = fsub(t, s);
    float err = fadd(fsub(s, fsub(t, bb)), fsub(ph, bb));
    s = t;
    e = fadd(e, fadd(err, pl));
}
// Same with the product negated.
__device__ __forceinline__ void df_acc_neg(float& s, float& e, df a, df b) {
    df na = {-a.h, -a.l};
    df_acc(s, e, na, b);
}
// Normalise (s, e) so that |lo| <= ulp(hi)/2 (Fast2Sum, |s| >= |e| holds here
// up to the rare exact cancellation, where the result is still exact).
__device__ __forceinline__ df df_norm(float s, float e) {
    float h = fadd(s, e);
    float l = fsub(e, fsub(h, s));
    return df{h, l};
}

// Start an accumulation with s + e = a * b (exact product, FP32 cross terms).
__device__ __forceinline__ void df_first(float& s, float& e, df a, df b) {
    s = fmul(a.h, b.h);
    e = __fmaf_rn(a.h, b.h, -s);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
}
// a + b and a - b for double-floats (TwoSum of the leading parts).
__device__ __forceinline__ df df_add(df a, df b) {
    float s = fadd(a.h, b.h);
    float bb = fsub(s, a.h);
    float e = fadd(fsub(a.h, fsub(s, bb)), fsub(b.h, bb));
    e = fadd(e, fadd(a.l, b.l));
    return df_norm(s, e);
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df{-b.h, -b.l}); }

// ------------------------------------------------------------ policies
// Each policy provides:
//   S        storage type of one amplitude (float2 / double2)
//   V        in-register / shared-memory value of one amplitude
//   M        matrix entry / twiddle (same type as V)
//   A        accumulator of a complex dot product
//   load(S) -> V, store(V) -> S, mat(re, im) -> M on the host,
//   from_d(re, im) -> M on the device, zero() -> A, mac(A&, M, V),
//   mac_first(A&, M, V) (the first term of a dot product, A uninitialised),
//   out(A) -> S, add/sub(V, V) -> V, cmul(M, V) -> V.
struct F32 {
    using S = float2;
    using V = float2;
    using M = float2;
    struct A { float re, im; };
    static constexpr int bytes = 8;
    __device__ __forceinline__ static V load(S s) { return s; }
    __device__ __forceinline__ static S store(V v) { return v; }
    __host__ __forceinline__ static M mat(double re, double im) {
        return make_float2((float)re, (float)im);
    }
    __device__ __forceinline__ static M from_d(double re, double im) {
        return make_float2((float)re, (float)im);
    }
    __device__ __forceinline__ static A zero() { return A{0.f, 0.f}; }
    __device__ __forceinline__ static void mac(A& a, M u, V v) {
        a.re = __fmaf_rn(u.x, v.x, a.re);
        a.re = __fmaf_rn(-u.y, v.y, a.re);
        a.im = __fmaf_rn(u.x, v.y, a.im);
        a.im = __fmaf_rn(u.y, v.x, a.im);
    }
    __device__ __forceinline__ static void mac_first(A& a, M u, V v) {
        a.re = __fmaf_rn(-u.y, v.y, fmul(u.x, v.x));
        a.im = __fmaf_rn(u.y, v.x, fmul(u.x, v.y));
    }
    __device__ __forceinline__ static S out(const A& a) { return make_float2(a.re, a.im); }
    __device__ __forceinline__ static V add(V a, V b) { return make_float2(fadd(a.x, b.x), fadd(a.y, b.y)); }
    __device__ __forceinline__ static V sub(V a, V b) { return make_float2(fsub(a.x, b.x), fsub(a.y, b.y)); }
    __device__ __forceinline__ static V cmul(M w, V v) {
        return make_float2(__fmaf_rn(w.x, v.x, -fmul(w.y, v.y)), __fmaf_rn(w.x, v.y, fmul(w.y, v.x)));
    }
};

struct F64 {
    using S = double2;
    using V = double2;
    using M = double2;
    struct A { double re, im; };
    static constexpr int bytes = 16;
    __device__ __forceinline__ static V load(S s) { return s; }
    __device__ __forceinline__ static S store(V v) { return v; }
    __host__ __forceinline__ static M mat(double re, double im) { return make_double2(re, im); }
    __device__ __forceinline__ static M from_d(double re, double im) { return make_double2(re, im); }
    __device__ __forceinline__ static A zero() { return A{0.0, 0.0}; }
    __device__ __forceinline__ static void mac(A& a, M u, V v) {
        a.re = __fma_rn(u.x, v.x, a.re);
        a.re = __fma_rn(-u.y, v.y, a.re);
        a.im = __fma_rn(u.x, v.y, a.im);
        a.im = __fma_rn(u.y, v.x, a.im);
    }
    __device__ __forceinline__ static void mac_first(A& a, M u, V v) {
        a.re = __fma_rn(-u.y, v.y, __dmul_rn(u.x, v.x));
        a.im = __fma_rn(u.y, v.x, __dmul_rn(u.x, v.y));
    }
    __device__ __forceinline__ static S out(const A& a) { return make_double2(a.re, a.im); }
    __device__ __forceinline__ static V add(V a, V b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
    __device__ __forceinline__ static V sub(V a, V b) { return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y)); }
    __device__ __forceinline__ static V cmul(M w, V v) {
        return make_double2(__fma_rn(w.x, v.x, -__dmul_rn(w.y, v.y)), __fma_rn(w.x, v.y, __dmul_rn(w.y, v.x)));
    }
};

struct DF {
    using S = double2;
    // 16-byte aligned so that a value moves in one 128-bit shared-memory access
    struct alignas(16) V { df re, im; };
    using M = V;
    struct A { float rs, re_, is, ie; };   // real (s,e), imaginary (s,e)
    static constexpr int bytes = 16;
    __device__ __forceinline__ static V load(S s) { return V{d2df(s.x), d2df(s.y)}; }
    __device__ __forceinline__ static S store(V v) {
        return make_double2(df2d(v.re.h, v.re.l), df2d(v.im.h, v.im.l));
    }
    __host__ __forceinline__ static M mat(double re, double im) {
        float rh = (float)re, ih = (float)im;
        return M{df{rh, (float)(re - (double)rh)}, df{ih, (float)(im - (double)ih)}};
    }
    __device__ __forceinline__ static M from_d(double re, double im) { return M{d2df(re), d2df(im)}; }
    __device__ __forceinline__ static A zero() { return A{0.f, 0.f, 0.f, 0.f}; }
    __device__ __forceinline__ static void mac(A& a, const M& u, const V& v) {
        df_acc(a.rs, a.re_, u.re, v.re);
        df_acc_neg(a.rs, a.re_, u.im, v.im);
        df_acc(a.is, a.ie, u.re, v.im);
        df_acc(a.is, a.ie, u.im, v.re);
    }
    // first product of a dot product: no addition, so no TwoSum
    __device__ __forceinline__ static void mac_first(A& a, const M& u, const V& v) {
        df_first(a.rs, a.re_, u.re, v.re);
        df_acc_neg(a.rs, a.re_, u.im, v.im);
        df_first(a.is, a.ie, u.re, v.im);
        df_acc(a.is, a.ie, u.im, v.re);
    }
    // (s, e) need no normalisation: one FP64 addition of the exactly
    // widened parts rounds s + e correctly
    __device__ __forceinline__ static S out(const A& a) {
        return make_double2(df2d(a.rs, a.re_), df2d(a.is, a.ie));
    }
    __device__ __forceinline__ static V add(const V& a, const V& b) { return V{df_add(a.re, b.re), df_add(a.im, b.im)}; }
    __device__ __forceinline__ static V sub(const V& a, const V& b) { return V{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
    __device__ __forceinline__ static V cmul(const M& w, const V& v) {
        float rs, re_, is, ie;
        df_first(rs, re_, w.re, v.re);
        df_acc_neg(rs, re_, w.im, v.im);
        df_first(is, ie, w.re, v.im);
        df_acc(is, ie, w.im, v.re);
        return V{df_norm(rs, re_), df_norm(is, ie)};
    }
};

// ------------------------------------------------------------ bit helpers
// Insert a zero bit at each position of sorted[0..cnt-1] (ascending).
__host__ __device__ __forceinline__ uint64_t insert_zero_bits(uint64_t t, const uint8_t* sorted, int cnt) {
    for (int j = 0; j < cnt; ++j) {
        uint64_t p = sorted[j];
        uint64_t low = t & ((1ull << p) - 1ull);
        t = ((t >> p) << (p + 1)) | low;
    }
    return t;
}

}  // namespace qe
