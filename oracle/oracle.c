/*
 * Oracle: a plain, slow, FP64 CPU restatement of what the state-vector path
 * of "High Performance Emulation of Quantum Circuits" (Haener, Steiger,
 * Smelyanskiy, Troyer, 2016) computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark load this library.  It shares no code, header or
 * table with the CUDA path and must never be used as a fallback for it.
 *
 * Conventions (readings of the paper, stated once here):
 *   - A state of n qubits is 2^n complex amplitudes alpha_i (Sec. II, the
 *     state-vector equation); qubit q is bit q of the index i (little-endian).
 *     Sec. II's Kronecker example writes qubit 0 as the leftmost factor; this
 *     library instead follows Sec. III-B, where the high-order qubits are the
 *     ones with large index stride.
 *   - A k-qubit gate is a 2^k x 2^k complex matrix, row-major, whose row and
 *     column index carries bit j <-> qubits[j].
 *   - Every function is the definition written out, loop by loop; sums of
 *     many terms use Neumaier's compensated summation.
 *   - Gate application may run its independent amplitude groups on several
 *     host threads (OpenMP, when the compiler provides it); each group is
 *     still computed by the same loop, so the arithmetic is unchanged.
 */
#define _USE_MATH_DEFINES
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Host threads used by the gate loops (1 without OpenMP). */
void or_set_threads(int t) {
#ifdef _OPENMP
    omp_set_num_threads(t > 0 ? t : 1);
#else
    (void)t;
#endif
}
int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Compensated summation (Neumaier 1974): s + c carries the running sum. */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nsum_val(const nsum* a) { return a->s + a->c; }

/* ------------------------------------------------------------------ */
/* Bit helpers: scatter the bits of c onto the positions qubits[0..k-1]. */
static uint64_t deposit(uint64_t c, int k, const int* qubits) {
    uint64_t x = 0;
    for (int j = 0; j < k; ++j)
        if ((c >> j) & 1u) x |= (uint64_t)1 << qubits[j];
    return x;
}
/* Gather the bits at positions qubits[0..k-1] of x into a k-bit value. */
static uint64_t extract(uint64_t x, int k, const int* qubits) {
    uint64_t c = 0;
    for (int j = 0; j < k; ++j)
        if ((x >> qubits[j]) & 1u) c |= (uint64_t)1 << j;
    return c;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its published
 * definition: 10 rounds of two 32x32->64 multiplications with the constants
 * M0 = 0xD2511F53, M1 = 0xCD9E8D57 and a Weyl key schedule with
 * W0 = 0x9E3779B9, W1 = 0xBB67AE85. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One complex Gaussian sample per amplitude index i: Philox with counter
 * (lo32(i), hi32(i), 0, 0) and key (lo32(seed), hi32(seed)); two 53-bit
 * uniforms u1 in (0,1], u2 in [0,1) from words (0,1) and (2,3); Box-Muller
 * gives re = r cos(2 pi u2), im = r sin(2 pi u2), r = sqrt(-2 ln u1). */
static cplx gaussian_amplitude(uint64_t seed, uint64_t i) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), 0u, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    uint64_t a = ((uint64_t)w[1] << 32) | w[0];
    uint64_t b = ((uint64_t)w[3] << 32) | w[2];
    double u1 = (double)((a >> 11) + 1) * 0x1.0p-53;
    double u2 = (double)(b >> 11) * 0x1.0p-53;
    double r = sqrt(-2.0 * log(u1));
    double th = 2.0 * M_PI * u2;
    return r * cos(th) + I * (r * sin(th));
}

/* Sum over i of |alpha_i|^2, compensated. */
double or_norm2(const cplx* psi, int n) {
    nsum acc = {0.0, 0.0};
    uint64_t dim = (uint64_t)1 << n;
    for (uint64_t i = 0; i < dim; ++i) {
        nsum_add(&acc, creal(psi[i]) * creal(psi[i]));
        nsum_add(&acc, cimag(psi[i]) * cimag(psi[i]));
    }
    return nsum_val(&acc);
}

/* |0...0>: alpha_0 = 1, all others 0 (Sec. II). */
void or_init_zero(cplx* psi, int n) {
    uint64_t dim = (uint64_t)1 << n;
    for (uint64_t i = 0; i < dim; ++i) psi[i] = 0.0;
    psi[0] = 1.0;
}

/* i.i.d. complex Gaussian amplitudes, then divided by the compensated norm
 * so that sum_i |alpha_i|^2 = 1 (Sec. II normalisation condition). */
void or_init_gaussian(cplx* psi, int n, uint64_t seed) {
    uint64_t dim = (uint64_t)1 << n;
    for (uint64_t i = 0; i < dim; ++i) psi[i] = gaussian_amplitude(seed, i);
    double inv = 1.0 / sqrt(or_norm2(psi, n));
    for (uint64_t i = 0; i < dim; ++i) psi[i] *= inv;
}

/* The same amplitudes for an index range [i0, i0+cnt), unnormalised, so
 * that samples of a state too large for host memory can be regenerated. */
void or_gaussian_slice(cplx* out, uint64_t seed, uint64_t i0, uint64_t cnt) {
    for (uint64_t t = 0; t < cnt; ++t) out[t] = gaussian_amplitude(seed, i0 + t);
}

/* ------------------------------------------------------------------ */
/* A k-qubit gate (Sec. II): the 2^n x 2^n matrix is the identity on every
 * qubit except qubits[], so it acts as U on each group of 2^k amplitudes
 * that agree on all other bits. */
void or_apply_gate(cplx* psi, int n, int k, const int* qubits, const cplx* U) {
    uint64_t dim = (uint64_t)1 << n, K = (uint64_t)1 << k;
    uint64_t gate_mask = deposit(K - 1, k, qubits);
#pragma omp parallel
    {
        cplx* v = (cplx*)malloc(K * sizeof(cplx));   /* this thread's copy of one group */
#pragma omp for schedule(static)
        for (uint64_t x = 0; x < dim; ++x) {
            if (x & gate_mask) continue;          /* x is the base of a group */
            for (uint64_t c = 0; c < K; ++c) v[c] = psi[x | deposit(c, k, qubits)];
            for (uint64_t r = 0; r < K; ++r) {
                cplx acc = 0.0;
                for (uint64_t c = 0; c < K; ++c) acc += U[r * K + c] * v[c];
                psi[x | deposit(r, k, qubits)] = acc;
            }
        }
        free(v);
    }
}

/* A gate U on targets[] applied only where every control qubit is 1
 * (Table I's CNOT and CR are the one-control cases). */
void or_apply_controlled(cplx* psi, int n, int nc, const int* controls, int k,
                         const int* targets, const cplx* U) {
    uint64_t dim = (uint64_t)1 << n, K = (uint64_t)1 << k;
    uint64_t cmask = 0;
    for (int j = 0; j < nc; ++j) cmask |= (uint64_t)1 << controls[j];
    uint64_t tmask = deposit(K - 1, k, targets);
#pragma omp parallel
    {
        cplx* v = (cplx*)malloc(K * sizeof(cplx));
#pragma omp for schedule(static)
        for (uint64_t x = 0; x < dim; ++x) {
            if ((x & tmask) || (x & cmask) != cmask) continue;
            for (uint64_t c = 0; c < K; ++c) v[c] = psi[x | deposit(c, k, targets)];
            for (uint64_t r = 0; r < K; ++r) {
                cplx acc = 0.0;
                for (uint64_t c = 0; c < K; ++c) acc += U[r * K + c] * v[c];
                psi[x | deposit(r, k, targets)] = acc;
            }
        }
        free(v);
    }
}

/* Multi-controlled NOT: where every control is 1, exchange the amplitudes
 * of the two basis states that differ in the target bit. */
void or_apply_mcx(cplx* psi, int n, int nc, const int* controls, int target) {
    uint64_t dim = (uint64_t)1 << n;
    uint64_t cmask = 0, t = (uint64_t)1 << target;
    for (int j = 0; j < nc; ++j) cmask |= (uint64_t)1 << controls[j];
#pragma omp parallel for schedule(static)
    for (uint64_t x = 0; x < dim; ++x) {
        if ((x & t) || (x & cmask) != cmask) continue;
        cplx tmp = psi[x];
        psi[x] = psi[x | t];
        psi[x | t] = tmp;
    }
}

/* ------------------------------------------------------------------ */
/* exp(+-2 pi i t / 2^m) for an integer 0 <= t < 2^m, with t reduced exactly
 * in integers so that the angle never carries the size of k*l. */
static cplx unit_root(uint64_t t, int m, int sign) {
    double th = 2.0 * M_PI * ldexp((double)t, -m);
    return cos(th) + I * (sign * sin(th));
}

/* QFT on the contiguous register [lo, lo+m) (Sec. III-B): for every
 * assignment of the other qubits, with register value k = sum_j bit(lo+j) 2^j,
 *   alpha_l -> 2^{-m/2} sum_k alpha_k exp(+2 pi i k l / 2^m),
 * and the inverse with the opposite sign.  Direct O(4^m) summation. */
void or_qft_dft(cplx* psi, int n, int lo, int m, int inverse) {
    uint64_t dim = (uint64_t)1 << n, M = (uint64_t)1 << m;
    uint64_t stride = (uint64_t)1 << lo;
    uint64_t reg_mask = (M - 1) << lo;
    int sign = inverse ? -1 : 1;
    double scale = 1.0 / sqrt((double)M);
    cplx* in = (cplx*)malloc(M * sizeof(cplx));
    for (uint64_t x = 0; x < dim; ++x) {
        if (x & reg_mask) continue;
        for (uint64_t k = 0; k < M; ++k) in[k] = psi[x + k * stride];
        for (uint64_t l = 0; l < M; ++l) {
            nsum re = {0, 0}, im = {0, 0};
            for (uint64_t k = 0; k < M; ++k) {
                cplx term = in[k] * unit_root((k * l) & (M - 1), m, sign);
                nsum_add(&re, creal(term));
                nsum_add(&im, cimag(term));
            }
            psi[x + l * stride] = scale * (nsum_val(&re) + I * nsum_val(&im));
        }
    }
    free(in);
}

/* One output amplitude of that QFT, at global index `index` (its register
 * bits give l), from the untouched input psi.  The phase
 * exp(2 pi i t / 2^m) is split as exp(2 pi i (t_hi 2^h) / 2^m) *
 * exp(2 pi i t_lo / 2^m) with two tables of 2^h and 2^(m-h) roots, which is
 * exponent addition and only changes rounding. */
void or_qft_amplitude(const cplx* psi, int n, int lo, int m, int inverse,
                      uint64_t index, double* out_re, double* out_im) {
    (void)n;
    uint64_t M = (uint64_t)1 << m, stride = (uint64_t)1 << lo;
    uint64_t reg_mask = (M - 1) << lo;
    uint64_t base = index & ~reg_mask;
    uint64_t l = (index & reg_mask) >> lo;
    int sign = inverse ? -1 : 1;
    int h = m / 2;
    uint64_t H = (uint64_t)1 << h, Lw = (uint64_t)1 << (m - h);
    cplx* thi = (cplx*)malloc(Lw * sizeof(cplx));
    cplx* tlo = (cplx*)malloc(H * sizeof(cplx));
    for (uint64_t a = 0; a < Lw; ++a) thi[a] = unit_root(a << h, m, sign);
    for (uint64_t b = 0; b < H; ++b) tlo[b] = unit_root(b, m, sign);
    nsum re = {0, 0}, im = {0, 0};
    for (uint64_t k = 0; k < M; ++k) {
        uint64_t t = (k * l) & (M - 1);
        cplx term = psi[base + k * stride] * (thi[t >> h] * tlo[t & (H - 1)]);
        nsum_add(&re, creal(term));
        nsum_add(&im, cimag(term));
    }
    double scale = 1.0 / sqrt((double)M);
    *out_re = scale * nsum_val(&re);
    *out_im = scale * nsum_val(&im);
    free(thi);
    free(tlo);
}

/* The QFT as the gate circuit of Sec. III-B: Hadamards and conditional
 * phase shifts CR(theta) = diag(1,1,1,e^{i theta}) (Table I), then the
 * qubit-order reversal that puts the output in natural order.  Register
 * qubit j is lo+j.  Forward: for j = m-1 down to 0, H on j, then CR with
 * control l < j and angle pi / 2^{j-l}; then swap j <-> m-1-j.  Inverse:
 * the adjoint, i.e. the same gates in reverse order with negated angles. */
static void apply_h(cplx* psi, int n, int q) {
    const double s = 1.0 / sqrt(2.0);
    cplx H[4] = {s, s, s, -s};
    or_apply_gate(psi, n, 1, &q, H);
}
static void apply_cr(cplx* psi, int n, int control, int target, double theta) {
    int c = control;
    cplx P[4] = {1.0, 0.0, 0.0, cos(theta) + I * sin(theta)};
    or_apply_controlled(psi, n, 1, &c, 1, &target, P);
}
static void apply_swap(cplx* psi, int n, int a, int b) {
    int q[2] = {a, b};
    cplx S[16] = {1, 0, 0, 0, 0, 0, 1, 0, 0, 1, 0, 0, 0, 0, 0, 1};
    or_apply_gate(psi, n, 2, q, S);
}
void or_qft_circuit(cplx* psi, int n, int lo, int m, int inverse) {
    if (!inverse) {
        for (int j = m - 1; j >= 0; --j) {
            apply_h(psi, n, lo + j);
            for (int l = j - 1; l >= 0; --l)
                apply_cr(psi, n, lo + l, lo + j, M_PI / ldexp(1.0, j - l));
        }
        for (int j = 0; j < m / 2; ++j) apply_swap(psi, n, lo + j, lo + m - 1 - j);
    } else {
        for (int j = 0; j < m / 2; ++j) apply_swap(psi, n, lo + j, lo + m - 1 - j);
        for (int j = 0; j < m; ++j) {
            for (int l = 0; l < j; ++l)
                apply_cr(psi, n, lo + l, lo + j, -M_PI / ldexp(1.0, j - l));
            apply_h(psi, n, lo + j);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Emulated addition of a classical constant (Sec. III-A): the register
 * value r (bit j <-> qubits[j]) becomes (r + c) mod 2^m, i.e. the amplitude
 * at basis index x moves to the index x' with that register value. */
void or_add_const(cplx* psi, int n, int m, const int* qubits, uint64_t c) {
    uint64_t dim = (uint64_t)1 << n;
    uint64_t M = (m >= 64) ? ~(uint64_t)0 : (((uint64_t)1 << m) - 1);
    uint64_t reg_mask = deposit(M, m, qubits);
    cplx* out = (cplx*)malloc(dim * sizeof(cplx));
    for (uint64_t x = 0; x < dim; ++x) {
        uint64_t r = extract(x, m, qubits);
        uint64_t r2 = (r + c) & M;
        uint64_t x2 = (x & ~reg_mask) | deposit(r2, m, qubits);
        out[x2] = psi[x];
    }
    memcpy(psi, out, dim * sizeof(cplx));
    free(out);
}

/* The same addition as a reversible gate circuit (the simulated baseline):
 * adding 2^j increments the sub-register (qubits[j], ..., qubits[m-1]) by
 * one, and an increment of a b-bit register flips bit i when all lower
 * bits are 1, taken from the top bit down.  One increment per set bit of c. */
void or_add_const_circuit(cplx* psi, int n, int m, const int* qubits, uint64_t c) {
    int* ctl = (int*)malloc((m > 0 ? m : 1) * sizeof(int));
    for (int j = 0; j < m; ++j) {
        if (!((c >> j) & 1u)) continue;
        for (int i = m - 1; i >= j; --i) {
            int nc = 0;
            for (int l = j; l < i; ++l) ctl[nc++] = qubits[l];
            or_apply_mcx(psi, n, nc, ctl, qubits[i]);
        }
    }
    free(ctl);
}

/* ------------------------------------------------------------------ */
/* Emulated multiplication and division (Sec. III-A).  Three registers a, b,
 * c of N qubits each (bit j of a value <-> qa[j], qb[j], qc[j]).
 *
 * Multiplication: the paper maps (a, b, 0) to (a, b, ab), the product kept to
 * the N bits of c.  On every basis state the emulator adds the product:
 * c -> (c + a b) mod 2^N, which is that map on c = 0, a permutation of the
 * basis states, and what the repeated add-and-shift circuit computes.
 *
 * Division: the paper maps (a, b, 0) to (r, b, a / b) with a = (a / b) b + r.
 * On every basis state the emulator runs the restoring division, for i from
 * N - 1 down to 0:  c_i ^= [b != 0 and a >= b 2^i];  then, if c_i = 1,
 * a -> (a - b 2^i) mod 2^N.  Each step is a permutation, so the whole map is
 * one; on c = 0 it leaves the quotient in c and the remainder in a (b = 0:
 * nothing changes). */
static uint64_t mul_target(uint64_t a, uint64_t b, uint64_t c, int N) {
    uint64_t mask = (N >= 64) ? ~(uint64_t)0 : (((uint64_t)1 << N) - 1);
    return (c + a * b) & mask;
}
static void div_target(uint64_t* a, uint64_t b, uint64_t* c, int N) {
    uint64_t mask = (N >= 64) ? ~(uint64_t)0 : (((uint64_t)1 << N) - 1);
    for (int i = N - 1; i >= 0; --i) {
        uint64_t bi = b << i;                               /* b 2^i, N + i < 64 bits */
        uint64_t t = (b != 0 && *a >= bi) ? 1u : 0u;
        *c ^= t << i;
        if ((*c >> i) & 1u) *a = (*a - bi) & mask;
    }
}
void or_mul(cplx* psi, int n, int N, const int* qa, const int* qb, const int* qc) {
    uint64_t dim = (uint64_t)1 << n, M = ((uint64_t)1 << N) - 1;
    uint64_t cmask = deposit(M, N, qc);
    cplx* out = (cplx*)malloc(dim * sizeof(cplx));
    for (uint64_t x = 0; x < dim; ++x) {
        uint64_t a = extract(x, N, qa), b = extract(x, N, qb), c = extract(x, N, qc);
        uint64_t x2 = (x & ~cmask) | deposit(mul_target(a, b, c, N), N, qc);
        out[x2] = psi[x];
    }
    memcpy(psi, out, dim * sizeof(cplx));
    free(out);
}
void or_div(cplx* psi, int n, int N, const int* qa, const int* qb, const int* qc) {
    uint64_t dim = (uint64_t)1 << n, M = ((uint64_t)1 << N) - 1;
    uint64_t amask = deposit(M, N, qa), cmask = deposit(M, N, qc);
    cplx* out = (cplx*)malloc(dim * sizeof(cplx));
    for (uint64_t x = 0; x < dim; ++x) {
        uint64_t a = extract(x, N, qa), b = extract(x, N, qb), c = extract(x, N, qc);
        div_target(&a, b, &c, N);
        uint64_t x2 = (x & ~(amask | cmask)) | deposit(a, N, qa) | deposit(c, N, qc);
        out[x2] = psi[x];
    }
    memcpy(psi, out, dim * sizeof(cplx));
    free(out);
}

/* The multiplication as a gate circuit (the simulated baseline, Sec. III-A's
 * repeated addition and shift): c += a b is c += 2^(i+j) for every pair of
 * set bits a_i, b_j with i + j < N, i.e. an increment of the sub-register
 * (qc[i+j], ..., qc[N-1]) under the two controls a_i, b_j; an increment
 * flips qc[k] when all lower bits of the sub-register are 1, from the top
 * bit down (multi-controlled NOTs). */
void or_mul_circuit(cplx* psi, int n, int N, const int* qa, const int* qb, const int* qc) {
    int* ctl = (int*)malloc((N + 2) * sizeof(int));
    for (int i = 0; i < N; ++i)
        for (int j = 0; i + j < N; ++j)
            for (int k = N - 1; k >= i + j; --k) {
                int nc = 0;
                ctl[nc++] = qa[i];
                ctl[nc++] = qb[j];
                for (int l = i + j; l < k; ++l) ctl[nc++] = qc[l];
                or_apply_mcx(psi, n, nc, ctl, qc[k]);
            }
    free(ctl);
}

/* ------------------------------------------------------------------ */
/* Expectation value of a Hermitian Pauli sum (Sec. III-D):
 *   <psi| sum_t w_t P_t |psi>,  P_t = tensor over q of
 *   I, X, Z, Y for (x_q, z_q) = (0,0), (1,0), (0,1), (1,1).
 * Each P_t |psi> is built by applying the 2x2 Pauli matrices one qubit at a
 * time, then <psi|P_t psi> is summed with compensation. */
double or_expectation(const cplx* psi, int n, int nterms, const uint64_t* xmask,
                      const uint64_t* zmask, const double* coeff) {
    uint64_t dim = (uint64_t)1 << n;
    const cplx X[4] = {0, 1, 1, 0};
    const cplx Y[4] = {0, -I, I, 0};
    const cplx Z[4] = {1, 0, 0, -1};
    cplx* phi = (cplx*)malloc(dim * sizeof(cplx));
    nsum total = {0, 0};
    for (int t = 0; t < nterms; ++t) {
        memcpy(phi, psi, dim * sizeof(cplx));
        for (int q = 0; q < n; ++q) {
            int xb = (int)((xmask[t] >> q) & 1u), zb = (int)((zmask[t] >> q) & 1u);
            if (xb && zb) or_apply_gate(phi, n, 1, &q, Y);
            else if (xb) or_apply_gate(phi, n, 1, &q, X);
            else if (zb) or_apply_gate(phi, n, 1, &q, Z);
        }
        nsum re = {0, 0};
        for (uint64_t x = 0; x < dim; ++x) {
            cplx p = conj(psi[x]) * phi[x];
            nsum_add(&re, creal(p));
        }
        nsum_add(&total, coeff[t] * nsum_val(&re));
    }
    free(phi);
    return nsum_val(&total);
}

/* Marginal probabilities of the qubits[] (Sec. II, Born rule |alpha_i|^2):
 * out[r] = sum over x whose bits at qubits[] spell r of |alpha_x|^2. */
void or_probs(const cplx* psi, int n, int m, const int* qubits, double* out) {
    uint64_t dim = (uint64_t)1 << n, M = (uint64_t)1 << m;
    nsum* acc = (nsum*)calloc(M, sizeof(nsum));
    for (uint64_t x = 0; x < dim; ++x) {
        uint64_t r = extract(x, m, qubits);
        nsum_add(&acc[r], creal(psi[x]) * creal(psi[x]));
        nsum_add(&acc[r], cimag(psi[x]) * cimag(psi[x]));
    }
    for (uint64_t r = 0; r < M; ++r) out[r] = nsum_val(&acc[r]);
    free(acc);
}

/* ------------------------------------------------------------------ */
/* Measurement (Sec. II): measuring the qubits[] yields the value r of their
 * bits with probability P(r), the sum of |alpha_x|^2 over the x whose bits
 * at qubits[] spell r (all n qubits in order: P(i) = |alpha_i|^2).  Sampling
 * by the inverse of the cumulative distribution, with the uniforms u[s] in
 * [0, 1) given: shot s is the smallest r whose cumulative probability
 * exceeds u[s] times the total; if rounding leaves none, the largest r with
 * P(r) > 0.  The cumulative sums are compensated. */
void or_sample(const cplx* psi, int n, int m, const int* qubits, int nshots, const double* u,
               uint64_t* out) {
    uint64_t M = (uint64_t)1 << m;
    double* P = (double*)malloc(M * sizeof(double));
    double* cum = (double*)malloc(M * sizeof(double));
    or_probs(psi, n, m, qubits, P);
    nsum acc = {0.0, 0.0};
    uint64_t last = 0;
    for (uint64_t r = 0; r < M; ++r) {
        nsum_add(&acc, P[r]);
        cum[r] = nsum_val(&acc);
        if (P[r] > 0.0) last = r;
    }
    double total = cum[M - 1];
    for (int s = 0; s < nshots; ++s) {
        double target = u[s] * total;
        uint64_t r = 0;
        while (r < M && !(cum[r] > target)) ++r;
        out[s] = (r < M) ? r : last;
    }
    free(P);
    free(cum);
}

/* The state after a measurement of qubits[] gave `outcome` (Sec. II's
 * collapse): amplitudes whose bits at qubits[] differ from the outcome
 * become 0, the others are divided by sqrt(p), p the outcome's probability
 * (compensated sum).  Returns p; for p = 0 the state is left unchanged. */
double or_collapse(cplx* psi, int n, int m, const int* qubits, uint64_t outcome) {
    uint64_t dim = (uint64_t)1 << n;
    nsum acc = {0.0, 0.0};
    for (uint64_t x = 0; x < dim; ++x) {
        if (extract(x, m, qubits) != outcome) continue;
        nsum_add(&acc, creal(psi[x]) * creal(psi[x]));
        nsum_add(&acc, cimag(psi[x]) * cimag(psi[x]));
    }
    double p = nsum_val(&acc);
    if (p == 0.0) return 0.0;
    double inv = 1.0 / sqrt(p);
    for (uint64_t x = 0; x < dim; ++x) {
        if (extract(x, m, qubits) != outcome) psi[x] = 0.0;
        else psi[x] *= inv;
    }
    return p;
}

/* ------------------------------------------------------------------ */
/* The cost model's network (a multilayer perceptron; not from the paper,
 * which chooses between emulation and simulation by performance models and
 * measured cross-overs, Sec. III-B and Sec. IV-D).  Layout of params:
 * W1[h1][d] b1[h1] W2[h2][h1] b2[h2] W3[h2] b3, tanh hidden units, linear
 * output:  y = W3 . tanh(W2 tanh(W1 x + b1) + b2) + b3.
 * Loss over a batch: L = (1/N) sum_s (y_s - t_s)^2. */
static void mlp_sizes(int d, int h1, int h2, int* o1, int* o2, int* o3, int* o4, int* o5, int* o6) {
    *o1 = 0;                 /* W1 */
    *o2 = *o1 + h1 * d;      /* b1 */
    *o3 = *o2 + h1;          /* W2 */
    *o4 = *o3 + h2 * h1;     /* b2 */
    *o5 = *o4 + h2;          /* W3 */
    *o6 = *o5 + h2;          /* b3 */
}

int or_mlp_param_count(int d, int h1, int h2) { return h1 * d + h1 + h2 * h1 + h2 + h2 + 1; }

void or_mlp_forward(const double* p, int d, int h1, int h2, const double* X, int n, double* y) {
    int oW1, ob1, oW2, ob2, oW3, ob3;
    mlp_sizes(d, h1, h2, &oW1, &ob1, &oW2, &ob2, &oW3, &ob3);
    double* a1 = (double*)malloc(sizeof(double) * h1);
    double* a2 = (double*)malloc(sizeof(double) * h2);
    for (int s = 0; s < n; ++s) {
        const double* x = X + (size_t)s * d;
        for (int j = 0; j < h1; ++j) {
            double z = p[ob1 + j];
            for (int i = 0; i < d; ++i) z += p[oW1 + j * d + i] * x[i];
            a1[j] = tanh(z);
        }
        for (int j = 0; j < h2; ++j) {
            double z = p[ob2 + j];
            for (int i = 0; i < h1; ++i) z += p[oW2 + j * h1 + i] * a1[i];
            a2[j] = tanh(z);
        }
        double out = p[ob3];
        for (int i = 0; i < h2; ++i) out += p[oW3 + i] * a2[i];
        y[s] = out;
    }
    free(a1);
    free(a2);
}

/* Gradient of L with respect to every parameter (backpropagation: the chain
 * rule applied layer by layer, d tanh(z)/dz = 1 - tanh(z)^2).  Returns L. */
double or_mlp_grad(const double* p, int d, int h1, int h2, const double* X, const double* t,
                   int n, double* grad) {
    int oW1, ob1, oW2, ob2, oW3, ob3;
    mlp_sizes(d, h1, h2, &oW1, &ob1, &oW2, &ob2, &oW3, &ob3);
    const int np = or_mlp_param_count(d, h1, h2);
    for (int k = 0; k < np; ++k) grad[k] = 0.0;
    double* a1 = (double*)malloc(sizeof(double) * h1);
    double* a2 = (double*)malloc(sizeof(double) * h2);
    double* d1 = (double*)malloc(sizeof(double) * h1);
    double* d2 = (double*)malloc(sizeof(double) * h2);
    double loss = 0.0;
    for (int s = 0; s < n; ++s) {
        const double* x = X + (size_t)s * d;
        for (int j = 0; j < h1; ++j) {
            double z = p[ob1 + j];
            for (int i = 0; i < d; ++i) z += p[oW1 + j * d + i] * x[i];
            a1[j] = tanh(z);
        }
        for (int j = 0; j < h2; ++j) {
            double z = p[ob2 + j];
            for (int i = 0; i < h1; ++i) z += p[oW2 + j * h1 + i] * a1[i];
            a2[j] = tanh(z);
        }
        double y = p[ob3];
        for (int i = 0; i < h2; ++i) y += p[oW3 + i] * a2[i];
        const double r = y - t[s];
        loss += r * r / n;
        const double dy = 2.0 * r / n;                 /* dL/dy */
        grad[ob3] += dy;
        for (int i = 0; i < h2; ++i) {
            grad[oW3 + i] += dy * a2[i];
            d2[i] = dy * p[oW3 + i] * (1.0 - a2[i] * a2[i]);
        }
        for (int j = 0; j < h2; ++j) {
            grad[ob2 + j] += d2[j];
            for (int i = 0; i < h1; ++i) grad[oW2 + j * h1 + i] += d2[j] * a1[i];
        }
        for (int i = 0; i < h1; ++i) {
            double acc = 0.0;
            for (int j = 0; j < h2; ++j) acc += p[oW2 + j * h1 + i] * d2[j];
            d1[i] = acc * (1.0 - a1[i] * a1[i]);
        }
        for (int j = 0; j < h1; ++j) {
            grad[ob1 + j] += d1[j];
            for (int i = 0; i < d; ++i) grad[oW1 + j * d + i] += d1[j] * x[i];
        }
    }
    free(a1);
    free(a2);
    free(d1);
    free(d2);
    return loss;
}
