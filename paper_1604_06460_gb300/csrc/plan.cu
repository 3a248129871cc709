// Analytic cross-over rule between emulation and simulation.
//
// Sec. III-B models the simulated QFT by its memory traffic, 4 N n^2 bytes
// for n^2/2 controlled phases that touch a quarter of the state plus the
// Hadamards, and the FFT by 5 N n flops at an FFT efficiency; the expected
// speedup is n * FLOPS_achieved / B_mem (Sec. IV-C).  On one GPU the network
// terms drop out.  The constants below are this device's measured copy
// bandwidth and the FP32-pipe throughput that the FFT butterflies use.
#include <algorithm>
#include <cmath>

#include "qe_mlp.h"
#include "qe_plan.h"

namespace qe {

namespace {
constexpr double kBandwidth = 6.7e12;      // bytes/s, device copy bandwidth
constexpr double kFp32Ops = 3.4e13;        // FP32-pipe instructions/s
constexpr double kFp64Ops = 5.9e11;        // FP64-pipe instructions/s
// Seconds of arithmetic per complex element per radix-2 FFT stage: about 46
// FP32-pipe instructions in double-float arithmetic, 5 in FP32, 4.5 FP64
// instructions in the FP64 mode.
double stage_time(const qe_state* s) {
    if (s->dtype == QE_C64) return 5.0 / kFp32Ops;
    return s->arith == QE_ARITH_FP64 ? 4.5 / kFp64Ops : 46.0 / kFp32Ops;
}
// Seconds of arithmetic per amplitude of a dense 1-qubit pass (8 FP64
// instructions in the FP64 mode; the FP32 pipes keep up with memory otherwise).
double one_qubit_alu(const qe_state* s) { return c128_f64(s) ? 8.0 / kFp64Ops : 0.0; }
}  // namespace

double analytic_qft_simulate(const qe_state* s, int m) {
    const double N = std::ldexp(1.0, s->n), B = s->dtype == QE_C128 ? 16.0 : 8.0;
    const double h = m * std::max(2.0 * N * B / kBandwidth, N * one_qubit_alu(s));    // m Hadamards
    const double cr_bytes = 0.5 * m * (m - 1) * 2.0 * (N / 4.0) * B;  // quarter-state phases
    const double rev_bytes = m > 1 ? 2.0 * N * B : 0.0;
    return h + (cr_bytes + rev_bytes) / kBandwidth;
}

double analytic_qft_emulate(const qe_state* s, int m) {
    const double N = std::ldexp(1.0, s->n), B = s->dtype == QE_C128 ? 16.0 : 8.0;
    // FP64 mode, digit passes on the tensor cores: G = m / d block passes,
    // G - 1 twiddle passes (about 6 FP64 instructions an amplitude) and the
    // digit reversal
    const int d = (m % 5 == 0) ? 5 : (m % 4 == 0) ? 4 : (m % 3 == 0) ? 3 : 0;
    if (c128_f64(s) && s->c128_tc && s->tensor_cores && s->n >= 12 && d > 0) {
        const int G = m / d;
        const double pass = 2.0 * N * B / kBandwidth;
        return G * pass + (G - 1) * std::max(pass, 6.0 * N / kFp64Ops) + (G > 1 ? pass : 0.0);
    }
    const int per_pass = s->dtype == QE_C128 ? 12 : 13;
    const int passes = (m + per_pass - 1) / per_pass + (m > per_pass ? 1 : 0);
    const double mem = passes * 2.0 * N * B / kBandwidth;
    const double alu = N * m * stage_time(s);
    return mem > alu ? mem : alu;
}

double analytic_add_simulate(const qe_state* s, int m, uint64_t c) {
    const double N = std::ldexp(1.0, s->n), B = s->dtype == QE_C128 ? 16.0 : 8.0;
    double bytes = 0.0;
    for (int j = 0; j < m; ++j) {
        if (!((c >> j) & 1ull)) continue;
        for (int i = m - 1; i >= j; --i) bytes += 2.0 * std::ldexp(N, -(i - j)) * B;
    }
    return bytes / kBandwidth;
}

double analytic_add_emulate(const qe_state* s, int m) {
    (void)m;
    const double N = std::ldexp(1.0, s->n), B = s->dtype == QE_C128 ? 16.0 : 8.0;
    return 2.0 * N * B / kBandwidth;
}

// The multiplication's gate circuit: for every pair i + j < N an increment
// of c[i+j ..] under controls a_i, b_j, i.e. multi-controlled NOTs on qubit
// c_k with 2 + (k - i - j) controls, each touching 2^-(controls) of the state.
double analytic_mul_simulate(const qe_state* s, int N) {
    const double Nn = std::ldexp(1.0, s->n), B = s->dtype == QE_C128 ? 16.0 : 8.0;
    double bytes = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; i + j < N; ++j)
            for (int k = N - 1; k >= i + j; --k) bytes += 2.0 * std::ldexp(Nn, -(2 + k - i - j)) * B;
    return bytes / kBandwidth;
}

// One permutation pass (two through the scratch buffer when a plane exceeds
// shared memory).
double analytic_mul_emulate(const qe_state* s, int N) {
    const double Nn = std::ldexp(1.0, s->n), B = s->dtype == QE_C128 ? 16.0 : 8.0;
    const double plane = std::ldexp(B, N);
    return (plane <= 65536.0 ? 2.0 : 4.0) * Nn * B / kBandwidth;
}

bool choose_emulate_mul(qe_state* s, int N) {
    if (s->policy == QE_POLICY_EMULATE) return true;
    if (s->policy == QE_POLICY_SIMULATE) return false;
    return analytic_mul_emulate(s, N) <= analytic_mul_simulate(s, N);
}

// Learned choice: predicted log-times of the two paths.
static bool model_prefers_first(qe_state* s, int op_a, int op_b, int lo, int hi, int m, uint64_t c) {
    float X[2 * kCostFeatures], y[2];
    cost_features(op_a, s->n, s->dtype, 0, lo, hi, m, c, X);
    cost_features(op_b, s->n, s->dtype, 0, lo, hi, m, c, X + kCostFeatures);
    mlp_predict(s->model, X, 2, y);
    return y[0] <= y[1];
}

bool choose_emulate_qft(qe_state* s, int lo, int m) {
    if (s->policy == QE_POLICY_EMULATE) return true;
    if (s->policy == QE_POLICY_SIMULATE) return false;
    if (s->policy == QE_POLICY_AUTO && s->model)
        return model_prefers_first(s, kOpQftEmulate, kOpQftSimulate, lo, lo + m - 1, m, 0);
    return analytic_qft_emulate(s, m) <= analytic_qft_simulate(s, m);
}

bool choose_emulate_add(qe_state* s, int m, const int* qubits, uint64_t c) {
    if (s->policy == QE_POLICY_EMULATE) return true;
    if (s->policy == QE_POLICY_SIMULATE) return false;
    if (s->policy == QE_POLICY_AUTO && s->model) {
        int lo = qubits[0], hi = qubits[0];
        for (int j = 1; j < m; ++j) { lo = std::min(lo, qubits[j]); hi = std::max(hi, qubits[j]); }
        return model_prefers_first(s, kOpAddEmulate, kOpAddSimulate, lo, hi, m, c);
    }
    return analytic_add_emulate(s, m) <= analytic_add_simulate(s, m, c);
}

}  // namespace qe
