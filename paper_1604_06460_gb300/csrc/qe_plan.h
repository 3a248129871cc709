// Emulate-vs-simulate choice for subroutines (Sec. III, Sec. IV-C).
#pragma once
#include "qe_internal.h"

namespace qe {

// Analytic single-GPU costs (seconds), restating the paper's performance
// models (Eq. for T_FFT and T_QFT, Sec. III-B) for one device: the network
// terms vanish, the memory terms count the bytes each pass moves.
double analytic_qft_simulate(const qe_state* s, int m);
double analytic_qft_emulate(const qe_state* s, int m);
double analytic_add_simulate(const qe_state* s, int m, uint64_t c);
double analytic_add_emulate(const qe_state* s, int m);

double analytic_mul_simulate(const qe_state* s, int N);
double analytic_mul_emulate(const qe_state* s, int N);

bool choose_emulate_qft(qe_state* s, int lo, int m);
bool choose_emulate_mul(qe_state* s, int N);
bool choose_emulate_add(qe_state* s, int m, const int* qubits, uint64_t c);

}  // namespace qe
