/*
 * qe.h -- C ABI of the GB300 state-vector emulator.
 *
 * The library updates one state vector of 2^n complex amplitudes resident in
 * GPU memory (Haener, Steiger, Smelyanskiy, Troyer, "High Performance
 * Emulation of Quantum Circuits", 2016, Sec. II).  Gates are applied as
 * dense 2^k x 2^k blocks; whole subroutines are emulated instead of being
 * simulated gate by gate (Sec. III): the QFT as an FFT (Sec. III-B), the
 * addition of a classical constant as an amplitude permutation (Sec. III-A),
 * and expectation values / probabilities computed directly (Sec. III-D).
 *
 * Conventions used by every call
 *   - qubit q is bit q of the amplitude index (little-endian); amplitudes are
 *     interleaved (re, im) in one contiguous allocation of 2^n elements;
 *   - QE_C128 stores complex128 (16 B/amplitude); by default it is computed
 *     in the FP64 mode (qe_set_arith: 53-bit FP64 arithmetic, dense blocks
 *     as exact products of 56-bit splittings on the tensor cores), or in the
 *     faster double-float mode on request.  QE_C64 stores complex64
 *     (8 B/amplitude) and is computed in FP32;
 *   - a k-qubit matrix is 2^k x 2^k complex, row-major, interleaved doubles
 *     (2 * 4^k values), host memory, whose row/column bit j <-> qubits[j];
 *   - all device work is enqueued on the state's CUDA stream; calls that
 *     return host values synchronise that stream; host arrays passed in are
 *     copied before the call returns, so the caller keeps ownership;
 *   - every call returns QE_OK (0) or a negative status; no C++ exception
 *     crosses the ABI; qe_last_error() describes the most recent failure of
 *     the calling thread.  Invalid arguments return QE_ERR_ARG and leave the
 *     state untouched.
 *   - gates may be queued for fusion; qe_flush() (and every call that reads
 *     or transforms the whole state) applies them first.
 */
#ifndef QE_H
#define QE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qe_state qe_state;

typedef enum { QE_C64 = 0, QE_C128 = 1 } qe_dtype;

typedef enum {
    QE_OK = 0,
    QE_ERR_ARG = -1,          /* invalid argument (range, duplicate qubit, NULL) */
    QE_ERR_OOM = -2,          /* device allocation failed */
    QE_ERR_CUDA = -3,         /* a CUDA call failed; see qe_last_error() */
    QE_ERR_TIMEOUT = -4,      /* a bounded device wait gave up */
    QE_ERR_STATE = -5,        /* handle unusable (freed, failed earlier) */
    QE_ERR_UNSUPPORTED = -6   /* a valid request the library does not implement */
} qe_status;

/* Planner policy for subroutines that can be emulated or simulated. */
typedef enum {
    QE_POLICY_AUTO = 0,       /* learned cost model if loaded, else analytic rule */
    QE_POLICY_ANALYTIC = 1,   /* analytic cross-over (Sec. III-B performance models) */
    QE_POLICY_EMULATE = 2,    /* always the classical shortcut */
    QE_POLICY_SIMULATE = 3    /* always the gate-by-gate circuit */
} qe_policy;

/* Allocate a state handle for n qubits (1 <= n <= 34) of the given dtype and
 * initialise it to |0...0>.  dev_ptr == NULL: the library allocates
 * 2^n * sizeof(amplitude) bytes and frees them in qe_free_state.  Otherwise
 * dev_ptr is caller-owned device memory of at least that many bytes (e.g. a
 * torch tensor's storage), 256-byte aligned, which the library borrows for
 * the handle's lifetime.  stream is a cudaStream_t (NULL = legacy default).
 * Sec. II: the state is a vector of 2^n amplitudes with sum |alpha_i|^2 = 1. */
int qe_alloc_state(int n, int dtype, void* dev_ptr, size_t bytes, void* stream,
                   qe_state** out);

/* Release the handle (and memory the library allocated).  NULL is a no-op. */
int qe_free_state(qe_state* s);

/* Report n, dtype and the device address of amplitude 0. */
int qe_state_info(const qe_state* s, int* n, int* dtype, void** dev_ptr);

/* Reset to the basis state |index> (Sec. II): alpha_index = 1, all others 0.
 * QE_ERR_ARG if index >= 2^n. */
int qe_init_basis(qe_state* s, uint64_t index);

/* Fill with i.i.d. standard complex Gaussian amplitudes and normalise by the
 * compensated FP64 norm.  Amplitude i draws Philox4x32-10 (Salmon et al.,
 * SC'11) with counter (lo32(i), hi32(i), 0, 0) and key (lo32(seed),
 * hi32(seed)); words (0,1) give u1 in (0,1], words (2,3) give u2 in [0,1)
 * (53-bit uniforms); Box-Muller: re + i im = sqrt(-2 ln u1) e^{2 pi i u2}. */
int qe_init_random(qe_state* s, uint64_t seed);

/* Copy count amplitudes between host memory (in the state's dtype,
 * interleaved) and the state, starting at amplitude offset.  Pending gates
 * are applied before a read and before an overwrite.  QE_ERR_ARG if
 * offset + count > 2^n, or host is NULL with count > 0. */
int qe_set_amplitudes(qe_state* s, const void* host, uint64_t offset, uint64_t count);
int qe_get_amplitudes(qe_state* s, void* host, uint64_t offset, uint64_t count);

/* Apply a k-qubit gate (1 <= k <= 5) given as a dense 2^k x 2^k matrix
 * (Sec. II; Table I lists the standard ones).  qubits[] are k distinct
 * qubits < n.  The planner exploits structure (Sec. II): a matrix that acts
 * as the identity unless some of its qubits are 1 runs as a controlled gate
 * touching only that fraction of the state; a diagonal matrix with a single
 * non-unit entry (e.g. CR(theta) = diag(1,1,1,e^{i theta})) touches only the
 * amplitudes of that entry (a quarter of the state, Sec. III-B); 0/1
 * permutation matrices (X, CNOT, SWAP) move amplitudes bit-exactly.
 * Consecutive gates are fused into blocks of up to max_k qubits
 * (qe_set_policy) and applied at the next flush. */
int qe_apply_gate(qe_state* s, int k, const int* qubits, const double* matrix);

/* Apply U (2^k x 2^k, 0 <= k <= 2) on targets[] only where every one of the
 * nc controls[] is 1 (multi-controlled gates such as the Toffoli / MCX used
 * by reversible arithmetic, Sec. III).  k = 0 multiplies the controlled
 * amplitudes by the scalar matrix[0].  QE_ERR_ARG for k > 2, a repeated
 * qubit, or a qubit that is both control and target. */
int qe_apply_controlled(qe_state* s, int nc, const int* controls, int k,
                        const int* targets, const double* matrix);

/* Quantum Fourier transform on the contiguous register [lo, lo+m)
 * (Sec. III-B): for every assignment of the other qubits, with register
 * value k = sum_j bit(lo+j) 2^j,
 *     alpha_l -> 2^{-m/2} sum_k alpha_k exp(+2 pi i k l / 2^m),
 * natural output order; inverse != 0 uses the opposite sign.  Emulated as an
 * in-place FFT, or simulated as m Hadamards, m(m-1)/2 CR gates and the
 * qubit reversal, as the policy decides.  QE_ERR_ARG unless m >= 1, lo >= 0
 * and lo + m <= n. */
int qe_apply_qft(qe_state* s, int lo, int m, int inverse);

/* Add the classical constant c to the m-qubit register qubits[] (bit j of
 * the register value <-> qubits[j]), modulo 2^m (Sec. III-A): the amplitude
 * at x moves to x' whose register value is (r + c) mod 2^m.  Emulated as one
 * in-place permutation (bit-exact), or simulated as a ripple of
 * multi-controlled NOTs, as the policy decides.  1 <= m <= n. */
int qe_apply_add_const(qe_state* s, int m, const int* qubits, uint64_t c);

/* Multiplication and division of two N-qubit registers into a third
 * (Sec. III-A), 1 <= N <= 16, the 3N qubits qa[], qb[], qc[] distinct and
 * < n (bit j of a register value <-> qa[j], qb[j], qc[j]).
 *   qe_apply_mul: c -> (c + a b) mod 2^N on every basis state: the paper's
 *     (a, b, 0) -> (a, b, ab) with the product kept to N bits, extended to
 *     c != 0 as the repeated add-and-shift circuit computes it.  Emulated as
 *     one permutation, or simulated as that circuit of multi-controlled NOTs
 *     (an increment of c[i+j ..] under controls a_i, b_j for every i + j < N),
 *     as the policy decides.
 *   qe_apply_div: the restoring division, for i = N-1 down to 0:
 *     c_i ^= [b != 0 and a >= b 2^i], then a -> (a - b 2^i) mod 2^N if c_i = 1;
 *     on c = 0 this is the paper's (a, b, 0) -> (a mod b, b, a div b) (b = 0
 *     leaves the state unchanged).  Emulated only: QE_ERR_UNSUPPORTED under
 *     QE_POLICY_SIMULATE.
 * Both are permutations of the amplitudes, bit-exact.  A permutation whose
 * plane (the 2^N values of c, or the 2^(2N) of (a, c)) exceeds 64 KB goes
 * through a device scratch buffer of at most 1 GiB owned by the state.
 * QE_ERR_ARG for N out of range, a qubit >= n, a repeated qubit or
 * overlapping registers. */
int qe_apply_mul(qe_state* s, int N, const int* qa, const int* qb, const int* qc);
int qe_apply_div(qe_state* s, int N, const int* qa, const int* qb, const int* qc);

/* <psi| sum_t coeff[t] P_t |psi> for Pauli strings P_t given by bit masks
 * over the qubits: (x,z) = (0,0) I, (1,0) X, (0,1) Z, (1,1) Y (Sec. III-D:
 * the expectation computed in one step instead of by repeated sampling).
 * complex128 states, terms whose X/Y bits below qubit 12 lie in one of the
 * triples {0,1,2} .. {9,10,11} and whose X/Y bits above it number at most
 * three (every term of a nearest-neighbour Ising or Heisenberg model): in
 * fixed point: every component rounded once to the nearest multiple of
 * 2^(e - 54), 2^e the power of two just above the largest component among
 * the 4096 amplitudes read with it (tiles below 2^-959 flush to zero),
 * products and tile sums exact in integers, tile results combined in FP64
 * with compensation.  Other terms and complex64 states: FP64 (FP64 mode) or
 * double-float products, compensated sums.  *out receives the real
 * value (0 for nterms = 0).  QE_ERR_ARG for nterms < 0, a mask naming a
 * qubit >= n or a non-finite coefficient; QE_ERR_TIMEOUT if a copy wait of
 * the fixed-point kernel ran out (bounded waits). */
int qe_expectation(qe_state* s, int nterms, const uint64_t* xmask,
                   const uint64_t* zmask, const double* coeff, double* out);

/* Marginal probabilities of the m qubits[] (Sec. II, |alpha_i|^2):
 * out[r] (host, 2^m doubles, 1 <= m <= 16) = sum over x whose bits at
 * qubits[] spell r of |alpha_x|^2.  FP64 compensated accumulation. */
int qe_probs(qe_state* s, int m, const int* qubits, double* out);

/* Phase estimation by emulation (Sec. III-C).  A dense 2^k x 2^k complex
 * matrix is held in a complex128 state of 2k qubits, column-major: entry
 * (i, j) is amplitude (j << k) | i.
 *   qe_init_identity: the identity matrix (s has 2 nsys qubits).  Applying a
 *     circuit's gates to qubits [0, nsys) of it afterwards applies them to
 *     every column, so the state becomes the circuit's dense matrix U: the
 *     emulator's O(G 2^(2n)) construction of U.
 *   qe_matmul: c = a b for three such states of the same width (c distinct
 *     from a and b): one squaring of the repeated squaring
 *     U^(2^i) = U^(2^(i-1)) U^(2^(i-1)), O(2^(3k)).  For k >= 6 on the
 *     tensor cores: every input rounded once to 56 bits of its row's (a's
 *     rows) or column's (b's columns) largest magnitude, exact digit
 *     products, exact 128-bit sums, one rounding to FP64 (each element within
 *     2^k rowmax colmax 2^-51 of the exact product; rows or columns below
 *     2^-920 flush to zero); the workspace (about 0.9 x the three matrices'
 *     bytes) is kept with c.  For k < 6, or with the environment variable
 *     QE_GEMM_F64=1, FP64 fused multiply-adds.  Synchronises c's stream;
 *     QE_ERR_TIMEOUT if a tensor-core wait ran out (bounded waits).
 *   qe_qpe_emulate: coherent phase estimation on s with the system register
 *     [0, nsys) and b ancillas [nsys, nsys + b) (nsys + b <= n): Hadamards on
 *     the ancillas, ancilla j applies U^(2^j) (u holds U, 2 nsys qubits) to
 *     the system register where it is 1 -- the powers by repeated squaring,
 *     each applied as one dense product -- then the inverse QFT on the
 *     ancillas (emulated).  With the ancillas in |0> and an eigenvector of U
 *     with eigenvalue exp(2 pi i k / 2^b), the ancilla register ends in |k>.
 *     The squarings are qe_matmul's (tensor cores for nsys >= 6, workspace
 *     kept with s); the controlled products run on the tensor cores too when
 *     nsys >= 6 and the rows they act on (2^(n - nsys - 1)) number at least
 *     128, else with FP64 fused multiply-adds.
 *     Allocates two temporary matrices (QE_ERR_OOM if that fails) and uses
 *     the state's scratch; synchronises the stream.
 * All three want complex128 states; QE_ERR_ARG for mismatched widths or a
 * result that would overwrite an input. */
int qe_init_identity(qe_state* s, int nsys);
int qe_matmul(qe_state* c, qe_state* a, qe_state* b);
int qe_qpe_emulate(qe_state* s, int nsys, int b, qe_state* u);

/* Measurement (Sec. II: the value r of the measured qubits' bits occurs with
 * probability P(r) = sum of |alpha_x|^2 over the x whose bits spell r;
 * Sec. III-D: an emulator draws all the samples it needs from one copy of
 * the state).
 *   qe_sample: nshots samples, by the inverse of the cumulative
 *     distribution with the caller's uniforms[s] in [0, 1) (host, nshots
 *     values; the caller owns the randomness, so samples are reproducible):
 *     outcomes[s] (host) is the smallest r whose cumulative probability
 *     exceeds uniforms[s] times the total, or, when rounding leaves none, the
 *     largest r with P(r) > 0.  m = 0 measures all n qubits (outcome = basis
 *     index, qubits ignored); 1 <= m <= 16 measures qubits[] (outcome bit j
 *     <-> qubits[j]).  Sums are FP64 in a fixed order; the state is not
 *     changed.  QE_ERR_ARG for m out of range, bad qubits, nshots < 0, NULL
 *     arrays with nshots > 0 or a uniform outside [0, 1).
 *   qe_collapse: the state after measuring qubits[] (1 <= m <= n) gave
 *     `outcome` (bit j <-> qubits[j]): amplitudes whose bits differ become 0,
 *     the others are divided by sqrt(p), p the outcome's probability (FP64
 *     sum), which *probability receives (may be NULL).  QE_ERR_ARG, state
 *     untouched, for bad qubits, outcome >= 2^m or p = 0. */
int qe_sample(qe_state* s, int m, const int* qubits, int nshots, const double* uniforms, uint64_t* outcomes);
int qe_collapse(qe_state* s, int m, const int* qubits, uint64_t outcome, double* probability);

/* sum_i |alpha_i|^2 in compensated FP64. */
int qe_norm2(qe_state* s, double* out);

/* Apply queued gates / wait for all work on the state's stream.  qe_flush
 * launches the fused passes as they are planned and, before returning, waits
 * for the last tensor-core pass: QE_ERR_TIMEOUT if one of them reported a
 * bounded wait that ran out (the remaining queued gates are then dropped). */
int qe_flush(qe_state* s);
int qe_sync(qe_state* s);

/* Choose the emulate-vs-simulate policy and the largest fused block width
 * (1 <= max_k <= 5) the gate fuser may form; max_k = 0 selects the default
 * (5 where the tensor cores take 3-5-qubit blocks, i.e. n >= 12, else 2 for
 * complex128 and 4 for complex64).  QE_ERR_ARG for other values. */
int qe_set_policy(qe_state* s, int policy, int max_k);

/* Arithmetic of a complex128 state.  The paper's CPU kernels compute in
 * double complex (Sec. IV-A); GB300 runs FP64 at about 1/64 of its FP32
 * rate, so the library offers two modes:
 *   QE_ARITH_FP64 (default): every operation at least as accurate as FP64
 *     arithmetic.  Dense 3-5-qubit blocks (n >= 12) run on the tensor cores
 *     as exact products of integer digits: every input is rounded to 2^-56 of
 *     its 32-amplitude group's scale and every matrix entry to 2^-56 of its
 *     row's, the digit products are summed exactly and each output is
 *     rounded once to a double, so an output is within 2^-50 of the product
 *     of the two scales -- inside the worst-case rounding error of an FP64
 *     dot product of the same 64 real terms.  1-2-qubit, diagonal,
 *     controlled and smaller-state gates, the FFT, expectation values and
 *     probabilities run in native FP64 (53-bit significands).
 *   QE_ARITH_DF64: the fast mode.  Values are split into pairs of floats
 *     (double-float, 47 significant bits; magnitudes below 2^-80 keep only
 *     the leading float, below 2^-126 become zero, and magnitudes of 2^127
 *     or more are not representable), dense 3-5-qubit blocks use 48-bit
 *     splittings on the tensor cores (inputs rounded to 2^-48 of their group's
 *     scale), and reductions sum float-float partials of about 44 bits.  For
 *     unitary gates on normalised states the results stay within 1e-12 of
 *     FP64 arithmetic over thousands of gates; other inputs get no such bound.
 * Both modes give bit-identical permutations.  Switching flushes the queued
 * gates and synchronises the stream; the fusion width follows the mode's
 * default unless one was set with qe_set_policy.  QE_ERR_ARG for another
 * value. */
typedef enum { QE_ARITH_FP64 = 0, QE_ARITH_DF64 = 1 } qe_arith;
int qe_set_arith(qe_state* s, int arith);
int qe_get_arith(const qe_state* s, int* arith);

/* Counters since the last reset: kernel launches, full-state passes, and the
 * algorithmic bytes those passes move (reads + writes, see Sec. III-B's
 * byte count for the controlled phase). */
typedef struct {
    uint64_t launches;
    uint64_t passes;
    double algorithmic_bytes;
    uint64_t gates_applied;
    uint64_t fused_blocks;
} qe_stats;
int qe_get_stats(const qe_state* s, qe_stats* out);
int qe_reset_stats(qe_state* s);

/* ---------------------------------------------------------------- batch
 * Many small parameterised circuits in one persistent launch, replayed as a
 * CUDA graph.  Circuit c acts on nqubits[c] qubits (1 <= n <= 23 for
 * QE_C128, <= 25 for QE_C64), starts from |0...0> and applies `layers` times:
 * RY(theta) then RZ(phi) on every qubit q (RY(t) = [[cos t/2, -sin t/2],
 * [sin t/2, cos t/2]], RZ as in Table I), then CZ on (q, q+1) for
 * q = 0..n-2.  angles holds, circuit after circuit, layer after layer, qubit
 * after qubit, the pair (theta, phi).  The result of circuit c is the energy
 * <psi_c| sum_{i<n-1} Z_i Z_{i+1} + hx sum_i X_i |psi_c> (open transverse-field
 * Ising chain; the expectation computed directly, Sec. III-D).  qe_batch_create
 * copies the inputs, allocates the device states of circuits too large for
 * one CTA's shared memory, builds the work queue and captures the graph.
 * qe_batch_run replays it, synchronises the stream and writes count energies
 * to host memory (energies may be NULL to discard them); it returns
 * QE_ERR_TIMEOUT if a work item's bounded wait for the items it depends on
 * ran out.  qe_batch_tune times the candidate tile schedules (tile bits,
 * tiles per work item, threads per CTA: 128, 256 or 512) reps times each and
 * keeps the fastest; the chosen plan is returned through the optional
 * pointers.  qe_batch_set_plan sets one: 4 <= tile_bits <= 12 (13 for
 * QE_C64) with 2 tile_bits - 1 >= the largest n, tiles_per_item >= 1.
 * qe_batch_info reports the algorithmic HBM bytes of one run and the number
 * of work items.  QE_ERR_ARG: count or layers < 1, NULL nqubits or angles, a
 * qubit count out of range, a non-finite angle or field, an unknown dtype, a
 * plan outside the ranges above, reps < 1.  The stream is borrowed (NULL =
 * legacy default stream); the batch owns its device memory, which
 * qe_batch_free releases. */
typedef struct qe_batch qe_batch;
int qe_batch_create(int count, const int* nqubits, int layers, const double* angles,
                    double hx, int dtype, void* stream, qe_batch** out);
int qe_batch_run(qe_batch* b, double* energies);
int qe_batch_tune(qe_batch* b, int reps, int* tile_bits, int* tiles_per_item, int* threads);
int qe_batch_set_plan(qe_batch* b, int tile_bits, int tiles_per_item, int threads);
/* Arithmetic of a complex128 batch: QE_ARITH_DF64 (the default; double-float
 * gates on the FP32 pipes and float-pair energy sums) or QE_ARITH_FP64
 * (native FP64 gates and FP64 energy sums; the FP64 pipe bounds it).  Rebuilds
 * the work queue and graph with the current plan; complex64 batches ignore
 * it.  QE_ERR_ARG for another value. */
int qe_batch_set_arith(qe_batch* b, int arith);
int qe_batch_info(const qe_batch* b, double* hbm_bytes, int* items);
int qe_batch_free(qe_batch* b);

/* ------------------------------------------------------------ cost model
 * A small network (16 features -> h1 -> h2 tanh units -> 1) that predicts
 * log(milliseconds) of an operation, trained on timings the emulator itself
 * measures.  With QE_POLICY_AUTO and a model attached (qe_set_cost_model) the
 * planner uses it to choose emulation or simulation for each QFT / addition
 * and the fusion width of each flushed gate sequence; without a model it
 * falls back to the analytic rule.  The choice never changes a result beyond
 * the arithmetic's rounding.  Forward, backward and Adam steps run in the
 * library's own kernels on a private stream.
 *   qe_cost_features: the 16 features of an operation: op (0 gate pass,
 *     1 QFT emulated, 2 QFT simulated, 3 addition emulated, 4 addition
 *     simulated), n, dtype, k (gate width), lo/hi (lowest/highest qubit
 *     touched), m (register size), c (the added constant): one-hot op, n/34,
 *     complex128 flag, k/5, log2 bytes/40, lo/n, hi/n, m/n, popcount(c)/m,
 *     the gate count of the subroutine's circuit / n^2 (m + m(m-1)/2 for a
 *     QFT, the sum of m - j over the set bits j of c for an addition), (n-m)/n
 *     and a constant 1;
 *   qe_cost_model_gradient: loss (mean squared error) and its gradient with
 *     respect to all parameters for the samples X[n][16], targets t[n];
 *   qe_cost_model_train: full-batch Adam for `epochs` steps at rate lr;
 *     *loss receives the final training loss;
 *   params: W1[h1][16] b1[h1] W2[h2][h1] b2[h2] W3[h2] b3 (float). */
typedef struct qe_cost_model qe_cost_model;
int qe_cost_model_create(int hidden1, int hidden2, uint64_t seed, qe_cost_model** out);
int qe_cost_model_param_count(const qe_cost_model* m, int* count);
int qe_cost_model_get_params(const qe_cost_model* m, float* params, int count);
int qe_cost_model_set_params(qe_cost_model* m, const float* params, int count);
int qe_cost_model_gradient(qe_cost_model* m, const float* X, const float* t, int n, float* grad,
                           float* loss);
int qe_cost_model_train(qe_cost_model* m, const float* X, const float* t, int n, int epochs,
                        float lr, float* loss);
int qe_cost_model_predict(qe_cost_model* m, const float* X, int n, float* y);
int qe_cost_model_free(qe_cost_model* m);
int qe_cost_features(int op, int n, int dtype, int k, int lo, int hi, int m, uint64_t c,
                     float* features);
/* Attach a model to a state (NULL detaches it) after flushing the queued
 * gates.  The state borrows the model: keep it alive, and do not pass it to
 * qe_cost_model_free, while a state holds it. */
int qe_set_cost_model(qe_state* s, qe_cost_model* model);
/* Fusion width the planner would use for the gates queued now (the state's
 * max_k, or the model's choice under QE_POLICY_AUTO), without applying them. */
int qe_planned_fusion_width(qe_state* s, int* k);

/* Host-only planning (no device work, no state): group ngates uncontrolled
 * gates on n qubits into fused blocks of at most max_k (1..5) qubits exactly
 * as the flush does (Sec. II, gate fusion): each block is the qubit set that
 * absorbs the most gates at the fronts of the per-qubit gate queues; a gate
 * wider than max_k stays a block of its own, and max_k = 1 applies every gate
 * as its own block.  Gate g acts on k[g] (1..5)
 * qubits qubits[5 g + j], j < k[g], with the row-major 2^k x 2^k complex
 * matrix (interleaved re, im doubles) at matrices + mat_offset[g] (doubles).
 * Outputs, for blocks b < *nblocks (in application order): width
 * block_k[b], qubits block_qubits[5 b + j] and matrix block_matrices +
 * 2048 b (row-major, interleaved, width block_k[b]).  QE_ERR_ARG for invalid
 * arguments or when more than cap blocks result (*nblocks then holds the
 * count needed). */
int qe_plan_fusion(int n, int ngates, const int* k, const int* qubits, const double* matrices,
                   const int64_t* mat_offset, int max_k, int cap, int* nblocks, int* block_k,
                   int* block_qubits, double* block_matrices);

/* Per-kernel timing with CUDA events recorded on the state's stream around
 * every launch (measurement aid; the events add a few microseconds per
 * launch).  qe_profile_enable(s, 1) clears earlier records and starts
 * recording; qe_profile_read synchronises the stream and reports, for each
 * kernel name, its launches, the summed event time and the algorithmic bytes
 * those launches move.  *count receives the number of kernel names (at most
 * max are written). */
typedef struct {
    char name[48];
    uint64_t launches;
    double total_ms;
    double bytes;
} qe_kernel_profile;
int qe_profile_enable(qe_state* s, int enable);
int qe_profile_read(qe_state* s, qe_kernel_profile* out, int max, int* count);

/* Marginal probabilities that allocate nothing.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory: code running while another component captures a CUDA graph,
 * processes whose GPU memory belongs entirely to another allocator or arena,
 * and hosts that forbid allocation after start-up.  It computes what
 * qe_probs computes, from a raw state pointer instead of a handle:
 *   state  device pointer to 2^n amplitudes of dtype (QE_C64 / QE_C128);
 *   qubits host array of m distinct qubits < n, 1 <= m <= 16;
 *   out    device pointer to 2^m doubles (written; caller-owned);
 *   stream cudaStream_t the work is enqueued on (NULL = legacy default).
 * It returns after enqueueing (synchronise the stream before reading out).
 * Block partial sums live in one static device array of 65536 (sum,
 * compensation) pairs, 1 MiB, which every GPU that loads the library keeps
 * until the process exits; requests needing more partials than that return
 * QE_ERR_ARG (with m <= 16 none does).  Every call looks up that array's
 * address on the current device (cudaGetSymbolAddress, which allocates
 * nothing); the first call on a device also loads the library's kernels
 * there, so make the first call on each device before any stream capture.  All
 * calls share the array: calls whose work overlaps on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  Every partial a
 * call reads is written earlier by the same call, so nothing needs clearing.
 * Status only (QE_ERR_ARG for bad arguments, QE_ERR_CUDA for a failed
 * launch, which includes an error an earlier CUDA call left pending on the
 * calling thread); qe_last_error() is not updated. */
int qe_probs_noalloc(const void* state, int n, int dtype, int m, const int* qubits,
                     double* out, void* stream);

/* Human-readable description of the calling thread's last failure. */
const char* qe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QE_H */
