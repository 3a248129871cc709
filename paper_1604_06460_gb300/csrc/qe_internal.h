// Host-side declarations shared by the translation units of libqe.
#pragma once
#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qe.h"

namespace qe {

using cd = std::complex<double>;

// Thrown inside the library, caught at the C boundary and turned into a status.
struct Error {
    int status;
    std::string msg;
};
[[noreturn]] void fail(int status, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
#define QE_CUDA(call) ::qe::check_cuda((call), #call)

// A queued (not yet applied) gate.
struct PendingGate {
    int k = 0;                  // number of target qubits
    int q[5] = {0, 0, 0, 0, 0}; // target qubits (matrix bit j <-> q[j])
    uint64_t cmask = 0;         // control qubits (all must be 1)
    std::vector<cd> U;          // 2^k x 2^k row-major
};

struct Stats {
    uint64_t launches = 0, passes = 0, gates = 0, blocks = 0;
    double bytes = 0.0;
};

struct ProfRec {
    const char* tag;
    cudaEvent_t start, stop;
    double bytes;
};

}  // namespace qe

struct qe_state {
    int n = 0;
    int dtype = QE_C128;
    void* d = nullptr;            // amplitudes
    size_t bytes = 0;
    bool owned = false;
    cudaStream_t stream = nullptr;
    int policy = QE_POLICY_AUTO;
    int max_k = 4;
    int arith = QE_ARITH_FP64;    // complex128 arithmetic (qe_set_arith)
    int c128_tc = 1;              // 0: complex128 blocks never on the tensor cores (native FP64 baseline)
    int force_tile = 0;           // 1: dense gates always through shared-memory tiles
    int tensor_cores = 1;         // 4-5 (complex64) / 1-5 or 3-5 (complex128) qubit blocks on tcgen05 (n >= 12)
    qe_cost_model* model = nullptr;   // learned cost model (borrowed), used by QE_POLICY_AUTO
    std::vector<qe::PendingGate> queue;
    // device scratch for reductions, grown on demand
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // digit planes of the tensor-core matrix product, grown on demand
    void* oz_ws = nullptr;
    size_t oz_ws_bytes = 0;
    // pinned host mirror of small results
    double* host_result = nullptr;
    qe::Stats stats;
    // status word of the last tensor-core launch (pinned host copy), checked
    // before the next such launch and at the end of every flush
    uint32_t* status_host = nullptr;
    bool status_pending = false;
    // optional per-launch event timing
    bool profile = false;
    std::vector<qe::ProfRec> prof;
    std::vector<cudaEvent_t> event_pool;
    int magic = 0x51E57A7E;
};

namespace qe {

inline uint64_t dim(const qe_state* s) { return 1ull << s->n; }

// Brackets one kernel launch: counts it, adds its algorithmic bytes and, when
// profiling is on, records CUDA events around it on the state's stream.
class Launch {
  public:
    Launch(qe_state* s, const char* tag, double bytes, bool full_pass = true);
    ~Launch();
  private:
    qe_state* s_;
    int idx_ = -1;
};
void profile_clear(qe_state* s);
inline int amp_bytes(const qe_state* s) { return s->dtype == QE_C128 ? 16 : 8; }
// complex128 computed in native FP64 (the FP64 mode) rather than double-float
inline bool c128_f64(const qe_state* s) { return s->dtype == QE_C128 && s->arith == QE_ARITH_FP64; }
// dense complex128 blocks of at least this many qubits run on the tensor cores
// (7-digit splitting in the FP64 mode, 6-digit in the double-float mode);
// 1-2-qubit blocks stay elementwise (native FP64 or double-float): widened to
// five qubits they would share one scale with 8-16 unrelated groups
inline int c128_tc_kmin(const qe_state*) { return 3; }
int num_sms();
void* ensure_scratch(qe_state* s, size_t bytes);
// the tensor-core matrix product's workspace (at least `bytes`; the state's
// stream is synchronised before an old one is freed)
void* ensure_oz_workspace(qe_state* s, size_t bytes);
// complex matrix products on the tensor cores (7-digit splitting, exact
// 128-bit sums): C (M x N, row-major, ldc) = A (M x K; logical row r is memory
// row r with a 1 inserted at a_rowbit when a_rowbit >= 0) B (K x N, row-major);
// false from the first when the shape is not supported (K a multiple of 32, N
// of 16) or QE_GEMM_F64=1 asks for the FP64 kernel
bool oz_gemm_available(int64_t M, int64_t K, int64_t N);
void oz_zgemm(qe_state* s, double2* C, int64_t ldc, const double2* A, int64_t M, int64_t K, int64_t lda, int a_rowbit,
              const double2* B, int64_t N, int64_t ldb);

// ---- kernels (each launcher enqueues on s->stream and updates s->stats)
void launch_init_basis(qe_state* s, uint64_t index);
void launch_init_random(qe_state* s, uint64_t seed);
void launch_scale(qe_state* s, double factor);

// dense k-qubit gate (1 <= k <= 5) through shared-memory tiles
void launch_gate_dense(qe_state* s, int k, const int* qubits, const cd* U);
// The tensor-core launchers copy their device status word into the state's
// pinned host word after the kernel and mark it pending; complete_pending()
// waits for the stream and raises QE_ERR_TIMEOUT if a launch reported one.
uint32_t* status_word_host(qe_state* s);
void complete_pending(qe_state* s);
// 5-qubit block on a complex64 state with tcgen05 tensor cores (n >= 12)
void launch_gate_tc5(qe_state* s, const int* qubits, const cd* U);
void launch_gate_tc5_c128(qe_state* s, const int* qubits, const cd* U);
// diagonal gate: amplitude x *= d[row(x)] for all x
void launch_gate_diag(qe_state* s, int k, const int* qubits, const cd* d);
// amplitudes with (x & mask) == value are multiplied by phase
void launch_phase_pattern(qe_state* s, uint64_t mask, uint64_t value, cd phase);
// U (k <= 2 targets) applied where all controls in cmask are 1
void launch_controlled(qe_state* s, uint64_t cmask, int k, const int* targets, const cd* U);
// 0/1 permutation within groups of targets, under controls: out[r] = in[perm[r]]
void launch_permute(qe_state* s, uint64_t cmask, int k, const int* targets, const int* perm);

// QFT on register [lo, lo+m) as an FFT
void launch_qft_fft(qe_state* s, int lo, int m, int inverse);
// register-value bit reversal of [lo, lo+m) (bit-exact)
void launch_bitrev(qe_state* s, int lo, int m);

// register + c mod 2^m, register bit j <-> qubits[j]
void launch_add_const(qe_state* s, int m, const int* qubits, uint64_t c);
// emulated multiplication c += a b and restoring division of N-qubit registers
void launch_mul(qe_state* s, int N, const int* qa, const int* qb, const int* qc);
void launch_div(qe_state* s, int N, const int* qa, const int* qb, const int* qc);

// batch of ansatz circuits (struct qe_batch is defined in batch.cu)
void batch_create(qe_batch* b);
void batch_run(qe_batch* b, double* energies);
void batch_set_plan(qe_batch* b, int T, int tiles_per_item, int threads);
void batch_set_arith(qe_batch* b, int arith);
void batch_destroy(qe_batch* b);

// planner
void flush(qe_state* s);
int choose_fusion_width(qe_state* s, const std::vector<PendingGate>& queue);

// reductions (synchronise the stream)
double reduce_norm2(qe_state* s);
double reduce_expectation(qe_state* s, int nterms, const uint64_t* xm, const uint64_t* zm,
                          const double* cf);
void reduce_probs(qe_state* s, int m, const int* qubits, double* out);
// the 2^m marginals into device memory (enqueued only); partial needs room for
// probs_partials_needed(s, m) block partials
uint64_t probs_partials_needed(const qe_state* s, int m);
void reduce_probs_device(qe_state* s, int m, const int* qubits, double2* partial, double* dout);

// phase estimation (Sec. III-C): identity matrix in a 2 nsys-qubit state,
// column-major complex products (FP64), a dense matrix applied to the system
// register [0, nsys) of the rows whose qubit ctrl is set
void launch_init_identity(qe_state* s, int nsys);
void launch_matmul(qe_state* acct, void* c, const void* a, const void* b, int k);
void launch_dense_controlled(qe_state* s, const void* mat, int nsys, int ctrl);

// measurement (Sec. II): inverse-CDF sampling with caller-given uniforms, and
// the collapse onto an outcome
void sample_shots(qe_state* s, int m, const int* qubits, int nshots, const double* u, uint64_t* out);
double collapse(qe_state* s, int m, const int* qubits, uint64_t outcome);

}  // namespace qe
