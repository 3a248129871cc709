// Host-side state of a batch of ansatz circuits (see batch.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/qe.h"

namespace qe {
// Tile schedule of the persistent batch kernel (chosen by qe_batch_tune).
struct BatchPlan {
    int T = 12;              // tile bits: circuits with n <= T run in shared memory
    int tiles_per_item = 4;  // tiles per work item of a large circuit's pass
    int threads = 256;       // threads per CTA
};
}  // namespace qe

struct qe_batch {
    int count = 0, layers = 0, dtype = QE_C128;
    int arith = QE_ARITH_DF64;   // complex128 arithmetic (qe_batch_set_arith)
    double hx = 0.7;
    cudaStream_t stream = nullptr;
    std::vector<int> n;
    std::vector<double> angles;
    qe::BatchPlan plan;
    // device memory
    void* states = nullptr;
    size_t state_bytes = 0;
    void* U = nullptr;
    void* items = nullptr;
    void* circ = nullptr;
    unsigned* sync = nullptr;   // head, status, counters[count]
    double2* partials = nullptr;
    double* energies = nullptr;
    double* host_energies = nullptr;   // pinned
    unsigned* host_status = nullptr;   // pinned
    int nitems = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;
    double hbm_bytes = 0.0;
    int magic = 0xBA7C4;
};
