// Host-side state of the learned cost model (see mlp.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/qe.h"

namespace qe {
constexpr int kCostFeatures = 16;
// operation codes of the feature vector
enum { kOpGatePass = 0, kOpQftEmulate = 1, kOpQftSimulate = 2, kOpAddEmulate = 3, kOpAddSimulate = 4 };
void cost_features(int op, int n, int dtype, int k, int lo, int hi, int m, uint64_t c, float* f);
}  // namespace qe

struct qe_cost_model {
    int d = 16, h1 = 32, h2 = 32, np = 0;
    cudaStream_t stream = nullptr;
    float* params = nullptr;
    float* grad = nullptr;
    float* mom1 = nullptr;
    float* mom2 = nullptr;
    float* loss = nullptr;
    int step = 0;
    // per-sample buffers
    int cap = 0;
    float* X = nullptr;
    float* T = nullptr;
    float* Y = nullptr;
    float* A1 = nullptr;
    float* A2 = nullptr;
    float* D1 = nullptr;
    float* D2 = nullptr;
    float* DY = nullptr;
    int magic = 0xC057;
};

namespace qe {
void mlp_create(qe_cost_model* m, uint64_t seed);
void mlp_destroy(qe_cost_model* m);
float mlp_gradient(qe_cost_model* m, const float* X, const float* T, int n, float* grad_host);
float mlp_train(qe_cost_model* m, const float* X, const float* T, int n, int epochs, float lr);
void mlp_predict(qe_cost_model* m, const float* X, int n, float* y_host);
}  // namespace qe
