// Learned cost model: a small multilayer perceptron (tanh hidden layers,
// linear output) that predicts log(time) of an operation from its features.
// Forward pass, backpropagation and the Adam update are hand-written kernels;
// training is full-batch on the GPU.  The planner asks it to choose between
// emulating and simulating a subroutine and to choose the gate-fusion width.
// (The paper picks between emulation and simulation with performance models
// and measured cross-over points, Sec. III-B, IV-C and IV-D; the analytic
// rule in plan.cu restates those models and remains the fallback.)
//
// Parameter layout: W1[h1][d] b1[h1] W2[h2][h1] b2[h2] W3[h2] b3.
#include <algorithm>
#include <cmath>
#include <vector>

#include "qe_internal.h"
#include "qe_mlp.h"

namespace qe {

namespace {

struct Offs {
    int W1, b1, W2, b2, W3, b3, np;
};
__host__ __device__ inline Offs offs(int d, int h1, int h2) {
    Offs o;
    o.W1 = 0;
    o.b1 = o.W1 + h1 * d;
    o.W2 = o.b1 + h1;
    o.b2 = o.W2 + h2 * h1;
    o.W3 = o.b2 + h2;
    o.b3 = o.W3 + h2;
    o.np = o.b3 + 1;
    return o;
}

// One thread per sample: hidden activations and output.
__global__ void k_mlp_forward(const float* __restrict__ p, int d, int h1, int h2,
                              const float* __restrict__ X, int n, float* __restrict__ A1,
                              float* __restrict__ A2, float* __restrict__ Y) {
    const Offs o = offs(d, h1, h2);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const float* x = X + (size_t)s * d;
        float* a1 = A1 + (size_t)s * h1;
        float* a2 = A2 + (size_t)s * h2;
        for (int j = 0; j < h1; ++j) {
            float z = p[o.b1 + j];
            for (int i = 0; i < d; ++i) z = fmaf(p[o.W1 + j * d + i], x[i], z);
            a1[j] = tanhf(z);
        }
        for (int j = 0; j < h2; ++j) {
            float z = p[o.b2 + j];
            for (int i = 0; i < h1; ++i) z = fmaf(p[o.W2 + j * h1 + i], a1[i], z);
            a2[j] = tanhf(z);
        }
        float y = p[o.b3];
        for (int i = 0; i < h2; ++i) y = fmaf(p[o.W3 + i], a2[i], y);
        Y[s] = y;
    }
}

// One thread per sample: output error dL/dy = 2 (y - t) / n and the
// back-propagated deltas of both hidden layers (through 1 - tanh^2).
__global__ void k_mlp_deltas(const float* __restrict__ p, int d, int h1, int h2,
                             const float* __restrict__ A1, const float* __restrict__ A2,
                             const float* __restrict__ Y, const float* __restrict__ T, int n,
                             float* __restrict__ DY, float* __restrict__ D1, float* __restrict__ D2) {
    const Offs o = offs(d, h1, h2);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const float dy = 2.0f * (Y[s] - T[s]) / (float)n;
        DY[s] = dy;
        const float* a1 = A1 + (size_t)s * h1;
        const float* a2 = A2 + (size_t)s * h2;
        float* d2 = D2 + (size_t)s * h2;
        float* d1 = D1 + (size_t)s * h1;
        for (int j = 0; j < h2; ++j) d2[j] = dy * p[o.W3 + j] * (1.0f - a2[j] * a2[j]);
        for (int i = 0; i < h1; ++i) {
            float acc = 0.f;
            for (int j = 0; j < h2; ++j) acc = fmaf(p[o.W2 + j * h1 + i], d2[j], acc);
            d1[i] = acc * (1.0f - a1[i] * a1[i]);
        }
    }
}

// One thread per parameter: its gradient summed over the samples in order
// (deterministic).
__global__ void k_mlp_param_grad(int d, int h1, int h2, const float* __restrict__ X,
                                 const float* __restrict__ A1, const float* __restrict__ A2,
                                 const float* __restrict__ DY, const float* __restrict__ D1,
                                 const float* __restrict__ D2, int n, float* __restrict__ G) {
    const Offs o = offs(d, h1, h2);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < o.np; k += gridDim.x * blockDim.x) {
        float g = 0.f;
        if (k < o.b1) {
            const int j = (k - o.W1) / d, i = (k - o.W1) % d;
            for (int s = 0; s < n; ++s) g = fmaf(D1[(size_t)s * h1 + j], X[(size_t)s * d + i], g);
        } else if (k < o.W2) {
            const int j = k - o.b1;
            for (int s = 0; s < n; ++s) g += D1[(size_t)s * h1 + j];
        } else if (k < o.b2) {
            const int j = (k - o.W2) / h1, i = (k - o.W2) % h1;
            for (int s = 0; s < n; ++s) g = fmaf(D2[(size_t)s * h2 + j], A1[(size_t)s * h1 + i], g);
        } else if (k < o.W3) {
            const int j = k - o.b2;
            for (int s = 0; s < n; ++s) g += D2[(size_t)s * h2 + j];
        } else if (k < o.b3) {
            const int i = k - o.W3;
            for (int s = 0; s < n; ++s) g = fmaf(DY[s], A2[(size_t)s * h2 + i], g);
        } else {
            for (int s = 0; s < n; ++s) g += DY[s];
        }
        G[k] = g;
    }
}

// Adam (Kingma & Ba, 2015) with bias correction.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int np, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

// Mean squared error of the current outputs (one block).
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, int n, float* out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const double r = (double)Y[s] - (double)T[s];
        acc += r * r;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)(sh[0] / n);
}

unsigned blocks_for(int n) { return (unsigned)std::max(1, std::min(1024, (n + 127) / 128)); }

void ensure_capacity(qe_cost_model* m, int n) {
    if (n <= m->cap) return;
    for (float* q : {m->X, m->T, m->Y, m->A1, m->A2, m->D1, m->D2, m->DY})
        if (q) cudaFree(q);
    const int c = std::max(n, 1024);
    QE_CUDA(cudaMalloc(&m->X, sizeof(float) * c * m->d));
    QE_CUDA(cudaMalloc(&m->T, sizeof(float) * c));
    QE_CUDA(cudaMalloc(&m->Y, sizeof(float) * c));
    QE_CUDA(cudaMalloc(&m->A1, sizeof(float) * c * m->h1));
    QE_CUDA(cudaMalloc(&m->A2, sizeof(float) * c * m->h2));
    QE_CUDA(cudaMalloc(&m->D1, sizeof(float) * c * m->h1));
    QE_CUDA(cudaMalloc(&m->D2, sizeof(float) * c * m->h2));
    QE_CUDA(cudaMalloc(&m->DY, sizeof(float) * c));
    m->cap = c;
}

void upload(qe_cost_model* m, const float* X, const float* T, int n) {
    ensure_capacity(m, n);
    QE_CUDA(cudaMemcpyAsync(m->X, X, sizeof(float) * n * m->d, cudaMemcpyHostToDevice, m->stream));
    if (T) QE_CUDA(cudaMemcpyAsync(m->T, T, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream));
}

void forward(qe_cost_model* m, int n) {
    k_mlp_forward<<<blocks_for(n), 128, 0, m->stream>>>(m->params, m->d, m->h1, m->h2, m->X, n, m->A1,
                                                        m->A2, m->Y);
}

void backward(qe_cost_model* m, int n) {
    k_mlp_deltas<<<blocks_for(n), 128, 0, m->stream>>>(m->params, m->d, m->h1, m->h2, m->A1, m->A2,
                                                       m->Y, m->T, n, m->DY, m->D1, m->D2);
    k_mlp_param_grad<<<blocks_for(m->np), 128, 0, m->stream>>>(m->d, m->h1, m->h2, m->X, m->A1, m->A2,
                                                               m->DY, m->D1, m->D2, n, m->grad);
}

}  // namespace

void mlp_create(qe_cost_model* m, uint64_t seed) {
    m->np = offs(m->d, m->h1, m->h2).np;
    QE_CUDA(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
    QE_CUDA(cudaMalloc(&m->params, sizeof(float) * m->np));
    QE_CUDA(cudaMalloc(&m->grad, sizeof(float) * m->np));
    QE_CUDA(cudaMalloc(&m->mom1, sizeof(float) * m->np));
    QE_CUDA(cudaMalloc(&m->mom2, sizeof(float) * m->np));
    QE_CUDA(cudaMalloc(&m->loss, sizeof(float)));
    // Glorot-uniform weights, zero biases; SplitMix64 (Steele et al. 2014) uniforms
    const Offs o = offs(m->d, m->h1, m->h2);
    std::vector<float> h(m->np, 0.f);
    uint64_t st = seed;
    auto uni = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * 0x1.0p-53;
    };
    auto fill = [&](int off, int fan_in, int fan_out) {
        const double a = std::sqrt(6.0 / (fan_in + fan_out));
        for (int i = 0; i < fan_in * fan_out; ++i) h[off + i] = (float)((2.0 * uni() - 1.0) * a);
    };
    fill(o.W1, m->d, m->h1);
    fill(o.W2, m->h1, m->h2);
    fill(o.W3, m->h2, 1);
    QE_CUDA(cudaMemcpy(m->params, h.data(), sizeof(float) * m->np, cudaMemcpyHostToDevice));
    QE_CUDA(cudaMemset(m->mom1, 0, sizeof(float) * m->np));
    QE_CUDA(cudaMemset(m->mom2, 0, sizeof(float) * m->np));
    m->step = 0;
}

void mlp_destroy(qe_cost_model* m) {
    for (float* q : {m->params, m->grad, m->mom1, m->mom2, m->loss, m->X, m->T, m->Y, m->A1, m->A2, m->D1, m->D2, m->DY})
        if (q) cudaFree(q);
    if (m->stream) cudaStreamDestroy(m->stream);
}

float mlp_gradient(qe_cost_model* m, const float* X, const float* T, int n, float* grad_host) {
    upload(m, X, T, n);
    forward(m, n);
    backward(m, n);
    k_mse<<<1, 256, 0, m->stream>>>(m->Y, m->T, n, m->loss);
    QE_CUDA(cudaGetLastError());
    float loss = 0.f;
    QE_CUDA(cudaMemcpyAsync(grad_host, m->grad, sizeof(float) * m->np, cudaMemcpyDeviceToHost, m->stream));
    QE_CUDA(cudaMemcpyAsync(&loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    QE_CUDA(cudaStreamSynchronize(m->stream));
    return loss;
}

float mlp_train(qe_cost_model* m, const float* X, const float* T, int n, int epochs, float lr) {
    upload(m, X, T, n);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int e = 0; e < epochs; ++e) {
        forward(m, n);
        backward(m, n);
        ++m->step;
        const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
        k_adam<<<blocks_for(m->np), 128, 0, m->stream>>>(m->params, m->grad, m->mom1, m->mom2, m->np, lr, b1,
                                                         b2, eps, c1, c2);
    }
    forward(m, n);
    k_mse<<<1, 256, 0, m->stream>>>(m->Y, m->T, n, m->loss);
    QE_CUDA(cudaGetLastError());
    float loss = 0.f;
    QE_CUDA(cudaMemcpyAsync(&loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    QE_CUDA(cudaStreamSynchronize(m->stream));
    return loss;
}

void mlp_predict(qe_cost_model* m, const float* X, int n, float* y_host) {
    if (n <= 0) return;
    upload(m, X, nullptr, n);
    forward(m, n);
    QE_CUDA(cudaGetLastError());
    QE_CUDA(cudaMemcpyAsync(y_host, m->Y, sizeof(float) * n, cudaMemcpyDeviceToHost, m->stream));
    QE_CUDA(cudaStreamSynchronize(m->stream));
}

// Features of an operation (the learned model's input, 16 values).
void cost_features(int op, int n, int dtype, int k, int lo, int hi, int m, uint64_t c, float* f) {
    for (int i = 0; i < kCostFeatures; ++i) f[i] = 0.f;
    if (op >= 0 && op < 5) f[op] = 1.f;
    const double nn = std::max(1, n);
    f[5] = (float)(n / 34.0);
    f[6] = dtype == QE_C128 ? 1.f : 0.f;
    f[7] = (float)(k / 5.0);
    f[8] = (float)((n + (dtype == QE_C128 ? 4 : 3)) / 40.0);   // log2 of the state's bytes
    f[9] = (float)(lo / nn);
    f[10] = (float)(hi / nn);
    f[11] = (float)(m / nn);
    f[12] = m > 0 ? (float)(__builtin_popcountll(c & ((m >= 64) ? ~0ull : ((1ull << m) - 1ull))) / (double)m) : 0.f;
    // size of the subroutine's gate circuit: m + m(m-1)/2 gates for a QFT,
    // m - j multi-controlled NOTs for every set bit j of an added constant
    double g = 0.0;
    if (op == kOpQftEmulate || op == kOpQftSimulate) g = m + 0.5 * m * (m - 1);
    if (op == kOpAddEmulate || op == kOpAddSimulate)
        for (int j = 0; j < m && j < 64; ++j)
            if ((c >> j) & 1ull) g += m - j;
    f[13] = (float)(g / (nn * nn));
    f[14] = (float)((n - m) / nn);
    f[15] = 1.f;
}

}  // namespace qe
