// Emulated quantum phase estimation (Sec. III-C): instead of applying the
// controlled powers U, U^2, U^4, ..., U^(2^(b-1)) gate by gate (O(G 2^(n+b))),
// the emulator builds the dense 2^n x 2^n matrix of U once (O(G 2^(2n))),
// squares it b - 1 times (O(2^(3n) b)) and applies each power as one dense
// matrix product on the state.
//
// Dense matrices live in states of 2n qubits, column-major: entry (i, j) is
// amplitude (j << n) | i.  The identity is one kernel; the circuit's gates
// applied to qubits [0, n) of that state then act on every column at once,
// so the gate path (fusion, tensor cores) builds U.  Products use one FP64
// complex matrix-multiply kernel: 64 x 64 tiles of C per CTA, K in steps of
// 16 staged in shared memory, a 4 x 4 register tile of complex accumulators
// per thread (fused multiply-adds in FP64).  A controlled power acts on the
// rows (system registers) whose control bit is set: those rows times M^T into
// a scratch buffer, then copied back.
#include <algorithm>
#include <cstring>

#include "qe_arith.cuh"
#include "qe_internal.h"

namespace qe {

namespace {

constexpr int kTM = 64, kTN = 64, kTK = 16, kGemmThreads = 256;

__global__ void __launch_bounds__(256) k_init_identity(double2* __restrict__ x, uint64_t dimx, int nsys) {
    const uint64_t lo = (1ull << nsys) - 1ull;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < dimx; i += (uint64_t)gridDim.x * blockDim.x)
        x[i] = make_double2(((i >> nsys) == (i & lo)) ? 1.0 : 0.0, 0.0);
}

struct GemmArgs {
    const double2* A;
    const double2* B;
    double2* C;
    int64_t M, N, K;         // C (M x N) = A (M x K) B (K x N), row-major
    int64_t lda, ldb, ldc;   // row strides in elements
    int a_rowbit;            // >= 0: logical row r of A is memory row r with a 1 inserted at this bit
};

__device__ __forceinline__ int64_t map_row(int64_t r, int bit) {
    if (bit < 0) return r;
    const int64_t low = r & ((1ll << bit) - 1);
    return ((r >> bit) << (bit + 1)) | (1ll << bit) | low;
}

__global__ void __launch_bounds__(kGemmThreads) k_zgemm(const __grid_constant__ GemmArgs a) {
    __shared__ double2 As[kTK][kTM];
    __shared__ double2 Bs[kTK][kTN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.y * kTM, col0 = (int64_t)blockIdx.x * kTN;
    double2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
    for (int64_t k0 = 0; k0 < a.K; k0 += kTK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + kGemmThreads * q;
            const int r = e >> 4, k = e & 15;         // A tile: 64 rows x 16 k
            const int64_t gr = row0 + r, gk = k0 + k;
            As[k][r] = (gr < a.M && gk < a.K) ? a.A[map_row(gr, a.a_rowbit) * a.lda + gk] : make_double2(0.0, 0.0);
            const int kb = e >> 6, c = e & 63;        // B tile: 16 k x 64 columns
            const int64_t gkb = k0 + kb, gc = col0 + c;
            Bs[kb][c] = (gkb < a.K && gc < a.N) ? a.B[gkb * a.ldb + gc] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kTK; ++kk) {
            double2 av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = __fma_rn(av[i].x, bv[j].x, __fma_rn(-av[i].y, bv[j].y, acc[i][j].x));
                    acc[i][j].y = __fma_rn(av[i].x, bv[j].y, __fma_rn(av[i].y, bv[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
            if (r < a.M && c < a.N) a.C[r * a.ldc + c] = acc[i][j];
        }
}

// rows of the state whose control bit is set <- the scratch rows
__global__ void __launch_bounds__(256) k_copy_rows(double2* __restrict__ x, const double2* __restrict__ scr,
                                                   uint64_t rows, int nsys, int bit) {
    const uint64_t total = rows << nsys;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = e >> nsys, i = e & ((1ull << nsys) - 1ull);
        x[((uint64_t)map_row((int64_t)r, bit) << nsys) | i] = scr[e];
    }
}

void gemm(qe_state* s, const GemmArgs& a, const char* tag) {
    const dim3 grid((unsigned)((a.N + kTN - 1) / kTN), (unsigned)((a.M + kTM - 1) / kTM));
    if (grid.y > 65535u) fail(QE_ERR_UNSUPPORTED, "matrix product too tall for one launch");
    Launch L(s, tag, (double)(a.M * a.K + a.K * a.N + a.M * a.N) * 16.0, false);
    k_zgemm<<<grid, kGemmThreads, 0, s->stream>>>(a);
    QE_CUDA(cudaGetLastError());
}

}  // namespace

void launch_init_identity(qe_state* s, int nsys) {
    const unsigned grid = (unsigned)std::min<uint64_t>((dim(s) + 255) / 256, (uint64_t)num_sms() * 8);
    Launch L(s, "init_identity", (double)dim(s) * amp_bytes(s));
    k_init_identity<<<grid, 256, 0, s->stream>>>(reinterpret_cast<double2*>(s->d), dim(s), nsys);
    QE_CUDA(cudaGetLastError());
}

// c = a b for 2^k x 2^k matrices stored column-major (entry (i, j) at
// (j << k) | i): as row-major arrays they are the transposes, and
// C^T = B^T A^T.  Enqueued on acct's stream, counted in its statistics.
void launch_matmul(qe_state* acct, void* c, const void* a, const void* b, int k) {
    const int64_t D = 1ll << k;
    if (acct->tensor_cores && k >= 6 && oz_gemm_available(D, D, D)) {
        // on the tensor cores: exact digit products, 128-bit sums
        oz_zgemm(acct, reinterpret_cast<double2*>(c), D, reinterpret_cast<const double2*>(b), D, D, D, -1,
                 reinterpret_cast<const double2*>(a), D, D);
        return;
    }
    GemmArgs g{};
    g.A = reinterpret_cast<const double2*>(b);
    g.B = reinterpret_cast<const double2*>(a);
    g.C = reinterpret_cast<double2*>(c);
    g.M = g.N = g.K = D;
    g.lda = g.ldb = g.ldc = D;
    g.a_rowbit = -1;
    gemm(acct, g, "zgemm");
}

// The rows of s (system register [0, nsys)) whose qubit ctrl is set times
// M^T: psi_row <- M psi_row.  M is held column-major in mat (2 nsys qubits),
// i.e. mat's amplitudes read row-major are M^T.  On the tensor cores from 128
// rows and nsys >= 6, else FP64 fused multiply-adds.
void launch_dense_controlled(qe_state* s, const void* mat, int nsys, int ctrl) {
    const int64_t D = 1ll << nsys;
    const uint64_t rows = 1ull << (s->n - nsys - 1);
    double2* scr = reinterpret_cast<double2*>(ensure_scratch(s, (size_t)(rows << nsys) * sizeof(double2)));
    if (s->tensor_cores && nsys >= 6 && rows >= 128 && oz_gemm_available((int64_t)rows, D, D)) {
        // on the tensor cores (rows padded to 128 inside the product)
        oz_zgemm(s, scr, D, reinterpret_cast<const double2*>(s->d), (int64_t)rows, D, D, ctrl - nsys,
                 reinterpret_cast<const double2*>(mat), D, D);
    } else {
        GemmArgs g{};
        g.A = reinterpret_cast<const double2*>(s->d);
        g.B = reinterpret_cast<const double2*>(mat);
        g.C = scr;
        g.M = (int64_t)rows;
        g.N = g.K = D;
        g.lda = g.ldb = g.ldc = D;
        g.a_rowbit = ctrl - nsys;
        gemm(s, g, "zgemm_controlled");
    }
    const uint64_t total = rows << nsys;
    const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, (uint64_t)num_sms() * 8);
    Launch L(s, "copy_rows", 2.0 * (double)total * 16.0, false);
    k_copy_rows<<<grid, 256, 0, s->stream>>>(reinterpret_cast<double2*>(s->d), scr, rows, nsys, ctrl - nsys);
    QE_CUDA(cudaGetLastError());
}

}  // namespace qe
