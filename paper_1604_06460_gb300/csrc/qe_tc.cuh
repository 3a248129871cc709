// Pieces shared by the tcgen05 gate kernels: shared-memory matrix
// descriptors, mbarrier waits with an iteration limit, and the tile geometry
// that makes the five gate qubits tile-local.
#pragma once
#include <algorithm>
#include <cstdint>

#include "qe_internal.h"

namespace qe {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor for a K-major operand in the 128-byte
// swizzle layout: start >> 4, leading offset (unused for swizzled K-major)
// 16 bytes, stride between 8-row groups 1024 bytes, descriptor version 1,
// layout SWIZZLE_128B (2).  Operands start on 1024-byte boundaries.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: D f32; A, B of type `ab` (kind::f16: 1 = bf16;
// kind::tf32: 2 = tf32), both K-major; N and M.
__host__ __device__ constexpr uint32_t idesc(uint32_t ab, uint32_t n, uint32_t m) {
    return (1u << 4) | (ab << 7) | (ab << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
}

// Wait for phase `phase` of an mbarrier; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, long long limit) {
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase));
        if (done) return true;
    }
    return false;
}

// Arrive on the mbarrier once every tcgen05.mma issued so far completes.
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(mbar)));
}

// Tile geometry of a 5-qubit block: 12 tile-local index bits, the low bits
// [0, L) (contiguous chunks of 2^L amplitudes) plus the kh gate qubits >= L;
// the five gate qubits sit at tile-local positions gpos[] and the other
// seven local bits index the 128 groups (rows) of a tile.
struct Geometry {
    int L = -1, kh = 0;
    uint8_t hq[8] = {};
    uint8_t gpos[5] = {};
};

inline Geometry tile_geometry(const int* qubits) {
    Geometry g;
    int srt[5];
    for (int j = 0; j < 5; ++j) srt[j] = qubits[j];
    std::sort(srt, srt + 5);
    for (int l = 12; l >= 0; --l) {
        int h = 0;
        for (int j = 0; j < 5; ++j) h += srt[j] >= l;
        if (l + h <= 12) {
            g.L = l;
            g.kh = h;
            break;
        }
    }
    if (g.L < 0) fail(QE_ERR_ARG, "no tensor-core tile geometry");
    int h = 0;
    for (int j = 0; j < 5; ++j)
        if (srt[j] >= g.L) g.hq[h++] = (uint8_t)srt[j];
    for (int j = 0; j < 5; ++j) {
        int q = qubits[j], pos = q;
        if (q >= g.L)
            for (int i = 0; i < g.kh; ++i)
                if (g.hq[i] == q) pos = g.L + i;
        g.gpos[j] = (uint8_t)pos;
    }
    return g;
}

}  // namespace tc
}  // namespace qe
