// Emulated arithmetic (Sec. III-A): adding a classical constant c to an
// m-qubit register is a permutation of the amplitudes, x -> x' where the
// register value r becomes (r + c) mod 2^m.  The emulator performs it as one
// in-place permutation: every amplitude is read once and written once, and
// the bits are moved unchanged (no arithmetic touches the values).
//
// For a fixed assignment of the non-register qubits (a "column") the map is a
// rotation by c of 2^m entries, which splits into g = gcd(c, 2^m) cycles of
// length 2^m / g.  In-place strategies:
//   bulk    - register [lo, lo+m), lo < 5, whose slice of 2^(lo+m) contiguous
//             amplitudes fits one CTA's (or a cluster of eight CTAs')
//             shared memory, with 16-byte-aligned rotation runs: each CTA
//             bulk-copies its contiguous part of the slice in, waits at the
//             cluster barrier until every part is held, and bulk-copies it
//             back out at its rotated place (one or two contiguous runs);
//   slice   - the same slices when the runs are not 16-byte aligned
//             (complex64 with an odd shift): load, write rotated;
//   cluster - slices up to 8x larger in that case: eight CTAs of a
//             thread-block cluster each stage 1/8 of the slice and read the
//             rotated source from the owner's shared memory;
//   walk    - otherwise every thread follows one cycle of one column,
//             prefetching several positions ahead (coalesced when the
//             lowest non-register qubits vary across the warp).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>

#include "qe_arith.cuh"
#include "qe_internal.h"
#include "qe_oz.cuh"

namespace cg = cooperative_groups;

namespace qe {

namespace {

template <class S>
struct WalkArgs {
    S* x;
    uint64_t columns;     // 2^(n-m)
    uint64_t g;           // cycles per column: gcd(c, 2^m)
    uint64_t nseg;        // segments per cycle
    uint64_t seg_len;     // cycle positions per segment
    uint64_t items;       // columns * g * nseg
    S* scratch;           // one saved element per item
    uint64_t c;           // constant mod 2^m
    uint64_t mmask;       // 2^m - 1
    uint64_t cycle_len;   // 2^m / g
    int m;
    int contiguous;       // register = [lo, lo+m) ascending
    int lo;
    uint8_t reg[64];      // register qubits (bit j <-> reg[j])
    uint8_t reg_sorted[64];   // register qubits ascending (for inserting zeros)
};

template <class S>
__device__ __forceinline__ uint64_t reg_deposit(const WalkArgs<S>& a, uint64_t r) {
    if (a.contiguous) return r << a.lo;
    uint64_t x = 0;
    for (int j = 0; j < a.m; ++j) x |= ((r >> j) & 1ull) << a.reg[j];
    return x;
}

// Cycle walks are split into S segments so that enough threads run even when
// there are few columns: a first kernel saves the last element of every
// segment to scratch, the second shifts each segment by one position along
// its cycle, seeding it with the saved element of the previous segment.
// Work item = ((segment * g) + cycle start) * columns + column.
template <class S>
__device__ __forceinline__ void walk_item(const WalkArgs<S>& a, uint64_t t, uint64_t& x0,
                                          uint64_t& start, uint64_t& seg) {
    const uint64_t col = t % a.columns;
    const uint64_t rest = t / a.columns;
    start = rest % a.g;
    seg = rest / a.g;
    x0 = insert_zero_bits(col, a.reg_sorted, a.m);
}

template <class S>
__global__ void __launch_bounds__(256) k_add_walk_save(const __grid_constant__ WalkArgs<S> a) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < a.items;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x0, start, seg;
        walk_item(a, t, x0, start, seg);
        const uint64_t last = min((seg + 1) * a.seg_len, a.cycle_len) - 1;
        const uint64_t r = (start + last * a.c) & a.mmask;
        a.scratch[t] = a.x[x0 | reg_deposit(a, r)];
    }
}

template <class S, int U>
__global__ void __launch_bounds__(256) k_add_walk(const __grid_constant__ WalkArgs<S> a) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < a.items;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x0, start, seg;
        walk_item(a, t, x0, start, seg);
        const uint64_t first = seg * a.seg_len;
        const uint64_t end = min(first + a.seg_len, a.cycle_len);
        // the element before this segment on the cycle was saved by the
        // previous segment's item (segment nseg-1 precedes segment 0)
        const uint64_t prev_seg = (seg == 0) ? a.nseg - 1 : seg - 1;
        S v = a.scratch[t + (prev_seg - seg) * a.g * a.columns];
        uint64_t r = (start + first * a.c) & a.mmask;
        for (uint64_t step = first; step < end; step += U) {
            const uint64_t left = end - step;
            const int cnt = left < (uint64_t)U ? (int)left : U;
            S buf[U];
            uint64_t pos[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (u < cnt) {
                    pos[u] = x0 | reg_deposit(a, r);
                    buf[u] = a.x[pos[u]];
                    r = (r + a.c) & a.mmask;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (u < cnt) a.x[pos[u]] = (u == 0) ? v : buf[u - 1];
            v = buf[cnt - 1];
        }
    }
}

// Chunks of 2^C contiguous amplitudes (C >= S: whole slices of 2^S) through
// shared memory, one per CTA pass; each slice rotated by c * 2^lo.
template <class S>
__global__ void __launch_bounds__(512) k_add_slice(S* __restrict__ x, uint64_t nchunks, int Cbits, int Sbits,
                                                   uint64_t shift) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* buf = reinterpret_cast<S*>(smem_raw);
    const uint32_t E = 1u << Cbits, mask = (1u << Sbits) - 1u;
    const uint32_t sh = (uint32_t)shift;
    for (uint64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        S* base = x + (ch << Cbits);
        for (uint32_t i = threadIdx.x; i < E; i += blockDim.x) buf[i] = base[i];
        __syncthreads();
        for (uint32_t p = threadIdx.x; p < E; p += blockDim.x) base[p] = buf[(p & ~mask) | ((p - sh) & mask)];
        __syncthreads();
    }
}

// Eight CTAs (one cluster) per slice of 2^S amplitudes, each holding 2^S/8.
template <class S>
__global__ void __launch_bounds__(512) k_add_cluster(S* __restrict__ x, int Sbits, uint64_t shift) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* buf = reinterpret_cast<S*>(smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t rank = cl.block_rank();
    const uint32_t nblk = cl.num_blocks();
    const uint32_t E = (1u << Sbits) / nblk;      // elements per CTA
    const uint32_t mask = (1u << Sbits) - 1u;
    const uint64_t slice = blockIdx.x / nblk;
    S* base = x + (slice << Sbits);
    for (uint32_t i = threadIdx.x; i < E; i += blockDim.x) buf[i] = base[rank * E + i];
    cl.sync();
    const uint32_t sh = (uint32_t)shift;
    for (uint32_t i = threadIdx.x; i < E; i += blockDim.x) {
        const uint32_t p = rank * E + i;
        const uint32_t src = (p - sh) & mask;
        const S* remote = cl.map_shared_rank(buf, src / E);
        base[p] = remote[src % E];
    }
    cl.sync();
}

// Status of the bulk path: set when a wait for a CTA's incoming copy ran out.
__device__ uint32_t g_add_status;

// One CTA (nblk = 1) or one cluster of nblk CTAs per slice of 2^S amplitudes;
// CTA `rank` holds the contiguous part [rank E, rank E + E), E = 2^S / nblk,
// and writes it back rotated by `shift` within the slice.
template <class S>
__global__ void __launch_bounds__(32) k_add_bulk(S* __restrict__ x, int Sbits, uint32_t shift, long long limit,
                                                 int stall_test) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t abort_flag;
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t nblk = cl.num_blocks(), rank = cl.block_rank();
    const uint32_t total = 1u << Sbits, E = total / nblk, mask = total - 1u;
    S* const base = x + ((uint64_t)(blockIdx.x / nblk) << Sbits);
    const uint32_t sm = oz::smem_u32(smem_raw);
    constexpr uint32_t kPiece = 16384;
    if (threadIdx.x == 0) {
        oz::mbar_init_count(&bar, 1);
        abort_flag = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        const uint32_t bytes = E * (uint32_t)sizeof(S);
        oz::mbar_expect_tx(&bar, bytes);
        const char* src = reinterpret_cast<const char*>(base + (uint64_t)rank * E);
        // (failure-path test: block 0 announces its part but copies none)
        if (!(stall_test && blockIdx.x == 0))
            for (uint32_t off = 0; off < bytes; off += kPiece)
                oz::bulk_g2s(sm + off, src + off, min(kPiece, bytes - off), &bar);
    }
    const bool ok = oz::wait_or_abort(oz::smem_u32(&bar), 0u, limit, &abort_flag);
    // every CTA of the cluster holds its part before any part is written back
    cl.sync();
    if (threadIdx.x == 0 && ok) {
        const uint32_t d0 = (rank * E + shift) & mask;
        const uint32_t first = min(E, total - d0);
        char* dst0 = reinterpret_cast<char*>(base + d0);
        for (uint32_t off = 0; off < first * (uint32_t)sizeof(S); off += kPiece)
            oz::bulk_s2g(dst0 + off, sm + off, min(kPiece, first * (uint32_t)sizeof(S) - off));
        const uint32_t rest = (E - first) * (uint32_t)sizeof(S), rest0 = first * (uint32_t)sizeof(S);
        char* dst1 = reinterpret_cast<char*>(base);
        for (uint32_t off = 0; off < rest; off += kPiece)
            oz::bulk_s2g(dst1 + off, sm + rest0 + off, min(kPiece, rest - off));
        oz::bulk_commit();
        oz::bulk_wait_all();
    }
    if (!ok && threadIdx.x == 0) atomicExch(&g_add_status, 1u);
}

template <class S>
void add_impl(qe_state* s, int m, const int* qubits, uint64_t c) {
    const uint64_t mmask = (m >= 64) ? ~0ull : ((1ull << m) - 1ull);
    c &= mmask;
    if (c == 0) return;
    bool contiguous = true;
    for (int j = 1; j < m; ++j) contiguous &= qubits[j] == qubits[0] + j;
    const int lo = qubits[0];
    const int n = s->n;
    const int Sbits = contiguous ? lo + m : 0;
    const int cap_bits = (sizeof(S) >= 16) ? 12 : 13;      // 64 KB per CTA
    const int ccap_bits = (sizeof(S) >= 16) ? 13 : 14;     // 128 KB per CTA, 8 per cluster
    S* x = reinterpret_cast<S*>(s->d);
    // bulk: parts of 32 KB to 128 KB per CTA (one CTA, or a cluster of
    // eight; smaller slices go through the chunked shared-memory kernel,
    // measured faster below 32 KB), and rotation runs on 16-byte boundaries
    const int bulk_bits = (sizeof(S) >= 16) ? 13 : 14;
    const int bulk_min = (sizeof(S) >= 16) ? 11 : 12;
    const uint64_t shift = c << lo;
    const int nblk = (contiguous && Sbits >= 3 && Sbits <= bulk_bits) ? 1 : 8;
    const bool use_bulk = contiguous && lo < 5 && Sbits >= bulk_min && Sbits <= bulk_bits + 3 &&
                          ((shift * sizeof(S)) % 16 == 0) && ((((uint64_t)sizeof(S) << Sbits) / nblk) % 16 == 0);
    if (use_bulk) {
        Launch L(s, nblk == 1 ? "add_bulk" : "add_bulk_cluster", 2.0 * dim(s) * amp_bytes(s));
        const uint64_t nslices = 1ull << (n - Sbits);
        const size_t smem = (sizeof(S) << Sbits) / nblk;
        QE_CUDA(cudaFuncSetAttribute(k_add_bulk<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        void* st_addr = nullptr;
        QE_CUDA(cudaGetSymbolAddress(&st_addr, g_add_status));
        QE_CUDA(cudaMemsetAsync(st_addr, 0, sizeof(uint32_t), s->stream));
        cudaLaunchConfig_t cfg = {};
        if (nslices * nblk > 0x7FFFFFFFull) fail(QE_ERR_UNSUPPORTED, "too many slices for one launch");
        cfg.gridDim = dim3((unsigned)(nslices * nblk));
        cfg.blockDim = dim3(32);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)nblk;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        // Failure-path test (QE_TEST_STALL_ADD=1): block 0's copy wait runs out
        // after a short limit (its cluster waits for it at the barrier), the
        // host reports QE_ERR_TIMEOUT; the state's contents are then undefined.
        const char* stall = std::getenv("QE_TEST_STALL_ADD");
        const int stall_test = (stall != nullptr && stall[0] == '1') ? 1 : 0;
        const long long limit = stall_test ? (1ll << 12) : (1ll << 20);   // polls of up to 1 us each
        QE_CUDA(cudaLaunchKernelEx(&cfg, k_add_bulk<S>, x, Sbits, (uint32_t)shift, limit, stall_test));
        QE_CUDA(cudaGetLastError());
        uint32_t st = 0;
        QE_CUDA(cudaMemcpyAsync(&st, st_addr, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream));
        QE_CUDA(cudaStreamSynchronize(s->stream));
        if (st != 0) fail(QE_ERR_TIMEOUT, "an add-constant copy wait ran out");
        return;
    }
    const bool use_slice = contiguous && lo < 5 && Sbits <= cap_bits;
    const bool use_cluster = !use_slice && contiguous && lo < 5 && Sbits <= ccap_bits + 3 && Sbits >= 3;
    Launch L(s, use_slice ? "add_slice" : use_cluster ? "add_cluster" : "add_walk",
             2.0 * dim(s) * amp_bytes(s));
    if (use_slice) {
        // 32 KB chunks (2^11 complex128 or 2^12 complex64 amplitudes), or the slice
        const int Cbits = std::min(n, std::max(Sbits, sizeof(S) >= 16 ? 11 : 12));
        const uint64_t nchunks = 1ull << (n - Cbits);
        size_t smem = sizeof(S) << Cbits;
        QE_CUDA(cudaFuncSetAttribute(k_add_slice<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int occ = 0;
        QE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_add_slice<S>, 512, smem));
        uint64_t grid = std::min<uint64_t>(nchunks, (uint64_t)num_sms() * std::max(occ, 1));
        k_add_slice<S><<<(unsigned)grid, 512, smem, s->stream>>>(x, nchunks, Cbits, Sbits, c << lo);
    } else if (use_cluster) {
        const uint64_t nslices = 1ull << (n - Sbits);
        size_t smem = sizeof(S) << (Sbits - 3);
        QE_CUDA(cudaFuncSetAttribute(k_add_cluster<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nslices * 8));
        cfg.blockDim = dim3(512);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 8;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (nslices * 8 > 0x7FFFFFFFull) fail(QE_ERR_UNSUPPORTED, "too many slices for one launch");
        QE_CUDA(cudaLaunchKernelEx(&cfg, k_add_cluster<S>, x, Sbits, (uint64_t)(c << lo)));
    } else {
        static thread_local WalkArgs<S> a;
        a.x = x;
        a.m = m;
        a.c = c;
        a.mmask = mmask;
        a.contiguous = contiguous;
        a.lo = lo;
        a.g = 1ull << __builtin_ctzll(c);   // gcd(c, 2^m), c != 0 mod 2^m
        a.columns = 1ull << (n - m);
        a.cycle_len = (mmask >> __builtin_ctzll(c)) + 1ull;
        // enough independent walks to fill the GPU, segments of >= 64 steps
        const uint64_t want = (uint64_t)num_sms() * 2048;
        const uint64_t base_items = a.columns * a.g;
        uint64_t nseg = (want + base_items - 1) / base_items;
        nseg = std::max<uint64_t>(1, std::min<uint64_t>(nseg, a.cycle_len / 64));
        a.seg_len = (a.cycle_len + nseg - 1) / nseg;
        a.nseg = (a.cycle_len + a.seg_len - 1) / a.seg_len;
        a.items = base_items * a.nseg;
        a.scratch = (S*)ensure_scratch(s, a.items * sizeof(S));
        for (int j = 0; j < m; ++j) a.reg[j] = (uint8_t)qubits[j];
        int tmp[64];
        for (int j = 0; j < m; ++j) tmp[j] = qubits[j];
        std::sort(tmp, tmp + m);
        for (int j = 0; j < m; ++j) a.reg_sorted[j] = (uint8_t)tmp[j];
        uint64_t grid = std::min<uint64_t>((a.items + 255) / 256, (uint64_t)num_sms() * 8);
        grid = std::max<uint64_t>(grid, 1);
        k_add_walk_save<S><<<(unsigned)grid, 256, 0, s->stream>>>(a);
        QE_CUDA(cudaGetLastError());
        k_add_walk<S, 8><<<(unsigned)grid, 256, 0, s->stream>>>(a);
    }
    QE_CUDA(cudaGetLastError());
}

}  // namespace

void launch_add_const(qe_state* s, int m, const int* qubits, uint64_t c) {
    if (s->dtype == QE_C128) add_impl<double2>(s, m, qubits, c);
    else add_impl<float2>(s, m, qubits, c);
}

}  // namespace qe
