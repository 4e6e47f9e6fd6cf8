// Blackwell tensor-core (tcgen05 + TMEM + TMA) BF16 GEMM for the density-fitted
// ppRPA sigma sandwich  O_k = sum_P L^P Zt_k L^P  (Sec. "ppRPA Equation" of the
// LibppRPA paper, evaluated with <pq|rs> = sum_P L^P_pr L^P_qs).
//
// Two stages, both "C = A * B^T" with K-major BF16 operands, FP32 accumulation
// in tensor memory:
//   stage 1:  T^P[a, (k, c)] = sum_d L^P[a, d] Zt_k[d, c]
//             M = naux * n_pad rows (P, a), N = k * nblock (vectors side by side),
//             K = nblock; stored as BF16 (hi, and lo = residual for the split form).
//   stage 2:  O_k[a, b] += sum_{P, q} T^P[a, (k, q)] L^P[q, b]
//             M, N = one pair block (virtual or occupied), K = naux * n_pad,
//             split over K across CTAs; FP32 atomic accumulation into O.
// The BF16x3 split form issues hi*hi + hi*lo + lo*hi per K step.
//
// Kernel organisation (one CTA per SM, persistent over a static work list):
//   warps 0-3  epilogue (TMEM lanes 0-127 -> registers -> global)
//   warp 4     TMA producer (one thread)
//   warp 5     TMEM allocator + MMA issuer (one thread)
// Shared-memory ring of STAGES operand slots (full/empty mbarriers) and two
// TMEM accumulators (full/empty mbarriers) so the epilogue of one tile
// overlaps the MMAs of the next.  Every wait is bounded; on expiry the kernel
// raises DEV_TIMEOUT in *status, drains its own copies and MMAs, frees TMEM
// and returns.
#include <cuda.h>

#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.h"
#include "tc.h"

namespace pprpa {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;  // one 128-byte swizzle row of BF16
// Warp roles: warps 0-7 epilogue (warp w reads TMEM lanes 32 * (w % 4) and one half of the
// tile's columns), warp 8 TMA producer, warp 9 MMA issuer and TMEM owner.
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_PRODUCER_WARP = 8;
constexpr int TC_MMA_WARP = 9;
constexpr int TC_THREADS = 32 * (TC_EPI_WARPS + 2);
constexpr int TC_SMEM_LIMIT = 227 * 1024;
constexpr int TC_EPI_BYTES = TC_EPI_WARPS * 32 * 128;  // stage-1 output staging
constexpr unsigned long long TC_WAIT_NS = 4000000000ull;  // 4 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait (limit_ns); returns false (and raises the abort flag) on expiry or abort.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* status, unsigned long long limit_ns) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*abort_flag) return false;
            if (gtimer() - t0 > limit_ns) {
                *abort_flag = 1;
                atomicOr(status, DEV_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* m, int x, int y,
                                       uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)m), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap* m, int x, int y, int z,
                                       uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3, %4}], [%5];" ::"r"(dst),
        "l"((uint64_t)m), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_4d(uint32_t dst, const CUtensorMap* m, int x, int y, int z,
                                       int w, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"((uint64_t)m), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
        : "memory");
}

// Multicast form: the box lands at the same shared-memory offset in every CTA of `mask`
// and completes bytes on the mbarrier at the same offset in each of them.
__device__ __forceinline__ void tma_2d_mc(uint32_t dst, const CUtensorMap* m, int x, int y,
                                          uint32_t bar, uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::"
        "cluster [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"((uint64_t)m), "r"(x), "r"(y), "r"(bar), "h"(mask)
        : "memory");
}

__device__ __forceinline__ void tma_3d_mc(uint32_t dst, const CUtensorMap* m, int x, int y, int z,
                                          uint32_t bar, uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::"
        "cluster [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
        "l"((uint64_t)m), "r"(x), "r"(y), "r"(z), "r"(bar), "h"(mask)
        : "memory");
}

// CTA-pair forms (tcgen05 cta_group::2): the copy lands in this CTA's shared memory and
// completes its bytes on the mbarrier at cluster address `bar` (the pair leader's).
__device__ __forceinline__ void tma_2d_pair(uint32_t dst, const CUtensorMap* m, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)m), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_3d_pair(uint32_t dst, const CUtensorMap* m, int x, int y, int z,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"((uint64_t)m), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_4d_pair(uint32_t dst, const CUtensorMap* m, int x, int y, int z,
                                            int w, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"((uint64_t)m), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
        : "memory");
}
// Bulk tensor store of a shared-memory box to global memory (bulk-group completion), and
// the waits on this thread's bulk groups: until their shared-memory reads are done, or
// until their writes are complete.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* m, uint32_t src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     (uint64_t)m),
                 "r"(x), "r"(y), "r"(z), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Address of the same shared variable in cluster CTA `rank`.
__device__ __forceinline__ uint32_t mapa_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
                 : "memory");
}
__device__ __forceinline__ void mma_bf16_pair(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_e4m3_pair(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}
// Completion of the pair's MMAs arrives on the barrier at the same offset in every CTA of
// `mask` (or only in this CTA for the unicast form).
__device__ __forceinline__ void mma_commit_pair_mc(uint32_t bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
        "[%0], %1;" ::"r"(bar), "h"(mask)
        : "memory");
}
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void mma_commit_mc(uint32_t bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
        "[%0], %1;" ::"r"(bar), "h"(mask)
        : "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (tcgen05 descriptor format, version 1).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major, M = 128 (256 for a
// CTA pair).
__host__ __device__ constexpr uint32_t idesc_bf16(int n, int m = TC_BM) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

// Instruction descriptor, kind::f8f6f4: E4M3 x E4M3 -> FP32, both K-major, M = 128 (256).
__host__ __device__ constexpr uint32_t idesc_e4m3(int n, int m = TC_BM) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Two 16-column loads in flight before one wait (the second only when `two`; warp-uniform).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, bool two, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    if (two) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
            "%11, %12, %13, %14, %15}, [%16];"
            : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
              "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr + 16u));
    } else {
#pragma unroll
        for (int i = 16; i < 32; ++i) r[i] = 0u;
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct ItemCoord {
    int m0, n0, batch, kb0, kb1, nw;  // nw: N of this item's MMAs and output columns
};

__device__ __forceinline__ ItemCoord decode_item(const TcParams& p, int item) {
    ItemCoord c;
    if (p.mode == 0) {
        const int nb = item % p.tiles_n;
        const int mb = item / p.tiles_n;
        c.m0 = mb * TC_BM;
        c.n0 = nb * p.BN;
        c.nw = p.BN;
        c.batch = 0;
        c.kb0 = 0;
        c.kb1 = p.kb_total;
    } else {
        // item = ((split * nbatch) + batch) * ntiles + tile : K-slices outermost so that
        // concurrently running CTAs share the same slice of L in L2.
        const int tile = item % p.ntiles;
        const int rest = item / p.ntiles;
        const int batch = rest % p.nbatch;
        const int split = rest / p.nbatch;
        const int4 t = p.tile_list[tile];
        c.m0 = t.x * TC_BM;
        c.n0 = t.y;
        c.nw = t.z;
        c.batch = batch;
        const int per = (p.kb_total + p.nsplit - 1) / p.nsplit;
        c.kb0 = split * per;
        c.kb1 = min(p.kb_total, c.kb0 + per);
    }
    return c;
}

// One kernel body for both launch forms.  Single: the tensor maps and the parameters are
// kernel parameters and work items are decoded arithmetically.  Batched: work item i is
// items[i]; it names a job (one molecule and stage block) whose tensor maps and epilogue
// parameters live in global memory, so molecules of different sizes and tile widths share
// one persistent launch.  p.slot_bn sizes the shared-memory slots (the widest B tile).
// CL > 1 (single launch only): the CL CTAs of a cluster share the B tile; each loads 1/CL of
// it and multicasts it to all of them.  Stage 1: neighbouring M tiles of one N tile.
// Stage 2: one output tile and K slice for CL neighbouring vectors.
// F8: stage-1 operands are E4M3 (kind::f8f6f4, 128 elements per 128-byte row); the
// epilogue multiplies by the row (per auxiliary index) and column (per vector) scales.
// PAIR (CL = 2): the two CTAs compute one 256-row tile with tcgen05 cta_group::2 MMAs issued
// by the leader (rank 0).  Each CTA holds its own 128 A rows and one half of the B tile
// (N / 2 rows) and completes its copies on the leader's full barrier; the leader's commits
// release the slots and publish the accumulators in both CTAs, and each epilogue warp of
// either CTA releases an accumulator with one arrive on the leader's barrier.
template <int NTERMS, bool BATCHED, int CL, bool F8 = false, bool PAIR = false>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA_hi,
                   const __grid_constant__ CUtensorMap tmA_lo,
                   const __grid_constant__ CUtensorMap tmB_hi,
                   const __grid_constant__ CUtensorMap tmB_lo,
                   const __grid_constant__ CUtensorMap tmT_hi,
                   const __grid_constant__ CUtensorMap tmT_lo, const TcParams p,
                   const TcJob* __restrict__ jobs, const TcItem* __restrict__ items) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[2 * TC_MAX_STAGES + 5];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int BKE = F8 ? 2 * TC_BK : TC_BK;  // elements per 128-byte K block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = p.stages;
    const uint32_t a_bytes = TC_BM * TC_BK * 2;
    static_assert(!PAIR || (CL == 2 && !BATCHED), "a CTA pair is a cluster of two");
    const uint32_t b_slot = (uint32_t)(PAIR ? p.slot_bn / 2 : p.slot_bn) * TC_BK * 2;
    const uint32_t slot_bytes = (a_bytes + b_slot) * (NTERMS == 3 ? 2 : 1);
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (TC_MAX_STAGES + s); };
    auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * TC_MAX_STAGES + a); };
    auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * TC_MAX_STAGES + 2 + a); };
    const uint32_t done_bar = bar0 + 8u * (2 * TC_MAX_STAGES + 4);

    const uint32_t crank = CL > 1 ? cluster_rank() : 0u;
    const bool leader = !PAIR || crank == 0;
    // persistent loop bounds: work items, or groups of CL items (one per cluster)
    const int first = (int)(blockIdx.x / CL);
    const int stride = (int)(gridDim.x / CL);
    const int count = p.total_items;
    // work item -> (coordinates, parameters, tensor maps)
    auto fetch = [&](int item, ItemCoord& c, const TcParams*& q, const CUtensorMap*& mA_hi,
                     const CUtensorMap*& mA_lo, const CUtensorMap*& mB_hi,
                     const CUtensorMap*& mB_lo) {
        if constexpr (CL > 1) {
            q = &p;
            mA_hi = &tmA_hi; mA_lo = &tmA_lo; mB_hi = &tmB_hi; mB_lo = &tmB_lo;
            if (PAIR && p.mode == 1) {
                // group = (K slice, vector, 256-row output tile); this CTA takes one half
                const int tile = item % p.ntiles;
                const int rest = item / p.ntiles;
                const int batch = rest % p.nbatch;
                const int split = rest / p.nbatch;
                const int4 t = p.tile_list[tile];
                c.m0 = t.x * (2 * TC_BM) + (int)crank * TC_BM;
                c.n0 = t.y;
                c.nw = t.z;
                c.batch = batch;
                const int per = (p.kb_total + p.nsplit - 1) / p.nsplit;
                c.kb0 = split * per;
                c.kb1 = min(p.kb_total, c.kb0 + per);
            } else if (p.mode == 0) {
                // group = (CL neighbouring M tiles, N tile)
                const int nb = item % p.tiles_n;
                const int mp = item / p.tiles_n;
                c.m0 = (CL * mp + (int)crank) * TC_BM;
                c.n0 = nb * p.BN;
                c.nw = p.BN;
                c.batch = 0;
                c.kb0 = 0;
                c.kb1 = p.kb_total;
            } else {
                // group = (K slice, CL neighbouring vectors, output tile): the CTAs share the
                // L^P tile; a CTA whose vector index passes nbatch computes on zero-filled A
                // and writes nothing
                const int nbg = (p.nbatch + CL - 1) / CL;
                const int tile = item % p.ntiles;
                const int rest = item / p.ntiles;
                const int bg = rest % nbg;
                const int split = rest / nbg;
                const int4 t = p.tile_list[tile];
                c.m0 = t.x * TC_BM;
                c.n0 = t.y;
                c.nw = t.z;
                c.batch = bg * CL + (int)crank;
                const int per = (p.kb_total + p.nsplit - 1) / p.nsplit;
                c.kb0 = split * per;
                c.kb1 = min(p.kb_total, c.kb0 + per);
            }
        } else if constexpr (BATCHED) {
            const TcItem it = items[item];
            const TcJob* jb = jobs + it.job;
            q = &jb->p;
            mA_hi = &jb->a_hi; mA_lo = &jb->a_lo; mB_hi = &jb->b_hi; mB_lo = &jb->b_lo;
            c.m0 = it.m0; c.n0 = it.n0; c.batch = it.batch; c.kb0 = it.kb0; c.kb1 = it.kb1;
            c.nw = it.nw;
        } else {
            q = &p;
            mA_hi = &tmA_hi; mA_lo = &tmA_lo; mB_hi = &tmB_hi; mB_lo = &tmB_lo;
            c = decode_item(p, item);
        }
    };

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(full_bar(s), 1);
            // every CTA of a multicast cluster releases a slot; a pair's leader releases both
            mbar_init(empty_bar(s), PAIR ? 1 : CL);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull_bar(a), 1);
            // pair: one arrive per epilogue warp of either CTA, on the leader's barrier
            mbar_init(tempty_bar(a), PAIR ? 2 * TC_EPI_WARPS : 32 * TC_EPI_WARPS);
        }
        mbar_init(done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == TC_MMA_WARP) {
        const uint32_t ncols = p.tmem_cols;
        if constexpr (PAIR) {
            // one warp of each CTA of the pair allocates the same columns in both
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&tmem_slot)),
                         "r"(ncols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&tmem_slot)),
                         "r"(ncols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if constexpr (CL > 1) cluster_sync_all();  // peer barriers initialised before multicast
    const uint32_t tmem_base = tmem_slot;

    if (warp == TC_PRODUCER_WARP) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            // last issued parity per slot (for draining on abort)
            uint32_t issued_mask = 0, issued_par = 0;
            bool ok = true;
            for (int item = first; item < count && ok; item += stride) {
                ItemCoord c;
                const TcParams* q;
                const CUtensorMap *mA_hi, *mA_lo, *mB_hi, *mB_lo;
                fetch(item, c, q, mA_hi, mA_lo, mB_hi, mB_lo);
                const uint32_t b_bytes = (uint32_t)q->BN * TC_BK * 2;
                // a pair's leader expects both CTAs' A rows and both halves of B
                const uint32_t tx = ((PAIR ? 2 : 1) * a_bytes + b_bytes) * (NTERMS == 3 ? 2 : 1);
                for (int kb = c.kb0; kb < c.kb1; ++kb) {
                    if (!mbar_wait(empty_bar(stage), phase ^ 1u, &abort_flag, p.status, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sbase = smem_u32(smem + (size_t)stage * slot_bytes);
                    const uint32_t fb = full_bar(stage);
                    if (leader) mbar_expect_tx(fb, tx);
                    const uint32_t a_hi = sbase, b_hi = sbase + a_bytes;
                    const uint32_t a_lo = sbase + a_bytes + b_slot,
                                   b_lo = sbase + 2 * a_bytes + b_slot;
                    if constexpr (PAIR) {
                        // own A rows and own half of B, completing on the leader's barrier
                        const uint32_t fbl = mapa_rank(fb, 0);
                        const int ybh = c.n0 + (int)crank * (c.nw / 2);
                        if (q->mode == 0) {
                            const int x = q->a_col_off + kb * BKE;
                            tma_2d_pair(a_hi, mA_hi, x, c.m0, fbl);
                            tma_2d_pair(b_hi, mB_hi, kb * BKE, ybh, fbl);
                            if (NTERMS == 3) {
                                tma_2d_pair(a_lo, mA_lo, x, c.m0, fbl);
                                tma_2d_pair(b_lo, mB_lo, kb * BKE, ybh, fbl);
                            }
                        } else {
                            const int P = kb / q->kq_blocks;
                            const int qq = (kb % q->kq_blocks) * TC_BK;
                            tma_4d_pair(a_hi, mA_hi, qq, c.batch, q->row_off + c.m0, P, fbl);
                            tma_3d_pair(b_hi, mB_hi, qq, q->col_off + ybh, P, fbl);
                            if (NTERMS == 3) {
                                tma_4d_pair(a_lo, mA_lo, qq, c.batch, q->row_off + c.m0, P, fbl);
                                tma_3d_pair(b_lo, mB_lo, qq, q->col_off + ybh, P, fbl);
                            }
                        }
                    } else if (q->mode == 0) {
                        const int x = q->a_col_off + kb * BKE;
                        tma_2d(a_hi, mA_hi, x, c.m0, fb);
                        if constexpr (CL > 1) {
                            // this CTA's 1/CL of the B tile, written into every CTA of the cluster
                            const int hrows = q->BN / CL;
                            const uint32_t hoff = crank * (uint32_t)hrows * (TC_BK * 2);
                            const uint16_t all = (uint16_t)((1u << CL) - 1u);
                            tma_2d_mc(b_hi + hoff, mB_hi, kb * BKE, c.n0 + (int)crank * hrows, fb, all);
                            if (NTERMS == 3) {
                                tma_2d(a_lo, mA_lo, x, c.m0, fb);
                                tma_2d_mc(b_lo + hoff, mB_lo, kb * BKE, c.n0 + (int)crank * hrows, fb, all);
                            }
                        } else {
                            tma_2d(b_hi, mB_hi, kb * BKE, c.n0, fb);
                            if (NTERMS == 3) {
                                tma_2d(a_lo, mA_lo, x, c.m0, fb);
                                tma_2d(b_lo, mB_lo, kb * BKE, c.n0, fb);
                            }
                        }
                    } else {
                        const int P = kb / q->kq_blocks;
                        const int qq = (kb % q->kq_blocks) * TC_BK;
                        tma_4d(a_hi, mA_hi, qq, c.batch, q->row_off + c.m0, P, fb);
                        if (NTERMS == 3) tma_4d(a_lo, mA_lo, qq, c.batch, q->row_off + c.m0, P, fb);
                        if constexpr (CL > 1) {
                            // this CTA's 1/CL of the L^P tile, written into every CTA
                            const int hrows = q->BN / CL;
                            const uint32_t hoff = crank * (uint32_t)hrows * (TC_BK * 2);
                            const uint16_t all = (uint16_t)((1u << CL) - 1u);
                            const int y = q->col_off + c.n0 + (int)crank * hrows;
                            tma_3d_mc(b_hi + hoff, mB_hi, qq, y, P, fb, all);
                            if (NTERMS == 3) tma_3d_mc(b_lo + hoff, mB_lo, qq, y, P, fb, all);
                        } else {
                            tma_3d(b_hi, mB_hi, qq, q->col_off + c.n0, P, fb);
                            if (NTERMS == 3) tma_3d(b_lo, mB_lo, qq, q->col_off + c.n0, P, fb);
                        }
                    }
                    issued_mask |= 1u << stage;
                    issued_par = (issued_par & ~(1u << stage)) | (phase << stage);
                    if (++stage == S) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (abort_flag && leader) {
                // let every copy this thread issued land before the CTA exits (a pair's
                // copies complete on the leader's barriers; the final cluster barrier holds
                // the other CTA until the leader has drained them)
                for (int s = 0; s < S; ++s) {
                    if (!(issued_mask & (1u << s))) continue;
                    const uint32_t par = (issued_par >> s) & 1u;
                    const unsigned long long t0 = gtimer();
                    while (!mbar_try(full_bar(s), par) && gtimer() - t0 < TC_WAIT_NS) {
                    }
                }
            }
        }
    } else if (warp == TC_MMA_WARP) {
        if (lane == 0 && leader) {
            // ---------------- MMA issuer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (int item = first; item < count && ok; item += stride) {
                ItemCoord c;
                const TcParams* q;
                const CUtensorMap *mA_hi, *mA_lo, *mB_hi, *mB_lo;
                fetch(item, c, q, mA_hi, mA_lo, mB_hi, mB_lo);
                const int bn = c.nw;
                constexpr int MM = PAIR ? 2 * TC_BM : TC_BM;
                const uint32_t idesc = F8 ? idesc_e4m3(bn, MM) : idesc_bf16(bn, MM);
                if (!mbar_wait(tempty_bar(acc), acc_phase ^ 1u, &abort_flag, p.status, p.wait_ns)) break;
                tc_fence_after();
                const uint32_t dt = tmem_base + (uint32_t)(acc * p.slot_bn);
                for (int kb = c.kb0; kb < c.kb1; ++kb) {
                    if (!mbar_wait(full_bar(stage), phase, &abort_flag, p.status, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sbase = smem_u32(smem + (size_t)stage * slot_bytes);
                    const uint32_t a_hi = sbase, b_hi = sbase + a_bytes;
                    const uint32_t a_lo = sbase + a_bytes + b_slot,
                                   b_lo = sbase + 2 * a_bytes + b_slot;
#pragma unroll
                    for (int k = 0; k < TC_BK / 16; ++k) {
                        const uint32_t off = k * 32;
                        const uint32_t first = (kb == c.kb0 && k == 0) ? 0u : 1u;
                        if constexpr (PAIR) {
                            if constexpr (F8) {
                                mma_e4m3_pair(dt, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, first);
                                continue;
                            }
                            mma_bf16_pair(dt, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, first);
                            if (NTERMS == 3) {
                                mma_bf16_pair(dt, sw128_desc(a_hi + off), sw128_desc(b_lo + off), idesc, 1u);
                                mma_bf16_pair(dt, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc, 1u);
                            }
                            continue;
                        }
                        if constexpr (F8) {
                            mma_e4m3(dt, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, first);
                            continue;
                        }
                        mma_bf16(dt, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, first);
                        if (NTERMS == 3) {
                            mma_bf16(dt, sw128_desc(a_hi + off), sw128_desc(b_lo + off), idesc, 1u);
                            mma_bf16(dt, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc, 1u);
                        }
                    }
                    if constexpr (PAIR) mma_commit_pair_mc(empty_bar(stage), (uint16_t)3u);
                    else if constexpr (CL > 1) mma_commit_mc(empty_bar(stage), (uint16_t)((1u << CL) - 1u));
                    else mma_commit(empty_bar(stage));
                    if (++stage == S) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                if constexpr (PAIR) mma_commit_pair_mc(tfull_bar(acc), (uint16_t)3u);
                else mma_commit(tfull_bar(acc));
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1u;
            }
            // all MMAs of this CTA (of the pair) complete before TMEM is released
            if constexpr (PAIR) mma_commit_pair(done_bar);
            else mma_commit(done_bar);
            const unsigned long long t0 = gtimer();
            while (!mbar_try(done_bar, 0) && gtimer() - t0 < TC_WAIT_NS) {
            }
        }
    } else {
        // ---------------- epilogue (warps 0-7) ----------------
        // warp w reads TMEM lanes 32 * (w % 4) .. + 31 (one output row per thread) and the
        // columns [cbeg, cend) of its half of the tile
        const int quarter = warp & 3, half = warp >> 2;
        bool bulk_pending = false;  // this warp's staging tile is being read by a bulk store
        int acc = 0;
        uint32_t acc_phase = 0;
        const int row = quarter * 32 + lane;
        for (int item = first; item < count; item += stride) {
            ItemCoord c;
            const TcParams* q;
            const CUtensorMap *mA_hi, *mA_lo, *mB_hi, *mB_lo;
            fetch(item, c, q, mA_hi, mA_lo, mB_hi, mB_lo);
            const int bn = c.nw;
            const int bn2 = ((bn / 2) + 15) / 16 * 16;  // half-tile split on a 16-column boundary
            const int cbeg = half == 0 ? 0 : bn2, cend = half == 0 ? min(bn2, bn) : bn;
            if (!mbar_wait(tfull_bar(acc), acc_phase, &abort_flag, p.status, p.wait_ns)) break;
            tc_fence_after();
            const uint32_t tbase =
                tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * p.slot_bn);
            if (q->mode == 0) {
                const int64_t R = (int64_t)c.m0 + row;
                const bool rok = R < q->M_rows;
                const int n_per_j = q->n_per_j, n_total = q->n_total, k_vec = q->k_vec;
                const int64_t n_pad = q->n_pad;
                // this row's output: T[R][j][t_col_off + cc]
                __nv_bfloat16* t_hi = q->t_hi + R * k_vec * n_pad + q->t_col_off;
                __nv_bfloat16* t_lo = NTERMS == 3 ? q->t_lo + R * k_vec * n_pad + q->t_col_off : nullptr;
                const float rs = (F8 && rok) ? q->row_scale[R / n_pad] : 1.0f;
                const bool aligned = (q->t_col_off & 7) == 0 && (n_per_j & 7) == 0;
                // 8-column groups never straddle two vectors (n_per_j is a multiple of 8), so
                // the vector j and the column cc inside it advance group by group
                int n = c.n0 + cbeg;
                int j = n / n_per_j;
                int cc = n - j * n_per_j;
                if (p.epi_stage && aligned) {
                    // Coalesced form.  Per 64-column chunk each lane packs its row into the
                    // warp's staging tile (32 rows x 128 bytes, 16-byte slot g of row r at
                    // slot g ^ (r & 7), so that neither pass has bank conflicts), then the warp
                    // writes 4 rows x 128 contiguous bytes per store instruction.
                    uint8_t* stg = smem + (size_t)S * slot_bytes + (size_t)warp * (32 * 128);
                    const int64_t R0 = (int64_t)c.m0 + quarter * 32;
                    const int gl = lane & 7;  // the 16-byte group this lane stores in the row pass
                    __nv_bfloat16* t_hi0 = q->t_hi + q->t_col_off;
                    __nv_bfloat16* t_lo0 = NTERMS == 3 ? q->t_lo + q->t_col_off : nullptr;
                    for (int c0 = cbeg; c0 < cend; c0 += 64) {
                        uint32_t lo_w[NTERMS == 3 ? 8 : 1][4];
#pragma unroll
                        for (int hc = 0; hc < 2; ++hc) {
                            const int cb = c0 + 32 * hc;
                            float v[32];
                            if (cb < cend) tmem_ld32(tbase + cb, cb + 16 < cend, v);
                            if (hc == 0 && bulk_pending) {
                                // the previous bulk store has read the staging tile
                                if (lane == 0) bulk_wait_read();
                                __syncwarp();
                                bulk_pending = false;
                            }
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                const int g = 4 * hc + h;
                                const float sc = (F8 && n < n_total) ? rs * q->col_scale[j] : 1.0f;
                                uint4 hv;
                                uint32_t* hw = (uint32_t*)&hv;
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    float x0 = v[8 * h + 2 * e], x1 = v[8 * h + 2 * e + 1];
                                    if (F8) {
                                        x0 *= sc;
                                        x1 *= sc;
                                    }
                                    const __nv_bfloat162 hb = __floats2bfloat162_rn(x0, x1);
                                    hw[e] = *(const uint32_t*)&hb;
                                    if constexpr (NTERMS == 3) {
                                        const float2 hf = __bfloat1622float2(hb);
                                        const __nv_bfloat162 lb = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
                                        lo_w[g][e] = *(const uint32_t*)&lb;
                                    }
                                }
                                if (cb < cend)
                                    *(uint4*)(stg + lane * 128 + ((g ^ (lane & 7)) << 4)) = hv;
                                n += 8;
                                cc += 8;
                                if (cc >= n_per_j) {
                                    cc -= n_per_j;
                                    ++j;
                                }
                            }
                        }
                        // the chunk's first column: vector jc, column ccc inside it
                        const int nc = c.n0 + c0;
                        const int jc = nc / n_per_j, ccc = nc - jc * n_per_j;
                        // whole chunk inside one vector and inside the tile: one bulk tensor
                        // store of the staged box (its layout is the 128-byte swizzle)
                        const bool bulk = p.t_store && c0 + 64 <= cend && ccc + 64 <= n_per_j &&
                                          nc + 64 <= n_total;
                        // row pass otherwise: lane writes group gl of rows 4 i + lane / 8
                        const int ng = nc + 8 * gl;
                        const bool gok = c0 + 8 * gl < cend && ng < n_total;
                        const int jg = ng / n_per_j;
                        const int64_t cg = (int64_t)jg * n_pad + (ng - jg * n_per_j);
#pragma unroll
                        for (int t = 0; t < (NTERMS == 3 ? 2 : 1); ++t) {
                            if (t == 1) {
                                if (bulk) {
                                    if (lane == 0) bulk_wait_read();
                                    __syncwarp();
                                }
#pragma unroll
                                for (int g = 0; g < 8; ++g)
                                    if constexpr (NTERMS == 3)
                                        *(uint4*)(stg + lane * 128 + ((g ^ (lane & 7)) << 4)) =
                                            make_uint4(lo_w[g][0], lo_w[g][1], lo_w[g][2], lo_w[g][3]);
                            }
                            if (bulk) {
                                fence_proxy_async_smem();
                                __syncwarp();
                                if (lane == 0 && R0 < q->M_rows) {
                                    tma_store_3d(t == 0 ? &tmT_hi : &tmT_lo, smem_u32(stg), ccc, jc, (int)R0);
                                    bulk_commit();
                                }
                                continue;
                            }
                            __syncwarp();
                            __nv_bfloat16* dst = t == 0 ? t_hi0 : t_lo0;
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const int r = 4 * i + (lane >> 3);
                                const uint4 val = *(const uint4*)(stg + r * 128 + ((gl ^ (r & 7)) << 4));
                                const int64_t R = R0 + r;
                                if (gok && R < q->M_rows) *(uint4*)(dst + R * k_vec * n_pad + cg) = val;
                            }
                            __syncwarp();
                        }
                        if (bulk) bulk_pending = true;
                    }
                } else
                for (int c0 = cbeg; c0 < cend; c0 += 32) {
                    float v[32];
                    tmem_ld32(tbase + c0, c0 + 16 < cend, v);
                    if (!rok) continue;
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        if (c0 + 8 * h < cend && n < n_total) {
                            const float sc = F8 ? rs * q->col_scale[j] : 1.0f;
                            const int64_t off = (int64_t)j * n_pad + cc;
                            if (aligned) {
                                uint4 hv, lv;
                                uint32_t* hw = (uint32_t*)&hv;
                                uint32_t* lw = (uint32_t*)&lv;
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    float x0 = v[8 * h + 2 * e], x1 = v[8 * h + 2 * e + 1];
                                    if (F8) {
                                        x0 *= sc;
                                        x1 *= sc;
                                    }
                                    const __nv_bfloat162 hb = __floats2bfloat162_rn(x0, x1);
                                    hw[e] = *(const uint32_t*)&hb;
                                    if (NTERMS == 3) {
                                        const float2 hf = __bfloat1622float2(hb);
                                        const __nv_bfloat162 lb = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
                                        lw[e] = *(const uint32_t*)&lb;
                                    }
                                }
                                *(uint4*)(t_hi + off) = hv;
                                if (NTERMS == 3) *(uint4*)(t_lo + off) = lv;
                            } else {
                                for (int e = 0; e < 8; ++e) {
                                    const int ne = n + e;
                                    if (ne >= n_total) break;
                                    const int je = ne / n_per_j;
                                    const int ce = ne - je * n_per_j;
                                    const int64_t o = (int64_t)je * n_pad + ce;
                                    const float x = F8 ? v[8 * h + e] * rs * q->col_scale[je] : v[8 * h + e];
                                    const __nv_bfloat16 hb = __float2bfloat16_rn(x);
                                    t_hi[o] = hb;
                                    if (NTERMS == 3) t_lo[o] = __float2bfloat16_rn(x - __bfloat162float(hb));
                                }
                            }
                        }
                        n += 8;
                        cc += 8;
                        if (cc >= n_per_j) {
                            cc -= n_per_j;
                            ++j;
                        }
                    }
                }
            } else {
                const int a = c.m0 + row;
                const bool rok = a < q->m_valid && c.batch < q->nbatch;
                const int n_valid = q->n_valid;
                float* Ob = q->O + (int64_t)c.batch * q->n_pad * q->n_pad +
                            (int64_t)(q->row_off + a) * q->n_pad + q->col_off;
                for (int c0 = cbeg; c0 < cend; c0 += 32) {
                    float v[32];
                    tmem_ld32(tbase + c0, c0 + 16 < cend, v);
                    if (!rok) continue;
                    // four columns per vector reduction (16-byte aligned: n_pad and the block
                    // offsets are multiples of 8 floats), single ones at a ragged edge
#pragma unroll
                    for (int e = 0; e < 32; e += 4) {
                        const int b = c.n0 + c0 + e;
                        if (c0 + e + 3 < cend && b + 3 < n_valid) {
                            atomicAdd(reinterpret_cast<float4*>(Ob + b), make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]));
                        } else {
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                if (c0 + e + u < cend && b + u < n_valid) atomicAdd(Ob + b + u, v[e + u]);
                        }
                    }
                }
            }
            tc_fence_before();
            if constexpr (PAIR) {
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(mapa_rank(tempty_bar(acc), 0));
            } else {
                mbar_arrive(tempty_bar(acc));
            }
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
        // the bulk stores of T are complete before the CTA exits
        if (lane == 0) bulk_wait_all();
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // no CTA leaves while its peer may still write into its shared memory or barriers
    if constexpr (CL > 1) cluster_sync_all();
    if (warp == TC_MMA_WARP) {
        __syncwarp();
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                         "r"((uint32_t)p.tmem_cols)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                         "r"((uint32_t)p.tmem_cols)
                         : "memory");
    }
}

// ---------------------------------------------------------------------------
// Host side: tensor maps through the driver entry point (no link to libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    });
    return fn;
}

}  // namespace

int make_tmap_bf16(CUtensorMap* map, const void* ptr, int rank, const uint64_t* dims,
                   const uint64_t* strides_bytes, const uint32_t* box) {
    return make_tmap(map, ptr, rank, dims, strides_bytes, box, 2);
}

int make_tmap(CUtensorMap* map, const void* ptr, int rank, const uint64_t* dims,
              const uint64_t* strides_bytes, const uint32_t* box, int elt_bytes) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return set_error(PPRPA_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    if (((uintptr_t)ptr & 15) != 0) return set_error(PPRPA_ERR_ARG, "tensor map base not 16-byte aligned");
    cuuint64_t d[5], s[4];
    cuuint32_t b[5], e[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        b[i] = box[i];
        e[i] = 1;
        if (i + 1 < rank) {
            s[i] = strides_bytes[i];
            if (s[i] % 16 != 0) return set_error(PPRPA_ERR_ARG, "tensor map stride not a multiple of 16 bytes");
        }
    }
    const CUtensorMapDataType dt = elt_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = fn(map, dt, (cuuint32_t)rank, const_cast<void*>(ptr),
                    d, s, b, e, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(PPRPA_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return PPRPA_OK;
}

int tc_stages_for(int BN, int nterms, bool epi_stage) {
    const int slot = (TC_BM * TC_BK * 2 + BN * TC_BK * 2) * (nterms == 3 ? 2 : 1);
    int s = (TC_SMEM_LIMIT - 2048 - (epi_stage ? TC_EPI_BYTES : 0)) / slot;
    if (s > TC_MAX_STAGES) s = TC_MAX_STAGES;
    return s;
}

static int slot_bytes_for(int BN, int nterms) {
    return (TC_BM * TC_BK * 2 + BN * TC_BK * 2) * (nterms == 3 ? 2 : 1);
}

// Pipeline depth and dynamic shared memory of a launch; the stage-1 staging tiles are
// reserved when `want_epi` and at least two pipeline slots still fit.
static size_t plan_smem(TcParams& p, int bn, int nterms, bool want_epi) {
    p.epi_stage = want_epi && tc_stages_for(bn, nterms, true) >= 2 ? 1 : 0;
    p.stages = tc_stages_for(bn, nterms, p.epi_stage != 0);
    return (size_t)slot_bytes_for(bn, nterms) * p.stages + 1024 + (p.epi_stage ? TC_EPI_BYTES : 0);
}

// Limit of the kernel's pipeline waits: PPRPA_TC_WAIT_NS nanoseconds when set (clamped to
// [1 us, 4 s]; a short limit makes a normal launch's waits run out, which is how the
// timeout path is tested), else 4 s.
static unsigned long long tc_wait_ns() {
    const char* v = getenv("PPRPA_TC_WAIT_NS");
    if (!v) return TC_WAIT_NS;
    const long long x = atoll(v);
    if (x < 1000) return 1000ull;
    return x > (long long)TC_WAIT_NS ? TC_WAIT_NS : (unsigned long long)x;
}

// Zero-filled stand-in for tensor-map parameters a launch does not use.
static const CUtensorMap& no_map() {
    static CUtensorMap m = [] {
        CUtensorMap z;
        std::memset(&z, 0, sizeof(z));
        return z;
    }();
    return m;
}

int tc_gemm_launch(const CUtensorMap& a_hi, const CUtensorMap& a_lo, const CUtensorMap& b_hi,
                   const CUtensorMap& b_lo, TcParams p, int nterms, int num_sms, cudaStream_t st,
                   bool f8, const CUtensorMap* t_hi, const CUtensorMap* t_lo) {
    if (p.total_items <= 0) return PPRPA_OK;
    p.wait_ns = tc_wait_ns();
    p.t_store = (p.mode == 0 && t_hi) ? 1 : 0;
    const CUtensorMap& th = t_hi ? *t_hi : no_map();
    const CUtensorMap& tl = t_lo ? *t_lo : th;
    if (p.BN < 16 || p.BN > 256 || (p.BN % 16) != 0)
        return set_error(PPRPA_ERR_ARG, "tc_gemm: BN must be a multiple of 16 in [16, 256]");
    p.slot_bn = p.BN;
    const size_t smem = plan_smem(p, p.BN, nterms, p.mode == 0);
    if (p.stages < 2) return set_error(PPRPA_ERR_ARG, "tc_gemm: tile too large for shared memory");
    int cols = 32;
    while (cols < 2 * p.BN) cols <<= 1;
    p.tmem_cols = cols;
    const int grid = p.total_items < num_sms ? p.total_items : num_sms;
    if (f8) {
        if (p.mode != 0 || nterms != 1) return set_error(PPRPA_ERR_ARG, "tc_gemm: FP8 is stage 1, one term");
        cudaFuncSetAttribute(tc_gemm_kernel<1, false, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tc_gemm_kernel<1, false, 1, true><<<grid, TC_THREADS, smem, st>>>(a_hi, a_lo, b_hi, b_lo, th, tl, p, nullptr, nullptr);
    } else if (nterms == 3) {
        cudaFuncSetAttribute(tc_gemm_kernel<3, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tc_gemm_kernel<3, false, 1><<<grid, TC_THREADS, smem, st>>>(a_hi, a_lo, b_hi, b_lo, th, tl, p, nullptr, nullptr);
    } else {
        cudaFuncSetAttribute(tc_gemm_kernel<1, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tc_gemm_kernel<1, false, 1><<<grid, TC_THREADS, smem, st>>>(a_hi, a_lo, b_hi, b_lo, th, tl, p, nullptr, nullptr);
    }
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// Stage 1 on clusters of CL CTAs sharing the B tile (TMA multicast).  Items are groups of
// CL M tiles; p.total_items is set here to the group count.  The B tensor maps must have
// boxes of BN / CL rows.
template <int NT, int CL, bool F8 = false, bool PAIR = false>
static cudaError_t launch_cluster(const CUtensorMap& a_hi, const CUtensorMap& a_lo,
                                  const CUtensorMap& b_hi, const CUtensorMap& b_lo,
                                  const CUtensorMap& t_hi, const CUtensorMap& t_lo, const TcParams& p,
                                  size_t smem, int groups, int num_sms, cudaStream_t st) {
    cudaFuncSetAttribute(tc_gemm_kernel<NT, false, CL, F8, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = std::min(groups, num_sms / CL);
    cfg.gridDim = dim3(CL * clusters);
    int maxc = 0;
    if (cudaOccupancyMaxActiveClusters(&maxc, tc_gemm_kernel<NT, false, CL, F8, PAIR>, &cfg) == cudaSuccess && maxc > 0)
        clusters = std::min(clusters, maxc);
    cfg.gridDim = dim3(CL * clusters);
    const TcJob* nj = nullptr;
    const TcItem* ni = nullptr;
    return cudaLaunchKernelEx(&cfg, tc_gemm_kernel<NT, false, CL, F8, PAIR>, a_hi, a_lo, b_hi, b_lo, t_hi,
                              t_lo, p, nj, ni);
}

int tc_gemm_launch_cluster(const CUtensorMap& a_hi, const CUtensorMap& a_lo,
                           const CUtensorMap& b_hi_part, const CUtensorMap& b_lo_part, TcParams p,
                           int nterms, int cl, int num_sms, cudaStream_t st, bool f8, bool pair,
                           const CUtensorMap* t_hi, const CUtensorMap* t_lo) {
    p.wait_ns = tc_wait_ns();
    p.t_store = (p.mode == 0 && t_hi) ? 1 : 0;
    const CUtensorMap& th = t_hi ? *t_hi : no_map();
    const CUtensorMap& tl = t_lo ? *t_lo : th;
    if (cl != 2 && cl != 4) return set_error(PPRPA_ERR_ARG, "tc_gemm_cluster: cluster size 2 or 4");
    if (pair && (cl != 2 || (p.BN % 32) != 0))
        return set_error(PPRPA_ERR_ARG, "tc_gemm_cluster: a CTA pair is a cluster of 2 with BN a multiple of 32");
    // each CTA loads BN / cl rows of the B tile: a whole number of 8-row swizzle atoms
    if (p.BN < 16 || p.BN > 256 || (p.BN % 16) != 0 || (p.BN % (8 * cl)) != 0)
        return set_error(PPRPA_ERR_ARG, "tc_gemm_cluster: BN must be a multiple of 16 and of 8 * cluster size");
    int64_t groups;
    if (p.mode == 0) {
        const int64_t mtiles = ceil_div(p.M_rows, TC_BM);
        groups = ceil_div(mtiles, cl) * p.tiles_n;
    } else {
        if (!p.tile_list || p.ntiles <= 0 || p.nbatch <= 0 || p.nsplit <= 0)
            return set_error(PPRPA_ERR_ARG, "tc_gemm_cluster: stage-2 parameters missing");
        // pair: one group per (256-row tile, vector, K slice); else CL vectors per group
        groups = (int64_t)p.ntiles * (pair ? p.nbatch : ceil_div(p.nbatch, cl)) * p.nsplit;
    }
    if (groups <= 0) return PPRPA_OK;
    if (groups > INT32_MAX) return set_error(PPRPA_ERR_ARG, "tc_gemm_cluster: too many tiles");
    p.total_items = (int)groups;
    p.slot_bn = p.BN;
    // a pair's CTA holds half of the B tile
    const size_t smem = plan_smem(p, pair ? p.BN / 2 : p.BN, nterms, p.mode == 0);
    if (p.stages < 2) return set_error(PPRPA_ERR_ARG, "tc_gemm_cluster: tile too large for shared memory");
    int cols = 32;
    while (cols < 2 * p.BN) cols <<= 1;
    p.tmem_cols = cols;
    cudaError_t e;
    if (pair) {
        if (f8 && nterms != 1) return set_error(PPRPA_ERR_ARG, "tc_gemm_cluster: FP8 is one term");
        e = f8 ? launch_cluster<1, 2, true, true>(a_hi, a_lo, b_hi_part, b_lo_part, th, tl, p, smem, (int)groups, num_sms, st)
           : nterms == 3 ? launch_cluster<3, 2, false, true>(a_hi, a_lo, b_hi_part, b_lo_part, th, tl, p, smem, (int)groups, num_sms, st)
                         : launch_cluster<1, 2, false, true>(a_hi, a_lo, b_hi_part, b_lo_part, th, tl, p, smem, (int)groups, num_sms, st);
    } else if (f8) {
        if (nterms != 1) return set_error(PPRPA_ERR_ARG, "tc_gemm_cluster: FP8 is one term");
        e = cl == 2 ? launch_cluster<1, 2, true>(a_hi, a_lo, b_hi_part, b_lo_part, th, tl, p, smem, (int)groups, num_sms, st)
                    : launch_cluster<1, 4, true>(a_hi, a_lo, b_hi_part, b_lo_part, th, tl, p, smem, (int)groups, num_sms, st);
    } else if (nterms == 3) {
        e = cl == 2 ? launch_cluster<3, 2>(a_hi, a_lo, b_hi_part, b_lo_part, th, tl, p, smem, (int)groups, num_sms, st)
                    : launch_cluster<3, 4>(a_hi, a_lo, b_hi_part, b_lo_part, th, tl, p, smem, (int)groups, num_sms, st);
    } else {
        e = cl == 2 ? launch_cluster<1, 2>(a_hi, a_lo, b_hi_part, b_lo_part, th, tl, p, smem, (int)groups, num_sms, st)
                    : launch_cluster<1, 4>(a_hi, a_lo, b_hi_part, b_lo_part, th, tl, p, smem, (int)groups, num_sms, st);
    }
    if (e != cudaSuccess) return set_error(PPRPA_ERR_CUDA, std::string("cluster launch: ") + cudaGetErrorString(e));
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

int tc_gemm_launch_batched(const TcJob* jobs, const TcItem* items, int total_items, int max_bn,
                           int nterms, int num_sms, int* status, cudaStream_t st) {
    if (total_items <= 0) return PPRPA_OK;
    if (max_bn < 16 || max_bn > 256 || (max_bn % 16) != 0)
        return set_error(PPRPA_ERR_ARG, "tc_gemm_batched: bad tile width");
    TcParams p;
    p.total_items = total_items;
    p.status = status;
    p.wait_ns = tc_wait_ns();
    p.slot_bn = max_bn;
    p.BN = max_bn;
    const size_t smem = plan_smem(p, max_bn, nterms, true);
    if (p.stages < 2) return set_error(PPRPA_ERR_ARG, "tc_gemm_batched: tile too large for shared memory");
    int cols = 32;
    while (cols < 2 * max_bn) cols <<= 1;
    p.tmem_cols = cols;
    const int grid = total_items < num_sms ? total_items : num_sms;
    CUtensorMap dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    if (nterms == 3) {
        cudaFuncSetAttribute(tc_gemm_kernel<3, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tc_gemm_kernel<3, true, 1><<<grid, TC_THREADS, smem, st>>>(dummy, dummy, dummy, dummy, dummy, dummy, p,
                                                                    jobs, items);
    } else {
        cudaFuncSetAttribute(tc_gemm_kernel<1, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tc_gemm_kernel<1, true, 1><<<grid, TC_THREADS, smem, st>>>(dummy, dummy, dummy, dummy, dummy, dummy, p,
                                                                    jobs, items);
    }
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

}  // namespace pprpa
