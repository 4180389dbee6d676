// tcgen05 tensor-core variants of the parametric GEMM for the low-precision
// forms (BF16, split BF16, per-tile scaled FP8 E4M3), FP32 accumulation in
// tensor memory.
//
// One persistent CTA per SM walks output tiles of BM x BN (BM = 128), or, for
// the CTA-pair variants, one two-CTA cluster per SM pair walks 256 x 256 tiles
// (each CTA stages and accumulates its 128 rows; the even CTA issues the MMAs
// with cta_group::2).  Warp roles:
//   warp 0  TMA producer: 128-byte-wide K slices of A (BM rows) and of B^T
//           (BN rows) land in a STAGES-deep ring of 128B-swizzled shared tiles,
//           completion tracked by mbarrier transaction counts;
//   warp 1  owns the tensor-memory allocation; one thread issues tcgen05.mma
//           (kind::f16 or kind::f8f6f4) into one of two accumulators and
//           releases each stage with tcgen05.commit;
//   warps 2.. epilogue: tcgen05.ld the accumulator (one TMEM lane per output
//           row), (FP8: scale each 128-deep chunk by sA*sB and add in
//           registers), store FP32 C, release the accumulator.
// The fused-conversion programs (128 x 64 tiles, N <= 64) add eight converter
// warps after the epilogue warps: the producer loads A in FP32 into a ring of its
// own and only B^T into the stages; the converters write A's BF16 tiles (hi, and
// lo for split) into the stages.  Their work units may be K slices of a tile,
// whose partial products k_slice_reduce sums in slice order.
// Every wait is bounded (globaltimer); on timeout the CTA sets the device
// error word, stops issuing, drains its own TMA and MMA work and frees TMEM.
//
// Operands are K-major: A is M x K and B is given transposed (N x K), as the
// preparation kernels write it.  Tails in M, N and K come from TMA's zero fill.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <mutex>
#include <vector>

#include "pgk_internal.cuh"

namespace pgk {

// MODE_SPLIT stages hi and lo of both operands together and issues the three
// products per K step; MODE_SPLIT3 runs three BF16-sized passes per K block
// ((lo_a, hi_b), (hi_a, lo_b), (hi_a, hi_b)) for a deeper pipeline.
enum { MODE_BF16 = 0, MODE_SPLIT = 1, MODE_FP8 = 2, MODE_SPLIT3 = 3 };

static constexpr unsigned long long WAIT_LIMIT_NS = 4000000000ULL;  // 4 s
// drains after an abort: copies and MMAs already issued finish within microseconds;
// a pair leader may also wait on a stage its peer never filled, so keep this short
static constexpr unsigned long long DRAIN_LIMIT_NS = 100000000ULL;  // 100 ms
static constexpr unsigned int ERR_TIMEOUT_PRODUCER = 0x1u;
static constexpr unsigned int ERR_TIMEOUT_MMA = 0x2u;
static constexpr unsigned int ERR_TIMEOUT_EPILOGUE = 0x4u;
static constexpr unsigned int ERR_TIMEOUT_DRAIN = 0x8u;
static constexpr unsigned int ERR_TIMEOUT_SELFTEST = 0x10u;

template <int MODE_, int BN_, int STAGES_, bool PAIR_ = false, int FSTAGES_ = 0>
struct TcCfg {
    static constexpr int MODE = MODE_, BN = BN_, STAGES = STAGES_;
    static constexpr bool PAIR = PAIR_;
    // Fused conversion (FSTAGES > 0): A arrives in FP32 through an FSTAGES-deep ring
    // (per K block two TMA boxes of 128 rows x 32 FP32, 128B-swizzled) and converter
    // warps write its BF16 tiles (hi, and lo for split) into the stage ring, so A is
    // read from memory once; only B^T (prepared, BF16) travels by TMA into the stages.
    static constexpr int FSTAGES = FSTAGES_;
    static constexpr bool FUSED = FSTAGES > 0;
    static constexpr int BM = 128;                          // rows of A staged (and accumulated) per CTA
    static constexpr int CTAS = PAIR ? 2 : 1;               // CTAs sharing one output tile
    static constexpr int TM = BM * CTAS;                    // rows of an output tile
    static constexpr int BNL = BN / CTAS;                   // rows of B^T staged per CTA
    static constexpr int BK = MODE == MODE_FP8 ? 128 : 64;   // elements per stage row (128 bytes)
    static constexpr int UK = MODE == MODE_FP8 ? 32 : 16;    // K per MMA instruction
    static constexpr int NKSUB = BK / UK;                   // MMAs per stage and product
    static constexpr int A_BYTES = BM * 128;
    static constexpr int B_BYTES = BNL * 128;
    static constexpr int NOPS = MODE == MODE_SPLIT ? 2 : 1; // hi/lo pairs per stage
    static constexpr int PASSES = MODE == MODE_SPLIT3 ? 3 : 1;  // stages per K block
    static constexpr int STAGE_BYTES = NOPS * (A_BYTES + B_BYTES);
    // K blocks accumulated in tensor memory before the epilogue folds the chunk
    // into FP32 registers (0 = whole K in tensor memory).  FP8: every 128-deep
    // chunk carries its own scales.  Split: 512-deep chunks bound the growth
    // of the tensor-core accumulator, the dominant error at large K.
    static constexpr int CHUNK =
        MODE == MODE_FP8 ? 1 : ((MODE == MODE_SPLIT || MODE == MODE_SPLIT3) ? 8 : 0);
    // epilogue warps: 8 fold the chunked forms' wide tiles; a fused 64-wide tile needs 4
    static constexpr int EPI_WARPS = (CHUNK == 0 || FSTAGES_ > 0) ? 4 : 8;
    // FP8 hands an accumulator to the epilogue every 128-deep chunk: the waits of
    // the producer, the MMA issuer and the epilogue poll (mbarrier.test_wait)
    // instead of suspending (try_wait), which shortens the round trip from an
    // MMA's completion to the reuse of its accumulator
    static constexpr bool POLL = MODE == MODE_FP8;
    static constexpr int CONV_WARPS = FUSED ? 8 : 0;        // warps after the epilogue warps
    static constexpr int THREADS = 64 + 32 * (EPI_WARPS + CONV_WARPS);
    static constexpr int F_BYTES = FUSED ? 2 * BM * 128 : 0;  // one FP32 K block of A (two boxes)
    // tensor-memory accumulators in flight: FP8 with 128-wide tiles keeps four
    // chunk accumulators so the MMA can run three chunks ahead of the epilogue
    static constexpr int ACC_BUFS = (MODE == MODE_FP8 && BN == 128) ? 4 : 2;
    static constexpr int TMEM_COLS = ACC_BUFS * BN;
    // epilogue staging: one 32 x 33 FP32 block per epilogue warp after the stage ring
    static constexpr int XPOSE_BYTES = EPI_WARPS * 32 * 33 * 4;
    static constexpr int SMEM_RAW = STAGES * STAGE_BYTES + FSTAGES * F_BYTES + XPOSE_BYTES + 1024;
    // at least 116 KB so that one CTA owns the SM (and its tensor memory)
    static constexpr int SMEM = SMEM_RAW > 118784 ? SMEM_RAW : 118784;
    static_assert(TMEM_COLS == 128 || TMEM_COLS == 256 || TMEM_COLS == 512,
                  "TMEM allocation is a power of two");
    static_assert(!FUSED || (!PAIR && (MODE == MODE_BF16 || MODE == MODE_SPLIT) && BN == 64),
                  "fused conversion: single-CTA BF16 and split tiles of 128 x 64");
    static_assert(SMEM <= 232448 - 512, "stage ring, staging blocks and barriers fit the opt-in shared memory");
    static_assert(CHUNK == 0 || BN / (EPI_WARPS / 4) <= 128, "promoted columns per warp");
    static_assert(!PAIR || (MODE != MODE_FP8 && BN == 256), "CTA pairs: kind::f16 forms, 256 x 256 tiles");
};

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test of the phase with parity `parity` (never suspends the thread).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with parity `parity`.  Returns false if the CTA
// was aborted by another warp or the limit expired (then the abort flag and
// the device error word are set).  POLL spins on test_wait instead of letting
// try_wait suspend the thread, for the waits on the critical path.
template <bool POLL = false>
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned int* err, unsigned int code,
                                          unsigned long long limit_ns = WAIT_LIMIT_NS) {
    if (POLL ? mbar_test_wait(bar, parity) : mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (POLL ? mbar_test_wait(bar, parity) : mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > limit_ns) {
                *abort_flag = 1;
                atomicOr(err, code);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tmap_prefetch(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)map) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// K-major operand tile in the canonical 128-byte swizzled layout: rows of 128
// bytes, groups of 8 rows 1024 bytes apart (stride byte offset), tile base
// 1024-byte aligned; version field 1 (bits 46-47), layout SWIZZLE_128B (2).
__device__ __forceinline__ uint64_t sdesc_k128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptors: D = F32 (bits 4-5 = 1), A/B formats (bits 7-9,
// 10-12), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// 32 TMEM lanes x 32 consecutive 32-bit columns -> 32 registers per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
}

// Paired FP32 arithmetic for the chunk fold: two IEEE fused multiply-adds
// (the rounding of fmaf) per instruction on a 64-bit register pair.
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_fma(uint64_t& acc, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
__device__ __forceinline__ float f2_lo(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2_hi(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------- CTA pairs (cta_group::2)
// Two CTAs of a cluster share one 256-row tile: each stages its own 128 rows of A
// and its own half of the B^T rows, the even CTA (the leader) issues the MMAs,
// which read both CTAs' shared tiles and write both CTAs' tensor memory.
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// First tile and tile stride of this CTA's work unit (a CTA, or a CTA pair).
template <bool PAIR>
__device__ __forceinline__ int tile_first() {
    return PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
}
template <bool PAIR>
__device__ __forceinline__ unsigned tile_stride() {
    return PAIR ? gridDim.x >> 1 : gridDim.x;
}
// rank of this CTA in its pair (0: the leader); 0 for single-CTA tiles
template <bool PAIR>
__device__ __forceinline__ uint32_t pair_rank() {
    if constexpr (PAIR) return cluster_ctarank();
    return 0u;
}

// shared::cluster address of the same shared-memory offset in CTA `rank`
__device__ __forceinline__ uint32_t mapa_shared(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// TMA tile load into this CTA's shared memory whose completion is counted on an
// mbarrier of either CTA of the pair (bar: shared::cluster address)
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint32_t bar, int x,
                                                 int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void mma_f16_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                             uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

// arrive on the mbarrier at this offset in both CTAs of the pair once the MMAs
// issued so far have completed
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)), "h"((unsigned short)3)
        : "memory");
}

// arrive on the leader's mbarrier only (the drain of an aborted launch)
__device__ __forceinline__ void mma_commit_pair_local(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// arrive on an mbarrier of either CTA of the cluster (bar: shared::cluster address)
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

// One problem of a grouped launch: its sizes, the first rows of its operands in
// the packed workspaces (A: M rows, B^T: N rows, both K-major with zeros from K
// to the next multiple of the K block) and its output.
struct TcProb {
    float* C;
    int M, N, K, ldc;
    int rowA, rowB;
};

struct TcParams {
    int M, N, K;
    float* C;
    int ldc;
    int beta;
    // tail balancing: the last `tail` tiles of the tile order run as two tiles of
    // BN/2 columns each (set when they would otherwise fill at most half a round)
    int tail;
    const float* sA;   // FP8: ceil(M/128) x ceil(K/128)
    const float* sB;   // FP8: ceil(K/128) x ceil(N/128)
    unsigned int* err;
    // grouped launch: tile t is (problem, tile row, tile column) = gtiles[t].x, .y, .z
    const int4* gtiles;
    const TcProb* gprobs;
    int ntiles_g;
    // fused-conversion programs split over K: work unit t is K slice t % kslices of tile
    // t / kslices (kper K blocks each, the last one shorter); slice s writes its partial
    // product to part + s M N (row stride N), summed into C by a second launch
    int kslices, kper;
    float* part;
};

// Tensor maps of one launch: A and B^T (hi, and lo for the split forms), and B^T
// with half-height boxes for the column halves of tail-balanced tiles.
struct TcMaps {
    CUtensorMap a, b, a2, b2, bh, b2h;
};

// TAIL: the instantiation that runs the last p.tail tiles as column halves; the
// others compile without any of that logic in their loops.
template <class Cfg, bool GROUPED = false, bool TAIL = false>
__global__ void __launch_bounds__(Cfg::THREADS, 1)
    k_tc_gemm(const __grid_constant__ TcMaps tm, TcParams p) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[Cfg::STAGES];
    __shared__ uint64_t empty_bar[Cfg::STAGES];
    __shared__ uint64_t accf_bar[Cfg::ACC_BUFS];
    __shared__ uint64_t acce_bar[Cfg::ACC_BUFS];
    __shared__ uint64_t drain_bar;
    // fused conversion: the FP32 ring of A (filled by TMA, emptied by the converters)
    __shared__ uint64_t ffull_bar[Cfg::FUSED ? Cfg::FSTAGES : 1];
    __shared__ uint64_t fempty_bar[Cfg::FUSED ? Cfg::FSTAGES : 1];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;

    constexpr bool PAIR = Cfg::PAIR;
    static_assert(!(PAIR && GROUPED), "grouped launches use single-CTA tiles");
    static_assert(!TAIL || (!GROUPED && Cfg::BN == 256 && Cfg::MODE != MODE_FP8),
                  "tail halves: 256-wide single launches of the BF16 and split forms");
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t* tiles = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    // CTA pairs: rank 0 (the leader) issues the MMAs; the pair walks the tiles as one
    // unit.  The unit's first tile, its stride and the CTA's rank are read where the
    // roles use them (tile_first, tile_stride, pair_rank): copies taken here, before
    // the barriers and the allocation, made every role about 10 % slower.

    const int tiles_m = (p.M + Cfg::TM - 1) / Cfg::TM;
    const int tiles_n = (p.N + Cfg::BN - 1) / Cfg::BN;
    const int nfull = tiles_m * tiles_n;
    const int tail = TAIL ? p.tail : 0;
    // work units: every tile, the last `tail` of them twice (one per column half)
    const int ksl = (Cfg::FUSED && p.kslices > 1) ? p.kslices : 1;
    const int ntiles = GROUPED ? p.ntiles_g : (nfull + tail) * ksl;
    const int nkb = (p.K + Cfg::BK - 1) / Cfg::BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            // fused: the producer's B^T copies and one arrival per converter warp
            mbar_init(&full_bar[s], 1 + Cfg::CONV_WARPS);
            mbar_init(&empty_bar[s], 1);
        }
        for (int s = 0; s < Cfg::FSTAGES; ++s) {
            mbar_init(&ffull_bar[s], 1);
            mbar_init(&fempty_bar[s], Cfg::CONV_WARPS);
        }
        for (int b = 0; b < Cfg::ACC_BUFS; ++b) {
            mbar_init(&accf_bar[b], 1);
            // one arrival per epilogue warp (of both CTAs of a pair, at the leader)
            mbar_init(&acce_bar[b], Cfg::EPI_WARPS * Cfg::CTAS);
        }
        mbar_init(&drain_bar, 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tmap_prefetch(&tm.a);
        tmap_prefetch(&tm.b);
        if (Cfg::MODE == MODE_SPLIT || Cfg::MODE == MODE_SPLIT3) {
            tmap_prefetch(&tm.a2);
            tmap_prefetch(&tm.b2);
        }
    }
    if (warp == 1) {
        // a pair allocates collectively: one warp of each CTA, the same columns in both
        if (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&tmem_base_sh)),
                         "r"((uint32_t)Cfg::TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&tmem_base_sh)),
                         "r"((uint32_t)Cfg::TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    // the peer's barriers are initialised before any copy, commit or arrival targets them
    if (PAIR) cluster_sync();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_sh;
    volatile int* abort_flag = &abort_sh;

    // tile t -> (tm, tn): groups of 2048 rows of tiles (16 single-CTA or 8 pair tile
    // rows) walked column by column, so that the tiles resident at once share
    // operand panels in L2
    auto coords = [&](int t, int& tm, int& tn) {
        const int G = 16 * Cfg::BM / Cfg::TM;
        const int per = G * tiles_n;
        const int g = t / per;
        const int first = g * G;
        const int gm = min(tiles_m - first, G);
        const int r = t - g * per;
        tm = first + r % gm;
        tn = r / gm;
    };
    // everything a warp needs about tile t: its position, its problem's sizes and
    // output, and where its operands start in the packed workspaces (grouped)
    struct TileInfo {
        int tm, tn, M, N, nkb, rowA, rowB, ldc;
        int half;   // -1: the whole tile; 0 or 1: its first or second BN/2 columns
        int kb0;    // first K block (a K slice of a fused-conversion program), else 0
        int beta;
        float* C;
    };
    auto tile_info = [&](int t) {
        TileInfo ti;
        if (GROUPED) {
            const int4 d = __ldg(p.gtiles + t);
            const TcProb* q = p.gprobs + d.x;
            ti.tm = d.y;
            ti.tn = d.z;
            ti.M = q->M;
            ti.N = q->N;
            ti.nkb = (q->K + Cfg::BK - 1) / Cfg::BK;
            ti.rowA = q->rowA;
            ti.rowB = q->rowB;
            ti.ldc = q->ldc;
            ti.C = q->C;
            ti.half = -1;
            ti.kb0 = 0;
            ti.beta = p.beta;
        } else {
            int tt = t;
            ti.half = -1;
            int sl = 0;
            if (Cfg::FUSED && ksl > 1) {
                sl = t % ksl;
                tt = t / ksl;
            }
            if (TAIL && t >= nfull - tail) {
                const int j = t - (nfull - tail);
                tt = nfull - tail + (j >> 1);
                ti.half = j & 1;
            }
            coords(tt, ti.tm, ti.tn);
            ti.M = p.M;
            ti.N = p.N;
            ti.nkb = nkb;
            ti.rowA = 0;
            ti.rowB = 0;
            ti.ldc = p.ldc;
            ti.C = p.C;
            ti.kb0 = 0;
            ti.beta = p.beta;
            if (Cfg::FUSED && ksl > 1) {
                ti.kb0 = sl * p.kper;
                ti.nkb = min(nkb - ti.kb0, p.kper);
                ti.C = p.part + (size_t)sl * p.M * p.N;
                ti.ldc = p.N;
                ti.beta = 0;
            }
        }
        return ti;
    };

    uint8_t* fring = tiles + (size_t)Cfg::STAGES * Cfg::STAGE_BYTES;   // FP32 ring (fused)
    if (Cfg::FUSED && warp == 0) {
        // ------------------------------------------------ producer (fused)
        // per K block: the FP32 slice of A (two 128-row x 32-column boxes) into the
        // FP32 ring, and B^T hi (and lo) into the stage the converters fill with A
        if (lane == 0) {
            int stage = 0, fs = 0;
            uint32_t phase = 0, fphase = 0;
            uint32_t issued = 0, parity = 0, fissued = 0, fparity = 0;
            bool ok = true;
            for (int t = tile_first<PAIR>(); t < ntiles && ok; t += tile_stride<PAIR>()) {
                const TileInfo ti = tile_info(t);
                const int ya = ti.tm * Cfg::TM;
                const int yb = ti.tn * Cfg::BN;
                for (int kb = 0; kb < ti.nkb && ok; ++kb) {
                    const int x = (ti.kb0 + kb) * Cfg::BK;
                    if (!mbar_wait<Cfg::POLL>(&fempty_bar[fs], fphase ^ 1u, abort_flag, p.err,
                                              ERR_TIMEOUT_PRODUCER)) {
                        ok = false;
                        break;
                    }
                    uint8_t* fd = fring + (size_t)fs * Cfg::F_BYTES;
                    mbar_arrive_expect_tx(&ffull_bar[fs], (uint32_t)Cfg::F_BYTES);
                    tma_load_2d(fd, &tm.a, &ffull_bar[fs], x, ya);
                    tma_load_2d(fd + Cfg::F_BYTES / 2, &tm.a, &ffull_bar[fs], x + 32, ya);
                    fissued |= 1u << fs;
                    fparity = (fparity & ~(1u << fs)) | (fphase << fs);
                    if (++fs == Cfg::FSTAGES) {
                        fs = 0;
                        fphase ^= 1u;
                    }
                    if (!mbar_wait<Cfg::POLL>(&empty_bar[stage], phase ^ 1u, abort_flag, p.err,
                                              ERR_TIMEOUT_PRODUCER)) {
                        ok = false;
                        break;
                    }
                    uint8_t* st = tiles + (size_t)stage * Cfg::STAGE_BYTES;
                    mbar_arrive_expect_tx(&full_bar[stage], (uint32_t)(Cfg::NOPS * Cfg::B_BYTES));
                    tma_load_2d(st + Cfg::A_BYTES, &tm.b, &full_bar[stage], x, yb);
                    if (Cfg::MODE == MODE_SPLIT)
                        tma_load_2d(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES, &tm.b2, &full_bar[stage], x, yb);
                    issued |= 1u << stage;
                    parity = (parity & ~(1u << stage)) | (phase << stage);
                    if (++stage == Cfg::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // drain: every issued copy must land before the CTA may exit.  A stage
                // barrier also waits for converter arrivals that an abort may withhold,
                // so its drain is bounded by the drain limit like every other.
                for (int s = 0; s < Cfg::FSTAGES; ++s)
                    if (fissued & (1u << s)) {
                        const unsigned long long t0 = globaltimer();
                        while (!mbar_try_wait(&ffull_bar[s], (fparity >> s) & 1u)) {
                            if (globaltimer() - t0 > DRAIN_LIMIT_NS) {
                                atomicOr(p.err, ERR_TIMEOUT_DRAIN);
                                break;
                            }
                        }
                    }
                for (int s = 0; s < Cfg::STAGES; ++s)
                    if (issued & (1u << s)) {
                        const unsigned long long t0 = globaltimer();
                        while (!mbar_try_wait(&full_bar[s], (parity >> s) & 1u)) {
                            if (globaltimer() - t0 > DRAIN_LIMIT_NS) {
                                atomicOr(p.err, ERR_TIMEOUT_DRAIN);
                                break;
                            }
                        }
                    }
            }
        }
    } else if (warp == 0) {
        // ------------------------------------------------------- producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued_mask = 0, last_parity = 0;
            bool ok = true;
            for (int t = tile_first<PAIR>(); t < ntiles && ok; t += tile_stride<PAIR>()) {
                const TileInfo ti = tile_info(t);
                const bool hf = ti.half >= 0;
                // B^T rows staged by this CTA: BNL, or BNL/2 for a column half
                const int nb = hf ? Cfg::BNL / 2 : Cfg::BNL;
                const uint32_t bytes = (uint32_t)(Cfg::NOPS * (Cfg::A_BYTES + nb * 128));
                // this CTA's rows of A and of B^T (a pair splits both between its CTAs)
                const int ya = ti.rowA + ti.tm * Cfg::TM + (int)pair_rank<PAIR>() * Cfg::BM;
                const int yb = ti.rowB + ti.tn * Cfg::BN + (hf ? ti.half * (Cfg::BN / 2) : 0) +
                               (int)pair_rank<PAIR>() * nb;
                const CUtensorMap* mbh = hf ? &tm.bh : &tm.b;     // B^T hi
                const CUtensorMap* mbl = hf ? &tm.b2h : &tm.b2;   // B^T lo
                for (int kb = 0; kb < ti.nkb && ok; ++kb)
                for (int v = 0; v < Cfg::PASSES; ++v) {
                    if (!mbar_wait<Cfg::POLL>(&empty_bar[stage], phase ^ 1u, abort_flag, p.err,
                                              ERR_TIMEOUT_PRODUCER)) {
                        ok = false;
                        break;
                    }
                    uint8_t* st = tiles + (size_t)stage * Cfg::STAGE_BYTES;
                    const int x = kb * Cfg::BK;
                    // passes of MODE_SPLIT3: 0 = (A lo, B hi), 1 = (A hi, B lo), 2 = (A hi, B hi)
                    const CUtensorMap* ma = (Cfg::MODE == MODE_SPLIT3 && v == 0) ? &tm.a2 : &tm.a;
                    const CUtensorMap* mb = (Cfg::MODE == MODE_SPLIT3 && v == 1) ? mbl : mbh;
                    if (PAIR) {
                        // both CTAs' copies complete on the leader's barrier, which
                        // the leader arms with the bytes of the pair
                        const uint32_t fb = mapa_shared(smem_u32(&full_bar[stage]), 0u);
                        if (pair_rank<PAIR>() == 0) mbar_arrive_expect_tx(&full_bar[stage], bytes * 2);
                        tma_load_2d_pair(st, ma, fb, x, ya);
                        tma_load_2d_pair(st + Cfg::A_BYTES, mb, fb, x, yb);
                        if (Cfg::MODE == MODE_SPLIT) {
                            tma_load_2d_pair(st + Cfg::A_BYTES + Cfg::B_BYTES, &tm.a2, fb, x, ya);
                            tma_load_2d_pair(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES, mbl, fb, x, yb);
                        }
                    } else {
                        mbar_arrive_expect_tx(&full_bar[stage], bytes);
                        tma_load_2d(st, ma, &full_bar[stage], x, ya);
                        tma_load_2d(st + Cfg::A_BYTES, mb, &full_bar[stage], x, yb);
                        if (Cfg::MODE == MODE_SPLIT) {
                            tma_load_2d(st + Cfg::A_BYTES + Cfg::B_BYTES, &tm.a2, &full_bar[stage], x,
                                        ya);
                            tma_load_2d(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES, mbl, &full_bar[stage],
                                        x, yb);
                        }
                    }
                    issued_mask |= 1u << stage;
                    last_parity = (last_parity & ~(1u << stage)) | (phase << stage);
                    if (++stage == Cfg::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok && PAIR && pair_rank<PAIR>() != 0) {
                // the peer's copies complete on the leader's barriers, which this CTA
                // cannot observe: give copies in flight a bounded time to land (a tile
                // copy takes microseconds) before the final cluster barrier
                const unsigned long long t0 = globaltimer();
                while (globaltimer() - t0 < 200000ULL) {
                }
            } else if (!ok) {
                // drain: every issued copy must land before the CTA may exit
                for (int s = 0; s < Cfg::STAGES; ++s)
                    if (issued_mask & (1u << s)) {
                        const unsigned long long t0 = globaltimer();
                        while (!mbar_try_wait(&full_bar[s], (last_parity >> s) & 1u)) {
                            if (globaltimer() - t0 > DRAIN_LIMIT_NS) {
                                atomicOr(p.err, ERR_TIMEOUT_DRAIN);
                                break;
                            }
                        }
                    }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA
        // one thread of the leader issues for the pair (M = 256: both CTAs' A rows,
        // N = BN: both CTAs' halves of B^T, accumulators in both CTAs' tensor memory)
        if (lane == 0 && pair_rank<PAIR>() == 0) {
            // instruction descriptors of whole tiles and of column halves (N = BN/2)
            const uint32_t idesc_full = Cfg::MODE == MODE_FP8 ? idesc_e4m3(Cfg::TM, Cfg::BN)
                                                              : idesc_bf16(Cfg::TM, Cfg::BN);
            const uint32_t idesc_half = Cfg::MODE == MODE_FP8 ? idesc_e4m3(Cfg::TM, Cfg::BN / 2)
                                                              : idesc_bf16(Cfg::TM, Cfg::BN / 2);
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            bool issued_any = false;
            for (int t = tile_first<PAIR>(); t < ntiles && ok; t += tile_stride<PAIR>()) {
                const TileInfo ti = tile_info(t);
                const int tnkb = ti.nkb;
                const uint32_t idesc = ti.half >= 0 ? idesc_half : idesc_full;
                if (Cfg::CHUNK == 0) {
                    if (!mbar_wait(&acce_bar[acc], acc_phase ^ 1u, abort_flag, p.err, ERR_TIMEOUT_MMA)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                }
                for (int kb = 0; kb < tnkb; ++kb) {
                    const int kin = Cfg::CHUNK > 0 ? kb % Cfg::CHUNK : kb;  // K block within the chunk
                    if (Cfg::CHUNK > 0 && kin == 0) {
                        // a fresh accumulator for each chunk, folded by the epilogue
                        if (!mbar_wait<Cfg::POLL>(&acce_bar[acc], acc_phase ^ 1u, abort_flag, p.err,
                                                  ERR_TIMEOUT_MMA)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    for (int v = 0; v < Cfg::PASSES; ++v) {
                        if (!mbar_wait<Cfg::POLL>(&full_bar[stage], phase, abort_flag, p.err,
                                                  ERR_TIMEOUT_MMA)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d = tmem_base + (uint32_t)(acc * Cfg::BN);
                        const uint32_t sa = smem_u32(tiles + (size_t)stage * Cfg::STAGE_BYTES);
                        const uint32_t sb = sa + Cfg::A_BYTES;
#pragma unroll
                        for (int ks = 0; ks < Cfg::NKSUB; ++ks) {
                            const uint32_t koff = (uint32_t)ks * 32u;  // 32 bytes of K per MMA
                            const uint64_t da = sdesc_k128(sa + koff);
                            const uint64_t db = sdesc_k128(sb + koff);
                            const uint32_t accum = (kin > 0 || v > 0 || ks > 0) ? 1u : 0u;
                            if (Cfg::MODE == MODE_FP8) {
                                mma_f8(d, da, db, idesc, accum);
                            } else if (PAIR && (Cfg::MODE == MODE_BF16 || Cfg::MODE == MODE_SPLIT3)) {
                                mma_f16_pair(d, da, db, idesc, accum);
                            } else if (Cfg::MODE == MODE_BF16 || Cfg::MODE == MODE_SPLIT3) {
                                mma_f16(d, da, db, idesc, accum);
                            } else if (PAIR) {
                                const uint32_t sa2 = sb + Cfg::B_BYTES;   // A lo
                                const uint32_t sb2 = sa2 + Cfg::A_BYTES;  // B lo
                                const uint64_t da2 = sdesc_k128(sa2 + koff);
                                const uint64_t db2 = sdesc_k128(sb2 + koff);
                                mma_f16_pair(d, da2, db, idesc, accum);
                                mma_f16_pair(d, da, db2, idesc, 1u);
                                mma_f16_pair(d, da, db, idesc, 1u);
                            } else {
                                const uint32_t sa2 = sb + Cfg::B_BYTES;   // A lo
                                const uint32_t sb2 = sa2 + Cfg::A_BYTES;  // B lo
                                const uint64_t da2 = sdesc_k128(sa2 + koff);
                                const uint64_t db2 = sdesc_k128(sb2 + koff);
                                // small terms first: lo*hi, hi*lo, then hi*hi
                                mma_f16(d, da2, db, idesc, accum);
                                mma_f16(d, da, db2, idesc, 1u);
                                mma_f16(d, da, db, idesc, 1u);
                            }
                        }
                        issued_any = true;
                        if (PAIR)
                            mma_commit_pair(&empty_bar[stage]);
                        else
                            mma_commit(&empty_bar[stage]);
                        if (++stage == Cfg::STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    if (Cfg::CHUNK > 0 && (kin == Cfg::CHUNK - 1 || kb == tnkb - 1)) {
                        if (PAIR)
                            mma_commit_pair(&accf_bar[acc]);
                        else
                            mma_commit(&accf_bar[acc]);
                        if (++acc == Cfg::ACC_BUFS) {
                            acc = 0;
                            acc_phase ^= 1u;
                        }
                    }
                }
                if (!ok) break;
                if (Cfg::CHUNK == 0) {
                    if (PAIR)
                        mma_commit_pair(&accf_bar[acc]);
                    else
                        mma_commit(&accf_bar[acc]);
                    if (++acc == Cfg::ACC_BUFS) {
                        acc = 0;
                        acc_phase ^= 1u;
                    }
                }
            }
            if (!ok && issued_any) {
                // drain: all MMAs issued by this thread must finish before TMEM is freed
                if (PAIR)
                    mma_commit_pair_local(&drain_bar);
                else
                    mma_commit(&drain_bar);
                const unsigned long long t0 = globaltimer();
                while (!mbar_try_wait(&drain_bar, 0)) {
                    if (globaltimer() - t0 > DRAIN_LIMIT_NS) {
                        atomicOr(p.err, ERR_TIMEOUT_DRAIN);
                        break;
                    }
                }
            }
        }
        __syncwarp();
    } else if (Cfg::FUSED && warp >= 2 + Cfg::EPI_WARPS) {
        // ------------------------------------------------------- converters
        // thread (r, h): row r of the 128-row block, FP32 box h (K columns 32h ..
        // 32h + 31 of the 64-deep block).  The 16-byte chunk i of a 128-byte row
        // sits at chunk i ^ (r mod 8) (128-byte swizzle) in the FP32 boxes and in
        // the BF16 operand tiles alike, so eight consecutive rows of a quarter warp
        // touch eight different chunks: no bank conflicts either way.
        const int ct = (int)threadIdx.x - 32 * (2 + Cfg::EPI_WARPS);
        const int r = ct & 127, h = ct >> 7;
        const int rx = r & 7;
        int stage = 0, fs = 0;
        uint32_t phase = 0, fphase = 0;
        bool ok = true;
        for (int t = tile_first<PAIR>(); t < ntiles && ok; t += tile_stride<PAIR>()) {
            const TileInfo ti = tile_info(t);
            for (int kb = 0; kb < ti.nkb; ++kb) {
                int w = 1;
                if (lane == 0)
                    w = (mbar_wait<Cfg::POLL>(&ffull_bar[fs], fphase, abort_flag, p.err,
                                              ERR_TIMEOUT_PRODUCER) &&
                         mbar_wait<Cfg::POLL>(&empty_bar[stage], phase ^ 1u, abort_flag, p.err,
                                              ERR_TIMEOUT_PRODUCER)) ? 1 : 0;
                w = __shfl_sync(0xffffffffu, w, 0);
                if (!w) {
                    ok = false;
                    break;
                }
                // every lane observes both completed phases (lane 0 already has)
                while (!mbar_test_wait(&ffull_bar[fs], fphase)) {
                }
                while (!mbar_test_wait(&empty_bar[stage], phase ^ 1u)) {
                }
                const uint8_t* src = fring + (size_t)fs * Cfg::F_BYTES + h * (Cfg::F_BYTES / 2) + r * 128;
                float4 v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    v[i] = *reinterpret_cast<const float4*>(src + ((i ^ rx) << 4));
                // the FP32 slot is free once every lane of every converter warp has read it
                __syncwarp();
                if (lane == 0) mbar_arrive(&fempty_bar[fs]);
                uint8_t* dhi = tiles + (size_t)stage * Cfg::STAGE_BYTES + r * 128;
                uint8_t* dlo = dhi + Cfg::A_BYTES + Cfg::B_BYTES;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    // K columns 32h + 8i .. 32h + 8i + 7 -> 16-byte chunk 4h + i of the BF16 row
                    const float x[8] = {v[2 * i].x, v[2 * i].y, v[2 * i].z, v[2 * i].w,
                                        v[2 * i + 1].x, v[2 * i + 1].y, v[2 * i + 1].z, v[2 * i + 1].w};
                    // a pair of columns per 32-bit word, lower column in the lower half:
                    // hi = bf16(x) and lo = bf16(x - hi), both rounded to nearest even
                    // (x - hi is exact in FP32)
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const __nv_bfloat162 hp = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
                        hw[j] = *reinterpret_cast<const uint32_t*>(&hp);
                        if (Cfg::MODE == MODE_SPLIT) {
                            const float2 hf = __bfloat1622float2(hp);
                            const __nv_bfloat162 lp =
                                __floats2bfloat162_rn(x[2 * j] - hf.x, x[2 * j + 1] - hf.y);
                            lw[j] = *reinterpret_cast<const uint32_t*>(&lp);
                        }
                    }
                    const int off = ((4 * h + i) ^ rx) << 4;
                    *reinterpret_cast<uint4*>(dhi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    if (Cfg::MODE == MODE_SPLIT)
                        *reinterpret_cast<uint4*>(dlo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
                // the tensor cores read the tiles through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&full_bar[stage]);
                if (++fs == Cfg::FSTAGES) {
                    fs = 0;
                    fphase ^= 1u;
                }
                if (++stage == Cfg::STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
        }
    } else {
        // -------------------------------------------------------- epilogue
        const int e = warp - 2;
        const int q = warp & 3;                       // TMEM lane quarter of this warp
        // a thread holds 32 consecutive columns of its own row after tcgen05.ld; the
        // block goes through this warp's shared staging (pitch 33: conflict-free both
        // ways) so that every store instruction covers 32 consecutive columns of a row
        float* xp = reinterpret_cast<float*>(tiles + (size_t)Cfg::STAGES * Cfg::STAGE_BYTES +
                                             (size_t)Cfg::FSTAGES * Cfg::F_BYTES) +
                    e * (32 * 33);
        auto store_block = [&](const float (&v)[32], int row0, int cb, int M, int N, float* C,
                               int ldc, int beta) {
#pragma unroll
            for (int j = 0; j < 32; ++j) xp[lane * 33 + j] = v[j];
            __syncwarp();
            const int col = cb + lane;
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
                const int row = row0 + rr;
                if (row < M && col < N) {
                    float* cp = C + (size_t)row * ldc + col;
                    const float x = xp[rr * 33 + lane];
                    *cp = beta ? *cp + x : x;
                }
            }
            __syncwarp();
        };
        const int ncol = Cfg::BN / (Cfg::EPI_WARPS / 4);  // columns handled by this warp
        const int col0 = (e >> 2) * ncol;
        // releases an accumulator: one arrival per warp at the MMA issuer's barrier
        // (the leader's, for the peer of a pair)
        auto release = [&](int a) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (PAIR)
                    mbar_arrive_cluster(mapa_shared(smem_u32(&acce_bar[a]), 0u));
                else
                    mbar_arrive(&acce_bar[a]);
            }
        };
        int acc = 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        for (int t = tile_first<PAIR>(); t < ntiles && ok; t += tile_stride<PAIR>()) {
            const TileInfo ti = tile_info(t);
            const int tm = ti.tm;
            // first of the 32 rows of this warp (TMEM lane quarter q of this CTA's rows)
            const int row0 = tm * Cfg::TM + (int)pair_rank<PAIR>() * Cfg::BM + q * 32;
            const int n0 = ti.tn * Cfg::BN + (ti.half >= 0 ? ti.half * (Cfg::BN / 2) : 0) + col0;
            const int tN = ti.N;
            // columns of this warp inside the tile (a column half holds BN/2; the tail
            // is only used with BN = 256, where the promoted forms' 128-column warps
            // fall wholly inside or outside it); an idle warp still waits and releases
            const int wcols = ti.half >= 0 ? max(0, min(ncol, Cfg::BN / 2 - col0)) : ncol;
            if (wcols == 0) {
                // an idle warp of a column half: releases each accumulator unread, so
                // that the hot loops below keep their compile-time shapes
                const int nrel = Cfg::CHUNK > 0 ? (ti.nkb + Cfg::CHUNK - 1) / max(Cfg::CHUNK, 1) : 1;
                for (int ch = 0; ch < nrel; ++ch) {
                    int w = 1;
                    if (lane == 0)
                        w = mbar_wait(&accf_bar[acc], acc_phase, abort_flag, p.err,
                                      ERR_TIMEOUT_EPILOGUE) ? 1 : 0;
                    w = __shfl_sync(0xffffffffu, w, 0);
                    if (!w) {
                        ok = false;
                        break;
                    }
                    while (!mbar_try_wait(&accf_bar[acc], acc_phase)) {
                    }
                    tc_fence_after();
                    release(acc);
                    if (++acc == Cfg::ACC_BUFS) {
                        acc = 0;
                        acc_phase ^= 1u;
                    }
                }
                continue;
            }
            if (Cfg::CHUNK > 0) {
                constexpr int NCOL = Cfg::BN / (Cfg::EPI_WARPS / 4);
                // running FP32 sums as pairs: acc2[j] holds columns 2j, 2j + 1
                uint64_t acc2[NCOL / 2];
#pragma unroll
                for (int j = 0; j < NCOL / 2; ++j) acc2[j] = 0ull;
                const int ksa = (p.K + 127) / 128, nsb = (p.N + 127) / 128;
                constexpr int CH = Cfg::CHUNK > 0 ? Cfg::CHUNK : 1;   // (this branch has CHUNK > 0)
                const int nchunks = (ti.nkb + CH - 1) / CH;
                // FP8 chunk factors sA * sB, 32 chunks per window: lane j holds the factor
                // of chunk 32 w + j of the current window (cur) and of the next one (nxt),
                // loaded a whole window before use, so that the global-load latency never
                // sits on the fold; each chunk takes its factor by a warp shuffle.  A warp
                // whose columns all lie beyond N stores nothing; its scale index is
                // clamped so that the loads stay inside the array.
                // scale blocks of this tile: its 128-row block of A and the 128-column block
                // of B^T (both offset by the problem's first block in a grouped launch)
                const int mblk = ti.rowA / 128 + tm * Cfg::CTAS + (int)pair_rank<PAIR>();
                const int nblk = ti.rowB / 128 + min(n0 / 128, (tN - 1) / 128);
                auto chunk_scale = [&](int c) {
                    return c < nchunks
                        ? __ldg(p.sA + (size_t)mblk * ksa + c) * __ldg(p.sB + (size_t)c * nsb + nblk)
                        : 0.f;
                };
                float sc_cur = 1.f, sc_nxt = 1.f;
                if (Cfg::MODE == MODE_FP8) {
                    sc_cur = chunk_scale(lane);
                    sc_nxt = chunk_scale(32 + lane);
                }
                for (int ch = 0; ch < nchunks; ++ch) {
                    int w = 1;
                    if (lane == 0)
                        w = mbar_wait<Cfg::POLL>(&accf_bar[acc], acc_phase, abort_flag, p.err,
                                                 ERR_TIMEOUT_EPILOGUE) ? 1 : 0;
                    w = __shfl_sync(0xffffffffu, w, 0);
                    if (!w) {
                        ok = false;
                        break;
                    }
                    // every lane observes the completed phase (lane 0 already has)
                    while (!(Cfg::POLL ? mbar_test_wait(&accf_bar[acc], acc_phase)
                                       : mbar_try_wait(&accf_bar[acc], acc_phase))) {
                    }
                    tc_fence_after();
                    const float sc = Cfg::MODE == MODE_FP8 ? __shfl_sync(0xffffffffu, sc_cur, ch & 31) : 1.f;
                    if (Cfg::MODE == MODE_FP8 && (ch & 31) == 31) {
                        sc_cur = sc_nxt;
                        sc_nxt = chunk_scale(ch + 33 + lane);
                    }
                    // sum += chunk * sc with one rounding per element: FP8 sc = sA * sB (the
                    // tile scales of this 128-deep chunk); split sc = 1, i.e. sum + chunk.
                    // Two 32-column loads are in flight per wait, except for the split
                    // form's 128-column slices (a fold every 8 K blocks, off the critical path)
                    const uint64_t sc2 = f2_pack(sc, sc);
                    constexpr int NB = (NCOL == 64 || Cfg::MODE == MODE_FP8) ? 2 : 1;
                    // the accumulator is released as soon as the warp's last batch of
                    // columns is in registers, before that batch's FMAs
#pragma unroll
                    for (int c0 = 0; c0 < NCOL / 32; c0 += NB) {
                        uint32_t r[NB][32];
#pragma unroll
                        for (int c = 0; c < NB; ++c)
                            tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) +
                                          (uint32_t)(acc * Cfg::BN + col0 + (c0 + c) * 32),
                                      r[c]);
                        tmem_ld_wait();
                        if (c0 + NB >= NCOL / 32) release(acc);
#pragma unroll
                        for (int c = 0; c < NB; ++c)
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                f2_fma(acc2[(c0 + c) * 16 + j],
                                       f2_pack(__uint_as_float(r[c][2 * j]), __uint_as_float(r[c][2 * j + 1])),
                                       sc2);
                    }
                    if (++acc == Cfg::ACC_BUFS) {
                        acc = 0;
                        acc_phase ^= 1u;
                    }
                }
                if (!ok) break;
#pragma unroll
                for (int g = 0; g < NCOL / 32; ++g) {
                    float v[32];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        v[2 * i] = f2_lo(acc2[g * 16 + i]);
                        v[2 * i + 1] = f2_hi(acc2[g * 16 + i]);
                    }
                    store_block(v, row0, n0 + g * 32, ti.M, tN, ti.C, ti.ldc, ti.beta);
                }
            } else {
                int w = 1;
                if (lane == 0)
                    w = mbar_wait(&accf_bar[acc], acc_phase, abort_flag, p.err, ERR_TIMEOUT_EPILOGUE)
                            ? 1 : 0;
                w = __shfl_sync(0xffffffffu, w, 0);
                if (!w) {
                    ok = false;
                    break;
                }
                while (!mbar_try_wait(&accf_bar[acc], acc_phase)) {
                }
                tc_fence_after();
                auto drain_block = [&](int c) {
                    uint32_t r[32];
                    tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) +
                                  (uint32_t)(acc * Cfg::BN + col0 + c * 32),
                              r);
                    tmem_ld_wait();
                    float v[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
                    store_block(v, row0, n0 + c * 32, ti.M, tN, ti.C, ti.ldc, ti.beta);
                };
                if (ti.half < 0) {
#pragma unroll 1
                    for (int c = 0; c < ncol / 32; ++c) drain_block(c);
                } else {
#pragma unroll 1
                    for (int c = 0; c < wcols / 32; ++c) drain_block(c);
                }
                release(acc);
                if (++acc == Cfg::ACC_BUFS) {
                    acc = 0;
                    acc_phase ^= 1u;
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    // neither CTA of a pair leaves while the other may still arrive on its barriers
    // or the leader's MMAs may still use its shared tiles and tensor memory
    if (PAIR) cluster_sync();
    tc_fence_after();
    if (warp == 1) {
        if (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                         "r"((uint32_t)Cfg::TMEM_COLS)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                         "r"((uint32_t)Cfg::TMEM_COLS)
                         : "memory");
    }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// arrives at, with a short limit; the wait gives up, sets the error word and the
// kernel returns normally.
__global__ void k_wait_selftest(unsigned int* err, unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort_sh;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_wait(&bar, 0, &abort_sh, err, ERR_TIMEOUT_SELFTEST, limit_ns);
    }
}

// Sum of the K-slice partials of a split fused-conversion launch, in slice order
// (deterministic): C = sum_s part[s] (beta = 0) or C += sum_s part[s] (beta = 1).
__global__ void k_slice_reduce(int M, int N, const float* __restrict__ part, int slices, float* C,
                               int ldc, int beta) {
    const long long total = (long long)M * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / N), c = (int)(i - (long long)r * N);
        float acc = part[i];
        for (int y = 1; y < slices; ++y) acc += part[(size_t)y * total + i];
        float* cp = C + (size_t)r * ldc + c;
        *cp = beta ? *cp + acc : acc;
    }
}

// ------------------------------------------------------------ host side
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_tc_mu;

static pgk_status get_encoder() {
    std::lock_guard<std::mutex> lk(g_tc_mu);
    if (g_encode) return PGK_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        if (e != cudaSuccess) cudaGetLastError();
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return PGK_ERR_CUDA;
    }
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return PGK_OK;
}

// 2D K-major tensor map: rows x K elements of esz bytes (1: E4M3 codes, 2: BF16,
// 4: FP32), row stride ld elements, box (128 bytes of K) x box_rows, 128-byte
// swizzle, zero fill out of bounds.
static pgk_status make_map(CUtensorMap* map, const void* base, int rows, int K, int ld, int esz,
                           int box_rows) {
    if (((uintptr_t)base & 15u) != 0 || ((long long)ld * esz) % 16 != 0) {
        set_error("tensor-core operand must be 16-byte aligned with a row stride multiple of 16 bytes");
        return PGK_ERR_ALIGNMENT;
    }
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType ty = esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                              : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    CUresult r = g_encode(map, ty,
                          2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for rows=%d K=%d ld=%d", (int)r, rows, K, ld);
        return PGK_ERR_CUDA;
    }
    return PGK_OK;
}

// Launches the persistent kernel over `tiles` output tiles on at most `sm_count`
// SMs: one CTA per tile slot, or for CTA pairs one two-CTA cluster per slot, as
// many clusters as can be resident at once.
typedef cudaError_t (*tc_launch_fn)(const TcMaps&, const TcParams&, long long tiles, int sm_count,
                                    cudaStream_t);

// Tail balancing: with U tile slots and T tiles, the last T mod U tiles would run
// as a partly filled round; when they fill at most half of it, each is run as two
// column halves (BN = 256 tiles of the BF16 and split forms), so that round takes
// about half as long.  Every output element is computed with the same products in
// the same order.
static int tail_tiles(long long tiles, long long slots, int BN) {
    if (BN != 256 || slots < 2) return 0;
    const long long rem = tiles % slots;
    return (rem > 0 && 2 * rem <= slots) ? (int)rem : 0;
}

template <class Cfg, bool GROUPED>
static cudaError_t launch_tc(const TcMaps& maps, const TcParams& p0, long long tiles, int sm_count,
                             cudaStream_t st) {
    const void* fn = (const void*)k_tc_gemm<Cfg, GROUPED>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    if (e != cudaSuccess) return e;
    TcParams p = p0;
    p.tail = 0;
    // the tail-balanced instantiation exists for 256-wide single launches of the
    // BF16 and split forms; the FP8 form's per-chunk fold takes as long for a
    // column half as for a whole tile, so halves would not shorten its last round
    constexpr bool CAN_TAIL = !GROUPED && Cfg::BN == 256 && Cfg::MODE != MODE_FP8;
    const void* fn_tail = fn;
    if constexpr (CAN_TAIL) {
        fn_tail = (const void*)k_tc_gemm<Cfg, false, true>;
        e = cudaFuncSetAttribute(fn_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
    }
    if (!Cfg::PAIR) {
        if (CAN_TAIL) p.tail = tail_tiles(tiles, sm_count, Cfg::BN);
        const int grid = (int)std::min<long long>(tiles + p.tail, sm_count);
        if constexpr (CAN_TAIL) {
            if (p.tail > 0) {
                k_tc_gemm<Cfg, false, true><<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(maps, p);
                return cudaGetLastError();
            }
        }
        k_tc_gemm<Cfg, GROUPED><<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(maps, p);
        return cudaGetLastError();
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(sm_count / 2 * 2), 1, 1);
    cfg.blockDim = dim3(Cfg::THREADS, 1, 1);
    cfg.dynamicSmemBytes = Cfg::SMEM;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // resident two-CTA clusters of this variant, queried once per device
    static std::atomic<int> resident[64];
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int clusters = dev >= 0 && dev < 64 ? resident[dev].load() : 0;
    if (clusters < 1) {
        e = cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg);
        if (e != cudaSuccess) return e;
        if (clusters < 1) return cudaErrorInvalidConfiguration;
        if (dev >= 0 && dev < 64) resident[dev].store(clusters);
    }
    clusters = std::min(clusters, sm_count / 2);
    if (CAN_TAIL) p.tail = tail_tiles(tiles, clusters, Cfg::BN);
    clusters = (int)std::min<long long>(tiles + p.tail, clusters);
    cfg.gridDim = dim3((unsigned)(2 * clusters), 1, 1);
    if constexpr (CAN_TAIL) {
        if (p.tail > 0) return cudaLaunchKernelEx(&cfg, k_tc_gemm<Cfg, false, true>, maps, p);
    }
    return cudaLaunchKernelEx(&cfg, k_tc_gemm<Cfg, GROUPED>, maps, p);
}

struct TcVariant {
    int family, BM, BN, stages, smem, threads, tmem_cols;
    int b_box;   // rows of B^T per tensor-map box (per CTA)
    int fused;   // 1: A is read in FP32 and converted inside the GEMM
    const void* func;
    tc_launch_fn launch;
};

template <int MODE, int BN, int ST, bool PAIR = false, int FST = 0>
static TcVariant tcv(int family) {
    typedef TcCfg<MODE, BN, ST, PAIR, FST> Cfg;
    TcVariant v = {family, Cfg::TM, BN, ST, Cfg::SMEM, Cfg::THREADS, Cfg::TMEM_COLS, Cfg::BNL,
                   Cfg::FUSED ? 1 : 0, (const void*)k_tc_gemm<Cfg>, launch_tc<Cfg, false>};
    return v;
}

// B0 = 128: one CTA per 128 x B1 tile; B0 = 256: a CTA pair per 256 x 256 tile;
// B1 = 64: the fused-conversion programs of the BF16 and split forms
static const TcVariant* tc_table(int* n) {
    static const TcVariant t[] = {
        tcv<MODE_BF16, 256, 4>(PGK_FAM_TC_BF16),   tcv<MODE_BF16, 128, 6>(PGK_FAM_TC_BF16),
        tcv<MODE_BF16, 256, 3>(PGK_FAM_TC_BF16),   tcv<MODE_BF16, 128, 4>(PGK_FAM_TC_BF16),
        tcv<MODE_SPLIT, 128, 3>(PGK_FAM_TC_SPLIT), tcv<MODE_SPLIT, 256, 2>(PGK_FAM_TC_SPLIT),
        tcv<MODE_SPLIT3, 256, 4>(PGK_FAM_TC_SPLIT), tcv<MODE_SPLIT3, 128, 6>(PGK_FAM_TC_SPLIT),
        tcv<MODE_FP8, 128, 6>(PGK_FAM_TC_FP8),     tcv<MODE_FP8, 256, 4>(PGK_FAM_TC_FP8),
        tcv<MODE_BF16, 256, 6, true>(PGK_FAM_TC_BF16),
        tcv<MODE_SPLIT3, 256, 6, true>(PGK_FAM_TC_SPLIT),
        tcv<MODE_SPLIT, 256, 3, true>(PGK_FAM_TC_SPLIT),
        // B1 = 64: A converted inside the GEMM (skinny products, N <= 64)
        tcv<MODE_SPLIT, 64, 3, false, 2>(PGK_FAM_TC_SPLIT),
        tcv<MODE_BF16, 64, 4, false, 3>(PGK_FAM_TC_BF16),
    };
    *n = (int)(sizeof(t) / sizeof(t[0]));
    return t;
}

static int tc_base_id = -1;  // registry index of the first tensor-core variant

void register_tc_variants(std::vector<Variant>& v) {
    int n;
    const TcVariant* t = tc_table(&n);
    tc_base_id = (int)v.size();
    for (int i = 0; i < n; ++i) {
        Variant x;
        x.info.family = t[i].family;
        x.info.s = t[i].stages;
        x.info.sr = 0;
        x.info.B0 = t[i].BM;
        x.info.B1 = t[i].BN;
        x.info.tile = 0;
        x.info.regopt = 0;
        x.info.regs = -1;
        x.info.max_threads = -1;
        x.func = t[i].func;
        x.launch = nullptr;
        x.smem_fixed = t[i].smem;
        v.push_back(x);
    }
}

static int family_of(pgk_dtype d) {
    return d == PGK_BF16 ? PGK_FAM_TC_BF16 : d == PGK_SPLIT_BF16 ? PGK_FAM_TC_SPLIT : PGK_FAM_TC_FP8;
}

pgk_status tc_select(const pgk_machine* m, int M, int N, int K, pgk_dtype dtype,
                     const pgk_params* prog, pgk_case* out) {
    (void)M; (void)N; (void)K;
    registry();
    int n;
    const TcVariant* t = tc_table(&n);
    const int fam = family_of(dtype);
    const int natural = dtype == PGK_FP8_E4M3 ? 128 : 64;
    if ((prog->B0 != 128 && prog->B0 != 256) || (prog->tile != 0 && prog->tile != natural) ||
        prog->s < 1) {
        set_error("tensor-core tiles are 128 x B1 (one CTA) or 256 x B1 (a CTA pair) with the natural "
                  "K depth (B0=%d tile=%d)", prog->B0, prog->tile);
        return PGK_ERR_UNSUPPORTED;
    }
    for (int i = 0; i < n; ++i) {
        if (t[i].family != fam || t[i].BM != prog->B0 || t[i].BN != prog->B1 ||
            t[i].stages != prog->s)
            continue;
        // resource counters of the variant against the machine parameters
        if (t[i].threads > m->max_threads_per_block || t[i].smem > m->smem_per_block_optin ||
            t[i].tmem_cols > 512 || m->cc_major != 10) {
            set_error("tensor-core variant does not fit this device (smem %d > %d or cc %d.%d)",
                      t[i].smem, m->smem_per_block_optin, m->cc_major, m->cc_minor);
            return PGK_ERR_INFEASIBLE;
        }
        // the fused program covers all N columns with one 64-wide tile, so every A
        // element is converted once
        if (t[i].fused && N > t[i].BN) {
            set_error("the fused-conversion program (B1 = %d) covers N <= %d, not N = %d", t[i].BN,
                      t[i].BN, N);
            return PGK_ERR_INFEASIBLE;
        }
        pgk_case c;
        memset(&c, 0, sizeof(c));
        c.leaf = PGK_LEAF_4A3A;
        c.variant_id = tc_base_id + i;
        c.family = fam;
        c.smem_bytes = t[i].smem;
        c.regs = -1;
        c.threads = t[i].threads;
        c.params = *prog;
        c.params.tile = natural;
        // sr: the K slices of a fused-conversion program (0: chosen for the shape)
        if (!t[i].fused) c.params.sr = 0;
        else if (c.params.sr < 0 || c.params.sr > 1024) {
            set_error("fused-conversion program: K slices (sr = %d) must lie in [0, 1024]", c.params.sr);
            return PGK_ERR_INVALID_ARG;
        }
        *out = c;
        return PGK_OK;
    }
    set_error("no tensor-core variant with B0=%d B1=%d stages=%d for this form", prog->B0, prog->B1,
              prog->s);
    return PGK_ERR_UNSUPPORTED;
}

pgk_status tc_gemm_launch(const pgk_case& c, int M, int N, int K, pgk_dtype dtype, const void* A,
                          int lda, const void* Bt, int ldbt, const void* A_lo, const void* Bt_lo,
                          const float* sA, const float* sB, float* C, int ldc, int beta,
                          cudaStream_t stream) {
    pgk_status st = get_encoder();
    if (st != PGK_OK) return st;
    int n;
    const TcVariant* t = tc_table(&n);
    const int i = c.variant_id - tc_base_id;
    if (i < 0 || i >= n || t[i].family != family_of(dtype)) {
        set_error("case does not name a tensor-core variant of this form");
        return PGK_ERR_INVALID_ARG;
    }
    if (t[i].fused) {
        set_error("the fused-conversion program (B1 = 64) takes FP32 A: call pgk_gemm");
        return PGK_ERR_UNSUPPORTED;
    }
    const int esz = dtype == PGK_FP8_E4M3 ? 1 : 2;
    TcMaps maps;
    if ((st = make_map(&maps.a, A, M, K, lda, esz, 128)) != PGK_OK) return st;
    if ((st = make_map(&maps.b, Bt, N, K, ldbt, esz, t[i].b_box)) != PGK_OK) return st;
    if ((st = make_map(&maps.bh, Bt, N, K, ldbt, esz, t[i].b_box / 2)) != PGK_OK) return st;
    if (dtype == PGK_SPLIT_BF16) {
        if (!A_lo || !Bt_lo) {
            set_error("split form needs the lo operands");
            return PGK_ERR_INVALID_ARG;
        }
        if ((st = make_map(&maps.a2, A_lo, M, K, lda, esz, 128)) != PGK_OK) return st;
        if ((st = make_map(&maps.b2, Bt_lo, N, K, ldbt, esz, t[i].b_box)) != PGK_OK) return st;
        if ((st = make_map(&maps.b2h, Bt_lo, N, K, ldbt, esz, t[i].b_box / 2)) != PGK_OK) return st;
    } else {
        maps.a2 = maps.a;
        maps.b2 = maps.b;
        maps.b2h = maps.bh;
    }
    if (dtype == PGK_FP8_E4M3 && (!sA || !sB)) {
        set_error("FP8 form needs the tile scales");
        return PGK_ERR_INVALID_ARG;
    }
    pgk_machine m;
    if ((st = current_machine(&m, NULL)) != PGK_OK) return st;
    TcParams p;
    memset(&p, 0, sizeof(p));
    p.M = M;
    p.N = N;
    p.K = K;
    p.C = C;
    p.ldc = ldc;
    p.beta = beta ? 1 : 0;
    p.sA = sA;
    p.sB = sB;
    p.err = device_error_word(&st);
    if (!p.err) return st;
    const long long tiles = (long long)((M + t[i].BM - 1) / t[i].BM) * ((N + t[i].BN - 1) / t[i].BN);
    cudaError_t e = t[i].launch(maps, p, tiles, m.sm_count, stream);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core GEMM launch");
    return PGK_OK;
}

// ------------------------------------------------------- grouped launches
struct TcGroupedVariant {
    pgk_dtype dtype;
    int BN, stages;
    tc_launch_fn launch;
};

// 128-wide tiles only: a group of uneven problems wastes less on ragged edges
// (256-wide grouped tiles measured no faster on the 512-problem group)
static const TcGroupedVariant* tcg_table(int* n) {
    static const TcGroupedVariant t[] = {
        {PGK_BF16, 128, 6, launch_tc<TcCfg<MODE_BF16, 128, 6>, true>},
        {PGK_SPLIT_BF16, 128, 3, launch_tc<TcCfg<MODE_SPLIT, 128, 3>, true>},
        {PGK_SPLIT_BF16, 128, 6, launch_tc<TcCfg<MODE_SPLIT3, 128, 6>, true>},
        {PGK_FP8_E4M3, 128, 6, launch_tc<TcCfg<MODE_FP8, 128, 6>, true>},
    };
    *n = (int)(sizeof(t) / sizeof(t[0]));
    return t;
}

int tc_grouped_variants(pgk_dtype dtype, pgk_params* out, int cap) {
    int n, k = 0;
    const TcGroupedVariant* t = tcg_table(&n);
    for (int i = 0; i < n; ++i)
        if (t[i].dtype == dtype) {
            if (out && k < cap)
                out[k] = pgk_params{128, t[i].BN, t[i].stages, 0, dtype == PGK_FP8_E4M3 ? 128 : 64};
            ++k;
        }
    return k;
}

pgk_status launch_quant_fp8_grouped(int transpose, const GQuant* probs, const int* prefix, int G,
                                    int total, uint8_t* dst, long long ldd, float* scales,
                                    int ld_scales, cudaStream_t st);

// G problems in a tensor-core form: one grouped conversion (BF16, split) or
// quantisation (FP8) of all A operands, one of all B operands (transposed), both
// into packed K-major workspaces, then one persistent tensor-core launch over the
// tiles of every problem, problems in decreasing K order.  Problem g's operands
// start at a multiple of 128 rows and are zero from K_g to the next multiple of the
// K block (64; 128 for FP8, whose 128 x 128 scale blocks then coincide with those of
// the problem alone), so every tile computes exactly what a single launch on that
// problem computes.
pgk_status tc_gemm_grouped(int G, const pgk_problem* pr, pgk_dtype dtype, const pgk_params* prog,
                           int beta, cudaStream_t s) {
    const bool fp8 = dtype == PGK_FP8_E4M3, split = dtype == PGK_SPLIT_BF16;
    const int kb = fp8 ? 128 : 64;            // K block of the form
    pgk_params pp = {128, 128, dtype == PGK_SPLIT_BF16 ? 3 : 6, 0, kb};
    if (prog) pp = *prog;
    if (pp.B0 != 128 || (pp.tile != 0 && pp.tile != kb)) {
        set_error("grouped tensor-core tiles are 128 x B1 x %d (B0=%d tile=%d)", kb, pp.B0, pp.tile);
        return PGK_ERR_UNSUPPORTED;
    }
    int nv;
    const TcGroupedVariant* tv = tcg_table(&nv);
    const TcGroupedVariant* v = nullptr;
    for (int i = 0; i < nv; ++i)
        if (tv[i].dtype == dtype && tv[i].BN == pp.B1 && tv[i].stages == pp.s) v = &tv[i];
    if (!v) {
        set_error("no grouped tensor-core variant with B1=%d stages=%d for this form", pp.B1, pp.s);
        return PGK_ERR_UNSUPPORTED;
    }
    pgk_status st = get_encoder();
    if (st != PGK_OK) return st;
    pgk_machine m;
    if ((st = current_machine(&m, NULL)) != PGK_OK) return st;

    std::vector<int> order(G);
    for (int i = 0; i < G; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pr[a].K > pr[b].K; });
    // items of the operand preparation: 64 x 64 tiles (BF16, split), 128 x 128 (FP8)
    const int it = fp8 ? 128 : 64;
    int kmax = 0;
    long long rowsA = 0, rowsB = 0, tiles = 0, itemsA = 0, itemsB = 0;
    for (int i = 0; i < G; ++i) {
        const pgk_problem& q = pr[i];
        kmax = std::max(kmax, q.K);
        rowsA += (q.M + 127) / 128 * 128;
        rowsB += (q.N + 127) / 128 * 128;
        tiles += (long long)((q.M + 127) / 128) * ((q.N + v->BN - 1) / v->BN);
        const long long kr = (q.K + kb - 1) / kb * kb / it;
        itemsA += (long long)((q.M + it - 1) / it) * kr;
        itemsB += kr * ((q.N + it - 1) / it);
    }
    const long long kst = (long long)(kmax + kb - 1) / kb * kb;   // row stride of the packed operands
    if (rowsA > INT_MAX - 256 || rowsB > INT_MAX - 256 || tiles > INT_MAX || itemsA > INT_MAX ||
        itemsB > INT_MAX || kst > INT_MAX) {
        set_error("grouped tensor-core problem set too large for one launch");
        return PGK_ERR_INVALID_ARG;
    }
    // host image of the tables: TcProb[G] | prep A[G] | prep B[G] | int4 tiles[T] |
    // int prefixA[G+1] | int prefixB[G+1]
    const size_t esz_prep = fp8 ? sizeof(GQuant) : sizeof(GCvt);
    const size_t off_gA = (sizeof(TcProb) * G + 15) / 16 * 16;
    const size_t off_gB = off_gA + (esz_prep * G + 15) / 16 * 16;
    const size_t off_t = off_gB + (esz_prep * G + 15) / 16 * 16;
    const size_t off_pA = off_t + sizeof(int4) * (size_t)tiles;
    const size_t off_pB = off_pA + (sizeof(int) * (G + 1) + 15) / 16 * 16;
    const size_t bytes = off_pB + sizeof(int) * (G + 1);
    std::vector<unsigned char> img(bytes, 0);
    TcProb* tp = reinterpret_cast<TcProb*>(img.data());
    int4* tl = reinterpret_cast<int4*>(img.data() + off_t);
    int* pa = reinterpret_cast<int*>(img.data() + off_pA);
    int* pb = reinterpret_cast<int*>(img.data() + off_pB);
    long long ra = 0, rb = 0, t = 0, ia = 0, ib = 0;
    for (int j = 0; j < G; ++j) {
        const pgk_problem& q = pr[order[j]];
        const int kr = (q.K + kb - 1) / kb * kb;
        tp[j] = TcProb{q.C, q.M, q.N, q.K, q.ldc, (int)ra, (int)rb};
        const int va = ((uintptr_t)q.A % 16 == 0) && q.lda % 4 == 0;
        const int vb = ((uintptr_t)q.B % 16 == 0) && q.ldb % 4 == 0;
        if (fp8) {
            reinterpret_cast<GQuant*>(img.data() + off_gA)[j] =
                GQuant{q.A, q.lda, q.M, q.K, kr, va, (int)(ra / 128), ra};
            reinterpret_cast<GQuant*>(img.data() + off_gB)[j] =
                GQuant{q.B, q.ldb, q.K, q.N, kr, vb, (int)(rb / 128), rb};
        } else {
            reinterpret_cast<GCvt*>(img.data() + off_gA)[j] = GCvt{q.A, q.lda, q.M, q.K, kr, va, 0, ra};
            reinterpret_cast<GCvt*>(img.data() + off_gB)[j] = GCvt{q.B, q.ldb, q.K, q.N, kr, vb, 0, rb};
        }
        pa[j] = (int)ia;
        pb[j] = (int)ib;
        ia += (long long)((q.M + it - 1) / it) * (kr / it);
        ib += (long long)(kr / it) * ((q.N + it - 1) / it);
        const int tm_n = (q.M + 127) / 128, tn_n = (q.N + v->BN - 1) / v->BN;
        for (int tm = 0; tm < tm_n; ++tm)
            for (int tn = 0; tn < tn_n; ++tn) tl[t++] = make_int4(j, tm, tn, 0);
        ra += (q.M + 127) / 128 * 128;
        rb += (q.N + 127) / 128 * 128;
    }
    pa[G] = (int)ia;
    pb[G] = (int)ib;

    unsigned char* dt = (unsigned char*)workspace(WS_TABLE, bytes, &st);
    if (!dt) return st;
    const int esz = fp8 ? 1 : 2;
    const size_t abytes = (size_t)rowsA * kst * esz, bbytes = (size_t)rowsB * kst * esz;
    void* a0 = workspace(WS_A0, abytes, &st);
    if (!a0) return st;
    void* b0 = workspace(WS_B0, bbytes, &st);
    if (!b0) return st;
    void* a1 = nullptr;
    void* b1 = nullptr;
    float* sa = nullptr;
    float* sb = nullptr;
    if (split) {
        if (!(a1 = workspace(WS_A1, abytes, &st))) return st;
        if (!(b1 = workspace(WS_B1, bbytes, &st))) return st;
    }
    if (fp8) {
        if (!(sa = (float*)workspace(WS_SA, (size_t)(rowsA / 128) * (kst / 128) * 4, &st))) return st;
        if (!(sb = (float*)workspace(WS_SB, (size_t)(kst / 128) * (rowsB / 128) * 4, &st))) return st;
    }
    PGK_CUDA_TRY(cudaMemcpyAsync(dt, img.data(), bytes, cudaMemcpyHostToDevice, s), "table upload");
    if (fp8) {
        if ((st = launch_quant_fp8_grouped(0, reinterpret_cast<const GQuant*>(dt + off_gA),
                                           reinterpret_cast<const int*>(dt + off_pA), G, (int)itemsA,
                                           (uint8_t*)a0, kst, sa, (int)(kst / 128), s)) != PGK_OK)
            return st;
        if ((st = launch_quant_fp8_grouped(1, reinterpret_cast<const GQuant*>(dt + off_gB),
                                           reinterpret_cast<const int*>(dt + off_pB), G, (int)itemsB,
                                           (uint8_t*)b0, kst, sb, (int)(rowsB / 128), s)) != PGK_OK)
            return st;
    } else {
        // one launch converts every A_g and every B_g (transposed)
        if ((st = launch_cvt_grouped(split ? 1 : 0, reinterpret_cast<const GCvt*>(dt + off_gA),
                                     reinterpret_cast<const int*>(dt + off_pA), (int)itemsA,
                                     (uint16_t*)a0, (uint16_t*)a1,
                                     reinterpret_cast<const GCvt*>(dt + off_gB),
                                     reinterpret_cast<const int*>(dt + off_pB), (int)itemsB,
                                     (uint16_t*)b0, (uint16_t*)b1, G, kst, s)) != PGK_OK)
            return st;
    }
    TcMaps maps;
    if ((st = make_map(&maps.a, a0, (int)rowsA, (int)kst, (int)kst, esz, 128)) != PGK_OK) return st;
    if ((st = make_map(&maps.b, b0, (int)rowsB, (int)kst, (int)kst, esz, v->BN)) != PGK_OK) return st;
    if (split) {
        if ((st = make_map(&maps.a2, a1, (int)rowsA, (int)kst, (int)kst, esz, 128)) != PGK_OK) return st;
        if ((st = make_map(&maps.b2, b1, (int)rowsB, (int)kst, (int)kst, esz, v->BN)) != PGK_OK) return st;
    } else {
        maps.a2 = maps.a;
        maps.b2 = maps.b;
    }
    maps.bh = maps.b;     // grouped launches run whole tiles only
    maps.b2h = maps.b2;
    TcParams p;
    memset(&p, 0, sizeof(p));
    // FP8: the scale arrays' row strides (ceil(K/128) and ceil(N/128) of a single launch)
    p.K = (int)kst;
    p.N = (int)rowsB;
    p.sA = sa;
    p.sB = sb;
    p.beta = beta ? 1 : 0;
    p.err = device_error_word(&st);
    if (!p.err) return st;
    p.gtiles = reinterpret_cast<const int4*>(dt + off_t);
    p.gprobs = reinterpret_cast<const TcProb*>(dt);
    p.ntiles_g = (int)tiles;
    cudaError_t e = v->launch(maps, p, tiles, m.sm_count, s);
    if (e != cudaSuccess) return cuda_fail(e, "grouped tensor-core GEMM launch");
    return PGK_OK;
}

pgk_status launch_cvt_bf16(int rows, int cols, const float* src, int lds, uint16_t* dst, int ldd,
                           int transpose, cudaStream_t st);
pgk_status launch_split_bf16(int rows, int cols, const float* src, int lds, uint16_t* hi,
                             uint16_t* lo, int ldd, int transpose, cudaStream_t st);
pgk_status launch_quant_fp8(int rows, int cols, const float* src, int lds, uint8_t* dst, int ldd,
                            float* scales, int ld_scales, int transpose, cudaStream_t st);

// The fused-conversion programs: B^T is prepared (BF16, or hi and lo) into a
// library workspace, A is read in FP32 by the kernel itself.
static pgk_status tc_gemm_fused(const TcVariant& v, int slices, int M, int N, int K,
                                pgk_dtype dtype, const float* A, int lda, const float* B, int ldb,
                                float* C, int ldc, int beta, cudaStream_t s, bool prep_b) {
    pgk_status st = get_encoder();
    if (st != PGK_OK) return st;
    if (((uintptr_t)A & 15u) != 0 || lda % 4 != 0) {
        set_error("the fused-conversion program reads A by TMA: A must be 16-byte aligned with lda "
                  "a multiple of 4");
        return PGK_ERR_ALIGNMENT;
    }
    const int Kp = (K + 15) / 16 * 16;
    void* b0 = workspace(WS_B0, (size_t)N * Kp * 2, &st);
    if (!b0) return st;
    void* b1 = nullptr;
    if (dtype == PGK_SPLIT_BF16 && !(b1 = workspace(WS_B1, (size_t)N * Kp * 2, &st))) return st;
    if (prep_b) {
        st = dtype == PGK_SPLIT_BF16
                 ? launch_split_bf16(K, N, B, ldb, (uint16_t*)b0, (uint16_t*)b1, Kp, 1, s)
                 : launch_cvt_bf16(K, N, B, ldb, (uint16_t*)b0, Kp, 1, s);
        if (st != PGK_OK) return st;
    }
    TcMaps maps;
    if ((st = make_map(&maps.a, A, M, K, lda, 4, 128)) != PGK_OK) return st;
    if ((st = make_map(&maps.b, b0, N, K, Kp, 2, v.b_box)) != PGK_OK) return st;
    if (b1) {
        if ((st = make_map(&maps.b2, b1, N, K, Kp, 2, v.b_box)) != PGK_OK) return st;
    } else {
        maps.b2 = maps.b;
    }
    maps.a2 = maps.a;
    maps.bh = maps.b;
    maps.b2h = maps.b2;
    pgk_machine m;
    if ((st = current_machine(&m, NULL)) != PGK_OK) return st;
    TcParams p;
    memset(&p, 0, sizeof(p));
    p.M = M;
    p.N = N;
    p.K = K;
    p.C = C;
    p.ldc = ldc;
    p.beta = beta ? 1 : 0;
    p.err = device_error_word(&st);
    if (!p.err) return st;
    // K slices: slices = 0 takes as many as fill the SMs when the 128-row tiles alone
    // do not, each at least 8 K blocks (512) deep; every slice gets at least one K block
    const int nkb = (K + 63) / 64;
    if (slices == 0) {
        const int tiles_m = (M + v.BM - 1) / v.BM;
        slices = tiles_m < m.sm_count ? std::min(m.sm_count / tiles_m, (K + 511) / 512) : 1;
    }
    int S = std::max(1, std::min(slices, nkb));
    const int kper = (nkb + S - 1) / S;
    S = (nkb + kper - 1) / kper;
    p.kslices = S;
    p.kper = kper;
    if (S > 1) {
        p.part = (float*)workspace(WS_SPLITK, sizeof(float) * (size_t)S * M * N, &st);
        if (!p.part) return st;
    }
    const long long tiles = (long long)((M + v.BM - 1) / v.BM) * ((N + v.BN - 1) / v.BN) * S;
    cudaError_t e = v.launch(maps, p, tiles, m.sm_count, s);
    if (e != cudaSuccess) return cuda_fail(e, "fused-conversion GEMM launch");
    if (S > 1) {
        const long long total = (long long)M * N;
        const int blocks = (int)std::min<long long>((total + 255) / 256, (long long)m.sm_count * 8);
        k_slice_reduce<<<blocks, 256, 0, s>>>(M, N, p.part, S, C, ldc, p.beta);
        PGK_CUDA_TRY(cudaGetLastError(), "K-slice reduction launch");
    }
    return PGK_OK;
}

// FP32 operands -> library workspaces (K padded to a multiple of 16 elements)
// -> tensor-core kernel; the fused-conversion programs read A in FP32 themselves.
pgk_status tc_gemm_fp32_inputs(const pgk_case& c, int M, int N, int K, pgk_dtype dtype,
                               const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                               int beta, cudaStream_t s, bool prep_b) {
    {
        int n;
        const TcVariant* t = tc_table(&n);
        const int i = c.variant_id - tc_base_id;
        if (i >= 0 && i < n && t[i].fused)
            return tc_gemm_fused(t[i], c.params.sr, M, N, K, dtype, A, lda, B, ldb, C, ldc, beta, s,
                                 prep_b);
    }
    const int Kp = (K + 15) / 16 * 16;
    const int esz = dtype == PGK_FP8_E4M3 ? 1 : 2;
    pgk_status st;
    void* a0 = workspace(WS_A0, (size_t)M * Kp * esz, &st);
    if (!a0) return st;
    void* b0 = workspace(WS_B0, (size_t)N * Kp * esz, &st);
    if (!b0) return st;
    if (dtype == PGK_BF16) {
        if ((st = launch_cvt_bf16(M, K, A, lda, (uint16_t*)a0, Kp, 0, s)) != PGK_OK) return st;
        if (prep_b && (st = launch_cvt_bf16(K, N, B, ldb, (uint16_t*)b0, Kp, 1, s)) != PGK_OK) return st;
        return tc_gemm_launch(c, M, N, K, dtype, a0, Kp, b0, Kp, nullptr, nullptr, nullptr, nullptr,
                              C, ldc, beta, s);
    }
    if (dtype == PGK_SPLIT_BF16) {
        void* a1 = workspace(WS_A1, (size_t)M * Kp * 2, &st);
        if (!a1) return st;
        void* b1 = workspace(WS_B1, (size_t)N * Kp * 2, &st);
        if (!b1) return st;
        if ((st = launch_split_bf16(M, K, A, lda, (uint16_t*)a0, (uint16_t*)a1, Kp, 0, s)) != PGK_OK)
            return st;
        if (prep_b &&
            (st = launch_split_bf16(K, N, B, ldb, (uint16_t*)b0, (uint16_t*)b1, Kp, 1, s)) != PGK_OK)
            return st;
        return tc_gemm_launch(c, M, N, K, dtype, a0, Kp, b0, Kp, a1, b1, nullptr, nullptr, C, ldc,
                              beta, s);
    }
    const int mt = (M + 127) / 128, kt = (K + 127) / 128, nt = (N + 127) / 128;
    float* sa = (float*)workspace(WS_SA, (size_t)mt * kt * 4, &st);
    if (!sa) return st;
    float* sb = (float*)workspace(WS_SB, (size_t)kt * nt * 4, &st);
    if (!sb) return st;
    if ((st = launch_quant_fp8(M, K, A, lda, (uint8_t*)a0, Kp, sa, kt, 0, s)) != PGK_OK) return st;
    if (prep_b && (st = launch_quant_fp8(K, N, B, ldb, (uint8_t*)b0, Kp, sb, nt, 1, s)) != PGK_OK)
        return st;
    return tc_gemm_launch(c, M, N, K, dtype, a0, Kp, b0, Kp, nullptr, nullptr, sa, sb, C, ldc, beta,
                          s);
}

}  // namespace pgk

using namespace pgk;

extern "C" pgk_status pgk_gemm_lowp(int M, int N, int K, pgk_dtype dtype, const void* A, int lda,
                                    const void* Bt, int ldbt, const void* A_lo, const void* Bt_lo,
                                    const float* scaleA, const float* scaleB, float* C, int ldc,
                                    int beta, const pgk_params* prog, void* stream) {
    if (M < 1 || N < 1 || K < 1 || !A || !Bt || !C || lda < K || ldbt < K || ldc < N) {
        set_error("bad tensor-core GEMM arguments");
        return PGK_ERR_INVALID_ARG;
    }
    if (dtype != PGK_BF16 && dtype != PGK_SPLIT_BF16 && dtype != PGK_FP8_E4M3) {
        set_error("pgk_gemm_lowp takes the BF16, split-BF16 or FP8 forms");
        return PGK_ERR_INVALID_ARG;
    }
    pgk_machine m;
    pgk_status st = current_machine(&m, NULL);
    if (st != PGK_OK) return st;
    pgk_params p;
    if (prog) {
        p = *prog;
    } else if (pgk_tune_cache_get(M, N, K, dtype, &p) != PGK_OK) {
        pgk_params d = {128, dtype == PGK_SPLIT_BF16 ? 128 : (dtype == PGK_BF16 ? 256 : 128),
                        dtype == PGK_SPLIT_BF16 ? 3 : (dtype == PGK_BF16 ? 4 : 6), 0, 0};
        p = d;
    }
    pgk_case c;
    st = tc_select(&m, M, N, K, dtype, &p, &c);
    if (st != PGK_OK) return st;
    return tc_gemm_launch(c, M, N, K, dtype, A, lda, Bt, ldbt, A_lo, Bt_lo, scaleA, scaleB, C, ldc,
                          beta, (cudaStream_t)stream);
}

extern "C" pgk_status pgk_selftest_bounded_wait(unsigned long long limit_ns, void* stream) {
    if (limit_ns == 0 || limit_ns > 2000000000ULL) {
        set_error("limit must be in (0, 2 s]");
        return PGK_ERR_INVALID_ARG;
    }
    pgk_status st;
    unsigned int* err = device_error_word(&st);
    if (!err) return st;
    k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(err, limit_ns);
    PGK_CUDA_TRY(cudaGetLastError(), "wait self-test launch");
    return PGK_OK;
}
