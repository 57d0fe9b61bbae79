// Tensor-core window search (uniform weights, T0 steps kMinSt .. kMaxSt).
//
// The in-transit sums of one duration (D points, T0 step st) are a
// contraction once the folded, padded curve is read as rows of sigma = g st
// points, g = 4 / gcd(st, 4) windows per row (so that every row starts on a
// 16-byte boundary):
//
//     A[rho][c]     = r[rho sigma + c]                      (c < sigma)
//     B[i g + q][c] = s_{i sigma + c - q st}   (0 where the index leaves [0, D))
//     G             = A B^T                     (M = rows, N = I g <= 32, K = sigma)
//     C1(rho g + q) = sum_{k < D} r[(rho g + q) st + k] s_k = sum_{i < I} G[rho + i][i g + q]
//
// with I = ceil((D + (g - 1) st) / sigma) row blocks.  That is the window sum
// C1 of Eq. (in) expanded: every product r s_k of a window appears once, so
// the MMA does the algorithmic work of the window-point evaluations, plus
// the padding of K to a multiple of 8 and of N to 32.  FP32 accuracy comes
// from the three-product split of both operands into TF32 halves (Ootomo &
// Yokota 2022): r = r_hi + r_lo, s = s_hi + s_lo, r s ~ r_hi s_hi + r_hi s_lo
// + r_lo s_hi, accumulated in FP32 by the tensor core; the dropped r_lo s_lo
// is below 2^-21 of r s.
//
// Work item = (period slot, duration), walked in M-tiles of 128 rows that
// overlap by I - 1 rows (so that every window's I rows lie in one tile) and
// K chunks of 32 columns.  One persistent CTA per SM (all 512 TMEM columns)
// runs three roles over a ring of kStages shared-memory stages, handing
// chunks over with mbarriers:
//   * a producer thread takes items from a device counter and, per chunk,
//     writes the chunk's description, then issues a TMA load of its 128 x 32
//     block of rows (a 3-D tensor map over (column, row, slot) of the chunk
//     scratch with row pitch sigma; columns past sigma and rows past the slot
//     read as zeros) into a 128-byte-swizzled stage and a bulk copy of the
//     chunk of B (host-built canonical K-major core matrices, hi and lo);
//   * four converter warps (TMEM lanes 0..127, one row per lane) read their
//     row of a stage (conflict free through the swizzle), split it into TF32
//     halves and write them to a TMEM stage (kTStages of them);
//   * four MMA threads (in four warps: the issue of one tcgen05.mma takes a
//     thread about 110 cycles, and the tensor core accepts four streams)
//     take one k-step of 8 columns of every chunk each and issue its three
//     tcgen05.mma.kind::tf32 (M 128, N 32, K 8; A from TMEM, B from shared
//     memory) into their own accumulator of the tile's D buffer (two buffers
//     alternate by tile); every thread commits every chunk to the barriers
//     that free the TMEM stage and B (four arrivals each), and at a tile's
//     end to the tile's D barrier.
// Four epilogue warps take every tile once its MMAs completed (the MMA
// thread of k-step 0 hands over the tile's description): every lane sums its
// row of the four accumulators (tcgen05.ld) into G = A B^T and writes it to
// shared memory (XOR-swizzled rows, conflict-free diagonals), and the g
// windows of its row get C1 = sum_i G[l + i][i g + q], S from the exact
// prefix sums, the depth, delta chi2 and the packed per-period minimum
// (64-bit atomicMin), as in the FP32 kernels.
//
// Every mbarrier wait is bounded (kWaitCycles); a wait that runs out records
// check 30 (reported as GTLS_ERR_TIMEOUT) and raises an abort flag that ends
// the other roles' waits; the converter and epilogue warps leave together
// (their barriers OR their failures), the producer and the MMA threads wait once
// more for their own copies and MMAs, and the CTA frees its TMEM before it
// returns.
#pragma once

namespace gtls {
namespace tc {

constexpr int kConvWarps = 4;      // TMEM lanes 0..127: one row each
constexpr int kMmaWarps = 4;       // one per MMA k-step of a chunk, each with its own accumulator
constexpr int kEpiWarps = 4;       // epilogue: one row of G per lane (TMEM lanes by warp % 4)
constexpr int kThreads = 32 * (kConvWarps + 1 + kMmaWarps + kEpiWarps);   // + a producer warp
constexpr int kRows = 128;         // MMA M: rows per tile
constexpr int kN = 32;             // MMA N: I g <= 32 template rows
constexpr int kChunk = 32;         // K columns per chunk (4 MMA k-steps of 8); 128 bytes of a row
constexpr int kStages = 8;         // shared-memory stages (rows 16 KB + B 8 KB each)
constexpr int kTStages = 4;        // TMEM stages of A (hi and lo, 64 columns each)
// T0 steps from which the search takes this kernel (GTLS_TC_MIN_ST overrides
// it per plan).  Off by default: on the Kepler-like search it measured slower
// than the FP32 kernels at every threshold (861 ms window stage at 24, 794 ms
// at 48, 723 ms without it): with N = 20..32 template rows an MMA carries
// little work, and the issue of one tcgen05.mma costs its thread ~110-136
// cycles (four issuing threads reach four times the rate).
constexpr int kMinStDefault = 1 << 30;
constexpr int kMaxSigma = 1024;    // longest row (points); the tensor maps cover sigma = 4, 8, .., 1024
constexpr int kMaps = kMaxSigma / 4;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kDCol = kTStages * 64;   // two D buffers of kMmaWarps x 32 columns after the A stages
constexpr long long kWaitCycles = 4000000000ll;   // about 2 s at 2 GHz
constexpr long long kTestWaitCycles = 2000000ll;  // the timeout test's wait
constexpr int kCheckTimeout = 30;  // check word of a wait that ran out
constexpr uint32_t kBytesA = kRows * kChunk * 4;      // 16 KB
constexpr uint32_t kBytesB = 2 * kN * kChunk * 4;     // 8 KB

// kind::tf32, D in FP32, A and B TF32, both K-major, N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kRows >> 4) << 24);

// What the converter and MMA warps need of a chunk (written by the producer
// before it arms the stage's barrier).
struct ChunkInfo {
    int32_t end;           // 1: no more chunks (the producer is done)
    int32_t kc, ksteps;    // column chunk, MMA k-steps in it
    int32_t kst_tile;      // MMA k-steps of the whole row (accumulators the tile fills: min(4, kst_tile))
    int32_t first, last;   // first / last chunk of its tile
    int32_t item_last;     // last chunk of its item
    int32_t tile;          // tile index inside the item
    int32_t lc, p, j, st, d, g, nblk, per_tile;
    int64_t nwin, slot;
    float w_uni, inv_sum_t, sum_t2;
};

struct alignas(1024) TcSmem {
    float a[kStages][kRows * kChunk];   // TMA stages, 128-byte swizzle (1024-byte aligned)
    float b[kStages][2 * kN * kChunk];  // [hi | lo] canonical K-major core matrices
    float g[kRows * kN];                // rows of G (XOR-swizzled) for the diagonal sums
    ChunkInfo info[kStages];
    unsigned long long full[kStages];   // rows + B landed (TMA / bulk transaction count)
    unsigned long long a_free[kStages]; // converters read the rows
    unsigned long long b_free[kStages]; // MMAs read B
    unsigned long long t_full[kTStages];  // converters wrote A to TMEM
    unsigned long long t_free[kTStages];  // MMAs read the TMEM stage
    unsigned long long d_full[2];       // a tile's MMAs completed
    unsigned long long d_free[2];       // the epilogue read the tile's accumulators
    unsigned long long i_full[2];       // the tile's description is in tinfo
    ChunkInfo tinfo[2];                 // description of the tile in each D buffer (from its last chunk)
    int abort;                          // a role gave up on a wait
};

constexpr size_t kSmemBytes = sizeof(TcSmem) + 1024;
constexpr int kSmemRequest = (int)kSmemBytes;
static_assert(kSmemBytes <= 227 * 1024, "tensor window kernel shared memory");
static_assert(kDCol + 2 * kMmaWarps * 32 <= kTmemCols, "TMEM columns");

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle, core matrices of 8
// rows x 16 bytes; lbo = byte step between core matrices along K, sbo =
// along M / N; bits 46-47 = 1 (descriptor version of tcgen05).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void bar_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Named barrier that also ORs a predicate over the participating threads:
// every thread gets the same answer, so control flow that follows it stays
// uniform.
__device__ __forceinline__ bool bar_sync_or(int id, int count, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity)
{
    uint32_t ok;
    // the thread may sleep in the instruction until the phase completes (the
    // hint bounds the sleep at 1 ms), instead of spinning on the issue slots
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}

// Waits until the phase of parity `parity` of the mbarrier completed, for at
// most `limit` SM cycles; false if it ran out (or, when `abort` is given,
// once another role has given up).
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, long long limit,
                                          const volatile int* abort = nullptr)
{
    const long long t0 = clock64();
    while (!mbar_try(addr, parity)) {
        if (clock64() - t0 > limit) return false;
        if (abort && *abort) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// 3-D tiled TMA load of the box {32 columns, 128 rows, 1 slot} at
// (c0, c1, c2) into shared memory; completes on `mbar` (expect_tx first).
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* map, int c0, int c1, int c2, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
        : "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// 32 consecutive TMEM columns of this thread's lane <- v[0..31]
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]),
        "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]),
        "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

// v[0..31] <- 32 consecutive TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace tc
}  // namespace gtls
