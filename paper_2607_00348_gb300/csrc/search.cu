// libgtls: the TLS period-grid search on one GPU (sm_103a).
//
// Pipeline of one search (all on `stream`; a batch runs the same kernels over
// many curves, see gtls_batch below):
//   k_curve_reset, k_curve_minmax, k_curve_prep, k_curve_reduce
//                      per-point derived arrays, chi2_0, input checks
//   for every wave (chunk) of periods:
//     k_fold_sort      fold on the exact phase lattice (Eq. phase), two-level
//                      bucket sort by (phase, index) (super-buckets in global
//                      memory, fine buckets in shared memory), gather the
//                      folded curve, pad it with its first D_m points
//                      (Sect. 2.3.2) and build the exact prefix sums that give
//                      every moving average (Eq. cumsum)
//     k_window_tiles   every duration and T0 start (Eq. N_skip): depth
//                      (Eqs. k, depth), chi2 - chi2_0 (Eqs. out, in),
//                      per-period minimum; staged tiles, window_tiles.cuh
//                      (k_window_search: one thread per window, for plans
//                      whose durations do not fit a tile)
//     k_period_finalize chi2(P), depth, T0 of each period's minimum
//   k_sr_stats_set, k_median_sde_set        SR, SDE_raw, SDE (Sect. 2.4)
//   k_topk + waves with T0 step 1           refinement of the best periods
//                                           (Sect. 2.5), then SR/SDE again
//   k_best                                  the candidate of largest SDE
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gtls_internal.h"

using namespace gtls;

namespace {

thread_local std::string g_last_error;

gtls_status fail(gtls_status s, const std::string& msg)
{
    g_last_error = msg;
    return s;
}

}  // namespace

gtls_status gtls::set_error(gtls_status s, const std::string& msg)
{
    return fail(s, msg);
}

namespace {

#define GTLS_CUDA(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? GTLS_ERR_OOM : GTLS_ERR_CUDA,   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

constexpr int kFoldThreads = 1024;
constexpr int kFoldMinBlocks = 1;     // fold CTAs per SM the register budget is sized for
constexpr int kFoldUnroll = 4;        // points whose loads a fold thread issues together
constexpr int kFoldSegKeys = 8192;    // sort keys (and folded rfx) staged in shared memory per run of buckets
constexpr int kRankBatch = 2;         // keys a fold thread ranks before issuing their gathers (1, 2, 4, 8: 240.0, 240.3, 245.9, 272.8 ms)
constexpr int kScanPer = 8;           // consecutive prefix-sum positions per fold thread
constexpr int kWeightedTilePairs = 24576;   // (w r, w) pairs staged per tile with per-point weights
constexpr int kSearchThreads = 256;
constexpr int kMedianThreads = 1024;
constexpr int kMedianCap = 8192;       // values a median block sorts in shared memory
constexpr double kRScale = 1099511627776.0;   // 2^40: fixed point of r = 1 - y
// zeros after the padded folded curve: the tensor-core window kernel reads
// whole rows of up to tc::kMaxSigma points (two rows and a T0 step past the
// last window's end; their template entries are zero, their values must be
// finite)
constexpr int64_t kPadMargin = 3 * 1024 + 64;

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long double_order_key(double v)
{
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ double double_from_order_key(unsigned long long k)
{
    unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)u);
}

__device__ __forceinline__ unsigned int float_order_key(float v)
{
    unsigned int u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float float_from_order_key(unsigned int k)
{
    unsigned int u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

// Record the first failed index check of a search; the access is then
// skipped (or redirected to index 0) so that the kernel never leaves its
// buffers.  The host turns a recorded check into GTLS_ERR_INTERNAL.
__device__ __noinline__ void record_check(unsigned int* w, unsigned int code, long long a, long long b)
{
    if (atomicCAS(w, 0u, code) == 0u) {
        w[1] = (unsigned int)a;
        w[2] = (unsigned int)b;
        w[3] = (unsigned int)(a >> 32);
    }
}

__device__ __forceinline__ bool in_range(unsigned int* w, unsigned int code, long long v, long long hi)
{
    if (v >= 0 && v < hi) return true;
    record_check(w, code, v, hi);
    return false;
}

__device__ __forceinline__ bool in_range32(unsigned int* w, unsigned int code, uint32_t v, uint32_t hi)
{
    if (v < hi) return true;
    record_check(w, code, v, hi);
    return false;
}

// Exact lattice phase rho = d mod P (0 <= d < 2^62, P > 0).  The float
// product gives the cycle count to within one; two integer corrections make
// it exact.
__device__ __forceinline__ long long lattice_rho(long long d, float d_f, long long p, float inv_p)
{
    long long c = (long long)floorf(d_f * inv_p);
    long long r = d - c * p;
    if (r < 0) r += p;
    else if (r >= p) r -= p;
    return r;
}

__device__ __forceinline__ uint32_t fold_bucket(long long rho, int sh, uint32_t mul)
{
    return (uint32_t)((((unsigned long long)rho >> sh) * (unsigned long long)mul) >> 32);
}

// Exclusive scan of one long long per thread over a 1024-thread block.
__device__ long long block_exclusive_scan(long long v, long long* warp_sums, long long* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        long long s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
        if (lane == nw - 1) *total = s;
    }
    __syncthreads();
    const long long base = warp > 0 ? warp_sums[warp - 1] : 0;
    const long long out = base + x - v;
    __syncthreads();
    return out;
}

// Exclusive scan of one long long per thread over the block with a single
// barrier: every warp scans the warp totals itself.  `total` receives the
// block sum.  The caller must pass a barrier before warp_sums is reused.
__device__ long long block_exclusive_scan1(long long v, long long* warp_sums, long long& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    long long t = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
    }
    total = __shfl_sync(0xffffffffu, t, 31);
    const long long base = __shfl_sync(0xffffffffu, t, (warp + 31) & 31);   // inclusive sum of warps < warp
    return (warp > 0 ? base : 0) + x - v;
}

// Light curve and period held by `slot` of a wave (segments ascend in
// slot0); false past the wave's slots or when the period index is out of
// range.
__device__ __forceinline__ bool resolve_slot(const DevSet& ds, const SlotMap& sm, int slot, int& lc, int& p)
{
    if (slot >= sm.slots) return false;
    int s = 0;
    while (s + 1 < sm.nseg && sm.seg[s + 1].slot0 <= slot) ++s;
    lc = sm.seg[s].lc;
    const int q = sm.seg[s].first + (slot - sm.seg[s].slot0);
    p = sm.from_list ? ds.outs[lc].plist[q] : q;
    return p >= 0 && p < ds.plans[lc].np;
}

// Work size of the per-curve preparation kernels for n points.
__host__ __device__ __forceinline__ int prep_blocks_for(int64_t n)
{
    const int64_t b = (n + 255) / 256;
    return (int)(b < 1024 ? b : 1024);
}

}  // namespace

#include "window_tiles.cuh"
#include "window_tc.cuh"

namespace {

// ---------------------------------------------------------------------------
// per-curve preparation
// ---------------------------------------------------------------------------

// Reset of the per-curve reduction words (block lc0 + b: curve lc0 + b).
__global__ void k_curve_reset(DevSet ds, int lc0)
{
    const DevCurve& dc = ds.curves[lc0 + blockIdx.x];
    if (threadIdx.x == 0) *dc.tmin_key = ~0ull;
    if (threadIdx.x == 1) *dc.flags = 0u;
    if (threadIdx.x >= 2 && threadIdx.x < 6) dc.check[threadIdx.x - 2] = 0u;
}

// Curve lc = lc0 + blockIdx.y holds points off[lc] .. off[lc+1] of t, y, dy;
// its blocks are the first prep_blocks_for(n) of the row.
__global__ void k_curve_minmax(const double* __restrict__ t, const double* __restrict__ y,
                               const double* __restrict__ dy, const int64_t* __restrict__ off,
                               DevSet ds, int lc0)
{
    const int lc = lc0 + blockIdx.y;
    const int64_t o = off[lc], n = off[lc + 1] - o;
    const int nb = prep_blocks_for(n);
    if ((int)blockIdx.x >= nb || n <= 0) return;
    t += o;
    y += o;
    dy += o;
    const DevCurve& dc = ds.curves[lc];
    unsigned long long kmin = ~0ull;
    unsigned int fl = 0;
    const double dy0 = dy[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)nb * blockDim.x) {
        const double ti = t[i], yi = y[i], di = dy[i];
        if (!isfinite(ti) || !isfinite(yi) || !isfinite(di)) fl |= 1u;
        if (!(di > 0.0)) fl |= 2u;
        if (di != dy0) fl |= 4u;
        const unsigned long long k = double_order_key(ti);
        kmin = k < kmin ? k : kmin;
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        unsigned long long k2 = __shfl_xor_sync(0xffffffffu, kmin, o2);
        kmin = k2 < kmin ? k2 : kmin;
        fl |= __shfl_xor_sync(0xffffffffu, fl, o2);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(dc.tmin_key, kmin);
        if (fl) atomicOr(dc.flags, fl);
    }
}

__global__ void k_curve_prep(const double* __restrict__ t, const double* __restrict__ y,
                             const double* __restrict__ dy, const int64_t* __restrict__ off,
                             DevSet ds, int lc0)
{
    __shared__ double red[32];
    const int lc = lc0 + blockIdx.y;
    const int64_t o = off[lc], n = off[lc + 1] - o;
    const int nb = prep_blocks_for(n);
    if ((int)blockIdx.x >= nb || n <= 0) return;
    t += o;
    y += o;
    dy += o;
    const DevCurve dc = ds.curves[lc];
    const int e = ds.plans[lc].time_exponent;
    const double t_ref = double_from_order_key(*dc.tmin_key);
    const double scale = ldexp(1.0, e);
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)nb * blockDim.x) {
        const double dt = t[i] - t_ref;
        const double r = 1.0 - y[i];
        const double w = 1.0 / (dy[i] * dy[i]);
        dc.d_lat[i] = __double2ll_rn(dt * scale);
        dc.d_f[i] = (float)dt;
        dc.pv[i] = PointVals{__double2ll_rn(r * kRScale), (float)r, (float)w};
        acc += w * r * r;
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        dc.part[blockIdx.x] = s;
    }
}

// One thread per curve (lc0 + global thread index < lc_end): chi2_0 from
// the block partials in block order, t_ref, the uniform weight; the
// validity flags go to flags_out[lc].
__global__ void k_curve_reduce(const double* __restrict__ dy, const int64_t* __restrict__ off, DevSet ds,
                               int lc0, int lc_end, unsigned int* flags_out)
{
    const int lc = lc0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (lc >= lc_end) return;
    const int64_t o = off[lc], n = off[lc + 1] - o;
    const DevCurve dc = ds.curves[lc];
    const int nparts = prep_blocks_for(n);
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += dc.part[i];
    const unsigned int fl = *dc.flags;
    dc.scal[0] = double_from_order_key(*dc.tmin_key);
    dc.scal[1] = s;
    dc.scal[2] = (fl & 4u) ? 0.0 : 1.0 / (dy[o] * dy[o]);
    flags_out[lc] = fl;
}

// ---------------------------------------------------------------------------
// fold + sort + gather + prefix sums (one block per period)
// ---------------------------------------------------------------------------
//
// The folded order is the order of the keys (rho << idx_bits | i).  Two
// monotone functions of rho split it into buckets: fold_bucket (2^bucket_log2
// buckets) and fold_fine (nsb 2^kFoldFineLog2 fine buckets, grouped into nsb
// super-buckets of 2^kFoldFineLog2 each; nsb is chosen so that a
// super-bucket holds about kFoldFillKeys points, seven eighths of its
// region, on average: fewer, fuller super-buckets mean fewer rounds of the
// barrier-separated steps below; measured on the Kepler-like search, a
// fill of 5120, 6144 and 7168 points gave 264, 254 and 246 ms, and the
// power-of-two count used before, about half full, 271 ms).
//
// Staged path (the common case): the keys are scattered once into global
// memory, each into its super-bucket's region of kFoldSegKeys slots -- a few
// dozen write streams that fill whole cache lines -- and every super-bucket
// is then bucket sorted, ranked, gathered and scanned in shared memory.
// Global path (a phase pile-up: some super-bucket too full for its region):
// the keys are scattered into global memory in bucket order and runs of
// whole buckets are ranked and scanned (in shared memory while a run fits,
// else in global memory).

constexpr int kFoldFineLog2 = 11;   // fine buckets per super-bucket (log2)
constexpr int kFoldMaxSbLog2 = 10;  // at most one super-bucket per fold thread
constexpr int kFoldFillKeys = 7168; // mean points per super-bucket the plan aims at

// Fine bucket of phase rho: floor((rho >> sh) mulf / 2^32) with
// mulf = floor(nsb 2^(kFoldFineLog2 + 32) / top), top > rho >> sh, is
// monotone in rho and below nsb 2^kFoldFineLog2.
__device__ __forceinline__ uint32_t fold_fine(long long rho, int sh, uint32_t mulf)
{
    return (uint32_t)((((unsigned long long)rho >> sh) * (unsigned long long)mulf) >> 32);
}

struct FoldOut {
    int32_t* sidx;
    float* rs;
    float* ws;
    float* wrs;
    long long* pf;
    bool uniform;
};

// Rank keys[q] (q < len, staged in shared memory in bucket order) inside
// their buckets, gather the folded curve into positions k0 + rank of the
// outputs and the folded rfx into srfx[rank].  bucket_of(q, key, b) gives the
// bucket b of keys[q] (false: skip the key); its keys occupy
// [e - cnt_of[b], e) of keys with e = end_of[b] - end_base.
template <typename BucketOf>
__device__ __forceinline__ void fold_rank_gather(const unsigned long long* keys, uint32_t len, uint32_t k0,
                                                 const uint32_t* cnt_of, const uint32_t* end_of,
                                                 uint32_t end_base, BucketOf bucket_of, int ib,
                                                 unsigned long long idx_mask,
                                                 int64_t n, const DevCurve& dc, const FoldOut& o,
                                                 long long* srfx)
{
    for (uint32_t q0 = threadIdx.x; q0 < len; q0 += kRankBatch * blockDim.x) {
        uint32_t pos[kRankBatch];
        int32_t idx[kRankBatch];
#pragma unroll
        for (int j = 0; j < kRankBatch; ++j) {
            pos[j] = 0xffffffffu;
            idx[j] = 0;
            const uint32_t q = q0 + j * blockDim.x;
            if (q >= len) continue;
            const unsigned long long key = keys[q];
            int b;
            if (!bucket_of(q, key, b)) continue;
            const uint32_t cnt = cnt_of[b], e = end_of[b] - end_base;
            if (!in_range32(dc.check, 6, e, len + 1) || !in_range32(dc.check, 6, cnt, e + 1)) continue;
            const uint32_t lo = e - cnt;
            uint32_t rank = 0;
            for (uint32_t u = 0; u < cnt; ++u) rank += keys[lo + u] < key ? 1u : 0u;
            const int32_t id = (int32_t)(key & idx_mask);
            if (!in_range32(dc.check, 7, lo + rank, len) || !in_range32(dc.check, 8, (uint32_t)id, (uint32_t)n))
                continue;
            pos[j] = lo + rank;
            idx[j] = id;
        }
        PointVals pv[kRankBatch];
#pragma unroll
        for (int j = 0; j < kRankBatch; ++j)
            pv[j] = pos[j] != 0xffffffffu ? dc.pv[idx[j]] : PointVals{0, 0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < kRankBatch; ++j) {
            if (pos[j] == 0xffffffffu) continue;
            const int64_t g = (int64_t)k0 + pos[j];
            o.sidx[g] = idx[j];
            o.rs[g] = pv[j].r;
            srfx[pos[j]] = pv[j].rfx;
            if (!o.uniform) {
                o.ws[g] = pv[j].w;
                o.wrs[g] = pv[j].w * pv[j].r;
            }
        }
    }
}

// pf[k0 + 1 + i] = carry + srfx[0] + ... + srfx[i] for i < len; carry
// advances by the run's total.
__device__ __forceinline__ void fold_scan_run(const long long* srfx, uint32_t len, uint32_t k0, long long* pf,
                                              long long& carry, long long* warp_sums, long long* total)
{
    const int64_t span = (int64_t)blockDim.x * kScanPer;
    for (int64_t base = 0; base < len; base += span) {
        const int64_t i0 = base + (int64_t)threadIdx.x * kScanPer;
        long long v[kScanPer];
        long long run = 0;
#pragma unroll
        for (int u = 0; u < kScanPer; ++u) {
            run += i0 + u < len ? srfx[i0 + u] : 0;
            v[u] = run;
        }
        const long long ex = block_exclusive_scan(run, warp_sums, total) + carry;
#pragma unroll
        for (int u = 0; u < kScanPer; ++u)
            if (i0 + u < len) pf[k0 + i0 + u + 1] = ex + v[u];
        carry += *total;
    }
}

// Staged path; false when a super-bucket holds more than kFoldSegKeys
// points (only keys have been written then).
__device__ bool fold_staged(unsigned char* smem, const DevPlan& dp, const DevCurve& dc, int p,
                            unsigned long long* keys, const FoldOut& o)
{
    const int64_t n = dp.n;
    const long long P = dp.p_lat[p];
    const float inv_p = dp.inv_p[p];
    const int sh = dp.bucket_shift[p];
    const int ib = dp.idx_bits;
    const unsigned long long idx_mask = (1ull << ib) - 1ull;
    const int nsb = dp.fold_nsb;
    const uint32_t mulf = (uint32_t)(((unsigned long long)nsb << (kFoldFineLog2 + 32)) /
                                     (((unsigned long long)P >> sh) + 1ull));
    constexpr uint32_t kFineMask = (1u << kFoldFineLog2) - 1u;
    static_assert((1 << kFoldFineLog2) % kFoldThreads == 0, "fine buckets split evenly over the threads");
    static_assert((1 << kFoldMaxSbLog2) <= kFoldThreads, "one super-bucket count per thread");
    static_assert(kFoldFineLog2 <= 16, "fine bucket indices are kept as 16-bit values");

    long long* warp_sums = reinterpret_cast<long long*>(smem);
    long long* total = warp_sums + 32;
    long long* srfx = reinterpret_cast<long long*>(total + 1);                  // rfx in final order (swizzled)
    unsigned long long* sorted = reinterpret_cast<unsigned long long*>(srfx + kFoldSegKeys);   // keys in fine-bucket order
    uint32_t* fcnt = reinterpret_cast<uint32_t*>(sorted + kFoldSegKeys);
    uint32_t* fcur = fcnt + (1 << kFoldFineLog2);
    uint32_t* sb_cnt = fcur + (1 << kFoldFineLog2);
    uint32_t* sb_start = sb_cnt + (1 << kFoldMaxSbLog2);
    uint16_t* inv = reinterpret_cast<uint16_t*>(sb_start + (1 << kFoldMaxSbLog2));       // final position -> sorted position
    uint16_t* sorted_f = inv + kFoldSegKeys;                                              // fine bucket of sorted[q]
    int* overflow = reinterpret_cast<int*>(sorted_f + kFoldSegKeys);

    for (int q = threadIdx.x; q < nsb; q += blockDim.x) sb_cnt[q] = 0;
    if (threadIdx.x == 0) *overflow = 0;
    __syncthreads();

    // A. super-bucket of every point; its key goes to the next slot of the
    // super-bucket's region (a shared-memory atomic per point: aggregating
    // the lanes of a warp with equal super-buckets first measured slower)
    const int64_t bs = blockDim.x;
    for (int64_t g0 = 0; g0 < n; g0 += kFoldUnroll * bs) {
        long long dl[kFoldUnroll];
        float df[kFoldUnroll];
#pragma unroll
        for (int u = 0; u < kFoldUnroll; ++u) {
            const int64_t i = g0 + u * bs + threadIdx.x;
            dl[u] = i < n ? dc.d_lat[i] : 0;
            df[u] = i < n ? dc.d_f[i] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kFoldUnroll; ++u) {
            const int64_t i = g0 + u * bs + threadIdx.x;
            const long long rho = lattice_rho(dl[u], df[u], P, inv_p);
            const uint32_t sb = fold_fine(rho, sh, mulf) >> kFoldFineLog2;
            const bool ok = i < n && in_range(dc.check, 2, rho, P) && in_range32(dc.check, 1, sb, nsb);
            if (ok) {
                const uint32_t slot = atomicAdd(&sb_cnt[sb], 1u);
                if (slot < (uint32_t)kFoldSegKeys)
                    keys[(int64_t)sb * kFoldSegKeys + slot] = ((unsigned long long)rho << ib) | (unsigned long long)i;
                else
                    *overflow = 1;
            }
        }
    }
    __syncthreads();
    if (*overflow) return false;
    {
        // positions of the super-buckets in the folded order
        const uint32_t c = threadIdx.x < nsb ? sb_cnt[threadIdx.x] : 0u;
        const long long st = block_exclusive_scan(c, warp_sums, total);
        if (threadIdx.x < nsb) sb_start[threadIdx.x] = (uint32_t)st;
    }
    __syncthreads();

    // B. each super-bucket in shared memory: the keys staged with their fine
    // bucket, counting-sorted by fine bucket and ranked inside it, which
    // gives inv[final position] = sorted position; then, in final-position
    // order, the folded curve gathered (coalesced stores), rfx scanned and
    // the prefix sums written.
    constexpr int kPerThread = kFoldSegKeys / kFoldThreads;
    static_assert(kFoldSegKeys % kFoldThreads == 0, "staged keys split evenly over the threads");
    static_assert(kPerThread == kScanPer, "one scan pass per super-bucket");
    static_assert(kPerThread % kRankBatch == 0, "gathers issued in whole batches");
    // srfx is read in blocks of kScanPer consecutive entries per thread; the
    // swizzle spreads the 16 lanes of a half-warp over 16 bank pairs
    auto swz = [](uint32_t i) { return i ^ ((i >> 4) & 7u); };
    long long carry = 0;
    if (threadIdx.x == 0) o.pf[0] = 0;
    for (int sb = 0; sb < nsb; ++sb) {
        const uint32_t k0 = sb_start[sb], len = sb_cnt[sb];
        if (len == 0) continue;
        const unsigned long long* region = keys + (int64_t)sb * kFoldSegKeys;
        for (int f = threadIdx.x; f < (1 << kFoldFineLog2); f += blockDim.x) fcnt[f] = 0;
        __syncthreads();
        // a thread's keys of the super-bucket and their fine buckets stay in
        // registers from the count to the scatter
        unsigned long long kv[kPerThread];
        uint32_t kf[kPerThread / 2];   // two 16-bit fine buckets per register
#pragma unroll
        for (int u = 0; u < kPerThread; ++u) {
            const uint32_t q = threadIdx.x + u * kFoldThreads;
            kv[u] = q < len ? __ldcs(region + q) : 0ull;   // last use of the staged key
        }
#pragma unroll
        for (int u = 0; u < kPerThread; ++u) {
            const uint32_t q = threadIdx.x + u * kFoldThreads;
            const uint32_t f = fold_fine((long long)(kv[u] >> ib), sh, mulf) & kFineMask;
            if (u & 1) kf[u >> 1] |= f << 16;
            else kf[u >> 1] = f;
            if (q < len) atomicAdd(&fcnt[f], 1u);
        }
        __syncthreads();
        // every staged key of the super-bucket is in registers now: drop the
        // region's lines from L2 without writing them back (the next period
        // writes the region again before reading it), so that the keys
        // cost no DRAM traffic when they stayed in L2
        {
            const uint32_t lines = (len * (uint32_t)sizeof(unsigned long long) + 127u) / 128u;
            for (uint32_t l = threadIdx.x; l < lines; l += blockDim.x)
                asm volatile("discard.global.L2 [%0], 128;" ::"l"(region + 16 * l) : "memory");
        }
        {
            constexpr int kPer = (1 << kFoldFineLog2) / kFoldThreads;
            const int f0 = threadIdx.x * kPer;
            long long local = 0;
#pragma unroll
            for (int u = 0; u < kPer; ++u) local += fcnt[f0 + u];
            long long sum;
            long long run = block_exclusive_scan1(local, warp_sums, sum);
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                fcur[f0 + u] = (uint32_t)run;
                run += fcnt[f0 + u];
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kPerThread; ++u) {
            const uint32_t q = threadIdx.x + u * kFoldThreads;
            if (q >= len) break;
            const uint32_t f = (kf[u >> 1] >> ((u & 1) * 16)) & 0xffffu;
            const uint32_t d = atomicAdd(&fcur[f], 1u);   // fcur[f] ends as the end of bucket f
            if (in_range32(dc.check, 5, d, len)) {
                sorted[d] = kv[u];
                sorted_f[d] = (uint16_t)f;
            }
        }
        __syncthreads();
        // rank inside the fine bucket: [fcur[f] - fcnt[f], fcur[f]) of sorted
        for (uint32_t q = threadIdx.x; q < len; q += blockDim.x) {
            const unsigned long long key = sorted[q];
            const uint32_t f = sorted_f[q];
            const uint32_t cnt = fcnt[f], e = fcur[f];
            if (!in_range32(dc.check, 6, e, len + 1) || !in_range32(dc.check, 6, cnt, e + 1)) continue;
            const uint32_t lo = e - cnt;
            uint32_t rank = 0;
            for (uint32_t u = 0; u < cnt; ++u) rank += sorted[lo + u] < key ? 1u : 0u;
            if (in_range32(dc.check, 7, lo + rank, len)) inv[lo + rank] = (uint16_t)q;
        }
        __syncthreads();
        // gather in final-position order (kRankBatch points' loads in flight;
        // batches past the super-bucket's length skipped, block-uniform)
#pragma unroll
        for (int h = 0; h < kPerThread; h += kRankBatch) {
            if ((uint32_t)h * kFoldThreads >= len) break;
            int32_t id[kRankBatch];
            bool ok[kRankBatch];
#pragma unroll
            for (int j = 0; j < kRankBatch; ++j) {
                const uint32_t i = threadIdx.x + (h + j) * kFoldThreads;
                ok[j] = false;
                id[j] = 0;
                if (i >= len) continue;
                const uint32_t q = inv[i];
                if (!in_range32(dc.check, 7, q, len)) continue;
                id[j] = (int32_t)(sorted[q] & idx_mask);
                ok[j] = in_range32(dc.check, 8, (uint32_t)id[j], (uint32_t)n);
            }
            PointVals pv[kRankBatch];
#pragma unroll
            for (int j = 0; j < kRankBatch; ++j) pv[j] = ok[j] ? dc.pv[id[j]] : PointVals{0, 0.0f, 0.0f};
#pragma unroll
            for (int j = 0; j < kRankBatch; ++j) {
                const uint32_t i = threadIdx.x + (h + j) * kFoldThreads;
                if (!ok[j]) continue;
                const int64_t g = (int64_t)k0 + i;
                // streaming stores: the window kernels read the folded curve
                // after the whole chunk is folded, from DRAM, so these lines
                // go first when L2 needs room (the super-bucket regions stay)
                __stcs(o.sidx + g, id[j]);
                __stcs(o.rs + g, pv[j].r);
                srfx[swz(i)] = pv[j].rfx;
                if (!o.uniform) {
                    __stcs(o.ws + g, pv[j].w);
                    __stcs(o.wrs + g, pv[j].w * pv[j].r);
                }
            }
        }
        __syncthreads();
        // inclusive prefix of rfx in final order, kScanPer consecutive
        // entries per thread, written back in place
        {
            const uint32_t i0 = threadIdx.x * kScanPer;
            long long v[kScanPer];
            long long run = 0;
#pragma unroll
            for (int u = 0; u < kScanPer; ++u) {
                run += i0 + u < len ? srfx[swz(i0 + u)] : 0;
                v[u] = run;
            }
            long long sum;
            const long long ex = block_exclusive_scan1(run, warp_sums, sum) + carry;
#pragma unroll
            for (int u = 0; u < kScanPer; ++u)
                if (i0 + u < len) srfx[swz(i0 + u)] = ex + v[u];
            carry += sum;
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) __stcs(o.pf + (int64_t)k0 + 1 + i, srfx[swz(i)]);
        __syncthreads();   // the next super-bucket overwrites the staged keys and rfx
    }
    return true;
}

// Global path (see above).
__device__ void fold_global(unsigned char* smem, const DevPlan& dp, const DevCurve& dc, int p,
                            unsigned long long* keys, const FoldOut& o)
{
    const int nb = 1 << dp.bucket_log2;
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem);
    uint32_t* start = hist + nb;
    long long* warp_sums = reinterpret_cast<long long*>(start + nb);
    long long* total = warp_sums + 32;

    const int64_t n = dp.n;
    const long long P = dp.p_lat[p];
    const float inv_p = dp.inv_p[p];
    const int sh = dp.bucket_shift[p];
    const uint32_t mul = dp.bucket_mul[p];
    const int ib = dp.idx_bits;
    const unsigned long long idx_mask = (1ull << ib) - 1ull;

    for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();

    // 1. bucket histogram (the loads of kFoldUnroll points are issued before
    // their arithmetic)
    const int64_t bs = blockDim.x;
    for (int64_t i0 = threadIdx.x; i0 < n; i0 += kFoldUnroll * bs) {
        long long dl[kFoldUnroll];
        float df[kFoldUnroll];
#pragma unroll
        for (int u = 0; u < kFoldUnroll; ++u) {
            const int64_t i = i0 + u * bs;
            dl[u] = i < n ? dc.d_lat[i] : 0;
            df[u] = i < n ? dc.d_f[i] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kFoldUnroll; ++u) {
            const int64_t i = i0 + u * bs;
            if (i >= n) break;
            const long long rho = lattice_rho(dl[u], df[u], P, inv_p);
            const uint32_t b = fold_bucket(rho, sh, mul);
            if (in_range(dc.check, 1, b, nb) && in_range(dc.check, 2, rho, P)) atomicAdd(&hist[b], 1u);
        }
    }
    __syncthreads();

    // 2. bucket starts (exclusive scan of the histogram)
    {
        const int per = (nb + blockDim.x - 1) / blockDim.x;
        const int b0 = threadIdx.x * per;
        long long local = 0;
        for (int b = b0; b < b0 + per && b < nb; ++b) local += hist[b];
        long long run = block_exclusive_scan(local, warp_sums, total);
        for (int b = b0; b < b0 + per && b < nb; ++b) {
            start[b] = (uint32_t)run;
            run += hist[b];
        }
    }
    __syncthreads();

    // 3. scatter keys (phase << idx_bits | index) into bucket order; the
    // arrival order inside a bucket does not matter (the keys are ranked
    // below), and start[b] ends as the end of bucket b
    for (int64_t i0 = threadIdx.x; i0 < n; i0 += kFoldUnroll * bs) {
        long long dl[kFoldUnroll];
        float df[kFoldUnroll];
#pragma unroll
        for (int u = 0; u < kFoldUnroll; ++u) {
            const int64_t i = i0 + u * bs;
            dl[u] = i < n ? dc.d_lat[i] : 0;
            df[u] = i < n ? dc.d_f[i] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kFoldUnroll; ++u) {
            const int64_t i = i0 + u * bs;
            if (i >= n) break;
            const long long rho = lattice_rho(dl[u], df[u], P, inv_p);
            const uint32_t b = fold_bucket(rho, sh, mul);
            if (!in_range(dc.check, 3, b, nb)) continue;
            const long long dst = (long long)atomicAdd(&start[b], 1u);
            if (in_range(dc.check, 4, dst, n))
                keys[dst] = ((unsigned long long)rho << ib) | (unsigned long long)i;
        }
    }
    __syncthreads();

    // 4. per run of whole buckets: rank inside the bucket -> folded position,
    // gather the folded curve, and the prefix sums of rfx in folded order
    // (pf[k+1] = sum_{u<=k} rfx).  A run holds at most kFoldSegKeys keys; its
    // keys and folded rfx are staged in shared memory, ranked and scanned
    // there, and pf is written once, coalesced.  A single bucket larger than
    // that is ranked and scanned in global memory.
    unsigned long long* const skeys = reinterpret_cast<unsigned long long*>(total + 1);
    long long* const srfx = reinterpret_cast<long long*>(skeys + kFoldSegKeys);
    const int64_t span = bs * kScanPer;
    long long carry = 0;   // sum of rfx over the folded positions before the run
    if (threadIdx.x == 0) o.pf[0] = 0;
    auto begin_of = [&](int b) -> uint32_t { return b < nb ? start[b] - hist[b] : (uint32_t)n; };
    for (int b_lo = 0; b_lo < nb;) {
        const uint32_t k0 = begin_of(b_lo);
        int b_hi = b_lo + 1;
        if (begin_of(b_hi) - k0 <= (uint32_t)kFoldSegKeys) {
            int lo = b_hi, hi = nb;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (begin_of(mid) - k0 <= (uint32_t)kFoldSegKeys) lo = mid;
                else hi = mid - 1;
            }
            b_hi = lo;
        }
        const uint32_t k1 = begin_of(b_hi);
        const uint32_t len = k1 - k0;
        if (len <= (uint32_t)kFoldSegKeys) {
            for (uint32_t q = threadIdx.x; q < len; q += blockDim.x) skeys[q] = keys[k0 + q];
            __syncthreads();
            auto bucket_of = [&](uint32_t, unsigned long long key, int& b) {
                b = (int)fold_bucket((long long)(key >> ib), sh, mul);
                return in_range(dc.check, 5, (long long)b - b_lo, b_hi - b_lo);
            };
            fold_rank_gather(skeys, len, k0, hist, start, k0, bucket_of, ib, idx_mask, n, dc, o, srfx);
            __syncthreads();
            fold_scan_run(srfx, len, k0, o.pf, carry, warp_sums, total);
            __syncthreads();   // the next run overwrites the staged keys and rfx
        } else {
            for (int64_t q = k0 + threadIdx.x; q < k1; q += blockDim.x) {
                const unsigned long long key = keys[q];
                const uint32_t b = fold_bucket((long long)(key >> ib), sh, mul);
                if (!in_range(dc.check, 5, (long long)b - b_lo, b_hi - b_lo)) continue;
                const uint32_t cnt = hist[b], lo = start[b] - cnt;
                if (!in_range(dc.check, 6, (long long)lo + cnt, (long long)k1 + 1)) continue;
                uint32_t rank = 0;
                for (uint32_t u = 0; u < cnt; ++u) rank += keys[lo + u] < key ? 1u : 0u;
                const uint32_t g = lo + rank;
                const int32_t id = (int32_t)(key & idx_mask);
                if (!in_range(dc.check, 7, g, n) || !in_range(dc.check, 8, id, n)) continue;
                const PointVals v = dc.pv[id];
                o.sidx[g] = id;
                o.rs[g] = v.r;
                o.pf[g + 1] = v.rfx;
                if (!o.uniform) {
                    o.ws[g] = v.w;
                    o.wrs[g] = v.w * v.r;
                }
            }
            __syncthreads();
            for (int64_t base = k0; base < k1; base += span) {
                const int64_t i0 = base + (int64_t)threadIdx.x * kScanPer;
                long long v[kScanPer];
                long long run = 0;
#pragma unroll
                for (int u = 0; u < kScanPer; ++u) {
                    run += i0 + u < k1 ? o.pf[i0 + u + 1] : 0;
                    v[u] = run;
                }
                const long long ex = block_exclusive_scan(run, warp_sums, total) + carry;
#pragma unroll
                for (int u = 0; u < kScanPer; ++u)
                    if (i0 + u < k1) o.pf[i0 + u + 1] = ex + v[u];
                carry += *total;
            }
            __syncthreads();
        }
        b_lo = b_hi;
    }
}

__global__ void __launch_bounds__(kFoldThreads, kFoldMinBlocks)
k_fold_sort(DevSet ds, const __grid_constant__ SlotMap smv, const SlotMap* smq, DevChunk dk)
{
    const SlotMap& sm = smq ? *smq : smv;
    extern __shared__ unsigned char smem[];
    const int slot_id = blockIdx.x;
    int lc, p;
    if (!resolve_slot(ds, sm, slot_id, lc, p)) return;
    unsigned long long* const keys = dk.keys + (int64_t)slot_id * dk.key_stride;
    const DevPlan& dp = ds.plans[lc];
    const DevCurve dc = ds.curves[lc];
    FoldOut o;
    o.sidx = dk.sidx + (int64_t)slot_id * dk.fold_stride;
    o.rs = dk.rs + (int64_t)slot_id * dk.pad_stride;
    o.ws = dk.ws ? dk.ws + (int64_t)slot_id * dk.pad_stride : nullptr;
    o.wrs = dk.wrs ? dk.wrs + (int64_t)slot_id * dk.pad_stride : nullptr;
    o.pf = dk.pf + (int64_t)slot_id * dk.pad_stride;
    o.uniform = dc.scal[2] > 0.0;
    if (threadIdx.x == 0) ds.outs[lc].best[p] = ~0ull;

    if (!fold_staged(smem, dp, dc, p, keys, o)) {
        __syncthreads();   // the global path reuses the shared memory
        fold_global(smem, dp, dc, p, keys, o);
    }

    // padding: the first D_m folded points repeat after position N-1
    const int64_t n = dp.n;
    const int64_t dm = dp.dmax_p[p];
    const long long tot = o.pf[n];
    for (int64_t k = threadIdx.x; k < dm + kPadMargin; k += blockDim.x) {
        const bool real = k < dm;
        o.rs[n + k] = real ? o.rs[k] : 0.0f;
        if (!o.uniform) {
            o.ws[n + k] = real ? o.ws[k] : 0.0f;
            o.wrs[n + k] = real ? o.wrs[k] : 0.0f;
        }
        if (real) o.pf[n + k + 1] = tot + o.pf[k + 1];
    }
}

// ---------------------------------------------------------------------------
// window search: one thread per (period, duration, T0 start)
// ---------------------------------------------------------------------------

__device__ __forceinline__ int kept_j(const DevPlan& dp, int p, int slot)
{
    const int lo = dp.jlo[p], hi = dp.jhi[p];
    int c = -1;
    for (int j = lo; j <= hi; ++j) {
        if (j > lo && dp.dpts[j] == dp.dpts[j - 1]) continue;
        if (++c == slot) return j;
    }
    return -1;
}

__global__ void __launch_bounds__(kSearchThreads)
k_window_search(DevSet ds, const __grid_constant__ SlotMap smv, const SlotMap* smq, DevChunk dk, int only_window_only)
{
    const SlotMap& sm = smq ? *smq : smv;
    __shared__ unsigned long long red[kSearchThreads / 32];
    const int slot_id = blockIdx.z;
    int lc, p;
    if (!resolve_slot(ds, sm, slot_id, lc, p)) return;
    const DevPlan& dp = ds.plans[lc];
    const DevCurve dc = ds.curves[lc];
    const int j = kept_j(dp, p, blockIdx.y);
    if (j < 0) return;
    if (only_window_only && dp.cfg_variant[j] != tiles::kWindowOnly) return;
    const int d = dp.dpts[j], st = dp.stride[j];
    const int64_t n = dp.n;
    const int64_t nwin = (n + st - 1) / st;
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if ((int64_t)blockIdx.x * blockDim.x >= nwin) return;  // whole block past the end
    unsigned long long packed = ~0ull;
    const bool ok = in_range(dc.check, 9, j, dp.nd) && in_range(dc.check, 10, d, dp.dmax_p[p] + 1) &&
                    in_range(dc.check, 11, dp.tmpl_off[j] + d, dp.tmpl_total + 1) &&
                    in_range(dc.check, 12, (nwin - 1) * st + d, dk.pad_stride);
    if (ok && m < nwin) {
        const int64_t s = m * st;
        const float* rs = dk.rs + (int64_t)slot_id * dk.pad_stride + s;
        const long long* pf = dk.pf + (int64_t)slot_id * dk.pad_stride;
        const float* tm = dp.tmpl + dp.tmpl_off[j];
        const double w_uni = dc.scal[2];
        const long long sfx = pf[s + d] - pf[s];
        const float sum_r = (float)((double)sfx * (1.0 / kRScale));
        const float depth = fmaxf(0.0f, sum_r * dp.inv_sum_t[j]);
        float dchi;
        if (w_uni > 0.0) {
            float c1 = 0.0f;
            for (int k = 0; k < d; ++k) c1 = fmaf(rs[k], tm[k], c1);
            dchi = (float)w_uni * depth * fmaf(depth, dp.sum_t2[j], -2.0f * c1);
        } else {
            const float* wr = dk.wrs + (int64_t)slot_id * dk.pad_stride + s;
            const float* ww = dk.ws + (int64_t)slot_id * dk.pad_stride + s;
            float c1 = 0.0f, c2 = 0.0f;
            for (int k = 0; k < d; ++k) {
                c1 = fmaf(wr[k], tm[k], c1);
                c2 = fmaf(ww[k] * tm[k], tm[k], c2);
            }
            dchi = depth * fmaf(depth, c2, -2.0f * c1);
        }
        packed = ((unsigned long long)float_order_key(dchi) << 32) |
                 ((unsigned long long)j << 24) | (unsigned long long)m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, packed, o);
        packed = v < packed ? v : packed;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = packed;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = red[0];
        for (int w = 1; w < kSearchThreads / 32; ++w) b = red[w] < b ? red[w] : b;
        atomicMin(&ds.outs[lc].best[p], b);
    }
}

// ---------------------------------------------------------------------------
// tiled window search (uniform weights): see window_tiles.cuh
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(tiles::kThreads, tiles::kCtasPerSm)
k_window_tiles(DevSet ds, const __grid_constant__ SlotMap smv, const SlotMap* smq, DevChunk dk, int buf, int weighted,
               unsigned int* counter)
{
    const SlotMap& sm = smq ? *smq : smv;
    using namespace tiles;
    extern __shared__ float tile_smem[];
    __shared__ DurTask dur[kMaxDur];
    __shared__ int s_item, s_ndur, s_total, s_task, s_lc, s_p, s_slot, s_x0, s_len, s_tau, s_tcount;
    __shared__ unsigned long long s_best[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = (int)atomicAdd(counter, 1u);
            s_item = item;
            if (item < sm.items) {
                int g = 0;
                while (g + 1 < sm.nseg && sm.seg[g + 1].item0 <= item) ++g;
                const int lcg = sm.seg[g].lc;
                const DevTiles tl = ds.tiles[lcg];
                const int tcount = weighted ? tl.count_w : tl.count;
                const int rel = item - sm.seg[g].item0;
                const int k = rel / tcount, tau = rel - k * tcount;
                const int q = sm.seg[g].first + k;
                int pp = sm.from_list ? ds.outs[lcg].plist[q] : q;
                if (!in_range(ds.curves[lcg].check, 22, pp, ds.plans[lcg].np)) pp = -1;
                s_lc = lcg;
                s_p = pp;
                s_slot = sm.seg[g].slot0 + k;
                s_x0 = tau * (weighted ? tl.len_w : tl.len);
                s_len = weighted ? tl.len_w : tl.len;
                s_tau = tau;
                s_tcount = tcount;
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item >= sm.items) break;
        const int lc = s_lc, p = s_p, slot = s_slot, x0 = s_x0, tile_len = s_len, tau = s_tau, tcount = s_tcount;
        if (p < 0) {   // block-uniform: a failed check skips the item
            __syncthreads();
            continue;
        }
        const DevPlan& dp = ds.plans[lc];
        unsigned int* const check = ds.curves[lc].check;
        const float w_uni = (float)ds.curves[lc].scal[2];
        const int64_t n = dp.n;

        // stage the folded, padded curve [x0, x0 + buf) (zeros past its end)
        const int valid = (int)min((int64_t)buf, n + (int64_t)dp.dmax_p[p] + kPadMargin - x0);
        if (weighted) {
            // (w r, w) pairs of the folded curve
            const float* swr = dk.wrs + (int64_t)slot * dk.pad_stride + x0;
            const float* sw = dk.ws + (int64_t)slot * dk.pad_stride + x0;
            float2* t2 = reinterpret_cast<float2*>(tile_smem);
            for (int i = threadIdx.x; i < buf; i += blockDim.x)
                t2[i] = i < valid ? make_float2(__ldg(swr + i), __ldg(sw + i)) : make_float2(0.0f, 0.0f);
        } else {
            const float* src = dk.rs + (int64_t)slot * dk.pad_stride + x0;
            const int v4 = valid >> 2;
            for (int i = threadIdx.x; i < v4; i += blockDim.x)
                reinterpret_cast<float4*>(tile_smem)[i] = __ldg(reinterpret_cast<const float4*>(src) + i);
            for (int i = (v4 << 2) + threadIdx.x; i < buf; i += blockDim.x)
                tile_smem[i] = i < valid ? src[i] : 0.0f;
        }

        // durations of the period, longest first, with their task ranges
        // (warp 0: one lane per candidate duration, ballot-compacted)
        if (warp == 0) {
            const int lo = dp.jlo[p], hi = dp.jhi[p];
            int kcount = 0;
            for (int base = 0; base <= hi - lo; base += 32) {
                const int j = hi - base - lane;
                const bool kept = j >= lo && (j == lo || dp.dpts[j] != dp.dpts[j - 1]);
                const unsigned int mask = __ballot_sync(0xffffffffu, kept);
                const int k = kcount + __popc(mask & ((1u << lane) - 1u));
                if (kept && in_range(check, 19, k, kMaxDur)) {
                    DurTask t;
                    t.j = j;
                    t.d = dp.dpts[j];
                    t.st = dp.stride[j];
                    t.m_total = (int)((n + t.st - 1) / t.st);
                    t.m_a = (x0 + t.st - 1) / t.st;
                    t.m_b = min(t.m_total, (x0 + tile_len + t.st - 1) / t.st);
                    t.variant = weighted ? (int)kWeighted15 : dp.cfg_variant[j];
                    t.nc = weighted ? dp.cfg_nc_w[j] : dp.cfg_nc[j];
                    t.w = variant_w(t.variant);
                    t.per_task = 32 * t.w / t.nc;
                    const int jrows = (t.d + t.st - 1) / t.st;
                    {
                        // whole tasks per tile where the staged buffers have room:
                        // the duration covers windows [tau K, (tau + 1) K) of tile
                        // tau, K a multiple of the task length with K st >= L (each
                        // tile starts inside its buffer) and K st <= L + room /
                        // tiles (the last tile's blocks and rows still fit), so
                        // that only its last tile has a partly filled task
                        const long long room =
                            (long long)buf - 32 - (long long)(jrows + t.w) * t.st - tile_len;
                        if (room > 0) {
                            const long long span = tile_len + room / tcount;
                            const long long k = span / t.st / t.per_task * t.per_task;
                            if (k * t.st >= tile_len) {
                                t.m_a = (int)min((long long)t.m_total, (long long)tau * k);
                                t.m_b = (int)min((long long)t.m_total, (long long)(tau + 1) * k);
                            }
                        }
                    }
                    const int nwin = max(0, t.m_b - t.m_a);
                    t.tasks = (!weighted && (t.variant == kWindowOnly || t.variant == kTensor))
                                  ? 0
                                  : (nwin + t.per_task - 1) / t.per_task;
                    t.jrows = jrows;
                    t.tg = dp.tmpl + dp.tmpl_off[j];
                    t.tg2 = weighted ? dp.tmplw + dp.tmplw_off[j] : dp.tmpl2 + dp.tmpl2_off[j];
                    t.inv_sum_t = dp.inv_sum_t[j] * (1.0f / 1099511627776.0f);  // 2^-40 fixed point
                    t.inv_sum_t_f = dp.inv_sum_t[j];
                    t.sum_t2 = dp.sum_t2[j];
                    // rows up to m + w + jrows - 1 and columns up to st + 31 must stay in the buffer
                    const int m_max_start = (x0 + buf - 32) / t.st - t.w - jrows;
                    t.hi_start = min(t.m_total - t.w, m_max_start);
                    if (t.tasks > 0) in_range(check, 20, (int64_t)t.m_a, (int64_t)m_max_start + 1);
                    t.first = 0;
                    dur[k] = t;
                }
                kcount += __popc(mask);
            }
            kcount = min(kcount, kMaxDur);
            __syncwarp();
            int run = 0;
            for (int base = 0; base < kcount; base += 32) {
                const int k = base + lane;
                const int tk = k < kcount ? dur[k].tasks : 0;
                int incl = tk;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (k < kcount) dur[k].first = run + incl - tk;
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) {
                s_ndur = kcount;
                s_total = run;
                s_task = 0;
            }
        }
        __syncthreads();

        unsigned long long best = ~0ull;
        const int ndur = s_ndur, total = s_total;
        for (;;) {
            int task = 0;
            if (lane == 0) task = atomicAdd(&s_task, 1);
            task = __shfl_sync(0xffffffffu, task, 0);
            if (task >= total) break;
            int lo_k = 0, hi_k = ndur - 1;   // last entry with first <= task
            while (lo_k < hi_k) {
                const int mid = (lo_k + hi_k + 1) >> 1;
                if (dur[mid].first <= task) lo_k = mid;
                else hi_k = mid - 1;
            }
            const int k = lo_k;
            const DurTask t = dur[k];
            WinCtx c;
            c.tile = tile_smem;
            c.tile2 = reinterpret_cast<const float2*>(tile_smem);
            c.x0 = x0;
            c.d = t.d;
            c.st = t.st;
            c.nc = t.nc;
            c.lg_nc = __ffs(t.nc) - 1;
            c.jrows = t.jrows;
            c.tg2 = t.tg2;
            c.m_first = t.m_a + (task - t.first) * t.per_task;
            c.m_a = t.m_a;
            c.m_b = t.m_b;
            c.hi_start = t.hi_start;
            c.m_total = t.m_total;
            c.tg = t.tg;
            c.inv_sum_t = t.inv_sum_t;
            c.inv_sum_t_f = t.inv_sum_t_f;
            c.sum_t2 = t.sum_t2;
            c.w_uni = w_uni;
            c.j = t.j;
            c.pf = dk.pf + (int64_t)slot * dk.pad_stride;
            switch (t.variant) {
            case kWin16: warp_task_winpair<16, 3>(c, lane, best); break;
            case kCol16: warp_task_colpair<16, 3>(c, lane, best); break;
            case kCol16R: warp_task_colpair_rot<16, 3>(c, lane, best); break;
            case kCol15: warp_task_colpair<15, 4>(c, lane, best); break;
            case kCol12: warp_task_colpair<12, 3>(c, lane, best); break;
            case kWeighted15: warp_task_weighted<15, 4>(c, lane, best); break;
            default: warp_task_scalar<15, 4>(c, lane, best); break;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
            best = v < best ? v : best;
        }
        if (lane == 0) s_best[warp] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long b = s_best[0];
            for (int w = 1; w < kWarps; ++w) b = s_best[w] < b ? s_best[w] : b;
            atomicMin(&ds.outs[lc].best[p], b);
        }
    }
}

// ---------------------------------------------------------------------------
// tensor-core window search (uniform weights): see window_tc.cuh
// ---------------------------------------------------------------------------

// Row pitch (points) of duration j on the tensor-core kernel: g = 4 / gcd(st, 4)
// windows per row, so that rows start on 16-byte boundaries.
__host__ __device__ __forceinline__ int tc_windows_per_row(int st) { return (st & 3) == 0 ? 1 : ((st & 1) ? 4 : 2); }

// Row blocks I of a window of d points: ceil((d + (g - 1) st) / sigma).
__host__ __device__ __forceinline__ int tc_row_blocks(int d, int st, int g)
{
    const int sigma = g * st;
    return (d + (g - 1) * st + sigma - 1) / sigma;
}

// Producer: items (slot, duration) from the device counter, item = slot *
// jspan + (j - jlo); per chunk the description, the TMA load of the rows and
// the bulk copy of B into the next stage of the ring; finally an end marker.
__device__ void tc_producer(const DevSet& ds, const SlotMap& sm, const DevChunk& dk, const void* maps, int jspan,
                            unsigned int* counter, tc::TcSmem& S, int test_wait)
{
    using namespace tc;
    volatile int* abort = &S.abort;
    const uint32_t a_base = smem_addr(&S.a[0][0]), b_base = smem_addr(&S.b[0][0]);
    const uint32_t full0 = smem_addr(&S.full[0]), af0 = smem_addr(&S.a_free[0]), bf0 = smem_addr(&S.b_free[0]);
    const int total = sm.slots * jspan;
    uint32_t c = 0;
    bool ok = true;
    if (test_wait) {
        // timeout test: a wait on a barrier phase that nothing completes (no
        // MMA can be committed before the first chunk is issued)
        if (!mbar_wait(smem_addr(&S.t_free[0]), 0u, kTestWaitCycles)) {
            record_check(ds.curves[0].check, kCheckTimeout, 1, 0);
            *abort = 1;
            ok = false;
        }
    }
    // a stage is free once the converters read its rows and the MMAs its B
    auto claim = [&](uint32_t cc) -> bool {
        if (cc < kStages) return true;
        const uint32_t s = cc % kStages, par = ((cc - kStages) / kStages) & 1u;
        if (mbar_wait(af0 + 8 * s, par, kWaitCycles, abort) && mbar_wait(bf0 + 8 * s, par, kWaitCycles, abort))
            return true;
        if (!*abort) record_check(ds.curves[0].check, kCheckTimeout, (long long)cc, 8);
        *abort = 1;
        return false;
    };
    while (ok) {
        const int item = (int)atomicAdd(counter, 1u);
        if (item >= total) break;
        const int slot = item / jspan, jj = item - slot * jspan;
        int lc = 0, p = 0;
        if (!resolve_slot(ds, sm, slot, lc, p)) continue;
        const DevPlan& dp = ds.plans[lc];
        const int j = dp.jlo[p] + jj;
        if (j > dp.jhi[p] || (jj > 0 && dp.dpts[j] == dp.dpts[j - 1]) || dp.cfg_variant[j] != tiles::kTensor)
            continue;
        unsigned int* const check = ds.curves[lc].check;
        const int64_t n = dp.n;
        const int d = dp.dpts[j], st = dp.stride[j];
        const int g = tc_windows_per_row(st);
        const int sigma = g * st;
        const int nblk = tc_row_blocks(d, st, g);
        const int ksteps = (sigma + 7) >> 3;
        const int nch = (ksteps + 3) >> 2;
        const int64_t nwin = (n + st - 1) / st;
        const int64_t wrows = (nwin + g - 1) / g;        // rows that start windows
        const int per_tile = kRows - (nblk - 1);
        const int64_t tiles_n = (wrows + per_tile - 1) / per_tile;
        if (!in_range(check, 31, nblk * g, kN + 1) || !in_range(check, 32, sigma / 4 - 1, kMaps) ||
            !in_range(check, 33, (wrows + nblk - 1) * (int64_t)sigma, n + dp.dmax_p[p] + kPadMargin + 1) ||
            !in_range(check, 34, d, dp.dmax_p[p] + 1) || !in_range(check, 35, tiles_n, 1ll << 24))
            continue;
        const void* map = static_cast<const unsigned char*>(maps) + (size_t)(sigma / 4 - 1) * 128;
        const float* tab = dp.tc_tab + dp.tc_off[j];
        ChunkInfo ci{};
        ci.end = 0;
        ci.lc = lc;
        ci.p = p;
        ci.j = j;
        ci.st = st;
        ci.d = d;
        ci.g = g;
        ci.nblk = nblk;
        ci.per_tile = per_tile;
        ci.nwin = nwin;
        ci.slot = slot;
        ci.w_uni = (float)ds.curves[lc].scal[2];
        ci.inv_sum_t = dp.inv_sum_t[j] * (1.0f / 1099511627776.0f);
        ci.sum_t2 = dp.sum_t2[j];
        for (int64_t t = 0; t < tiles_n && ok; ++t) {
            for (int kc = 0; kc < nch; ++kc) {
                if (!claim(c)) {
                    ok = false;
                    break;
                }
                const uint32_t s = c % kStages;
                ci.kc = kc;
                ci.ksteps = min(4, ksteps - kc * 4);
                ci.kst_tile = ksteps;
                ci.first = kc == 0;
                ci.last = kc == nch - 1;
                ci.item_last = ci.last && t == tiles_n - 1;
                ci.tile = (int)t;
                S.info[s] = ci;
                mbar_expect_tx(full0 + 8 * s, kBytesA + kBytesB);
                tma_load_3d(a_base + s * kBytesA, map, kc * kChunk, (int)(t * per_tile), slot, full0 + 8 * s);
                bulk_load(b_base + s * kBytesB, tab + (size_t)kc * 2 * kN * kChunk, kBytesB, full0 + 8 * s);
                ++c;
            }
        }
    }
    bool marked = false;
    if (ok && claim(c)) {
        const uint32_t s = c % kStages;
        S.info[s].end = 1;
        mbar_arrive(full0 + 8 * s);
        marked = true;
    }
    // copies in flight land before the CTA frees its memory (the stage that
    // took the end marker has moved on by one phase: its last chunk is done)
    const uint32_t lo = c >= kStages ? c - kStages + (marked ? 1u : 0u) : 0u;
    for (uint32_t cc = lo; cc < c; ++cc)
        mbar_wait(full0 + 8 * (cc % kStages), (cc / kStages) & 1u, kWaitCycles);
}

// MMA thread w (0..3): k-step w of every chunk, its three tcgen05.mma (A
// from the chunk's TMEM stage, B from its shared-memory stage) into
// accumulator w of the tile's D buffer; every chunk is committed to the
// barriers that free the TMEM stage and B, and a tile's last chunk to the
// tile's D barrier (each of them counts the four threads).
__device__ void tc_mma(tc::TcSmem& S, uint32_t tmem, unsigned int* check0, int w)
{
    using namespace tc;
    volatile int* abort = &S.abort;
    const uint32_t b_base = smem_addr(&S.b[0][0]);
    const uint32_t full0 = smem_addr(&S.full[0]), bf0 = smem_addr(&S.b_free[0]);
    const uint32_t tf0 = smem_addr(&S.t_full[0]), tr0 = smem_addr(&S.t_free[0]);
    const uint32_t df0 = smem_addr(&S.d_full[0]), dr0 = smem_addr(&S.d_free[0]);
    const uint32_t if0 = smem_addr(&S.i_full[0]);
    uint32_t tile_seq = 0, committed = 0;
    bool ok = true;
    int where = 0;
    for (uint32_t c = 0;; ++c) {
        const uint32_t s = c % kStages, ts = c % kTStages;
        if (!mbar_wait(full0 + 8 * s, (c / kStages) & 1u, kWaitCycles, abort)) {
            ok = false;
            where = 5;
            break;
        }
        // a copy: the stage (and its description) is refilled as soon as
        // the four threads commit it to b_free
        const ChunkInfo ci = S.info[s];
        if (ci.end) {
            if (w == 0) {
                // end marker for the epilogue, once it left this D buffer
                const uint32_t db = tile_seq & 1u;
                if (tile_seq >= 2 && !mbar_wait(dr0 + 8 * db, ((tile_seq - 2) >> 1) & 1u, kWaitCycles, abort)) {
                    ok = false;
                    where = 9;
                    break;
                }
                S.tinfo[db].end = 1;
                mbar_arrive(if0 + 8 * db);
            }
            break;
        }
        const int kc = ci.kc, ksteps = ci.ksteps, first = ci.first, last = ci.last;
        if (!mbar_wait(tf0 + 8 * ts, (c / kTStages) & 1u, kWaitCycles, abort)) {
            ok = false;
            where = 6;
            break;
        }
        const uint32_t db = tile_seq & 1u;
        if (first && tile_seq >= 2 && !mbar_wait(dr0 + 8 * db, ((tile_seq - 2) >> 1) & 1u, kWaitCycles, abort)) {
            ok = false;
            where = 7;
            break;
        }
        fence_after();
        if (w < ksteps) {
            const uint32_t a_col = tmem + ts * 64u + (uint32_t)(w * 8);
            const uint32_t d_col = tmem + kDCol + db * (kMmaWarps * 32u) + (uint32_t)(w * 32);
            const uint32_t bh = b_base + s * kBytesB + (uint32_t)(w * 256), bl = bh + kBytesB / 2;
            const uint64_t dh = smem_desc(bh, 128, 1024);
            const uint64_t dl = smem_desc(bl, 128, 1024);
            mma_tf32(d_col, a_col, dh, kc > 0 ? 1u : 0u);
            mma_tf32(d_col, a_col, dl, 1u);
            mma_tf32(d_col, a_col + 32, dh, 1u);
        }
        mma_commit(tr0 + 8 * ts);
        mma_commit(bf0 + 8 * s);
        if (last) {
            mma_commit(df0 + 8 * db);
            if (w == 0) {
                S.tinfo[db] = ci;
                mbar_arrive(if0 + 8 * db);
            }
            ++tile_seq;
        }
        committed = c + 1;
    }
    if (!ok) {
        if (!*abort) record_check(check0, kCheckTimeout, (long long)committed, where * 10 + w);
        *abort = 1;
    }
    // the MMAs complete before the CTA frees TMEM
    if (committed > 0) {
        const uint32_t c = committed - 1, ts = c % kTStages;
        mbar_wait(tr0 + 8 * ts, (c / kTStages) & 1u, kWaitCycles);
    }
}

// Converter warps (TMEM lanes 0..127): the rows of every chunk to a TMEM
// stage in TF32 halves.
__device__ void tc_convert(const DevSet& ds, tc::TcSmem& S, uint32_t tmem)
{
    using namespace tc;
    volatile int* abort = &S.abort;
    unsigned int* const check0 = ds.curves[0].check;
    const int l = threadIdx.x;   // 0..127
    const uint32_t lane_field = (uint32_t)((l >> 5) * 32) << 16;
    const uint32_t full0 = smem_addr(&S.full[0]), af0 = smem_addr(&S.a_free[0]);
    const uint32_t tf0 = smem_addr(&S.t_full[0]), tr0 = smem_addr(&S.t_free[0]);
    bool fail = false;
    for (uint32_t c = 0;; ++c) {
        const uint32_t s = c % kStages, ts = c % kTStages;
        if (!fail && !mbar_wait(full0 + 8 * s, (c / kStages) & 1u, kWaitCycles, abort)) {
            fail = true;
            record_check(check0, kCheckTimeout, (long long)c, 1);
            *abort = 1;
        }
        const int end = S.info[s].end;
        float v[32];
        {
            const float4* row = reinterpret_cast<const float4*>(&S.a[s][l * kChunk]);
#pragma unroll
            for (int c4 = 0; c4 < 8; ++c4) {
                const float4 x = row[c4 ^ (l & 7)];
                v[4 * c4] = x.x;
                v[4 * c4 + 1] = x.y;
                v[4 * c4 + 2] = x.z;
                v[4 * c4 + 3] = x.w;
            }
        }
        // the MMAs of chunk c - kTStages read this TMEM stage
        if (!fail && c >= kTStages &&
            !mbar_wait(tr0 + 8 * ts, ((c - kTStages) / kTStages) & 1u, kWaitCycles, abort)) {
            fail = true;
            record_check(check0, kCheckTimeout, (long long)c, 2);
            *abort = 1;
        }
        const uint32_t a_col = tmem + ts * 64u + lane_field;
        {
            uint32_t h[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) h[k] = __float_as_uint(v[k]) & 0xffffe000u;
            tmem_st32(a_col, h);
#pragma unroll
            for (int k = 0; k < 32; ++k) h[k] = __float_as_uint(v[k] - __uint_as_float(h[k]));
            tmem_st32(a_col + 32, h);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        fence_before();
        if (bar_sync_or(1, 128, fail)) break;
        if (end) break;    // every lane read the same marker
        if (l == 0) {
            mbar_arrive(af0 + 8 * s);
            mbar_arrive(tf0 + 8 * ts);
        }
    }
}

// Epilogue warps: every tile once its MMAs completed.  Lane l of warp w owns
// row 32 (w % 4) + l (the TMEM lanes its warp may read).
__device__ void tc_epilogue(const DevSet& ds, const SlotMap& sm, const DevChunk& dk, tc::TcSmem& S, uint32_t tmem,
                            int quad)
{
    using namespace tc;
    volatile int* abort = &S.abort;
    unsigned int* const check0 = ds.curves[0].check;
    const int l = quad * 32 + (threadIdx.x & 31);
    const uint32_t lane_field = (uint32_t)(quad * 32) << 16;
    const uint32_t df0 = smem_addr(&S.d_full[0]), dr0 = smem_addr(&S.d_free[0]);
    const uint32_t if0 = smem_addr(&S.i_full[0]);
    bool fail = false;
    unsigned long long best = ~0ull;
    for (uint32_t tile_seq = 0;; ++tile_seq) {
        const uint32_t db = tile_seq & 1u, par = (tile_seq >> 1) & 1u;
        if (!fail && !mbar_wait(if0 + 8 * db, par, kWaitCycles, abort)) {
            fail = true;
            record_check(check0, kCheckTimeout, (long long)tile_seq, 3);
            *abort = 1;
        }
        const ChunkInfo pi = S.tinfo[db];
        // the description must name a slot of this wave and the curve and
        // period that slot holds (checked before any memory access it steers)
        bool valid = false;
        if (!fail && !pi.end) {
            int lc2 = -1, p2 = -1;
            valid = pi.slot >= 0 && pi.slot < sm.slots && resolve_slot(ds, sm, (int)pi.slot, lc2, p2) &&
                    lc2 == pi.lc && p2 == pi.p;
            if (!valid && l == 0) record_check(check0, 36, pi.slot, pi.p);
        }
        // prefix sums of the windows of this lane's row
        long long pa[4] = {0, 0, 0, 0}, pb[4] = {0, 0, 0, 0};
        if (valid) {
            const long long* pf = dk.pf + pi.slot * dk.pad_stride;
            const int64_t rho = (int64_t)pi.tile * pi.per_tile + l;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t m = rho * pi.g + q;
                if (q < pi.g && l < pi.per_tile && m < pi.nwin) {
                    pa[q] = pf[m * pi.st];
                    pb[q] = pf[m * pi.st + pi.d];
                }
            }
        }
        if (!fail && !pi.end && !mbar_wait(df0 + 8 * db, par, kWaitCycles, abort)) {
            fail = true;
            record_check(check0, kCheckTimeout, (long long)tile_seq, 4);
            *abort = 1;
        }
        float gsum[32];
        if (!fail && !pi.end) {
            fence_after();
            uint32_t gv[32];
            const uint32_t dcol = tmem + kDCol + db * (kMmaWarps * 32u) + lane_field;
            tmem_ld32(dcol, gv);
#pragma unroll
            for (int c = 0; c < 32; ++c) gsum[c] = __uint_as_float(gv[c]);
            const int nacc = min(kMmaWarps, pi.kst_tile);
            for (int a = 1; a < nacc; ++a) {
                tmem_ld32(dcol + (uint32_t)(a * 32), gv);
#pragma unroll
                for (int c = 0; c < 32; ++c) gsum[c] += __uint_as_float(gv[c]);
            }
            fence_before();
        }
        // every lane read its accumulators (and the last tile's G was used)
        if (bar_sync_or(2, 128, fail)) break;
        if (pi.end) break;
        if (l == 0) mbar_arrive(dr0 + 8 * db);
#pragma unroll
        for (int c = 0; c < 32; ++c) S.g[l * 32 + (c ^ (l & 31))] = gsum[c];
        bar_sync(2, 128);
        if (valid && l < pi.per_tile) {
            const int64_t rho = (int64_t)pi.tile * pi.per_tile + l;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t m = rho * pi.g + q;
                if (q < pi.g && m < pi.nwin) {
                    float c1 = 0.0f;
                    for (int i = 0; i < pi.nblk; ++i) {
                        const int r = l + i;
                        c1 += S.g[r * 32 + ((i * pi.g + q) ^ (r & 31))];
                    }
                    const float depth = fmaxf(0.0f, tiles::fixed_to_float(pb[q] - pa[q]) * pi.inv_sum_t);
                    const float dchi = pi.w_uni * depth * fmaf(depth, pi.sum_t2, -2.0f * c1);
                    const unsigned long long key = ((unsigned long long)float_order_key(dchi) << 32) |
                                                   ((unsigned long long)pi.j << 24) | (unsigned long long)m;
                    best = key < best ? key : best;
                }
            }
        }
        if (pi.item_last) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
                best = w < best ? w : best;
            }
            if ((l & 31) == 0 && best != ~0ull && valid) atomicMin(&ds.outs[pi.lc].best[pi.p], best);
            best = ~0ull;
        }
    }
}

__global__ void __launch_bounds__(tc::kThreads, 1)
k_window_tc(DevSet ds, const __grid_constant__ SlotMap smv, const SlotMap* smq, DevChunk dk, const void* maps,
            int jspan, unsigned int* counter, int test_wait)
{
    const SlotMap& sm = smq ? *smq : smv;
    using namespace tc;
    extern __shared__ unsigned char tc_smem_raw[];
    __shared__ uint32_t s_tmem;
    TcSmem& S = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        S.tinfo[0].end = 0;
        S.tinfo[1].end = 0;
        auto init = [](unsigned long long* b, int n, int count) {
            for (int i = 0; i < n; ++i)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b + i)), "r"(count) : "memory");
        };
        init(S.full, kStages, 1);
        init(S.a_free, kStages, 1);
        init(S.b_free, kStages, kMmaWarps);
        init(S.t_full, kTStages, 1);
        init(S.t_free, kTStages, kMmaWarps);
        init(S.d_full, 2, kMmaWarps);
        init(S.d_free, 2, 1);
        init(S.i_full, 2, 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    if (warp < kConvWarps) {
        tc_convert(ds, S, tmem);
    } else if (warp == kConvWarps) {
        if (lane == 0) tc_producer(ds, sm, dk, maps, jspan, counter, S, test_wait);
    } else if (warp < kConvWarps + 1 + kMmaWarps) {
        if (lane == 0) tc_mma(S, tmem, ds.curves[0].check, warp - kConvWarps - 1);
    } else {
        tc_epilogue(ds, sm, dk, S, tmem, warp % 4);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---------------------------------------------------------------------------
// per-period result: chi2(P), depth, T0 of the minimum
// ---------------------------------------------------------------------------

__global__ void k_period_finalize(DevSet ds, const __grid_constant__ SlotMap smv, const SlotMap* smq, DevChunk dk)
{
    const SlotMap& sm = smq ? *smq : smv;
    const int slot_id = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot_id >= sm.slots) return;
    int lc, p;
    if (!resolve_slot(ds, sm, slot_id, lc, p)) return;
    const DevPlan& dp = ds.plans[lc];
    const DevCurve dc = ds.curves[lc];
    const DevPeriod dq = ds.outs[lc];
    const unsigned long long b = dq.best[p];
    const float dchi = float_from_order_key((unsigned int)(b >> 32));
    const int j = (int)((b >> 24) & 0xffull);
    const int64_t m = (int64_t)(b & 0xffffffull);
    if (!in_range(dc.check, 13, j, dp.nd)) return;
    const int d = dp.dpts[j], st = dp.stride[j];
    const int64_t s = m * st;
    const int64_t n = dp.n;
    if (!in_range(dc.check, 14, s + d, dk.pad_stride)) return;
    const long long* pf = dk.pf + (int64_t)slot_id * dk.pad_stride;
    const double sum_r = (double)(pf[s + d] - pf[s]) * (1.0 / kRScale);
    const double depth = fmax(0.0, sum_r / dp.sum_t[j]);
    const int64_t c = (s + d / 2) % n;
    const int32_t idx = dk.sidx[(int64_t)slot_id * dk.fold_stride + c];
    if (!in_range(dc.check, 15, idx, n)) return;
    const long long rho = lattice_rho(dc.d_lat[idx], dc.d_f[idx], dp.p_lat[p], dp.inv_p[p]);
    dq.chi2[p] = dc.scal[1] + (double)dchi;
    dq.dur[p] = j;
    dq.t0i[p] = (int32_t)s;
    dq.depth[p] = depth;
    dq.t0[p] = dc.scal[0] + ldexp((double)rho, -dp.time_exponent);
}

// ---------------------------------------------------------------------------
// device work queue of the batched search: waves cut on the device
// ---------------------------------------------------------------------------
//
// The periods of a batch are a list of (curve, first, count) runs; a wave
// takes the next at most `wave_slots` periods of the list in at most kMaxSeg
// segments.  k_wave_next cuts the next wave from the queue's cursor into
// device memory, clears the wave's window-kernel counters and, when the
// queue is empty after it, sets the condition of the enclosing graph loop to
// zero, so that one loop node replays the wave kernels until the queue is
// drained: the graph has the same nodes for any number of curves.

struct QueueRun {
    int32_t lc, first, count, tiles_pp;
};

struct WaveQueue {
    const QueueRun* runs;
    int32_t nruns;
    int32_t wave_slots;
    int32_t from_list;
    int32_t* cursor;              // [0] run, [1] periods of that run taken, [2] waves cut
    SlotMap* wave;                // the wave being searched
    unsigned int* counters;       // the window kernels' item counters (2)
    cudaGraphConditionalHandle cond;
};

__global__ void k_wave_next(WaveQueue q)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int r = q.cursor[0], off = q.cursor[1];
    SlotMap& sm = *q.wave;
    int nseg = 0, slots = 0, items = 0;
    while (slots < q.wave_slots && nseg < kMaxSeg && r < q.nruns) {
        const QueueRun u = q.runs[r];
        const int take = min(u.count - off, q.wave_slots - slots);
        sm.seg[nseg++] = WaveSeg{u.lc, u.first + off, slots, items};
        slots += take;
        items += take * u.tiles_pp;
        off += take;
        if (off >= u.count) {
            ++r;
            off = 0;
        }
    }
    sm.nseg = nseg;
    sm.slots = slots;
    sm.items = items;
    sm.from_list = q.from_list;
    q.cursor[0] = r;
    q.cursor[1] = off;
    q.cursor[2] += 1;
    q.counters[0] = 0;
    q.counters[1] = 0;
    cudaGraphSetConditional(q.cond, r < q.nruns ? 1u : 0u);
}

// Rewinds the cursors of `n` queues (3 words each).
__global__ void k_queue_reset(int32_t* cursors, int n)
{
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) cursors[i] = 0;
}

// ---------------------------------------------------------------------------
// SR, SDE_raw (one block), median detrending, argmax
// ---------------------------------------------------------------------------

__device__ double block_sum_fixed(double v, double* sh)
{
    // fixed-order tree over the block: deterministic for a given block size
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ void sr_stats_body(int np, const DevPeriod& dq, double* sh)
{
    double mn = INFINITY;
    for (int i = threadIdx.x; i < np; i += blockDim.x) mn = fmin(mn, dq.chi2[i]);
    sh[threadIdx.x] = mn;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    const double cmin = sh[0];
    __syncthreads();
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const double c = dq.chi2[i];
        const double sr = c > 0.0 ? cmin / c : 1.0;
        dq.sr[i] = sr;
        acc += sr;
    }
    const double mean = block_sum_fixed(acc, sh) / (double)np;
    acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const double dd = dq.sr[i] - mean;
        acc += dd * dd;
    }
    const double var = block_sum_fixed(acc, sh) / (double)np;
    const double sd = sqrt(var);
    for (int i = threadIdx.x; i < np; i += blockDim.x)
        dq.sde_raw[i] = sd > 1e-12 ? (dq.sr[i] - mean) / sd : 0.0;
    if (threadIdx.x == 0) {
        dq.stats[0] = cmin;
        dq.stats[1] = mean;
        dq.stats[2] = sd;
    }
}

__global__ void __launch_bounds__(1024) k_sr_stats(int np, DevPeriod dq)
{
    __shared__ double sh[1024];
    sr_stats_body(np, dq, sh);
}

// One block per curve lc0 + blockIdx.x.
__global__ void __launch_bounds__(1024) k_sr_stats_set(DevSet ds, int lc0)
{
    __shared__ double sh[1024];
    const int lc = lc0 + blockIdx.x;
    const DevPeriod dq = ds.outs[lc];
    sr_stats_body(ds.plans[lc].np, dq, sh);
}

// Lower running median of sde_raw over [i-h, i+h] (truncated), one block per
// `outs` consecutive outputs: the block sorts the union of its windows once
// (bitonic, by value then position) and every thread walks the sorted list.
__device__ void median_body(int np, int h, int outs, int blk, const DevPeriod& dq, unsigned char* smem)
{
    double* val = reinterpret_cast<double*>(smem);
    int* pos = reinterpret_cast<int*>(val + kMedianCap);
    const int i0 = blk * outs;
    const int lo = max(0, i0 - h);
    const int hi = min(np - 1, i0 + outs - 1 + h);
    const int len = hi - lo + 1;
    if (len > kMedianCap) {   // block-uniform: the whole block leaves
        if (threadIdx.x == 0) record_check(dq.check, 16, len, kMedianCap);
        return;
    }
    int cap = 1;
    while (cap < len) cap <<= 1;
    for (int k = threadIdx.x; k < cap; k += blockDim.x) {
        if (k < len) {
            val[k] = dq.sde_raw[lo + k];
            pos[k] = lo + k;
        } else {
            val[k] = INFINITY;
            pos[k] = 0x7fffffff;
        }
    }
    __syncthreads();
    for (int size = 2; size <= cap; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = threadIdx.x; k < cap; k += blockDim.x) {
                const int l = k ^ stride;
                if (l > k) {
                    const bool up = (k & size) == 0;
                    const bool gt = val[k] > val[l] || (val[k] == val[l] && pos[k] > pos[l]);
                    if (gt == up) {
                        const double tv = val[k];
                        val[k] = val[l];
                        val[l] = tv;
                        const int tp = pos[k];
                        pos[k] = pos[l];
                        pos[l] = tp;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < outs; t += blockDim.x) {
        const int i = i0 + t;
        if (i >= np) break;
        const int wlo = max(0, i - h), whi = min(np - 1, i + h);
        const int want = (whi - wlo) / 2;  // lower median: index (cnt-1)/2
        int seen = 0;
        double med = 0.0;
        for (int k = 0; k < len; ++k) {
            const int q = pos[k];
            if (q >= wlo && q <= whi) {
                if (seen == want) {
                    med = val[k];
                    break;
                }
                ++seen;
            }
        }
        dq.sde[i] = dq.sde_raw[i] - med;
    }
}

__global__ void __launch_bounds__(kMedianThreads) k_median_sde(int np, int h, int outs, DevPeriod dq)
{
    extern __shared__ unsigned char smem[];
    median_body(np, h, outs, blockIdx.x, dq, smem);
}

// Outputs per block of the running median for half width h.
__host__ __device__ __forceinline__ int median_outs(int h)
{
    const int o = kMedianCap - 2 * h;
    return (o < 1024 ? o : 1024) & ~31;
}

// Row blockIdx.y: curve lc0 + blockIdx.y; its blocks are the first
// ceil(np / median_outs(h)) of the row.
__global__ void __launch_bounds__(kMedianThreads) k_median_sde_set(DevSet ds, int lc0)
{
    extern __shared__ unsigned char smem[];
    const int lc = lc0 + blockIdx.y;
    const int np = ds.plans[lc].np, h = ds.plans[lc].median_half;
    const int outs = median_outs(h);
    if (outs < 32 || (int)blockIdx.x * outs >= np) return;
    const DevPeriod dq = ds.outs[lc];
    median_body(np, h, outs, blockIdx.x, dq, smem);
}

// Curve lc0 + blockIdx.x: clears its refined flags, then takes the
// refine_k periods with the largest SDE (ties: lower index first) into its
// plist in ascending period order and flags them.  A radix select over the
// order-preserving 64-bit keys of SDE (eight passes of 8-bit histograms)
// finds the key T of the k-th largest; every key above T is taken, and of
// the keys equal to T the lowest indices (a block-wide scan in index order).
__global__ void __launch_bounds__(1024) k_topk(DevSet ds, int lc0)
{
    __shared__ unsigned int hist[256];
    __shared__ long long warp_sums[33];
    __shared__ unsigned long long s_prefix, s_mask;
    __shared__ long long s_need;
    const int lc = lc0 + blockIdx.x;
    const int np = ds.plans[lc].np, k = ds.plans[lc].refine_k;
    const DevPeriod dq = ds.outs[lc];
    for (int i = threadIdx.x; i < np; i += blockDim.x) dq.refined[i] = 0;
    if (k <= 0) return;
    if (threadIdx.x == 0) {
        s_prefix = 0ull;
        s_mask = 0ull;
        s_need = k;
    }
    __syncthreads();
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
        __syncthreads();
        const unsigned long long prefix = s_prefix, mask = s_mask;
        for (int i = threadIdx.x; i < np; i += blockDim.x) {
            const unsigned long long u = double_order_key(dq.sde[i]);
            if ((u & mask) == prefix) atomicAdd(&hist[(u >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long above = 0;
            int b = 255;
            for (; b > 0; --b) {
                if (above + hist[b] >= s_need) break;
                above += hist[b];
            }
            s_need -= above;
            s_prefix = prefix | ((unsigned long long)b << shift);
            s_mask = mask | (255ull << shift);
        }
        __syncthreads();
    }
    const unsigned long long thr = s_prefix;
    const long long need_eq = s_need;   // keys equal to thr to take, lowest indices first
    // selection in index order: contiguous chunk per thread, two block scans
    long long* total = warp_sums + 32;
    const int chunk = (np + (int)blockDim.x - 1) / (int)blockDim.x;
    const int i0 = threadIdx.x * chunk, i1 = min(np, i0 + chunk);
    long long gt = 0, eq = 0;
    for (int i = i0; i < i1; ++i) {
        const unsigned long long u = double_order_key(dq.sde[i]);
        gt += u > thr ? 1 : 0;
        eq += u == thr ? 1 : 0;
    }
    const long long gt_before = block_exclusive_scan(gt, warp_sums, total);
    const long long eq_before = block_exclusive_scan(eq, warp_sums, total);
    long long pos = gt_before + min(eq_before, need_eq);
    long long eq_seen = eq_before;
    for (int i = i0; i < i1; ++i) {
        const unsigned long long u = double_order_key(dq.sde[i]);
        bool take = u > thr;
        if (u == thr) {
            take = eq_seen < need_eq;
            ++eq_seen;
        }
        if (!take) continue;
        if (in_range(dq.check, 21, pos, k)) {
            dq.plist[pos] = i;
            dq.refined[i] = 1;
        }
        ++pos;
    }
}

// Curve lc0 + blockIdx.x: the candidate of largest SDE into its result
// (and results[lc], checks[4 lc ..] when given).
__global__ void __launch_bounds__(1024) k_best(DevSet ds, int lc0, gtls_result* results, unsigned int* checks)
{
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    const int lc = lc0 + blockIdx.x;
    const DevPlan& dp = ds.plans[lc];
    const DevCurve dc = ds.curves[lc];
    const DevPeriod dq = ds.outs[lc];
    double v = -INFINITY;
    int idx = 0x7fffffff;
    for (int i = threadIdx.x; i < dp.np; i += blockDim.x) {
        const double s = dq.sde[i];
        if (s > v) {
            v = s;
            idx = i;
        }
    }
    bv[threadIdx.x] = v;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double ov = bv[threadIdx.x + s];
            const int oi = bi[threadIdx.x + s];
            if (ov > bv[threadIdx.x] || (ov == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = ov;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int b = bi[0];
        gtls_result r{};
        const int j = in_range(dc.check, 17, b, dp.np) ? dq.dur[b] : -1;
        if (j < 0 || !in_range(dc.check, 18, j, dp.nd)) {
            if (checks)
                for (int u = 0; u < 4; ++u) checks[4 * lc + u] = dc.check[u];
            return;
        }
        r.period = dp.periods[b];
        r.duration_days = dp.q[j] * dp.periods[b];
        r.t0 = dq.t0[b];
        r.depth = dq.depth[b];
        r.sde = dq.sde[b];
        r.chi2 = dq.chi2[b];
        r.chi2_min = dq.stats[0];
        r.chi2_0 = dc.scal[1];
        r.period_idx = b;
        r.dur_idx = j;
        r.dur_points = dp.dpts[j];
        r.t0_idx = dq.t0i[b];
        r.uniform_dy = dc.scal[2] > 0.0 ? 1 : 0;
        r.refined = dp.refine_k;
        r.snr = sqrt(fmax(0.0, r.chi2_0 - r.chi2));
        *dq.result = r;
        if (results) results[lc] = r;
        if (checks)
            for (int u = 0; u < 4; ++u) checks[4 * lc + u] = dc.check[u];
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <class T>
gtls_status dev_alloc(gtls_plan* pl, T** ptr, size_t count)
{
    *ptr = nullptr;
    if (count == 0) count = 1;
    if (pl->n_allocs >= (int)(sizeof(pl->allocs) / sizeof(pl->allocs[0])))
        return fail(GTLS_ERR_INTERNAL, "too many plan allocations");
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(GTLS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    pl->allocs[pl->n_allocs++] = p;
    pl->device_bytes += (int64_t)(count * sizeof(T));
    *ptr = static_cast<T*>(p);
    return GTLS_OK;
}

template <class T>
gtls_status upload(gtls_plan* pl, T** ptr, const std::vector<T>& v)
{
    gtls_status s = dev_alloc(pl, ptr, v.size());
    if (s != GTLS_OK) return s;
    if (!v.empty()) GTLS_CUDA(cudaMemcpy(*ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return GTLS_OK;
}

#define GTLS_TRY(x)                     \
    do {                                \
        gtls_status s_ = (x);           \
        if (s_ != GTLS_OK) return s_;   \
    } while (0)

// Window-kernel variant and phase lanes for a duration of d points, T0 step
// st and about `nwin` windows per tile: the candidates keep W st = nc * odd
// (mod 32) (bank conflict free); the one with the lowest predicted time per
// window-point evaluation wins.  Predicted time = intrinsic cost of the
// variant / (useful fraction of lane slots x filled fraction of the last
// task x share of a window's time spent on its points).  The intrinsic
// costs are warp cycles per 1000 issued FMA lanes, fitted to clock64
// timings of every task of a Kepler-like search: 15-window column pairs
// 220, 16-window 255, 12-window and window pairs 320, rotated 16-window
// pairs 280 (swept on the bench's window stage); the (C1, S) pairs
// spend two lanes per evaluation and their nc = st lanes per block a
// recursive halving that grows with st (280 + 13 st per 1000 evaluations)
// but finish a window without prefix-sum reads.  A window's epilogue
// (reduction, two 8-byte prefix reads, the packed minimum) costs about as
// much as 80 evaluations (about 20 for the (C1, S) pairs).
void pick_config_host(int d, int st, int nwin, int32_t& variant, int32_t& nc_out)
{
    // column pairs with rotated rounds: their two-way bank conflicts priced
    // against the conflict-free 16-window variant (GTLS_COL16R_BASE
    // overrides it; 0 disables the variant)
    double kCol16RBase = 280.0;
    if (const char* e = std::getenv("GTLS_COL16R_BASE")) kCol16RBase = std::atof(e);
    int v = 0;
    while (v < 5 && ((st >> v) & 1) == 0) ++v;
    double best = 1e300;
    variant = tiles::kWin16;
    nc_out = 32;
    auto consider = [&](int var, int nc) {
        if (nc > 32 || nc < 1) return;
        const int w = tiles::variant_w(var);
        const int cols = tiles::variant_colpair(var) ? 2 * nc : nc;
        const int rounds = (st + cols - 1) / cols;
        const double util = (double)st / (double)(cols * rounds);
        const int per = 32 * w / nc;
        const int tasks = (nwin + per - 1) / per;
        const double fill = (double)nwin / (double)(tasks * per);
        double base, epi;
        switch (var) {
        case tiles::kCol15: base = 220.0; epi = 80.0; break;
        case tiles::kCol16: base = 255.0; epi = 80.0; break;
        case tiles::kCol16R: base = kCol16RBase; epi = 80.0; break;
        case tiles::kCol12: base = 320.0; epi = 80.0; break;
        case tiles::kWin16: base = 320.0; epi = 80.0; break;
        default: base = 280.0 + 13.0 * st; epi = 20.0; break;   // (C1, S) pairs: two lanes per evaluation
        }
        const double cost = base / (util * fill * ((double)d / (d + epi)));
        if (cost < best - 1e-9) {
            best = cost;
            variant = var;
            nc_out = nc;
        }
    };
    // variants built into the kernel: scalar15 (nc = 2^v), winpair16 (nc = 32),
    // colpair 16 / 15 / 12 (W st = nc * odd)
    consider(tiles::kWin16, 32);
    consider(tiles::kCol16, 32);
    if (v <= 4) {
        consider(tiles::kScalar15, 1 << v);
        consider(tiles::kCol15, 1 << v);
    }
    if (v + 2 <= 5) consider(tiles::kCol12, 1 << (v + 2));
    if (v + 4 <= 5) consider(tiles::kCol16, 1 << (v + 4));
    // (measured per T0-step class on the Kepler-like and 3000-day searches:
    // 260-290 cycles per 1000 evaluations at steps 32-127, slower than the
    // other variants below and above that range)
    if (v >= 1 && kCol16RBase > 0.0 && st >= 32 && st < 128)
        for (int nc = 2; nc <= 16; nc <<= 1) consider(tiles::kCol16R, nc);
}

int fold_smem_bytes(int bucket_log2)
{
    // global path: histogram and starts, scan scratch, staged keys and folded rfx
    const int global_path = (2 << bucket_log2) * (int)sizeof(uint32_t) + 33 * (int)sizeof(long long) +
                            kFoldSegKeys * (int)(sizeof(unsigned long long) + sizeof(long long));
    // staged path: scan scratch, rfx in final order, keys in fine-bucket
    // order, fine-bucket counts and ends, super-bucket counts and starts,
    // inverse permutation, fine buckets of the sorted keys, overflow flag
    const int staged = 33 * (int)sizeof(long long) + 2 * kFoldSegKeys * (int)sizeof(unsigned long long) +
                       (2 << kFoldFineLog2) * (int)sizeof(uint32_t) +
                       2 * (1 << kFoldMaxSbLog2) * (int)sizeof(uint32_t) +
                       2 * kFoldSegKeys * (int)sizeof(uint16_t) + (int)sizeof(int);
    return std::max(global_path, staged);
}

int topk_smem_bytes(int, int)
{
    return 0;   // the selection uses static shared memory only
}

constexpr int kMedianSmem = kMedianCap * (int)(sizeof(double) + sizeof(int));

// Every kernel with dynamic shared memory may use up to the device's opt-in
// limit (set once per device, so that plans of any size coexist).
gtls_status configure_kernels(int dev)
{
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return GTLS_OK;
    int optin = 0;
    GTLS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    auto allow = [&](const void* fn) -> gtls_status {
        cudaFuncAttributes a{};
        GTLS_CUDA(cudaFuncGetAttributes(&a, fn));
        GTLS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       optin - (int)a.sharedSizeBytes));
        return GTLS_OK;
    };
    GTLS_TRY(allow((const void*)k_fold_sort));
    GTLS_TRY(allow((const void*)k_window_tiles));
    GTLS_TRY(allow((const void*)k_median_sde));
    GTLS_TRY(allow((const void*)k_median_sde_set));
    GTLS_TRY(allow((const void*)k_topk));
    GTLS_CUDA(cudaFuncSetAttribute((const void*)k_window_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   tc::kSmemRequest));
    done.push_back(dev);
    return GTLS_OK;
}

gtls_status create_device(gtls_plan* pl)
{
    const PlanHost& h = pl->host;
    GTLS_CUDA(cudaGetDevice(&pl->device));
    DevPlan& dp = pl->dp;
    dp.n = h.n;
    dp.np = (int32_t)h.periods.size();
    dp.nd = (int32_t)h.q.size();
    dp.time_exponent = h.time_exponent;
    dp.idx_bits = h.idx_bits;
    dp.bucket_log2 = h.bucket_log2;
    {
        // super-buckets of the staged fold: about kFoldFillKeys points each
        // on average (regions of kFoldSegKeys slots)
        const int64_t nsb = (h.n + kFoldFillKeys - 1) / kFoldFillKeys;
        dp.fold_nsb = (int32_t)std::max<int64_t>(1, std::min<int64_t>(nsb, 1 << kFoldMaxSbLog2));
    }
    dp.max_kept = h.max_kept;
    dp.median_half = h.median_window / 2;
    if (median_outs(dp.median_half) < 32)
        return fail(GTLS_ERR_INVALID_ARG, "median window too large for the device median");
    dp.refine_k = std::min<int>(h.prm.refine_periods, dp.np);
    pl->tc_test_wait = (h.prm.test_flags & 1) ? 1 : 0;
    GTLS_TRY(configure_kernels(pl->device));
    std::vector<float> inv_sum_t(dp.nd), sum_t2f(dp.nd);
    for (int j = 0; j < dp.nd; ++j) {
        inv_sum_t[j] = (float)(1.0 / h.sum_t[j]);
        sum_t2f[j] = (float)h.sum_t2[j];
    }
    GTLS_TRY(upload(pl, const_cast<double**>(&dp.periods), h.periods));
    GTLS_TRY(upload(pl, const_cast<int64_t**>(&dp.p_lat), h.p_lat));
    GTLS_TRY(upload(pl, const_cast<float**>(&dp.inv_p), h.inv_p));
    GTLS_TRY(upload(pl, const_cast<int32_t**>(&dp.bucket_shift), h.bucket_shift));
    GTLS_TRY(upload(pl, const_cast<uint32_t**>(&dp.bucket_mul), h.bucket_mul));
    GTLS_TRY(upload(pl, const_cast<int32_t**>(&dp.jlo), h.jlo));
    GTLS_TRY(upload(pl, const_cast<int32_t**>(&dp.jhi), h.jhi));
    GTLS_TRY(upload(pl, const_cast<int32_t**>(&dp.dmax_p), h.dmax_p));
    GTLS_TRY(upload(pl, const_cast<int32_t**>(&dp.dpts), h.dpts));
    GTLS_TRY(upload(pl, const_cast<int32_t**>(&dp.stride), h.stride));
    {
        // every template is followed by (kMaxRing + 2) st + 64 zeros: the
        // window kernels run ceil(D / st) rows for every phase column and
        // fetch template rows up to kMaxRing rows ahead without bounds tests
        std::vector<int64_t> off(dp.nd);
        int64_t pos = 0;
        for (int j = 0; j < dp.nd; ++j) {
            off[j] = pos;
            pos += h.dpts[j] + (tiles::kMaxRing + 2) * (int64_t)h.stride[j] + 64;
        }
        std::vector<float> tmpl_pad((size_t)pos, 0.0f);
        for (int j = 0; j < dp.nd; ++j)
            std::copy(h.tmpl.begin() + h.tmpl_off[j], h.tmpl.begin() + h.tmpl_off[j] + h.dpts[j],
                      tmpl_pad.begin() + off[j]);
        GTLS_TRY(upload(pl, const_cast<float**>(&dp.tmpl), tmpl_pad));
        GTLS_TRY(upload(pl, const_cast<int64_t**>(&dp.tmpl_off), off));
        dp.tmpl_total = pos;
        pl->tmpl_pad = std::move(tmpl_pad);
        pl->tmpl_pad_off = std::move(off);
    }
    GTLS_TRY(upload(pl, const_cast<float**>(&dp.inv_sum_t), inv_sum_t));
    GTLS_TRY(upload(pl, const_cast<float**>(&dp.sum_t2), sum_t2f));
    GTLS_TRY(upload(pl, const_cast<double**>(&dp.sum_t), h.sum_t));
    GTLS_TRY(upload(pl, const_cast<double**>(&dp.q), h.q));

    const int64_t n = h.n;
    DevCurve& dc = pl->dc;
    GTLS_TRY(dev_alloc(pl, &dc.d_lat, n));
    GTLS_TRY(dev_alloc(pl, &dc.d_f, n));
    GTLS_TRY(dev_alloc(pl, &dc.pv, n));
    GTLS_TRY(dev_alloc(pl, &dc.scal, 8));
    GTLS_TRY(dev_alloc(pl, &dc.tmin_key, 1));
    GTLS_TRY(dev_alloc(pl, &dc.flags, 1));
    GTLS_TRY(dev_alloc(pl, &dc.part, 1024));
    GTLS_TRY(dev_alloc(pl, &dc.check, 4));

    DevChunk& dk = pl->dk;
    dk.fold_stride = (n + 31) & ~int64_t(31);
    dk.key_stride = std::max<int64_t>(dk.fold_stride, (int64_t)kFoldSegKeys * dp.fold_nsb);
    dk.pad_stride = (n + h.dmax + kPadMargin + 31) & ~int64_t(31);
    const int64_t per_period = dk.key_stride * 8 + dk.fold_stride * 4 + dk.pad_stride * (4 + 4 + 4 + 8);
    // 8 GiB of chunk scratch (measured on the Kepler-like search: 1024,
    // 1520 and 3040 periods per chunk took 1013, 994 and 980 ms)
    const int64_t budget = int64_t(8) << 30;
    int64_t chunk = std::max<int64_t>(1, budget / per_period);
    chunk = std::min<int64_t>(chunk, 4096);
    {
        // whole waves of the fold (one CTA per period and SM): a multiple of
        // the SM count when at least one wave fits
        int dev = 0, sms = 0;
        GTLS_CUDA(cudaGetDevice(&dev));
        GTLS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (sms > 0 && chunk >= sms) chunk = chunk / sms * sms;
    }
    if (h.prm.periods_per_chunk > 0) chunk = h.prm.periods_per_chunk;
    chunk = std::min<int64_t>(chunk, dp.np);
    dk.chunk = (int32_t)chunk;   // allocated by the first single-curve search

    DevPeriod& dq = pl->dq;
    const int64_t np_ = dp.np;
    GTLS_TRY(dev_alloc(pl, &dq.best, np_));
    GTLS_TRY(dev_alloc(pl, &dq.chi2, np_));
    GTLS_TRY(dev_alloc(pl, &dq.dur, np_));
    GTLS_TRY(dev_alloc(pl, &dq.t0i, np_));
    GTLS_TRY(dev_alloc(pl, &dq.depth, np_));
    GTLS_TRY(dev_alloc(pl, &dq.t0, np_));
    GTLS_TRY(dev_alloc(pl, &dq.sr, np_));
    GTLS_TRY(dev_alloc(pl, &dq.sde_raw, np_));
    GTLS_TRY(dev_alloc(pl, &dq.sde, np_));
    GTLS_TRY(dev_alloc(pl, &dq.stats, 4));
    GTLS_TRY(dev_alloc(pl, &dq.result, 1));
    dq.check = dc.check;

    // tiled window search: staged buffer, tile length, tiles per period
    {
        int dev = 0;
        GTLS_CUDA(cudaGetDevice(&dev));
        GTLS_CUDA(cudaDeviceGetAttribute(&pl->n_sm, cudaDevAttrMultiProcessorCount, dev));
        int smem_optin = 0;
        GTLS_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        const int static_bytes = 8192;  // duration table and reduction scratch, rounded up
        // floats of folded curve staged per tile; the rest of the SM's
        // unified L1/shared memory caches the template tables
        int want = 32768;   // measured best on the Kepler-like curve (vs 49152, 40960, 24576, 16384)
        if (const char* e = std::getenv("GTLS_TILE_FLOATS")) want = std::max(4096, std::atoi(e));
        int buf = std::min(want, (smem_optin - static_bytes) / 4) & ~63;
        {
            // the largest T0 step must fit one register block of rows
            int need = 0;
            for (int j = 0; j < dp.nd; ++j) {
                const int jrows = (h.dpts[j] + h.stride[j] - 1) / h.stride[j];
                need = std::max(need, (16 + jrows + 2) * h.stride[j] + 32);
            }
            const int need_len = (int)std::min<int64_t>(h.n, 4096);
            int st_mx = 1;
            for (int v : h.stride) st_mx = std::max(st_mx, v);
            need = std::max<int64_t>(need, need_len + h.dmax + 3 * (int64_t)st_mx + 96 + 63);
            buf = std::max(buf, std::min((int)((need + 63) & ~63), (smem_optin - static_bytes) / 4 & ~63));
        }
        // durations whose register block of rows and a 64-window tile fit the
        // staged buffer take the tiled kernel; longer ones are marked for the
        // one-thread-per-window kernel
        int st_max = 1, dmax_fit = 0;
        std::vector<uint8_t> fit(dp.nd, 0);
        for (int j = 0; j < dp.nd; ++j) {
            const int st = h.stride[j], d = h.dpts[j];
            const int jrows = (d + st - 1) / st;
            fit[j] = buf > 0 && (int64_t)(16 + jrows + 2) * st + 32 <= buf &&
                     (int64_t)d + 3 * st + 96 + 64 <= buf;
            if (!fit[j]) continue;
            st_max = std::max(st_max, st);
            dmax_fit = std::max(dmax_fit, d);
        }
        const int64_t len = ((int64_t)buf - dmax_fit - 3 * (int64_t)st_max - 96) & ~int64_t(63);
        pl->tile_ok = dmax_fit > 0 && len >= 64;
        std::vector<int32_t> var(dp.nd, tiles::kWin16), ncs(dp.nd, 32);
        std::vector<int64_t> off2(dp.nd, 0);
        std::vector<float2> t2;
        if (pl->tile_ok) {
            pl->tile_buf = buf;
            pl->tile_len = (int)len;
            pl->tile_count = (int)((n + len - 1) / len);
            int64_t pos2 = 0;
            for (int j = 0; j < dp.nd; ++j) {
                const int st = h.stride[j];
                const int64_t m_total = (n + st - 1) / st;
                const int nwin = (int)std::min<int64_t>(m_total, (len + st - 1) / st);
                pick_config_host(h.dpts[j], st, nwin, var[j], ncs[j]);
                if (!fit[j]) {
                    var[j] = tiles::kWindowOnly;
                    ncs[j] = 32;
                    pl->has_window_only = true;
                }
                off2[j] = pos2;
                if (tiles::variant_colpair(var[j]) || var[j] == tiles::kScalar15)
                    pos2 += h.dpts[j] + (tiles::kMaxRing + 2) * (int64_t)st + 64;
            }
            t2.assign((size_t)std::max<int64_t>(pos2, 1), make_float2(0.0f, 0.0f));
            for (int j = 0; j < dp.nd; ++j) {
                if (var[j] == tiles::kScalar15) {
                    // (s_k, 1): one FFMA2 gives C1 and the window sum S
                    const int st = h.stride[j], d = h.dpts[j];
                    const float* tj = pl->tmpl_pad.data() + pl->tmpl_pad_off[j];
                    const int64_t len2 = d + (tiles::kMaxRing + 2) * (int64_t)st + 64;
                    for (int64_t k = 0; k < len2; ++k)
                        t2[(size_t)(off2[j] + k)] = k < d ? make_float2(tj[k], 1.0f) : make_float2(0.0f, 0.0f);
                    continue;
                }
                if (!tiles::variant_colpair(var[j])) continue;
                const int st = h.stride[j], d = h.dpts[j], nc = ncs[j];
                const float* tj = pl->tmpl_pad.data() + pl->tmpl_pad_off[j];
                const int64_t len2 = d + (tiles::kMaxRing + 2) * (int64_t)st + 64;
                for (int64_t k = 0; k < len2; ++k) {
                    const int rho = (int)(k % st);
                    const float x = k < d ? tj[k] : 0.0f;
                    const float y = (rho + nc < st && k + nc < d) ? tj[k + nc] : 0.0f;
                    t2[(size_t)(off2[j] + k)] = make_float2(x, y);
                }
            }
        }
        // uniform-weight durations whose T0 step is at least the tensor-core
        // threshold, whose rows (sigma = g st points, g = 4 / gcd(st, 4)) are
        // at most tc::kMaxSigma long and whose window spans I g <= 32 template
        // rows go to the tensor-core kernel; its table holds, per duration and
        // K chunk of 32 columns, B[i g + q][c] = s_{i sigma + c - q st} (zero
        // outside the template and past sigma), split into TF32 halves (round
        // to nearest) in the canonical K-major core-matrix layout: element
        // (row, c) at float (row / 8) 256 + (c / 4) 32 + (row % 8) 4 + c % 4
        std::vector<int64_t> tc_off(dp.nd, 0);
        std::vector<float> tc_tab;
        {
            int tc_min = tc::kMinStDefault;
            if (const char* e = std::getenv("GTLS_TC_MIN_ST")) tc_min = std::max(2, std::atoi(e));
            pl->has_tensor = false;
            pl->has_window_only = false;
            auto tf32_rn = [](float x) {
                uint32_t b;
                std::memcpy(&b, &x, 4);
                b = (b + 0x1000u) & 0xffffe000u;
                float y;
                std::memcpy(&y, &b, 4);
                return y;
            };
            for (int j = 0; j < dp.nd && pl->tile_ok; ++j) {
                const int st = h.stride[j], d = h.dpts[j];
                const int g = tc_windows_per_row(st), sigma = g * st;
                const int nblk = sigma <= tc::kMaxSigma ? tc_row_blocks(d, st, g) : tc::kN + 1;
                if (st >= tc_min && sigma <= tc::kMaxSigma && nblk * g <= tc::kN && d <= h.n) {
                    var[j] = tiles::kTensor;
                    ncs[j] = 32;
                    const int ksteps = (sigma + 7) / 8, nch = (ksteps + 3) / 4;
                    tc_off[j] = (int64_t)tc_tab.size();
                    tc_tab.resize(tc_tab.size() + (size_t)nch * 2 * tc::kN * tc::kChunk, 0.0f);
                    float* tb = tc_tab.data() + tc_off[j];
                    const float* tj = h.tmpl.data() + h.tmpl_off[j];
                    for (int kc = 0; kc < nch; ++kc)
                        for (int i = 0; i < nblk; ++i)
                            for (int q = 0; q < g; ++q)
                                for (int c = 0; c < tc::kChunk; ++c) {
                                    const int row = i * g + q, col = kc * tc::kChunk + c;
                                    const int64_t k = (int64_t)i * sigma + col - (int64_t)q * st;
                                    const float v = (col < sigma && k >= 0 && k < d) ? tj[k] : 0.0f;
                                    const float hi = tf32_rn(v);
                                    const float lo = tf32_rn(v - hi);
                                    const size_t e = (size_t)(row / 8) * 256 + (size_t)(c / 4) * 32 + (row % 8) * 4 +
                                                     c % 4;
                                    tb[(size_t)kc * 2 * tc::kN * tc::kChunk + e] = hi;
                                    tb[(size_t)kc * 2 * tc::kN * tc::kChunk + tc::kN * tc::kChunk + e] = lo;
                                }
                    pl->has_tensor = true;
                }
                if (var[j] == tiles::kWindowOnly) pl->has_window_only = true;
            }
            int span = 1;
            for (int p = 0; p < dp.np; ++p) span = std::max(span, h.jhi[p] - h.jlo[p] + 1);
            pl->tc_jspan = span;
            if (tc_tab.empty()) tc_tab.assign(4, 0.0f);
        }
        GTLS_TRY(upload(pl, const_cast<int64_t**>(&dp.tc_off), tc_off));
        GTLS_TRY(upload(pl, const_cast<float**>(&dp.tc_tab), tc_tab));
        GTLS_TRY(upload(pl, const_cast<int32_t**>(&dp.cfg_variant), var));
        pl->variant_host = var;
        GTLS_TRY(upload(pl, const_cast<int32_t**>(&dp.cfg_nc), ncs));
        GTLS_TRY(upload(pl, const_cast<int64_t**>(&dp.tmpl2_off), off2));
        if (t2.empty()) t2.assign(1, make_float2(0.0f, 0.0f));
        GTLS_TRY(upload(pl, const_cast<float2**>(&dp.tmpl2), t2));

        // per-point weights: (s_k, s_k^2) pair tables (zero padded like the
        // templates), lanes per window block, and the tile shape in
        // (w r, w) pairs
        {
            std::vector<int64_t> offw(dp.nd);
            std::vector<int32_t> ncw(dp.nd, 1);
            int64_t posw = 0;
            for (int j = 0; j < dp.nd; ++j) {
                offw[j] = posw;
                posw += h.dpts[j] + (tiles::kMaxRing + 2) * (int64_t)h.stride[j] + 64;
            }
            std::vector<float2> tw((size_t)std::max<int64_t>(posw, 1), make_float2(0.0f, 0.0f));
            for (int j = 0; j < dp.nd; ++j) {
                const float* tj = pl->tmpl_pad.data() + pl->tmpl_pad_off[j];
                for (int k = 0; k < h.dpts[j]; ++k) tw[(size_t)(offw[j] + k)] = make_float2(tj[k], tj[k] * tj[k]);
            }
            GTLS_TRY(upload(pl, const_cast<float2**>(&dp.tmplw), tw));
            GTLS_TRY(upload(pl, const_cast<int64_t**>(&dp.tmplw_off), offw));
            const int bufw = std::min(kWeightedTilePairs, (smem_optin - static_bytes) / 8) & ~63;
            bool fits_w = bufw > 0;
            for (int j = 0; j < dp.nd; ++j) {
                const int jrows = (h.dpts[j] + h.stride[j] - 1) / h.stride[j];
                if ((int64_t)(16 + jrows + 2) * h.stride[j] + 32 > bufw) fits_w = false;
            }
            const int64_t len_w = ((int64_t)bufw - h.dmax - 3 * (int64_t)st_max - 96) & ~int64_t(63);
            pl->tile_w_ok = fits_w && len_w >= 64;
            if (pl->tile_w_ok) {
                pl->tile_buf_w = bufw;
                pl->tile_len_w = (int)len_w;
                pl->tile_count_w = (int)((n + len_w - 1) / len_w);
                // lanes per window block: 2^min(v, 4) for st = 2^v odd (distinct banks
                // across blocks), or 16 / 32 (one block per half-warp / warp: adjacent
                // columns); the largest column use x task fill wins
                for (int j = 0; j < dp.nd; ++j) {
                    const int st = h.stride[j];
                    int v = 0;
                    while (v < 4 && ((st >> v) & 1) == 0) ++v;
                    const int64_t m_total = (n + st - 1) / st;
                    const int nwin = (int)std::min<int64_t>(m_total, (len_w + st - 1) / st);
                    double best = -1.0;
                    for (int nc : {1 << v, 16, 32}) {
                        const int rounds = (st + nc - 1) / nc;
                        const double util = (double)st / (double)(nc * rounds);
                        const int per = 32 * tiles::variant_w(tiles::kWeighted15) / nc;
                        const int tasks = (nwin + per - 1) / per;
                        const double fill = (double)nwin / (double)(tasks * per);
                        if (util * fill > best + 1e-9) {
                            best = util * fill;
                            ncw[j] = nc;
                        }
                    }
                }
            }
            GTLS_TRY(upload(pl, const_cast<int32_t**>(&dp.cfg_nc_w), ncw));
        }

        // refinement stage: every duration with T0 step 1 through the (C1, S)
        // variant (one column per lane)
        pl->refine_k = dp.refine_k;
        GTLS_TRY(dev_alloc(pl, &pl->dq.refined, dp.np));
        if (pl->refine_k > 0) {
            pl->dp_ref = dp;
            std::vector<int32_t> ones(dp.nd, 1), var1(dp.nd, tiles::kScalar15);
            std::vector<int64_t> off1(dp.nd);
            int64_t pos1 = 0;
            for (int j = 0; j < dp.nd; ++j) {
                off1[j] = pos1;
                pos1 += h.dpts[j] + (tiles::kMaxRing + 2) + 64;
            }
            std::vector<float2> t21((size_t)pos1, make_float2(0.0f, 0.0f));
            for (int j = 0; j < dp.nd; ++j) {
                const float* tj = pl->tmpl_pad.data() + pl->tmpl_pad_off[j];
                for (int k = 0; k < h.dpts[j]; ++k) t21[(size_t)(off1[j] + k)] = make_float2(tj[k], 1.0f);
            }
            GTLS_TRY(upload(pl, const_cast<int32_t**>(&pl->dp_ref.stride), ones));
            GTLS_TRY(upload(pl, const_cast<int32_t**>(&pl->dp_ref.cfg_nc), ones));
            GTLS_TRY(upload(pl, const_cast<int64_t**>(&pl->dp_ref.tmpl2_off), off1));
            GTLS_TRY(upload(pl, const_cast<float2**>(&pl->dp_ref.tmpl2), t21));
            GTLS_TRY(dev_alloc(pl, &pl->dq.plist, pl->refine_k));
            if (pl->tile_ok) {
                // T0 step 1: durations whose rows or 64-window tile do not fit are
                // searched by the one-thread-per-window kernel
                int dmax1 = 0;
                for (int j = 0; j < dp.nd; ++j) {
                    const int d = h.dpts[j];
                    if ((int64_t)(16 + d + 2) + 32 <= pl->tile_buf && (int64_t)d + 3 + 96 + 64 <= pl->tile_buf)
                        dmax1 = std::max(dmax1, d);
                    else {
                        var1[j] = tiles::kWindowOnly;
                        pl->has_window_only_ref = true;
                    }
                }
                const int64_t len1 = ((int64_t)pl->tile_buf - dmax1 - 3 - 96) & ~int64_t(63);
                if (dmax1 == 0 || len1 < 64)
                    return fail(GTLS_ERR_INVALID_ARG, "durations too long for the refinement tiles");
                pl->tile_len_ref = (int)len1;
                pl->tile_count_ref = (int)((n + len1 - 1) / len1);
            }
            GTLS_TRY(upload(pl, const_cast<int32_t**>(&pl->dp_ref.cfg_variant), var1));
        }
        GTLS_TRY(dev_alloc(pl, &pl->tile_counter, 1));
        GTLS_TRY(dev_alloc(pl, &pl->tc_counter, 1));
    }

    // one-entry descriptor sets of this plan's own searches
    {
        DevPlan* d_plans = nullptr;
        DevCurve* d_curves = nullptr;
        DevPeriod* d_outs = nullptr;
        DevTiles* d_tiles = nullptr;
        GTLS_TRY(upload(pl, &d_plans, std::vector<DevPlan>{dp, pl->refine_k > 0 ? pl->dp_ref : dp}));
        GTLS_TRY(upload(pl, &d_curves, std::vector<DevCurve>{dc}));
        GTLS_TRY(upload(pl, &d_outs, std::vector<DevPeriod>{pl->dq}));
        GTLS_TRY(upload(pl, &d_tiles,
                        std::vector<DevTiles>{DevTiles{pl->tile_len, pl->tile_count, pl->tile_len_w, pl->tile_count_w},
                                              DevTiles{pl->tile_len_ref, pl->tile_count_ref, 0, 0}}));
        pl->set = DevSet{d_plans, d_curves, d_outs, d_tiles};
        pl->set_ref = DevSet{d_plans + 1, d_curves, d_outs, d_tiles + 1};
        GTLS_TRY(upload(pl, &pl->prep_off, std::vector<int64_t>{0, n}));
    }
    return GTLS_OK;
}

// TMA descriptors of the tensor-core window kernel over the folded curves of
// a chunk scratch: map k reads dk.rs as rows of sigma = 4 (k + 1) points,
// 3-D (column < sigma, row < pad_stride / sigma, slot < chunk), boxes of 32
// columns x 128 rows x 1 slot into 128-byte-swizzled shared memory; columns
// and rows outside read as zeros.  Written to `dev` (tc::kMaps x 128 bytes).
gtls_status make_tc_maps(const DevChunk& dk, void* dev)
{
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!encode) {
            void* fn = nullptr;
            cudaDriverEntryPointQueryResult q{};
            GTLS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
            if (!fn || q != cudaDriverEntryPointSuccess)
                return fail(GTLS_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        }
    }
    std::vector<CUtensorMap> maps(tc::kMaps);
    for (int k = 0; k < tc::kMaps; ++k) {
        const uint64_t sigma = 4ull * (uint64_t)(k + 1);
        const cuuint64_t dims[3] = {sigma, (cuuint64_t)dk.pad_stride / sigma, (cuuint64_t)dk.chunk};
        const cuuint64_t strides[2] = {sigma * 4ull, (cuuint64_t)dk.pad_stride * 4ull};
        const cuuint32_t box[3] = {(cuuint32_t)tc::kChunk, (cuuint32_t)tc::kRows, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        const CUresult r = encode(&maps[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, dk.rs, dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return fail(GTLS_ERR_CUDA, "cuTensorMapEncodeTiled failed for a row pitch of " + std::to_string(sigma) +
                                           " points (error " + std::to_string((int)r) + ")");
    }
    GTLS_CUDA(cudaMemcpy(dev, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    return GTLS_OK;
}

// The chunk scratch of a plan's own searches (batches bring their own).
gtls_status ensure_chunk(gtls_plan* pl)
{
    if (pl->chunk_ready) return GTLS_OK;
    DevChunk& dk = pl->dk;
    const int64_t chunk = dk.chunk;
    const int64_t bytes0 = pl->device_bytes;
    GTLS_TRY(dev_alloc(pl, &dk.keys, chunk * dk.key_stride));
    GTLS_TRY(dev_alloc(pl, &dk.sidx, chunk * dk.fold_stride));
    GTLS_TRY(dev_alloc(pl, &dk.rs, chunk * dk.pad_stride));
    GTLS_TRY(dev_alloc(pl, &dk.ws, chunk * dk.pad_stride));
    GTLS_TRY(dev_alloc(pl, &dk.wrs, chunk * dk.pad_stride));
    GTLS_TRY(dev_alloc(pl, &dk.pf, chunk * dk.pad_stride));
    if (pl->has_tensor) {
        unsigned char* maps = nullptr;
        GTLS_TRY(dev_alloc(pl, &maps, (size_t)tc::kMaps * sizeof(CUtensorMap)));
        GTLS_TRY(make_tc_maps(dk, maps));
        pl->tc_maps = maps;
    }
    pl->chunk_ready = true;
    pl->chunk_bytes = pl->device_bytes - bytes0;
    return GTLS_OK;
}

// Frees the chunk scratch.
gtls_status trim_chunk(gtls_plan* pl)
{
    if (!pl->chunk_ready) return GTLS_OK;
    GTLS_CUDA(cudaDeviceSynchronize());
    const void* mine[] = {pl->dk.keys, pl->dk.sidx, pl->dk.rs, pl->dk.ws, pl->dk.wrs, pl->dk.pf, pl->tc_maps};
    int kept = 0;
    for (int i = 0; i < pl->n_allocs; ++i) {
        bool chunk = false;
        for (const void* m : mine) chunk = chunk || (m && m == pl->allocs[i]);
        if (chunk) cudaFree(pl->allocs[i]);
        else pl->allocs[kept++] = pl->allocs[i];
    }
    for (int i = kept; i < pl->n_allocs; ++i) pl->allocs[i] = nullptr;
    pl->n_allocs = kept;
    pl->device_bytes -= pl->chunk_bytes;
    pl->chunk_bytes = 0;
    const int32_t chunk = pl->dk.chunk;
    pl->dk.keys = nullptr;
    pl->dk.sidx = nullptr;
    pl->dk.rs = pl->dk.ws = pl->dk.wrs = nullptr;
    pl->dk.pf = nullptr;
    pl->dk.chunk = chunk;
    pl->tc_maps = nullptr;
    pl->chunk_ready = false;
    return GTLS_OK;
}

enum Stage { kStagePrepare = 0, kStageFold, kStageWindow, kStageFinalize, kStageSrSde, kStageCount };

// Record the end of a stage interval on the search stream (profiling only).
gtls_status mark(gtls_plan* pl, cudaStream_t st, int stage, size_t& used)
{
    if (!pl->profiling) return GTLS_OK;
    if (used == pl->events.size()) {
        cudaEvent_t e;
        GTLS_CUDA(cudaEventCreate(&e));
        pl->events.push_back(e);
        pl->event_stage.push_back(stage);
    }
    pl->event_stage[used] = stage;
    GTLS_CUDA(cudaEventRecord(pl->events[used], st));
    ++used;
    return GTLS_OK;
}

gtls_status collect_profile(gtls_plan* pl, size_t used)
{
    double ms[kStageCount] = {0, 0, 0, 0, 0};
    for (size_t i = 1; i < used; ++i) {
        float dt = 0.0f;
        GTLS_CUDA(cudaEventElapsedTime(&dt, pl->events[i - 1], pl->events[i]));
        const int sg = pl->event_stage[i];
        if (sg >= 0 && sg < kStageCount) ms[sg] += dt;
    }
    pl->profile.ms_prepare = ms[kStagePrepare];
    pl->profile.ms_fold_sort = ms[kStageFold];
    pl->profile.ms_window_search = ms[kStageWindow];
    pl->profile.ms_finalize = ms[kStageFinalize];
    pl->profile.ms_sr_sde = ms[kStageSrSde];
    pl->profile.enabled = 1;
    return GTLS_OK;
}

// Launch context of one search: a plan's own (one curve) or a batch's.
struct Ctx {
    DevSet set{}, set_ref{};
    DevChunk dk{};
    int n_lc = 1;
    int fold_smem = 0;
    int tile_buf = 0;
    int tile_buf_w = 0;      // (w r, w) pairs per tile with per-point weights
    int n_sm = 0;
    int median_blocks = 1;   // widest row of the running-median grid
    int topk_smem = 0;
    cudaStream_t st = nullptr;
    const void* tc_maps = nullptr;   // tensor-core kernel: TMA maps of dk.rs (tc::kMaps rows pitches)
    int tc_jspan = 1;        // tensor-core kernel: work items per period slot
    int tc_test = 0;         // tensor-core kernel: run the timeout test
    int64_t launches = 0, window_launches = 0;
    gtls_plan* prof = nullptr;   // stage marks (single search with profiling on)
    size_t ev = 0;
};

gtls_status stage_mark(Ctx& c, int stage)
{
    return c.prof ? mark(c.prof, c.st, stage, c.ev) : GTLS_OK;
}

// One wave: fold + sort, every window, per-period results.  `counter` must
// be zero when the window kernel starts (reset here when reset_counter).
// With smq (a wave cut on the device, see k_wave_next) the kernels read the
// wave from device memory; sm.slots then only sizes the grids (the most
// slots a wave of the queue can hold).
gtls_status wave_pass(Ctx& c, bool ref, const SlotMap& sm, bool tiled, bool weighted, bool window_only,
                      unsigned int* counter, bool reset_counter, int64_t max_n, int max_kept, bool tensor = false,
                      unsigned int* tc_counter = nullptr, const SlotMap* smq = nullptr)
{
    const DevSet& ds = ref ? c.set_ref : c.set;
    k_fold_sort<<<sm.slots, kFoldThreads, c.fold_smem, c.st>>>(ds, sm, smq, c.dk);
    GTLS_CUDA(cudaGetLastError());
    GTLS_TRY(stage_mark(c, kStageFold));
    if (tiled) {
        if (reset_counter) GTLS_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned int), c.st));
        const int buf = weighted ? c.tile_buf_w : c.tile_buf;
        const int bytes = buf * (int)(weighted ? sizeof(float2) : sizeof(float));
        k_window_tiles<<<c.n_sm * tiles::kCtasPerSm, tiles::kThreads, bytes, c.st>>>(ds, sm, smq, c.dk, buf,
                                                                                   weighted ? 1 : 0, counter);
        if (tensor && !weighted && tc_counter) {
            // the durations marked kTensor (the tiled kernel gave them no tasks)
            GTLS_CUDA(cudaGetLastError());
            if (reset_counter) GTLS_CUDA(cudaMemsetAsync(tc_counter, 0, sizeof(unsigned int), c.st));
            if (!c.tc_maps) return fail(GTLS_ERR_INTERNAL, "tensor-core window kernel without tensor maps");
            k_window_tc<<<c.n_sm, tc::kThreads, tc::kSmemRequest, c.st>>>(ds, sm, smq, c.dk, c.tc_maps, c.tc_jspan,
                                                                        tc_counter, c.tc_test);
            c.launches += 1;
        }
    }
    if (!tiled || window_only) {
        // every duration, or (next to the tiled kernel) those marked kWindowOnly
        dim3 grid((unsigned)((max_n + kSearchThreads - 1) / kSearchThreads), (unsigned)max_kept,
                  (unsigned)sm.slots);
        k_window_search<<<grid, kSearchThreads, 0, c.st>>>(ds, sm, smq, c.dk, tiled ? 1 : 0);
        if (tiled) {
            GTLS_CUDA(cudaGetLastError());
            c.launches += 1;
        }
    }
    GTLS_CUDA(cudaGetLastError());
    GTLS_TRY(stage_mark(c, kStageWindow));
    k_period_finalize<<<(sm.slots + 127) / 128, 128, 0, c.st>>>(ds, sm, smq, c.dk);
    GTLS_CUDA(cudaGetLastError());
    GTLS_TRY(stage_mark(c, kStageFinalize));
    c.launches += 3;
    c.window_launches += 1;
    return GTLS_OK;
}

// SR, SDE_raw and the median-detrended SDE of every curve.
gtls_status sr_sde_pass(Ctx& c)
{
    k_sr_stats_set<<<c.n_lc, 1024, 0, c.st>>>(c.set, 0);
    GTLS_CUDA(cudaGetLastError());
    k_median_sde_set<<<dim3((unsigned)c.median_blocks, (unsigned)c.n_lc), kMedianThreads, kMedianSmem, c.st>>>(
        c.set, 0);
    GTLS_CUDA(cudaGetLastError());
    c.launches += 2;
    return stage_mark(c, kStageSrSde);
}

// Curve preparation: reset, min(t) and flags, derived arrays and block
// partials of chi2_0, then the per-curve reduction (flags to flags_out).
gtls_status prep_pass(Ctx& c, const double* t, const double* y, const double* dy, const int64_t* off_dev,
                      int64_t max_n, unsigned int* flags_out)
{
    k_curve_reset<<<c.n_lc, 32, 0, c.st>>>(c.set, 0);
    GTLS_CUDA(cudaGetLastError());
    const dim3 grid((unsigned)std::max(1, prep_blocks_for(max_n)), (unsigned)c.n_lc);
    k_curve_minmax<<<grid, 256, 0, c.st>>>(t, y, dy, off_dev, c.set, 0);
    GTLS_CUDA(cudaGetLastError());
    k_curve_prep<<<grid, 256, 0, c.st>>>(t, y, dy, off_dev, c.set, 0);
    GTLS_CUDA(cudaGetLastError());
    k_curve_reduce<<<(c.n_lc + 127) / 128, 128, 0, c.st>>>(dy, off_dev, c.set, 0, c.n_lc, flags_out);
    GTLS_CUDA(cudaGetLastError());
    c.launches += 4;
    return GTLS_OK;
}

SlotMap single_wave(int first, int cnt, int tiles_per_period, bool from_list)
{
    SlotMap sm{};
    sm.nseg = 1;
    sm.slots = cnt;
    sm.items = cnt * tiles_per_period;
    sm.from_list = from_list ? 1 : 0;
    sm.seg[0] = WaveSeg{0, first, 0, 0};
    return sm;
}

gtls_status check_words(const unsigned int* chk, const std::string& where)
{
    if (chk[0] == 0) return GTLS_OK;
    if (chk[0] == (unsigned int)tc::kCheckTimeout)
        return fail(GTLS_ERR_TIMEOUT, where + "a tensor-core window kernel wait ran out (index " +
                                          std::to_string(chk[1]) + ", wait " + std::to_string(chk[2]) + ")");
    return fail(GTLS_ERR_INTERNAL, where + "device index check " + std::to_string(chk[0]) + " failed (value " +
                                       std::to_string(((long long)chk[3] << 32) | chk[1]) + ", limit " +
                                       std::to_string(chk[2]) + ")");
}

// Per-period outputs of the plan's last search into caller device arrays.
gtls_status copy_period_outputs(const gtls_plan* pl, const gtls_period_outputs* per, cudaStream_t st)
{
    const DevPeriod& dq = pl->dq;
    const size_t np_ = (size_t)pl->dp.np;
    if (per->chi2) GTLS_CUDA(cudaMemcpyAsync(per->chi2, dq.chi2, np_ * 8, cudaMemcpyDeviceToDevice, st));
    if (per->dur_idx) GTLS_CUDA(cudaMemcpyAsync(per->dur_idx, dq.dur, np_ * 4, cudaMemcpyDeviceToDevice, st));
    if (per->t0_idx) GTLS_CUDA(cudaMemcpyAsync(per->t0_idx, dq.t0i, np_ * 4, cudaMemcpyDeviceToDevice, st));
    if (per->depth) GTLS_CUDA(cudaMemcpyAsync(per->depth, dq.depth, np_ * 8, cudaMemcpyDeviceToDevice, st));
    if (per->t0) GTLS_CUDA(cudaMemcpyAsync(per->t0, dq.t0, np_ * 8, cudaMemcpyDeviceToDevice, st));
    if (per->sr) GTLS_CUDA(cudaMemcpyAsync(per->sr, dq.sr, np_ * 8, cudaMemcpyDeviceToDevice, st));
    if (per->sde_raw) GTLS_CUDA(cudaMemcpyAsync(per->sde_raw, dq.sde_raw, np_ * 8, cudaMemcpyDeviceToDevice, st));
    if (per->sde) GTLS_CUDA(cudaMemcpyAsync(per->sde, dq.sde, np_ * 8, cudaMemcpyDeviceToDevice, st));
    if (per->refined) GTLS_CUDA(cudaMemcpyAsync(per->refined, dq.refined, np_ * 4, cudaMemcpyDeviceToDevice, st));
    return GTLS_OK;
}

gtls_status run_search(gtls_plan* pl, const double* t, const double* y, const double* dy,
                       int64_t n, cudaStream_t st, gtls_result* out,
                       const gtls_period_outputs* per)
{
    const PlanHost& h = pl->host;
    if (n != h.n)
        return fail(GTLS_ERR_INVALID_ARG, "n (" + std::to_string(n) + ") differs from the plan's n_points (" +
                                              std::to_string(h.n) + ")");
    if (!t || !y || !dy || !out) return fail(GTLS_ERR_INVALID_ARG, "null pointer argument");
    int dev = -1;
    GTLS_CUDA(cudaGetDevice(&dev));
    if (dev != pl->device) return fail(GTLS_ERR_INVALID_ARG, "current device differs from the plan's device");
    GTLS_TRY(ensure_chunk(pl));

    const DevPlan& dp = pl->dp;
    const DevChunk& dk = pl->dk;
    const DevPeriod& dq = pl->dq;
    Ctx c;
    c.set = pl->set;
    c.set_ref = pl->set_ref;
    c.dk = dk;
    c.n_lc = 1;
    c.fold_smem = fold_smem_bytes(h.bucket_log2);
    c.tile_buf = pl->tile_buf;
    c.tile_buf_w = pl->tile_buf_w;
    c.n_sm = pl->n_sm;
    c.median_blocks = (dp.np + median_outs(dp.median_half) - 1) / median_outs(dp.median_half);
    c.topk_smem = topk_smem_bytes(dp.np, pl->refine_k);
    c.st = st;
    c.tc_jspan = pl->tc_jspan;
    c.tc_test = pl->tc_test_wait;
    c.tc_maps = pl->tc_maps;
    pl->profile = gtls_profile{};
    if (pl->profiling) c.prof = pl;

    GTLS_TRY(stage_mark(c, -1));
    GTLS_TRY(prep_pass(c, t, y, dy, pl->prep_off, n, pl->dc.flags));
    GTLS_TRY(stage_mark(c, kStagePrepare));
    unsigned int flags = 0;
    GTLS_CUDA(cudaMemcpyAsync(&flags, pl->dc.flags, sizeof flags, cudaMemcpyDeviceToHost, st));
    GTLS_CUDA(cudaStreamSynchronize(st));
    if (flags & 1u) return fail(GTLS_ERR_INVALID_ARG, "t, y or dy holds a NaN or infinity");
    if (flags & 2u) return fail(GTLS_ERR_INVALID_ARG, "dy must be > 0 everywhere");

    const bool uniform = !(flags & 4u);
    const bool tiled = pl->tile_ok && uniform;
    const bool wtiled = pl->tile_w_ok && !uniform;   // per-point weights, (w r, w) tiles
    for (int p0 = 0; p0 < dp.np; p0 += dk.chunk) {
        const int cnt = std::min<int>(dk.chunk, dp.np - p0);
        GTLS_TRY(wave_pass(c, false, single_wave(p0, cnt, wtiled ? pl->tile_count_w : pl->tile_count, false),
                           tiled || wtiled, wtiled, tiled && pl->has_window_only, pl->tile_counter, true, n,
                           h.max_kept, tiled && pl->has_tensor, pl->tc_counter));
    }
    GTLS_TRY(sr_sde_pass(c));
    // two-stage T0 search (Sect. 2.5): the refine_k best periods by SDE(P)
    // again with T0 step 1, then SR / SDE once more (k_topk also clears the
    // refined flags when refine_k is 0)
    k_topk<<<1, 1024, c.topk_smem, st>>>(c.set, 0);
    GTLS_CUDA(cudaGetLastError());
    c.launches += 1;
    GTLS_TRY(stage_mark(c, kStageSrSde));
    const int kref = pl->refine_k;
    if (kref > 0) {
        for (int r0 = 0; r0 < kref; r0 += dk.chunk) {
            const int cnt = std::min<int>(dk.chunk, kref - r0);
            GTLS_TRY(wave_pass(c, true, single_wave(r0, cnt, pl->tile_count_ref, true), tiled, false,
                               tiled && pl->has_window_only_ref, pl->tile_counter, true, n, h.max_kept));
        }
        GTLS_TRY(sr_sde_pass(c));
    }
    k_best<<<1, 1024, 0, st>>>(c.set, 0, nullptr, nullptr);
    GTLS_CUDA(cudaGetLastError());
    c.launches += 1;
    GTLS_TRY(stage_mark(c, kStageSrSde));
    if (per) GTLS_TRY(copy_period_outputs(pl, per, st));
    unsigned int chk[4] = {0, 0, 0, 0};
    GTLS_CUDA(cudaMemcpyAsync(chk, pl->dc.check, sizeof chk, cudaMemcpyDeviceToHost, st));
    GTLS_CUDA(cudaMemcpyAsync(out, dq.result, sizeof(gtls_result), cudaMemcpyDeviceToHost, st));
    GTLS_CUDA(cudaStreamSynchronize(st));
    GTLS_TRY(check_words(chk, ""));
    pl->profile.kernel_launches = c.launches;
    pl->profile.window_search_launches = c.window_launches;
    if (pl->profiling) GTLS_TRY(collect_profile(pl, c.ev));
    return GTLS_OK;
}

// ---------------------------------------------------------------------------
// batched search: many light curves, one shared chunk scratch, waves of
// (curve, period range) segments, replayed from a captured CUDA graph
// ---------------------------------------------------------------------------

struct BatchWave {
    SlotMap sm;
    bool tiled;
    bool weighted;
    bool window_only;   // some curve of the wave has durations marked kWindowOnly
    bool tensor;        // some curve of the wave has durations marked kTensor
    bool ref;
    int64_t max_n;
    int max_kept;
};

struct BatchCfg {
    int wave_slots = 0;
    int tile_buf = 0;
};

}  // namespace

struct gtls_batch {
    std::vector<gtls_plan*> plans;
    int device = -1;
    int n_lc = 0;
    std::vector<int64_t> off;          // host offsets (n_lc + 1, from 0)
    int64_t max_n = 0;
    int max_kept = 0;
    int fold_smem = 0, topk_smem = 0, median_blocks = 1, n_sm = 0;
    int max_slots = 0;                 // chunk scratch slots allocated
    int tile_buf_max = 0;              // the smallest staged tile of the tiled plans (their own choice)
    int tile_buf_cap = 0;              // largest staged tile the device's shared memory allows
    gtls::DevChunk dk{};
    gtls::DevSet set{}, set_ref{};
    gtls::DevTiles* d_tiles = nullptr;   // 2 n_lc entries: coarse, refinement
    int64_t* off_dev = nullptr;
    unsigned int* flags = nullptr;     // per curve validity flags
    unsigned int* checks = nullptr;    // 4 words per curve
    gtls_result* results = nullptr;
    unsigned int* counters = nullptr;  // two per tiled wave (autotuner probes) or per graph loop
    int n_counters = 0;
    // device work queues of the graph's loops: their (curve, first, count,
    // tiles per period) runs, the wave each loop is searching and the cursors
    int32_t* q_runs = nullptr;         // 4 words per run, at most 2 n_lc runs
    gtls::SlotMap* q_waves = nullptr;  // kMaxLoops
    int32_t* q_cursors = nullptr;      // 3 words per loop
    cudaStream_t body_stream = nullptr;   // stream the loop bodies are captured on
    BatchCfg cfg;
    bool tuned = false;
    // graph of everything after the curve preparation, for one set of
    // per-curve kernel classes (uniform dy and tile fit)
    std::vector<uint8_t> graph_class;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr; // private stream the graph is captured on
    int graph_kernels = 0;             // kernels in the graph (a loop body counted once)
    int64_t graph_launches = 0;        // kernels one replay launches
    int waves = 0;
    int64_t last_launches = 0;         // kernels of the last search
    int64_t total_periods = 0;         // coarse plus refinement periods
    double tuned_rate = 0.0;           // probe window flop/s of the chosen configuration
    std::vector<gtls::DevTiles> tiles_host;   // 2 n_lc entries
    std::vector<uint8_t> fits, fits_ref;      // curve fits the tiled kernel at cfg.tile_buf
    std::vector<uint8_t> fits_w;              // ... with per-point weights at tile_buf_w pairs
    int tile_buf_w = 0;                       // (w r, w) pairs per tile of the weighted waves
    const void* tc_maps = nullptr;            // TMA maps of dk.rs for the tensor-core window kernel
    std::vector<void*> allocs;
    int64_t device_bytes = 0;
};

namespace {

template <class T>
gtls_status batch_alloc(gtls_batch* b, T** ptr, size_t count)
{
    *ptr = nullptr;
    if (count == 0) count = 1;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(GTLS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    b->allocs.push_back(p);
    b->device_bytes += (int64_t)(count * sizeof(T));
    *ptr = static_cast<T*>(p);
    return GTLS_OK;
}

void batch_release(gtls_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    b->cap_stream = nullptr;
    if (b->body_stream) cudaStreamDestroy(b->body_stream);
    b->body_stream = nullptr;
    for (void* p : b->allocs) cudaFree(p);
    b->allocs.clear();
}

// Tile shape of every curve for a staged buffer of `buf` floats; curves
// whose durations do not fit take the one-thread-per-window kernel.
void batch_tiles(gtls_batch* b, int buf)
{
    b->tiles_host.assign(2 * (size_t)b->n_lc, DevTiles{0, 0, 0, 0});
    b->fits.assign(b->n_lc, 0);
    b->fits_ref.assign(b->n_lc, 0);
    b->fits_w.assign(b->n_lc, 0);
    for (int i = 0; i < b->n_lc; ++i) {
        const gtls_plan* pl = b->plans[i];
        const PlanHost& h = pl->host;
        b->fits_w[i] = pl->tile_w_ok && pl->tile_buf_w == b->tile_buf_w ? 1 : 0;
        if (b->fits_w[i]) {
            b->tiles_host[i].len_w = pl->tile_len_w;
            b->tiles_host[i].count_w = pl->tile_count_w;
        }
        if (!pl->tile_ok) continue;
        // the plan's tiled durations (not kWindowOnly) must fit this buffer
        int st_max = 1, dmax_t = 0, dmax1 = 0;
        bool fits = true, fits1 = true;
        for (size_t j = 0; j < h.dpts.size(); ++j) {
            const int st = h.stride[j], d = h.dpts[j];
            if (pl->variant_host[j] != tiles::kWindowOnly && pl->variant_host[j] != tiles::kTensor) {
                st_max = std::max(st_max, st);
                dmax_t = std::max(dmax_t, d);
                const int jrows = (d + st - 1) / st;
                if ((int64_t)(16 + jrows + 2) * st + 32 > buf || (int64_t)d + 3 * st + 96 + 64 > buf) fits = false;
            }
            if ((int64_t)(16 + d + 2) + 32 <= buf && (int64_t)d + 3 + 96 + 64 <= buf) dmax1 = std::max(dmax1, d);
            else fits1 = false;   // every duration must fit the refinement tiles at this buffer
        }
        if (pl->has_window_only_ref) fits1 = false;   // refinement tiles sized at the plan's own buffer only
        const int64_t len = ((int64_t)buf - dmax_t - 3 * (int64_t)st_max - 96) & ~int64_t(63);
        const int64_t len1 = ((int64_t)buf - dmax1 - 3 - 96) & ~int64_t(63);
        if (dmax1 == 0) fits1 = false;
        if (fits && len >= 64) {
            b->fits[i] = 1;
            b->tiles_host[i].len = (int32_t)len;
            b->tiles_host[i].count = (int32_t)((h.n + len - 1) / len);
        }
        if (fits1 && len1 >= 64) {
            b->fits_ref[i] = 1;
            b->tiles_host[b->n_lc + i] = DevTiles{(int32_t)len1, (int32_t)((h.n + len1 - 1) / len1), 0, 0};
        }
    }
}

// Waves over the given (curve, first, count) runs, in order: at most
// wave_slots slots and kMaxSeg segments each; a run may span waves.
struct Run {
    int lc, first, count;
};

void build_waves(const gtls_batch* b, const std::vector<Run>& runs, bool tiled, bool weighted, bool ref,
                 int wave_slots, std::vector<BatchWave>& out)
{
    BatchWave w{};
    auto flush = [&]() {
        if (w.sm.slots > 0) out.push_back(w);
        w = BatchWave{};
        w.tiled = tiled;
        w.weighted = weighted;
        w.window_only = false;
        w.tensor = false;
        w.ref = ref;
        w.sm.from_list = ref ? 1 : 0;
    };
    flush();
    for (const Run& r : runs) {
        int done = 0;
        const DevTiles& tl = b->tiles_host[(ref ? b->n_lc : 0) + r.lc];
        const int tiles_pp = tiled ? (weighted ? tl.count_w : tl.count) : 0;
        const PlanHost& h = b->plans[r.lc]->host;
        while (done < r.count) {
            if (w.sm.slots == wave_slots || w.sm.nseg == kMaxSeg) flush();
            const int take = std::min(r.count - done, wave_slots - w.sm.slots);
            WaveSeg g{r.lc, r.first + done, w.sm.slots, w.sm.items};
            w.sm.seg[w.sm.nseg++] = g;
            w.sm.slots += take;
            w.sm.items += take * tiles_pp;
            w.max_n = std::max<int64_t>(w.max_n, h.n);
            w.max_kept = std::max(w.max_kept, h.max_kept);
            const gtls_plan* pl = b->plans[r.lc];
            if (tiled && !weighted && (ref ? pl->has_window_only_ref : pl->has_window_only)) w.window_only = true;
            if (tiled && !weighted && !ref && pl->has_tensor) w.tensor = true;
            done += take;
        }
    }
    flush();
}

// Per-curve kernel class: 1 = tiled window kernel, 2 = tiled with per-point
// weights, 0 = one thread per window.
std::vector<uint8_t> batch_classes(const gtls_batch* b, const std::vector<unsigned int>& flags)
{
    std::vector<uint8_t> c(b->n_lc);
    for (int i = 0; i < b->n_lc; ++i) {
        const bool uniform = !(flags[i] & 4u);
        c[i] = uniform ? (b->fits[i] ? 1 : 0) : (b->fits_w[i] ? 2 : 0);
    }
    return c;
}

Ctx batch_ctx(const gtls_batch* b, cudaStream_t st)
{
    Ctx c;
    c.set = b->set;
    c.set_ref = b->set_ref;
    c.dk = b->dk;
    c.n_lc = b->n_lc;
    c.fold_smem = b->fold_smem;
    c.tile_buf = b->cfg.tile_buf;
    c.tile_buf_w = b->tile_buf_w;
    c.n_sm = b->n_sm;
    c.median_blocks = b->median_blocks;
    c.topk_smem = b->topk_smem;
    c.st = st;
    for (const gtls_plan* pl : b->plans) {
        c.tc_jspan = std::max(c.tc_jspan, pl->tc_jspan);
        c.tc_test = std::max(c.tc_test, pl->tc_test_wait);
    }
    c.tc_maps = b->tc_maps;
    return c;
}

gtls_status batch_upload_tiles(gtls_batch* b)
{
    GTLS_CUDA(cudaMemcpy(b->d_tiles, b->tiles_host.data(), b->tiles_host.size() * sizeof(DevTiles),
                         cudaMemcpyHostToDevice));
    return GTLS_OK;
}

// Makes sure there are two window-kernel counters (tiled, tensor-core) for
// each of n waves or loops.
gtls_status batch_counters(gtls_batch* b, int n)
{
    if (2 * n <= b->n_counters) return GTLS_OK;
    const int m = std::max(2 * n, 2 * b->n_counters);
    GTLS_TRY(batch_alloc(b, &b->counters, m));
    b->n_counters = m;
    return GTLS_OK;
}

// One loop of the batch graph: the runs of one kernel class, coarse or
// refinement, and what its wave kernels need.
constexpr int kMaxLoops = 6;   // classes 1, 2, 0 for the coarse and the refinement pass
struct LoopSpec {
    bool tiled = false, weighted = false, window_only = false, tensor = false, ref = false;
    int64_t max_n = 0;
    int max_kept = 0;
    int run0 = 0, nruns = 0;   // runs[run0, run0 + nruns) of the queue table
    int waves = 0;             // waves the device will cut (the host's build_waves count)
    int body_kernels = 0;      // kernels per wave
};

void add_loop_spec(const gtls_batch* b, const std::vector<Run>& rs, bool tiled, bool weighted, bool ref,
                   std::vector<QueueRun>& runs, std::vector<LoopSpec>& loops)
{
    if (rs.empty()) return;
    LoopSpec L;
    L.tiled = tiled;
    L.weighted = weighted;
    L.ref = ref;
    L.run0 = (int)runs.size();
    for (const Run& r : rs) {
        const gtls_plan* pl = b->plans[r.lc];
        const DevTiles& tl = b->tiles_host[(ref ? b->n_lc : 0) + r.lc];
        const int tiles_pp = tiled ? (weighted ? tl.count_w : tl.count) : 0;
        runs.push_back(QueueRun{r.lc, r.first, r.count, tiles_pp});
        L.max_n = std::max<int64_t>(L.max_n, pl->host.n);
        L.max_kept = std::max(L.max_kept, pl->host.max_kept);
        if (tiled && !weighted && (ref ? pl->has_window_only_ref : pl->has_window_only)) L.window_only = true;
        if (tiled && !weighted && !ref && pl->has_tensor) L.tensor = true;
    }
    L.nruns = (int)rs.size();
    std::vector<BatchWave> w;
    build_waves(b, rs, tiled, weighted, ref, b->cfg.wave_slots, w);
    L.waves = (int)w.size();
    loops.push_back(L);
}

// The loops of the graph in order (coarse classes 1, 2, 0, then the
// refinement) and the queue table of their runs.
void batch_loops(const gtls_batch* b, const std::vector<uint8_t>& cls, std::vector<QueueRun>& runs,
                 std::vector<LoopSpec>& coarse, std::vector<LoopSpec>& refine)
{
    for (int k = 0; k < 3; ++k) {
        const int klass = k == 2 ? 0 : k + 1;
        std::vector<Run> rc, rr;
        for (int i = 0; i < b->n_lc; ++i) {
            const gtls_plan* pl = b->plans[i];
            if (cls[i] == klass) rc.push_back(Run{i, 0, pl->dp.np});
            const int klass_ref = (cls[i] == 1 && b->fits_ref[i]) ? 1 : 0;
            if (pl->refine_k > 0 && klass_ref == klass) rr.push_back(Run{i, 0, pl->refine_k});
        }
        add_loop_spec(b, rc, klass != 0, klass == 2, false, runs, coarse);
        add_loop_spec(b, rr, klass != 0, klass == 2, true, runs, refine);
    }
}

// Appends, at the capture position of c.st, a while-loop node whose body
// cuts the next wave of queue `qi` (k_wave_next) and searches it; the body
// is captured on the batch's second stream.
gtls_status capture_loop(gtls_batch* b, Ctx& c, LoopSpec& L, int qi)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    GTLS_CUDA(cudaStreamGetCaptureInfo(c.st, &cs, nullptr, &g, &deps, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive || !g) return fail(GTLS_ERR_INTERNAL, "batch graph capture is not active");
    cudaGraphConditionalHandle h{};
    GTLS_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};   // aggregate: every other byte zero
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    GTLS_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    GTLS_CUDA(cudaStreamUpdateCaptureDependencies(c.st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = np.conditional.phGraph_out[0];

    WaveQueue q{};
    q.runs = reinterpret_cast<const QueueRun*>(b->q_runs) + L.run0;
    q.nruns = L.nruns;
    q.wave_slots = b->cfg.wave_slots;
    q.from_list = L.ref ? 1 : 0;
    q.cursor = b->q_cursors + 3 * qi;
    q.wave = b->q_waves + qi;
    q.counters = b->counters + 2 * qi;
    q.cond = h;
    GTLS_CUDA(cudaStreamBeginCaptureToGraph(b->body_stream, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
    Ctx cb = c;
    cb.st = b->body_stream;
    cb.launches = 0;
    k_wave_next<<<1, 32, 0, cb.st>>>(q);
    gtls_status s = cudaGetLastError() == cudaSuccess ? GTLS_OK : fail(GTLS_ERR_CUDA, "k_wave_next launch");
    SlotMap grid{};   // grid sizes: the most slots a wave can hold
    grid.slots = b->cfg.wave_slots;
    if (s == GTLS_OK)
        s = wave_pass(cb, L.ref, grid, L.tiled, L.weighted, L.window_only, q.counters, false, L.max_n, L.max_kept,
                      L.tensor, q.counters + 1, q.wave);
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->body_stream, &out);
    if (s != GTLS_OK) return s;
    if (e != cudaSuccess) return fail(GTLS_ERR_CUDA, std::string("loop body capture: ") + cudaGetErrorString(e));
    L.body_kernels = (int)cb.launches + 1;
    c.launches += L.body_kernels;
    return GTLS_OK;
}

// Everything after the curve preparation: the coarse loops, SR / SDE and
// the refinement list, the refinement loops, SR / SDE and the best
// candidate of every curve.
gtls_status batch_enqueue(gtls_batch* b, Ctx& c, std::vector<LoopSpec>& coarse, std::vector<LoopSpec>& refine)
{
    const int nloops = (int)(coarse.size() + refine.size());
    k_queue_reset<<<1, 32, 0, c.st>>>(b->q_cursors, nloops);
    GTLS_CUDA(cudaGetLastError());
    c.launches += 1;
    int qi = 0;
    for (LoopSpec& L : coarse) GTLS_TRY(capture_loop(b, c, L, qi++));
    GTLS_TRY(sr_sde_pass(c));
    k_topk<<<c.n_lc, 1024, c.topk_smem, c.st>>>(c.set, 0);
    GTLS_CUDA(cudaGetLastError());
    c.launches += 1;
    if (!refine.empty()) {
        for (LoopSpec& L : refine) GTLS_TRY(capture_loop(b, c, L, qi++));
        GTLS_TRY(sr_sde_pass(c));
    }
    k_best<<<c.n_lc, 1024, 0, c.st>>>(c.set, 0, b->results, b->checks);
    GTLS_CUDA(cudaGetLastError());
    c.launches += 1;
    return GTLS_OK;
}

gtls_status batch_capture(gtls_batch* b, cudaStream_t st, const std::vector<uint8_t>& cls)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_class.clear();
    std::vector<QueueRun> runs;
    std::vector<LoopSpec> coarse, refine;
    batch_loops(b, cls, runs, coarse, refine);
    if (coarse.size() + refine.size() > (size_t)kMaxLoops || runs.size() > 2 * (size_t)b->n_lc)
        return fail(GTLS_ERR_INTERNAL, "batch queue table overflow");
    GTLS_TRY(batch_counters(b, kMaxLoops));
    if (!runs.empty())
        GTLS_CUDA(cudaMemcpy(b->q_runs, runs.data(), runs.size() * sizeof(QueueRun), cudaMemcpyHostToDevice));
    // captured on the batch's own stream (the caller's may be the legacy
    // default stream, which cannot be captured); launched on the caller's
    (void)st;
    Ctx c = batch_ctx(b, b->cap_stream);
    GTLS_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    gtls_status s = batch_enqueue(b, c, coarse, refine);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (s != GTLS_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return fail(GTLS_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    b->graph = g;
    GTLS_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    b->graph_class = cls;
    b->graph_kernels = (int)c.launches;
    // kernels one replay launches: the fixed ones and every wave's body
    int64_t per_search = c.launches, waves = 0;
    for (const std::vector<LoopSpec>* v : {&coarse, &refine})
        for (const LoopSpec& L : *v) {
            per_search += (int64_t)(L.waves - 1) * L.body_kernels;
            waves += L.waves;
        }
    b->graph_launches = per_search;
    b->waves = (int)waves;
    return GTLS_OK;
}

gtls_status batch_check_inputs(const gtls_batch* b, const double* t, const double* y, const double* dy,
                               const int64_t* offsets)
{
    if (!t || !y || !dy || !offsets) return fail(GTLS_ERR_INVALID_ARG, "null pointer argument");
    for (int i = 0; i < b->n_lc; ++i)
        if (offsets[i + 1] - offsets[i] != b->plans[i]->host.n)
            return fail(GTLS_ERR_INVALID_ARG, "light curve " + std::to_string(i) + " has " +
                                                  std::to_string(offsets[i + 1] - offsets[i]) +
                                                  " points; its plan was made for " +
                                                  std::to_string(b->plans[i]->host.n));
    int dev = -1;
    GTLS_CUDA(cudaGetDevice(&dev));
    if (dev != b->device) return fail(GTLS_ERR_INVALID_ARG, "current device differs from the batch's device");
    return GTLS_OK;
}

// Curve preparation of the whole batch and its validity check (one sync).
gtls_status batch_prepare(gtls_batch* b, const double* t, const double* y, const double* dy, cudaStream_t st,
                          std::vector<unsigned int>& flags, int64_t& launches)
{
    Ctx c = batch_ctx(b, st);
    GTLS_TRY(prep_pass(c, t, y, dy, b->off_dev, b->max_n, b->flags));
    launches += c.launches;
    flags.assign(b->n_lc, 0u);
    GTLS_CUDA(cudaMemcpyAsync(flags.data(), b->flags, b->n_lc * sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    GTLS_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < b->n_lc; ++i) {
        if (flags[i] & 1u)
            return fail(GTLS_ERR_INVALID_ARG, "light curve " + std::to_string(i) + ": t, y or dy holds a NaN or infinity");
        if (flags[i] & 2u)
            return fail(GTLS_ERR_INVALID_ARG, "light curve " + std::to_string(i) + ": dy must be > 0 everywhere");
    }
    return GTLS_OK;
}

gtls_status batch_search(gtls_batch* b, const double* t, const double* y, const double* dy,
                         const int64_t* offsets, cudaStream_t st, gtls_result* out)
{
    GTLS_TRY(batch_check_inputs(b, t, y, dy, offsets));
    if (!out) return fail(GTLS_ERR_INVALID_ARG, "null pointer argument");
    const int64_t o0 = offsets[0];
    std::vector<unsigned int> flags;
    int64_t launches = 0;
    GTLS_TRY(batch_prepare(b, t + o0, y + o0, dy + o0, st, flags, launches));
    const std::vector<uint8_t> cls = batch_classes(b, flags);
    if (!b->exec || cls != b->graph_class) GTLS_TRY(batch_capture(b, st, cls));
    GTLS_CUDA(cudaGraphLaunch(b->exec, st));
    std::vector<unsigned int> chk(4 * (size_t)b->n_lc);
    GTLS_CUDA(cudaMemcpyAsync(chk.data(), b->checks, chk.size() * sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    GTLS_CUDA(cudaMemcpyAsync(out, b->results, b->n_lc * sizeof(gtls_result), cudaMemcpyDeviceToHost, st));
    GTLS_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < b->n_lc; ++i)
        GTLS_TRY(check_words(&chk[4 * (size_t)i], "light curve " + std::to_string(i) + ": "));
    b->last_launches = launches + b->graph_launches;
    return GTLS_OK;
}

gtls_status batch_create(gtls_plan* const* plans, int64_t n_lc, int32_t wave_slots, gtls_batch* b)
{
    if (n_lc < 1 || n_lc > 65535) return fail(GTLS_ERR_INVALID_ARG, "n_lc must be in [1, 65535]");
    GTLS_CUDA(cudaGetDevice(&b->device));
    GTLS_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    GTLS_CUDA(cudaStreamCreateWithFlags(&b->body_stream, cudaStreamNonBlocking));
    b->n_lc = (int)n_lc;
    b->plans.assign(plans, plans + n_lc);
    b->off.assign(1, 0);
    int bucket_log2 = 0, max_np_blocks = 1, topk = 0, buf_max = 1 << 30;
    int64_t fold_stride = 32, key_stride = 32, pad_stride = 32;
    bool any_tiled = false;
    for (int i = 0; i < b->n_lc; ++i) {
        gtls_plan* pl = plans[i];
        if (!pl) return fail(GTLS_ERR_INVALID_ARG, "null plan in the batch");
        if (pl->device != b->device) return fail(GTLS_ERR_INVALID_ARG, "plans of a batch must share its device");
        for (int k = 0; k < i; ++k)
            if (plans[k] == pl) return fail(GTLS_ERR_INVALID_ARG, "a plan may appear once in a batch");
        const PlanHost& h = pl->host;
        b->off.push_back(b->off.back() + h.n);
        b->max_n = std::max<int64_t>(b->max_n, h.n);
        b->max_kept = std::max(b->max_kept, h.max_kept);
        bucket_log2 = std::max(bucket_log2, h.bucket_log2);
        fold_stride = std::max<int64_t>(fold_stride, pl->dk.fold_stride);
        key_stride = std::max<int64_t>(key_stride, pl->dk.key_stride);
        pad_stride = std::max<int64_t>(pad_stride, pl->dk.pad_stride);
        const int mo = median_outs(pl->dp.median_half);
        max_np_blocks = std::max(max_np_blocks, (pl->dp.np + mo - 1) / mo);
        topk = std::max(topk, topk_smem_bytes(pl->dp.np, pl->refine_k));
        if (pl->tile_ok) {
            buf_max = std::min(buf_max, pl->tile_buf);
            any_tiled = true;
        }
    }
    b->fold_smem = fold_smem_bytes(bucket_log2);
    b->topk_smem = topk;
    b->median_blocks = max_np_blocks;
    b->n_sm = plans[0]->n_sm;
    b->tile_buf_max = any_tiled ? buf_max : 0;
    for (int i = 0; i < b->n_lc && b->tile_buf_w == 0; ++i)
        if (plans[i]->tile_w_ok) b->tile_buf_w = plans[i]->tile_buf_w;
    {
        int optin = 0;
        GTLS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
        b->tile_buf_cap = ((optin - 8192) / 4) & ~63;
    }
    b->cfg.tile_buf = b->tile_buf_max;

    // chunk scratch shared by all curves: slots of the largest curve's strides
    DevChunk& dk = b->dk;
    dk.fold_stride = fold_stride;
    dk.key_stride = key_stride;
    dk.pad_stride = pad_stride;
    const int64_t per_slot = key_stride * 8 + fold_stride * 4 + pad_stride * (4 + 4 + 4 + 8);
    const int64_t budget = int64_t(16) << 30;
    int64_t slots = std::min<int64_t>(4096, std::max<int64_t>(1, budget / per_slot));
    if (b->n_sm > 0 && slots >= 4 * b->n_sm) slots = slots / (4 * b->n_sm) * (4 * b->n_sm);   // whole fold waves at 1, 1/2, 1/4
    if (wave_slots > 0) slots = wave_slots;
    b->max_slots = (int)slots;
    b->cfg.wave_slots = (int)slots;
    dk.chunk = (int32_t)slots;
    GTLS_TRY(batch_alloc(b, &dk.keys, slots * key_stride));
    GTLS_TRY(batch_alloc(b, &dk.sidx, slots * fold_stride));
    GTLS_TRY(batch_alloc(b, &dk.rs, slots * pad_stride));
    GTLS_TRY(batch_alloc(b, &dk.ws, slots * pad_stride));
    GTLS_TRY(batch_alloc(b, &dk.wrs, slots * pad_stride));
    GTLS_TRY(batch_alloc(b, &dk.pf, slots * pad_stride));
    {
        bool any_tensor = false;
        for (int i = 0; i < n_lc; ++i) any_tensor = any_tensor || plans[i]->has_tensor;
        if (any_tensor) {
            unsigned char* maps = nullptr;
            GTLS_TRY(batch_alloc(b, &maps, (size_t)tc::kMaps * sizeof(CUtensorMap)));
            GTLS_TRY(make_tc_maps(dk, maps));
            b->tc_maps = maps;
        }
    }

    // per-curve descriptors
    std::vector<DevPlan> hp(2 * (size_t)n_lc);
    std::vector<DevCurve> hc(n_lc);
    std::vector<DevPeriod> hq(n_lc);
    int64_t total_periods = 0;
    for (int i = 0; i < b->n_lc; ++i) {
        hp[i] = plans[i]->dp;
        hp[n_lc + i] = plans[i]->refine_k > 0 ? plans[i]->dp_ref : plans[i]->dp;
        hc[i] = plans[i]->dc;
        hq[i] = plans[i]->dq;
        total_periods += plans[i]->dp.np + plans[i]->refine_k;
    }
    DevPlan* d_plans = nullptr;
    DevCurve* d_curves = nullptr;
    DevPeriod* d_outs = nullptr;
    GTLS_TRY(batch_alloc(b, &d_plans, hp.size()));
    GTLS_TRY(batch_alloc(b, &d_curves, hc.size()));
    GTLS_TRY(batch_alloc(b, &d_outs, hq.size()));
    GTLS_TRY(batch_alloc(b, &b->d_tiles, 2 * (size_t)n_lc));
    GTLS_CUDA(cudaMemcpy(d_plans, hp.data(), hp.size() * sizeof(DevPlan), cudaMemcpyHostToDevice));
    GTLS_CUDA(cudaMemcpy(d_curves, hc.data(), hc.size() * sizeof(DevCurve), cudaMemcpyHostToDevice));
    GTLS_CUDA(cudaMemcpy(d_outs, hq.data(), hq.size() * sizeof(DevPeriod), cudaMemcpyHostToDevice));
    b->set = DevSet{d_plans, d_curves, d_outs, b->d_tiles};
    b->set_ref = DevSet{d_plans + n_lc, d_curves, d_outs, b->d_tiles + n_lc};
    GTLS_TRY(batch_alloc(b, &b->off_dev, b->off.size()));
    GTLS_CUDA(cudaMemcpy(b->off_dev, b->off.data(), b->off.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    GTLS_TRY(batch_alloc(b, &b->flags, n_lc));
    GTLS_TRY(batch_alloc(b, &b->checks, 4 * (size_t)n_lc));
    GTLS_TRY(batch_alloc(b, &b->results, n_lc));
    GTLS_TRY(batch_alloc(b, &b->q_runs, 4 * 2 * (size_t)n_lc));
    GTLS_TRY(batch_alloc(b, &b->q_waves, (size_t)kMaxLoops));
    GTLS_TRY(batch_alloc(b, &b->q_cursors, 3 * (size_t)kMaxLoops));
    b->total_periods = total_periods;
    batch_tiles(b, b->cfg.tile_buf);
    GTLS_TRY(batch_upload_tiles(b));
    return GTLS_OK;
}

// Window-point evaluations of period p of a plan's coarse pass.
double period_wpe(const PlanHost& h, int p)
{
    double w = 0.0;
    for (int j = h.jlo[p]; j <= h.jhi[p]; ++j) {
        if (j > h.jlo[p] && h.dpts[j] == h.dpts[j - 1]) continue;
        w += (double)((h.n + h.stride[j] - 1) / h.stride[j]) * h.dpts[j];
    }
    return w;
}

// Picks the wave size and the staged tile size: every candidate runs the
// coarse pass of a probe (runs of 256 periods spread over the grids of the
// first tiled curves) once untimed and twice timed; the score is window-point
// evaluations per second.
gtls_status batch_autotune(gtls_batch* b, const double* t, const double* y, const double* dy,
                           const int64_t* offsets, cudaStream_t st)
{
    GTLS_TRY(batch_check_inputs(b, t, y, dy, offsets));
    const int64_t o0 = offsets[0];
    std::vector<unsigned int> flags;
    int64_t launches = 0;
    GTLS_TRY(batch_prepare(b, t + o0, y + o0, dy + o0, st, flags, launches));
    std::vector<uint8_t> cls = batch_classes(b, flags);
    std::vector<Run> probe;
    double probe_wpe = 0.0;
    for (int i = 0, used = 0; i < b->n_lc && used < 4; ++i) {
        if (!cls[i]) continue;
        ++used;
        const PlanHost& h = b->plans[i]->host;
        const int np = (int)h.periods.size();
        for (int k = 0; k < 4; ++k) {
            const int cnt = std::min(256, np);
            const int first = std::max(0, std::min(np - cnt, (int)((k + 0.5) * np / 4.0) - cnt / 2));
            probe.push_back(Run{i, first, cnt});
            for (int p = first; p < first + cnt; ++p) probe_wpe += period_wpe(h, p);
        }
    }
    if (probe.empty()) return GTLS_OK;   // no curve takes the tiled kernel: nothing to tune
    std::vector<int> slot_c, buf_c;
    for (int sc : {b->max_slots, b->max_slots / 2, b->max_slots / 4})
        if (sc >= 128 && std::find(slot_c.begin(), slot_c.end(), sc) == slot_c.end()) slot_c.push_back(sc);
    if (slot_c.empty()) slot_c.push_back(b->max_slots);
    // the staged tile stays the plans' own: the tile decomposition decides
    // which warp block evaluates a window, and the rotated column-pair
    // variant sums a window's column rounds in an order that depends on its
    // block, so another tile size would change results in the last bits
    // against the curves searched alone
    buf_c.push_back(b->tile_buf_max);
    cudaEvent_t e0, e1;
    GTLS_CUDA(cudaEventCreate(&e0));
    GTLS_CUDA(cudaEventCreate(&e1));
    BatchCfg best = b->cfg;
    double best_rate = -1.0;
    gtls_status s = GTLS_OK;
    for (int bc : buf_c) {
        batch_tiles(b, bc);
        bool ok = true;
        for (const Run& r : probe) ok = ok && b->fits[r.lc];
        if (!ok) continue;
        if ((s = batch_upload_tiles(b)) != GTLS_OK) break;
        for (int sc : slot_c) {
            std::vector<BatchWave> waves;
            build_waves(b, probe, true, false, false, sc, waves);
            if ((s = batch_counters(b, (int)waves.size())) != GTLS_OK) break;
            Ctx c = batch_ctx(b, st);
            c.tile_buf = bc;
            float ms = 0.0f;
            for (int rep = 0; rep < 3 && s == GTLS_OK; ++rep) {
                if (rep == 1 && cudaEventRecord(e0, st) != cudaSuccess) s = fail(GTLS_ERR_CUDA, "cudaEventRecord");
                int ci = 0;
                for (const BatchWave& w : waves) {
                    unsigned int* cnt = b->counters + 2 * ci++;
                    s = wave_pass(c, false, w.sm, true, false, false, cnt, true, w.max_n, w.max_kept, w.tensor,
                                  cnt + 1);
                    if (s != GTLS_OK) break;
                }
            }
            if (s != GTLS_OK) break;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                s = fail(GTLS_ERR_CUDA, "timing the autotuner probe failed");
                break;
            }
            const double rate = 2.0 * probe_wpe / (ms * 1e-3);
            if (rate > best_rate) {
                best_rate = rate;
                best.wave_slots = sc;
                best.tile_buf = bc;
            }
        }
        if (s != GTLS_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cfg = best;
    batch_tiles(b, best.tile_buf);
    GTLS_TRY(batch_upload_tiles(b));
    if (s != GTLS_OK) return s;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_class.clear();
    b->tuned = true;
    b->tuned_rate = best_rate;
    return GTLS_OK;
}

void release(gtls_plan* pl)
{
    if (!pl) return;
    for (cudaEvent_t e : pl->events) cudaEventDestroy(e);
    pl->events.clear();
    for (int i = 0; i < pl->n_allocs; ++i) cudaFree(pl->allocs[i]);
    pl->n_allocs = 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

void gtls_plan_params_default(gtls_plan_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->m_star = 1.0;
    p->r_star = 1.0;
    p->oversampling = 3.0;
    p->k_min = 20.05;
    p->k_max = 620.84;
    p->q_cap = 0.15;
    p->dur_ratio = 1.1;
    p->dt0 = 0.05;
    p->u1 = 0.4;
    p->u2 = 0.25;
}

gtls_status gtls_plan_create(const gtls_plan_params* p, gtls_plan** out)
{
    if (!p || !out) return fail(GTLS_ERR_INVALID_ARG, "null pointer argument");
    *out = nullptr;
    gtls_plan* pl = new (std::nothrow) gtls_plan();
    if (!pl) return fail(GTLS_ERR_OOM, "host allocation of the plan failed");
    std::string err;
    try {
        if (!build_plan_host(*p, pl->host, err)) {
            delete pl;
            return fail(GTLS_ERR_INVALID_ARG, err);
        }
    } catch (const std::bad_alloc&) {
        delete pl;
        return fail(GTLS_ERR_OOM, "host allocation failed while building the grids");
    }
    gtls_status s = create_device(pl);
    if (s != GTLS_OK) {
        release(pl);
        delete pl;
        return s;
    }
    *out = pl;
    return GTLS_OK;
}

gtls_status gtls_plan_get_info(const gtls_plan* pl, gtls_plan_info* o)
{
    if (!pl || !o) return fail(GTLS_ERR_INVALID_ARG, "null pointer argument");
    const PlanHost& h = pl->host;
    o->n_periods = (int64_t)h.periods.size();
    o->n_points = h.n;
    o->n_durations = (int32_t)h.q.size();
    o->time_exponent = h.time_exponent;
    o->max_duration_points = h.dmax;
    o->n_windows = h.n_windows;
    o->wpe = h.wpe;
    o->device_bytes = pl->device_bytes;
    o->median_window = h.median_window;
    o->periods_per_chunk = pl->dk.chunk;
    return GTLS_OK;
}

gtls_status gtls_plan_get_periods(const gtls_plan* pl, double* o)
{
    if (!pl || !o) return fail(GTLS_ERR_INVALID_ARG, "null pointer argument");
    std::memcpy(o, pl->host.periods.data(), pl->host.periods.size() * sizeof(double));
    return GTLS_OK;
}

gtls_status gtls_plan_get_durations(const gtls_plan* pl, double* q, int32_t* pts)
{
    if (!pl) return fail(GTLS_ERR_INVALID_ARG, "null plan");
    if (q) std::memcpy(q, pl->host.q.data(), pl->host.q.size() * sizeof(double));
    if (pts) std::memcpy(pts, pl->host.dpts.data(), pl->host.dpts.size() * sizeof(int32_t));
    return GTLS_OK;
}

gtls_status gtls_plan_get_ranges(const gtls_plan* pl, int32_t* jlo, int32_t* jhi)
{
    if (!pl) return fail(GTLS_ERR_INVALID_ARG, "null plan");
    if (jlo) std::memcpy(jlo, pl->host.jlo.data(), pl->host.jlo.size() * sizeof(int32_t));
    if (jhi) std::memcpy(jhi, pl->host.jhi.data(), pl->host.jhi.size() * sizeof(int32_t));
    return GTLS_OK;
}

gtls_status gtls_search(gtls_plan* pl, const double* t, const double* y, const double* dy,
                        int64_t n, void* stream, gtls_result* out, const gtls_period_outputs* per)
{
    if (!pl) return fail(GTLS_ERR_INVALID_ARG, "null plan");
    g_last_error.clear();
    return run_search(pl, t, y, dy, n, static_cast<cudaStream_t>(stream), out, per);
}

gtls_status gtls_search_host(gtls_plan* pl, const double* t, const double* y, const double* dy,
                             int64_t n, void* stream, gtls_result* out)
{
    if (!pl) return fail(GTLS_ERR_INVALID_ARG, "null plan");
    if (!t || !y || !dy || !out) return fail(GTLS_ERR_INVALID_ARG, "null pointer argument");
    if (n != pl->host.n) return fail(GTLS_ERR_INVALID_ARG, "n differs from the plan's n_points");
    g_last_error.clear();
    if (!pl->in_t) {
        GTLS_TRY(dev_alloc(pl, &pl->in_t, n));
        GTLS_TRY(dev_alloc(pl, &pl->in_y, n));
        GTLS_TRY(dev_alloc(pl, &pl->in_dy, n));
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GTLS_CUDA(cudaMemcpyAsync(pl->in_t, t, n * sizeof(double), cudaMemcpyHostToDevice, st));
    GTLS_CUDA(cudaMemcpyAsync(pl->in_y, y, n * sizeof(double), cudaMemcpyHostToDevice, st));
    GTLS_CUDA(cudaMemcpyAsync(pl->in_dy, dy, n * sizeof(double), cudaMemcpyHostToDevice, st));
    return run_search(pl, pl->in_t, pl->in_y, pl->in_dy, n, st, out, nullptr);
}

gtls_status gtls_batch_create(gtls_plan* const* plans, int64_t n_lc, int32_t wave_slots, gtls_batch** out)
{
    if (!plans || !out) return fail(GTLS_ERR_INVALID_ARG, "null pointer argument");
    *out = nullptr;
    if (wave_slots < 0 || wave_slots > 65535) return fail(GTLS_ERR_INVALID_ARG, "wave_slots must be in [0, 65535]");
    g_last_error.clear();
    gtls_batch* b = new (std::nothrow) gtls_batch();
    if (!b) return fail(GTLS_ERR_OOM, "host allocation of the batch failed");
    gtls_status s;
    try {
        s = batch_create(plans, n_lc, wave_slots, b);
    } catch (const std::bad_alloc&) {
        s = fail(GTLS_ERR_OOM, "host allocation failed while building the batch");
    }
    if (s != GTLS_OK) {
        batch_release(b);
        delete b;
        return s;
    }
    *out = b;
    return GTLS_OK;
}

gtls_status gtls_batch_search(gtls_batch* b, const double* t, const double* y, const double* dy,
                              const int64_t* offsets, void* stream, gtls_result* out)
{
    if (!b) return fail(GTLS_ERR_INVALID_ARG, "null batch");
    g_last_error.clear();
    try {
        return batch_search(b, t, y, dy, offsets, static_cast<cudaStream_t>(stream), out);
    } catch (const std::bad_alloc&) {
        return fail(GTLS_ERR_OOM, "host allocation failed during the batch search");
    }
}

gtls_status gtls_batch_autotune(gtls_batch* b, const double* t, const double* y, const double* dy,
                                const int64_t* offsets, void* stream)
{
    if (!b) return fail(GTLS_ERR_INVALID_ARG, "null batch");
    g_last_error.clear();
    try {
        return batch_autotune(b, t, y, dy, offsets, static_cast<cudaStream_t>(stream));
    } catch (const std::bad_alloc&) {
        return fail(GTLS_ERR_OOM, "host allocation failed during autotuning");
    }
}

gtls_status gtls_batch_get_info(const gtls_batch* b, gtls_batch_info* o)
{
    if (!b || !o) return fail(GTLS_ERR_INVALID_ARG, "null pointer argument");
    std::memset(o, 0, sizeof *o);
    o->n_lc = b->n_lc;
    o->n_points = b->off.back();
    for (const gtls_plan* pl : b->plans) {
        o->n_periods += pl->dp.np;
        o->wpe += pl->host.wpe;
    }
    o->waves = b->waves;
    o->wave_slots = b->cfg.wave_slots;
    o->tile_floats = b->cfg.tile_buf;
    o->graph_kernels = b->graph_kernels;
    o->last_launches = b->last_launches;
    o->device_bytes = b->device_bytes;
    o->tuned = b->tuned ? 1 : 0;
    o->tuned_flops = b->tuned_rate;
    return GTLS_OK;
}

gtls_status gtls_batch_get_period_outputs(const gtls_batch* b, int64_t lc, const gtls_period_outputs* per,
                                          void* stream)
{
    if (!b || !per) return fail(GTLS_ERR_INVALID_ARG, "null pointer argument");
    if (lc < 0 || lc >= b->n_lc) return fail(GTLS_ERR_INVALID_ARG, "light curve index out of range");
    return copy_period_outputs(b->plans[(size_t)lc], per, static_cast<cudaStream_t>(stream));
}

void gtls_batch_destroy(gtls_batch* b)
{
    if (!b) return;
    int cur = -1;
    const bool switch_dev = cudaGetDevice(&cur) == cudaSuccess && cur != b->device && b->device >= 0;
    if (switch_dev) cudaSetDevice(b->device);
    batch_release(b);
    if (switch_dev) cudaSetDevice(cur);
    delete b;
}

gtls_status gtls_search_batch(gtls_plan* const* plans, int64_t n_lc, const double* t, const double* y,
                              const double* dy, const int64_t* offsets, void* stream, gtls_result* out)
{
    gtls_batch* b = nullptr;
    GTLS_TRY(gtls_batch_create(plans, n_lc, 0, &b));
    const gtls_status s = gtls_batch_search(b, t, y, dy, offsets, stream, out);
    const std::string err = g_last_error;
    gtls_batch_destroy(b);
    g_last_error = err;
    return s;
}

void gtls_plan_destroy(gtls_plan* pl)
{
    if (!pl) return;
    int cur = -1;
    const bool switch_dev = cudaGetDevice(&cur) == cudaSuccess && cur != pl->device && pl->device >= 0;
    if (switch_dev) cudaSetDevice(pl->device);
    release(pl);
    if (switch_dev) cudaSetDevice(cur);
    delete pl;
}

gtls_status gtls_plan_reserve(gtls_plan* pl)
{
    if (!pl) return fail(GTLS_ERR_INVALID_ARG, "null plan");
    g_last_error.clear();
    int dev = -1;
    GTLS_CUDA(cudaGetDevice(&dev));
    if (dev != pl->device) return fail(GTLS_ERR_INVALID_ARG, "current device differs from the plan's device");
    return ensure_chunk(pl);
}

gtls_status gtls_plan_trim(gtls_plan* pl)
{
    if (!pl) return fail(GTLS_ERR_INVALID_ARG, "null plan");
    g_last_error.clear();
    int dev = -1;
    GTLS_CUDA(cudaGetDevice(&dev));
    if (dev != pl->device) return fail(GTLS_ERR_INVALID_ARG, "current device differs from the plan's device");
    return trim_chunk(pl);
}

gtls_status gtls_plan_set_profiling(gtls_plan* pl, int32_t on)
{
    if (!pl) return fail(GTLS_ERR_INVALID_ARG, "null plan");
    pl->profiling = on != 0;
    return GTLS_OK;
}

gtls_status gtls_plan_get_profile(const gtls_plan* pl, gtls_profile* out)
{
    if (!pl || !out) return fail(GTLS_ERR_INVALID_ARG, "null pointer argument");
    *out = pl->profile;
    return GTLS_OK;
}

const char* gtls_last_error(void) { return g_last_error.c_str(); }

const char* gtls_status_string(gtls_status s)
{
    switch (s) {
    case GTLS_OK: return "GTLS_OK";
    case GTLS_ERR_INVALID_ARG: return "GTLS_ERR_INVALID_ARG";
    case GTLS_ERR_CUDA: return "GTLS_ERR_CUDA";
    case GTLS_ERR_OOM: return "GTLS_ERR_OOM";
    case GTLS_ERR_TIMEOUT: return "GTLS_ERR_TIMEOUT";
    case GTLS_ERR_INTERNAL: return "GTLS_ERR_INTERNAL";
    }
    return "GTLS_UNKNOWN";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free SR / SDE reduction
// ---------------------------------------------------------------------------
//
// For callers that cannot allocate device memory (for example code running
// inside a pre-sized memory pool, or a host process that hands all of its
// allocations to another framework): the reduction of Sect. 2.4 over a
// caller-owned chi2(P) spectrum, with its scratch (statistics, check words,
// argmax, and SR / SDE_raw when the caller passes no buffer for them) in a
// fixed file-scope device array instead of memory from cudaMalloc.  Every
// GPU that loads this library holds the array until the process exits.

namespace {

constexpr int64_t kNoAllocMaxPeriods = int64_t(1) << 19;  // 524,288 trial periods
constexpr int64_t kNoAllocHead = 32;                        // doubles before the SR / SDE_raw areas
// [0..4) stats  [4..8) check words  [8] best SDE  [9] best index (bits)
// [32 .. 32+max) SR   [32+max .. 32+2 max) SDE_raw
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocHead + 2 * kNoAllocMaxPeriods];

std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[64] = {};   // device address of g_noalloc_scratch per device

// Argmax of SDE (ties: lower index) and a check of the caller's chi2(P): every
// value must be finite and >= 0 (check 18); an argmax that finds no index
// (every SDE NaN) records check 17.
__global__ void __launch_bounds__(1024) k_argmax_noalloc(int np, const double* __restrict__ chi2,
                                                         const double* __restrict__ sde, double* head)
{
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    unsigned int* check = reinterpret_cast<unsigned int*>(head + 4);
    double v = -INFINITY;
    int idx = 0x7fffffff;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const double c = chi2[i];
        if (!(c >= 0.0 && c <= DBL_MAX)) record_check(check, 18, i, np);
        const double x = sde[i];
        if (x > v || (x == v && i < idx)) {
            v = x;
            idx = i;
        }
    }
    bv[threadIdx.x] = v;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double ov = bv[threadIdx.x + s];
            const int oi = bi[threadIdx.x + s];
            if (ov > bv[threadIdx.x] || (ov == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = ov;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (bi[0] < 0 || bi[0] >= np) record_check(check, 17, bi[0], np);
        head[8] = bv[0];
        head[9] = __longlong_as_double((long long)bi[0]);
    }
}

// Where `p` lives: device memory of the current device (or managed memory)
// is accepted, anything else rejected.  cudaPointerGetAttributes allocates
// nothing.
gtls_status noalloc_pointer(const void* p, int dev, const char* what)
{
    if (!p) return GTLS_OK;
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GTLS_ERR_INVALID_ARG, std::string(what) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(GTLS_ERR_INVALID_ARG, std::string(what) + " must be device memory");
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
        return fail(GTLS_ERR_INVALID_ARG, std::string(what) + " lives on device " + std::to_string(a.device) +
                                              ", not on the current device " + std::to_string(dev));
    return GTLS_OK;
}

// Device address of the scratch array on the current device; the first call
// on a device looks it up (and sets the median kernel's shared-memory limit).
gtls_status noalloc_scratch(int dev, double** out)
{
    if (dev < 0 || dev >= 64) return fail(GTLS_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        GTLS_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        GTLS_CUDA(cudaFuncSetAttribute(k_median_sde, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kMedianCap * (int)(sizeof(double) + sizeof(int))));
        g_noalloc_ptr[dev] = static_cast<double*>(ptr);
    }
    *out = g_noalloc_ptr[dev];
    return GTLS_OK;
}

}  // namespace

extern "C" gtls_status gtls_sr_sde_noalloc(const double* chi2, int64_t n_periods, int32_t median_window,
                                           void* stream, double* sr_out, double* sde_raw_out, double* sde_out,
                                           int64_t* best_idx, double* best_sde)
{
    g_last_error.clear();
    if (!chi2 || !sde_out) return fail(GTLS_ERR_INVALID_ARG, "chi2 and sde_out are required");
    if (n_periods < 1 || n_periods > kNoAllocMaxPeriods)
        return fail(GTLS_ERR_INVALID_ARG, "n_periods must be in [1, " + std::to_string(kNoAllocMaxPeriods) +
                                              "] for the allocation-free reduction");
    if (median_window < 0 || (median_window > 0 && median_window % 2 == 0))
        return fail(GTLS_ERR_INVALID_ARG, "median_window must be 0 or odd");
    const int np = (int)n_periods;
    const int win = median_window > 0 ? median_window : std::max(3, 2 * (np / 200) + 1);
    const int hwin = win / 2;
    const int outs = std::min(1024, kMedianCap - 2 * hwin) & ~31;
    if (outs < 32) return fail(GTLS_ERR_INVALID_ARG, "median window too large for the device median");
    int dev = -1;
    GTLS_CUDA(cudaGetDevice(&dev));
    GTLS_TRY(noalloc_pointer(chi2, dev, "chi2"));
    GTLS_TRY(noalloc_pointer(sde_out, dev, "sde_out"));
    GTLS_TRY(noalloc_pointer(sr_out, dev, "sr_out"));
    GTLS_TRY(noalloc_pointer(sde_raw_out, dev, "sde_raw_out"));
    double* head = nullptr;
    GTLS_TRY(noalloc_scratch(dev, &head));
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    DevPeriod dq{};
    dq.chi2 = const_cast<double*>(chi2);
    dq.sr = sr_out ? sr_out : head + kNoAllocHead;
    dq.sde_raw = sde_raw_out ? sde_raw_out : head + kNoAllocHead + kNoAllocMaxPeriods;
    dq.sde = sde_out;
    dq.stats = head;
    dq.check = reinterpret_cast<unsigned int*>(head + 4);
    // the array keeps the previous call's contents: clear the check words
    GTLS_CUDA(cudaMemsetAsync(head + 4, 0, 4 * sizeof(double), st));
    k_sr_stats<<<1, 1024, 0, st>>>(np, dq);
    GTLS_CUDA(cudaGetLastError());
    k_median_sde<<<(np + outs - 1) / outs, kMedianThreads, kMedianCap * (int)(sizeof(double) + sizeof(int)), st>>>(
        np, hwin, outs, dq);
    GTLS_CUDA(cudaGetLastError());
    k_argmax_noalloc<<<1, 1024, 0, st>>>(np, chi2, sde_out, head);
    GTLS_CUDA(cudaGetLastError());
    double res[2] = {0.0, 0.0};
    unsigned int chk[4] = {0, 0, 0, 0};
    GTLS_CUDA(cudaMemcpyAsync(res, head + 8, sizeof res, cudaMemcpyDeviceToHost, st));
    GTLS_CUDA(cudaMemcpyAsync(chk, head + 4, sizeof chk, cudaMemcpyDeviceToHost, st));
    GTLS_CUDA(cudaStreamSynchronize(st));
    if (chk[0] == 18)
        return fail(GTLS_ERR_INVALID_ARG, "chi2[" + std::to_string(chk[1]) + "] is not finite and >= 0");
    if (chk[0] != 0)
        return fail(GTLS_ERR_INTERNAL, "device index check " + std::to_string(chk[0]) + " failed");
    long long bidx = 0;
    std::memcpy(&bidx, &res[1], sizeof bidx);
    if (best_idx) *best_idx = bidx;
    if (best_sde) *best_sde = res[0];
    return GTLS_OK;
}
