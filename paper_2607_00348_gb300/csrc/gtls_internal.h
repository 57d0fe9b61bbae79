// Internal structures of libgtls shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "gtls.h"
#include "plan_host.h"

namespace gtls {

// Read-only plan tables on the device (passed to kernels by value).
struct DevPlan {
    int64_t n;
    int32_t np;           // periods
    int32_t nd;           // T14/P grid points
    int32_t time_exponent;
    int32_t idx_bits;
    int32_t bucket_log2;
    int32_t fold_nsb;      // super-buckets of the staged fold
    int32_t max_kept;
    const double* periods;
    const int64_t* p_lat;
    const float* inv_p;
    const int32_t* bucket_shift;
    const uint32_t* bucket_mul;
    const int32_t* jlo;
    const int32_t* jhi;
    const int32_t* dmax_p;
    const int32_t* dpts;
    const int32_t* stride;
    const int64_t* tmpl_off;
    const float* tmpl;
    const float* inv_sum_t;   // 1 / sum_k s_k
    const float* sum_t2;      // sum_k s_k^2
    const double* sum_t;      // FP64 sum_k s_k
    const double* q;
    int64_t tmpl_total;       // floats in tmpl
    const int32_t* cfg_variant; // window-kernel variant per duration (see window_tiles.cuh)
    const int32_t* cfg_nc;      // phase-column lanes per window block per duration
    const int64_t* tmpl2_off;   // offset of duration j in tmpl2 (float2 units)
    const float2* tmpl2;        // template pairs (s_k, s_{k+nc}) of column-pair durations
    const int64_t* tmplw_off;   // offset of duration j in tmplw (float2 units)
    const float2* tmplw;        // per-point weights: template pairs (s_k, s_k^2), zero padded
    const int32_t* cfg_nc_w;    // per-point weights: lanes per window block per duration
    int32_t median_half;        // half width h of the running-median window
    int32_t refine_k;           // periods re-searched with T0 step 1 (0: none)
    const int64_t* tc_off;      // offset of duration j in tc_tab (floats; kTensor durations)
    const float* tc_tab;        // tensor-core template chunks: [chunk][hi, lo][32 x 32 core-matrix layout]
};

// What the fold gathers for one point, in one 16-byte load.
struct alignas(16) PointVals {
    long long rfx;            // rint((1 - y) 2^40): exact window sums of r
    float r;                  // float(1 - y)
    float w;                  // float(1 / dy^2)
};

// Per-light-curve derived arrays (n long unless noted).
struct DevCurve {
    int64_t* d_lat;           // rint((t - t_ref) 2^e)
    float* d_f;               // float(t - t_ref) (days): coarse cycle estimate
    PointVals* pv;            // rfx, r, w of every point
    double* scal;             // [0] t_ref [1] chi2_0 [2] uniform weight w (0 if not uniform)
    unsigned long long* tmin_key;  // ordered key of min(t)
    unsigned int* flags;      // bit0 non-finite, bit1 dy <= 0, bit2 dy not uniform
    double* part;             // block partials of chi2_0
    unsigned int* check;      // [0] first failed device check (0 = none), [1..3] its values
};

// Per-chunk scratch: `chunk` periods in flight.
struct DevChunk {
    int32_t chunk;
    int64_t fold_stride;      // >= n
    int64_t key_stride;       // >= n and >= the super-bucket regions of the fold
    int64_t pad_stride;       // >= n + dmax + margin (folded, padded arrays)
    unsigned long long* keys; // fold keys (super-bucket regions, or bucket order)
    int32_t* sidx;            // folded order -> original index
    float* rs;                // folded r, padded by the period's first D_m points
    float* ws;                // folded w (per-point weights only)
    float* wrs;               // folded w r (per-point weights only)
    long long* pf;            // prefix sums of rfx over the padded folded curve
};

// Per-period outputs (np long) and the reduction scratch.
struct DevPeriod {
    unsigned long long* best; // packed (delta-chi2 key, j, window) minimum
    double* chi2;
    int32_t* dur;
    int32_t* t0i;
    double* depth;
    double* t0;
    double* sr;
    double* sde_raw;
    double* sde;
    double* stats;            // [0] chi2_min [1] mean SR [2] std SR
    unsigned int* check;      // same words as DevCurve::check
    int32_t* refined;         // 1 where the period was re-searched with T0 step 1
    int32_t* plist;           // the refine_k periods to re-search, in rank order
    gtls_result* result;      // device copy of the best candidate
};

// Tile shape of one light curve in the tiled window kernel.
struct DevTiles {
    int32_t len;              // window starts per tile (L)
    int32_t count;            // tiles per period
    int32_t len_w;            // the same for per-point weights (tiles of (w r, w) pairs)
    int32_t count_w;
};

// Per-light-curve descriptors of a search (device arrays, one entry per
// curve; a single search uses one entry).
struct DevSet {
    const DevPlan* plans;
    const DevCurve* curves;
    const DevPeriod* outs;
    const DevTiles* tiles;
};

// Which (light curve, period) each slot of a wave holds: a wave is up to
// kMaxSeg segments of consecutive periods (or consecutive positions of the
// curve's refinement list), passed by value.
constexpr int kMaxSeg = 32;
struct WaveSeg {
    int32_t lc;               // light curve
    int32_t first;            // first period (or refinement-list position)
    int32_t slot0;            // first slot of the segment in the wave
    int32_t item0;            // first window-tile item of the segment
};
struct SlotMap {
    int32_t nseg;
    int32_t slots;            // slots in the wave
    int32_t items;            // window-tile items in the wave
    int32_t from_list;        // periods are refinement-list positions
    WaveSeg seg[kMaxSeg];
};

// Records `msg` as the calling thread's last error and returns s (shared by
// the translation units behind the C ABI).
gtls_status set_error(gtls_status s, const std::string& msg);

}  // namespace gtls

struct gtls_plan {
    gtls::PlanHost host;
    int device = -1;
    gtls::DevPlan dp{};
    gtls::DevCurve dc{};
    gtls::DevChunk dk{};
    gtls::DevPeriod dq{};
    double* in_t = nullptr;   // plan-owned input buffers of gtls_search_host
    double* in_y = nullptr;
    double* in_dy = nullptr;
    int64_t device_bytes = 0;
    // tiled window search (uniform weights; per-point weights: tile_w_*, in
    // (w r, w) pairs)
    bool tile_ok = false;
    int tile_buf = 0, tile_len = 0, tile_count = 0;
    bool tile_w_ok = false;
    int tile_buf_w = 0, tile_len_w = 0, tile_count_w = 0;
    // durations too long for a tile (marked kWindowOnly): searched by the
    // one-thread-per-window kernel in the same waves
    bool has_window_only = false, has_window_only_ref = false;
    // durations on the tensor-core window kernel (kTensor), the widest
    // [jlo, jhi] span of a period (work items per period of that kernel),
    // its counter, and the timeout test (a wait that nothing completes)
    bool has_tensor = false;
    int tc_jspan = 0;
    unsigned int* tc_counter = nullptr;
    int tc_test_wait = 0;
    const void* tc_maps = nullptr;      // TMA maps of dk.rs (made with the chunk scratch)
    std::vector<int32_t> variant_host;   // window-kernel variant per duration (host copy)
    int n_sm = 0;
    unsigned int* tile_counter = nullptr;
    // refinement stage (T0 step 1 on the best periods): plan tables with
    // stride 1 and the (s_k, 1) pair tables, its tile configuration and the
    // device list of periods to re-search
    int refine_k = 0;
    gtls::DevPlan dp_ref{};
    int tile_len_ref = 0, tile_count_ref = 0;
    // one-entry device descriptor sets of the coarse and refinement passes
    gtls::DevSet set{}, set_ref{};
    int64_t* prep_off = nullptr;        // device {0, n}: the curve's offsets
    bool chunk_ready = false;           // dk allocated (first single search or gtls_plan_reserve)
    int64_t chunk_bytes = 0;            // device bytes of the chunk scratch
    std::vector<float> tmpl_pad;        // host copy of the zero-padded template table
    std::vector<int64_t> tmpl_pad_off;
    // stage profiling: events recorded on the search stream when enabled
    bool profiling = false;
    std::vector<cudaEvent_t> events;
    std::vector<int> event_stage;   // stage of the interval ending at event i
    gtls_profile profile{};
    void* allocs[96] = {};
    int n_allocs = 0;
};
