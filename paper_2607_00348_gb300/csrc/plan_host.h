// Host-side search plan: period grid, duration grid, templates, phase lattice.
// Pure C++17 in FP64; no CUDA.  Built into libgtls.so by the package build.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "gtls.h"

namespace gtls {

struct PlanHost {
    gtls_plan_params prm{};          // copy of the user parameters (periods pointer cleared)
    int64_t n = 0;                   // points per light curve
    double baseline_days = 0.0;

    // period grid (ascending) and its exact phase lattice
    std::vector<double> periods;     // days
    std::vector<int64_t> p_lat;      // rint(P 2^e)
    std::vector<float> inv_p;        // float(1 / P) (days^-1): coarse cycle estimate
    std::vector<int32_t> bucket_shift;   // see fold bucket map in search.cu
    std::vector<uint32_t> bucket_mul;
    int time_exponent = 0;           // e
    int idx_bits = 0;                // bits of the point index in a fold key
    int bucket_log2 = 0;             // log2 of fold buckets per period

    // global T14/P grid
    std::vector<double> q;           // q_j
    std::vector<int32_t> dpts;       // D_j
    std::vector<int32_t> stride;     // max(1, floor(D_j dt0))
    std::vector<int64_t> tmpl_off;   // offset of template j in tmpl
    std::vector<float> tmpl;         // s_k of every j, FP32
    std::vector<double> sum_t;       // sum_k s_k (FP64 of the FP32 values)
    std::vector<double> sum_t2;      // sum_k s_k^2

    // per-period duration range [jlo, jhi] and derived sizes
    std::vector<int32_t> jlo, jhi;
    std::vector<int32_t> dmax_p;     // largest D of the period (padding length)
    int32_t max_kept = 0;            // most distinct durations of any period
    int64_t dmax = 0;                // largest D of any period
    int64_t n_windows = 0;
    double wpe = 0.0;
    int32_t median_window = 0;
};

// Build the plan; returns false and sets err on invalid parameters.
bool build_plan_host(const gtls_plan_params& p, PlanHost& out, std::string& err);

// 1 if duration j is the first of its D inside [jlo, jhi] (duplicates are skipped).
inline bool kept_duration(const PlanHost& h, int32_t j, int32_t jlo)
{
    return j == jlo || h.dpts[j] != h.dpts[j - 1];
}

}  // namespace gtls
