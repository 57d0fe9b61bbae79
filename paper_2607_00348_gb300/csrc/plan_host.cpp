// Host-side plan of the TLS period search: grids, template table, phase lattice.
//
// Period grid: the cubic frequency sampling of Ofir (2014) as given in
// Sect. 2.2.1, Eqs. (f_min), (f_max), (f_i), (C, A), (N).  Duration grid:
// the envelope k_min P^(-2/3) <= T14/P <= min(q_cap, k_max P^(-2/3)) of
// Sect. 2.2.2, Eqs. (upper), (lower), sampled by one geometric T14/P grid.
// Template: central small-planet transit with quadratic limb darkening.
// Everything here is FP64 host arithmetic; the device receives the tables.
#include "plan_host.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>

namespace gtls {

namespace {

constexpr double kGMSun = 1.3271244e20;  // m^3 s^-2, IAU 2015 nominal
constexpr double kRSun = 6.957e8;        // m, IAU 2015 nominal
constexpr double kDay = 86400.0;         // s
constexpr double kPi = 3.141592653589793;

std::string fmt(const char* f, double a, double b = 0.0)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, f, a, b);
    return buf;
}

int bit_length(uint64_t v)
{
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

}  // namespace

bool build_plan_host(const gtls_plan_params& p, PlanHost& h, std::string& err)
{
    h = PlanHost{};
    h.prm = p;
    h.prm.periods_days = nullptr;
    h.n = p.n_points;
    h.baseline_days = p.baseline_days;
    if (p.n_points < 2) { err = "n_points must be >= 2"; return false; }
    if (p.n_points > (int64_t(1) << 24)) { err = "n_points must be <= 2^24"; return false; }
    if (!(p.baseline_days > 0.0) || !std::isfinite(p.baseline_days)) {
        err = "baseline_days must be > 0"; return false;
    }
    if (!(p.oversampling > 0.0) || !(p.m_star > 0.0) || !(p.r_star > 0.0)) {
        err = "oversampling, m_star, r_star must be > 0"; return false;
    }
    if (!(p.k_min > 0.0) || !(p.k_max > p.k_min) || !(p.q_cap > 0.0) || p.q_cap > 1.0) {
        err = "need 0 < k_min < k_max and 0 < q_cap <= 1"; return false;
    }
    if (!(p.dur_ratio > 1.0) || !(p.dt0 > 0.0) || p.dt0 > 1.0) {
        err = "need dur_ratio > 1 and 0 < dt0 <= 1"; return false;
    }
    if (p.refine_periods < 0 || p.refine_periods > 65535) {
        err = "refine_periods must be in [0, 65535]"; return false;
    }
    if (p.periods_per_chunk < 0 || p.periods_per_chunk > 65535) {
        err = "periods_per_chunk must be in [0, 65535]"; return false;
    }
    if (p.median_window < 0 || (p.median_window > 0 && p.median_window % 2 == 0)) {
        err = "median_window must be 0 or odd"; return false;
    }

    // ---- period grid ------------------------------------------------------
    if (p.periods_days && p.n_periods > 0) {
        h.periods.assign(p.periods_days, p.periods_days + p.n_periods);
        for (double v : h.periods)
            if (!(v > 0.0) || !std::isfinite(v)) { err = "explicit periods must be > 0"; return false; }
        std::sort(h.periods.begin(), h.periods.end());
    } else {
        const double s_sec = p.baseline_days * kDay;
        const double gm = kGMSun * p.m_star;
        const double rad = kRSun * p.r_star;
        const double f_min = p.period_max_days > 0.0 ? 1.0 / (p.period_max_days * kDay) : 2.0 / s_sec;
        const double f_max = p.period_min_days > 0.0
                                 ? 1.0 / (p.period_min_days * kDay)
                                 : std::sqrt(gm / std::pow(3.0 * rad, 3.0)) / (2.0 * kPi);
        if (!(f_max > f_min)) {
            err = fmt("empty period range: P_min %.9g d >= P_max %.9g d", 1.0 / (f_max * kDay),
                      1.0 / (f_min * kDay));
            return false;
        }
        const double a = std::pow(2.0 * kPi, 2.0 / 3.0) / kPi * rad / std::cbrt(gm) /
                         (s_sec * p.oversampling);
        const double c = std::cbrt(f_min) - a / 3.0;
        const double n_real = (std::cbrt(f_max) - std::cbrt(f_min) + a / 3.0) * 3.0 / a;
        if (!(n_real < 5.0e7)) { err = "period grid larger than 5e7 points"; return false; }
        const int64_t n_int = (int64_t)std::ceil(n_real);
        const double lo_f = f_min * (1.0 - 1e-12), hi_f = f_max * (1.0 + 1e-12);
        std::vector<double> f;
        f.reserve((size_t)n_int);
        for (int64_t i = 1; i <= n_int; ++i) {
            const double x = a / 3.0 * (double)i + c;
            const double fi = x * x * x;
            if (fi >= lo_f && fi <= hi_f) f.push_back(fi);
        }
        h.periods.resize(f.size());
        for (size_t i = 0; i < f.size(); ++i) h.periods[i] = 1.0 / (f[i] * kDay);
        std::sort(h.periods.begin(), h.periods.end());
    }
    const int64_t np_ = (int64_t)h.periods.size();
    if (np_ < 1) { err = "period grid is empty"; return false; }
    const double p_max = h.periods.back();
    const double p_min = h.periods.front();

    // ---- phase lattice ------------------------------------------------------
    h.idx_bits = std::max(1, bit_length((uint64_t)(h.n - 1)));
    {
        int ex = 0;
        const double m = std::frexp(p_max, &ex);  // p_max = m 2^ex, m in [0.5, 1)
        const int ceil_log2 = (m == 0.5) ? ex - 1 : ex;
        h.time_exponent = std::min(40, 64 - h.idx_bits - 1 - ceil_log2);
    }
    if (h.time_exponent < 8) { err = "periods too long for the phase lattice"; return false; }
    // the float cycle estimate is off by at most one when S/P_min < 2^22
    if (p.baseline_days / p_min > 4.0e6) { err = "baseline / P_min exceeds 4e6 cycles"; return false; }
    const double scale = std::ldexp(1.0, h.time_exponent);
    h.bucket_log2 = std::min(13, std::max(6, bit_length((uint64_t)h.n) - 1));
    const uint64_t nbuckets = uint64_t(1) << h.bucket_log2;
    h.p_lat.resize(np_);
    h.inv_p.resize(np_);
    h.bucket_shift.resize(np_);
    h.bucket_mul.resize(np_);
    for (int64_t i = 0; i < np_; ++i) {
        const int64_t pl = (int64_t)std::llrint(h.periods[i] * scale);
        if (pl < (int64_t(1) << 32)) { err = "periods too short for the phase lattice"; return false; }
        h.p_lat[i] = pl;
        h.inv_p[i] = (float)(1.0 / h.periods[i]);
        const int sh = std::max(0, bit_length((uint64_t)pl) - 32);
        const uint64_t top = ((uint64_t)pl >> sh) + 1;  // > every (rho >> sh)
        h.bucket_shift[i] = sh;
        h.bucket_mul[i] = (uint32_t)((nbuckets << 32) / top);
    }

    // ---- duration grid ------------------------------------------------------
    std::vector<double> lo(np_), hi(np_);
    double q_top = 0.0;
    for (int64_t i = 0; i < np_; ++i) {
        const double p23 = std::pow(h.periods[i] * kDay, -2.0 / 3.0);
        lo[i] = p.k_min * p23;
        hi[i] = std::min(p.q_cap, p.k_max * p23);
        q_top = std::max(q_top, hi[i]);
    }
    const double q_lo = lo[np_ - 1];  // k_min P_max^(-2/3), the smallest lower bound
    for (int j = 0;; ++j) {
        const double qj = q_lo * std::pow(p.dur_ratio, (double)j);
        if (qj > q_top) break;
        h.q.push_back(qj);
        if (h.q.size() > 4096) { err = "duration grid larger than 4096 points"; return false; }
    }
    const int32_t nd = (int32_t)h.q.size();
    if (nd < 1) { err = "duration grid is empty"; return false; }
    if (nd > 255) { err = "more than 255 durations (raise dur_ratio)"; return false; }
    h.dpts.resize(nd);
    h.stride.resize(nd);
    for (int32_t j = 0; j < nd; ++j) {
        const int64_t d = std::max<int64_t>(1, (int64_t)std::floor(h.q[j] * (double)h.n + 0.5));
        h.dpts[j] = (int32_t)std::min<int64_t>(d, h.n);
        h.stride[j] = (int32_t)std::max<int64_t>(1, (int64_t)std::floor((double)h.dpts[j] * p.dt0));
    }
    h.jlo.resize(np_);
    h.jhi.resize(np_);
    h.dmax_p.resize(np_);
    for (int64_t i = 0; i < np_; ++i) {
        // first q_j >= lo, last q_j <= hi (the grid is increasing)
        const int32_t a = (int32_t)(std::lower_bound(h.q.begin(), h.q.end(), lo[i]) - h.q.begin());
        const int32_t b = (int32_t)(std::upper_bound(h.q.begin(), h.q.end(), hi[i]) - h.q.begin()) - 1;
        if (a > b) {
            err = fmt("period %.9g d has no admissible duration (raise k_max or lower dur_ratio)",
                      h.periods[i]);
            return false;
        }
        h.jlo[i] = a;
        h.jhi[i] = b;
        int32_t kept = 0, dm = 0;
        for (int32_t j = a; j <= b; ++j) {
            if (!kept_duration(h, j, a)) continue;
            ++kept;
            dm = std::max(dm, h.dpts[j]);
            const int64_t m = (h.n + h.stride[j] - 1) / h.stride[j];
            h.n_windows += m;
            h.wpe += (double)m * (double)h.dpts[j];
        }
        h.dmax_p[i] = dm;
        h.max_kept = std::max(h.max_kept, kept);
        h.dmax = std::max<int64_t>(h.dmax, dm);
    }

    // ---- templates (one per grid point j, FP64 -> FP32) ----------------------
    h.tmpl_off.resize(nd);
    h.sum_t.resize(nd);
    h.sum_t2.resize(nd);
    int64_t off = 0;
    for (int32_t j = 0; j < nd; ++j) {
        h.tmpl_off[j] = off;
        off += h.dpts[j];
    }
    h.tmpl.resize((size_t)off);
    for (int32_t j = 0; j < nd; ++j) {
        const int32_t d = h.dpts[j];
        double s1 = 0.0, s2 = 0.0;
        for (int32_t k = 0; k < d; ++k) {
            const double x = ((double)k + 0.5) / (double)d;
            const double rr = std::fabs(2.0 * x - 1.0);
            const double mu = std::sqrt(1.0 - rr * rr);
            const double om = 1.0 - mu;
            const double s = 1.0 - p.u1 * om - p.u2 * (om * om);
            const float sf = (float)s;
            h.tmpl[(size_t)(h.tmpl_off[j] + k)] = sf;
            s1 += (double)sf;
            s2 += (double)sf * (double)sf;
        }
        h.sum_t[j] = s1;
        h.sum_t2[j] = s2;
        if (!(s1 > 0.0)) { err = "template with a non-positive sum (check u1, u2)"; return false; }
    }

    h.median_window = p.median_window > 0 ? p.median_window
                                          : (int32_t)std::max<int64_t>(3, 2 * (np_ / 200) + 1);
    return true;
}

}  // namespace gtls
