/*
 * FP64 CPU oracle of the TLS period search (test infrastructure only).
 *
 * This file is test infrastructure.  Only tests/, __graft_entry__.smoke()
 * and bench.py's cpu_baseline / reference legs may build, load or call it.
 * It shares no code with the CUDA library.
 *
 * For every requested trial period it follows the steps of Sect. 2.3 in the
 * paper's order, in double precision, with no blocking or fusion:
 *   1. fold: phase of every point on the exact 2^-e-day lattice
 *      (Eq. phase; rho_i = d_i mod P_int, phase = rho_i / P_int);
 *   2. sort by phase, ties by original index (a stable sort);
 *   3. pad: append the first D_m folded points (Sect. 2.3.2, Fig. patch),
 *      D_m = the largest duration this period searches;
 *   4. edge term chi2_edge over the first D_m folded points (Eq. edge,
 *      index read as the duplicated points 1..D_m);
 *   5. cumulative sum F_cum of the padded flux; moving average
 *      F_avg = (F_cum(s+D) - F_cum(s)) / D (Eq. cumsum);
 *   6. depth: delta = max(0, (1 - F_avg) / mean(template)) (Eqs. k, depth:
 *      the mean in-window flux deficit scaled by the template's mean);
 *   7. out-of-transit chi2 = chi2_out_a + chi2_out_b - chi2_edge (Eq. out)
 *      from running sums of ((f - 1)/dy)^2 over the padded curve;
 *   8. in-transit chi2 as a direct point-by-point sum (Eq. in);
 *   9. chi2(P) = min over durations (ascending) and T0 starts
 *      s = 0, st, 2 st, ... < N, st = max(1, floor(D dt0)) (Eq. N_skip);
 *      a later candidate replaces the best only when strictly smaller.
 * The running median used to detrend SDE (Sect. 2.4) is also here.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t rho;
    int64_t idx;
} fold_key;

static int cmp_fold_key(const void* a, const void* b)
{
    const fold_key* x = (const fold_key*)a;
    const fold_key* y = (const fold_key*)b;
    if (x->rho != y->rho) return x->rho < y->rho ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

/* Search one trial period.  Outputs the minimum chi2 and where it occurs. */
static void search_one_period(int64_t n, const double* y, const double* dy,
                              const int64_t* d_lat, int64_t p_int,
                              int64_t jlo, int64_t jhi, const int64_t* dur_pts,
                              const int64_t* tmpl_off, const double* tmpl,
                              double dt0, fold_key* keys, double* f, double* e,
                              double* fcum, double* r2cum,
                              double* chi2_out, int64_t* j_out, int64_t* s_out,
                              double* depth_out, int64_t* rho_c_out)
{
    /* 1-2. fold and stable sort by phase */
    for (int64_t i = 0; i < n; i++) {
        keys[i].rho = d_lat[i] % p_int;
        keys[i].idx = i;
    }
    qsort(keys, (size_t)n, sizeof(fold_key), cmp_fold_key);

    /* largest duration of this period */
    int64_t d_m = 0;
    for (int64_t j = jlo; j <= jhi; j++)
        if (dur_pts[j] > d_m) d_m = dur_pts[j];
    if (d_m > n) d_m = n;

    /* 3. padded folded curve, N_p = N + D_m */
    const int64_t np_ = n + d_m;
    for (int64_t k = 0; k < n; k++) {
        f[k] = y[keys[k].idx];
        e[k] = dy[keys[k].idx];
    }
    for (int64_t k = 0; k < d_m; k++) {
        f[n + k] = f[k];
        e[n + k] = e[k];
    }

    /* 4. edge term over the duplicated points */
    double chi2_edge = 0.0;
    for (int64_t k = 0; k < d_m; k++) {
        const double z = (1.0 - f[k]) / e[k];
        chi2_edge += z * z;
    }

    /* 5. cumulative sums of flux and of the out-of-transit residual^2 */
    fcum[0] = 0.0;
    r2cum[0] = 0.0;
    for (int64_t k = 0; k < np_; k++) {
        const double z = (f[k] - 1.0) / e[k];
        fcum[k + 1] = fcum[k] + f[k];
        r2cum[k + 1] = r2cum[k] + z * z;
    }

    double best = INFINITY;
    int64_t best_j = -1, best_s = -1;
    double best_depth = 0.0;
    for (int64_t j = jlo; j <= jhi; j++) {
        if (j > jlo && dur_pts[j] == dur_pts[j - 1]) continue; /* first of equal D */
        const int64_t d = dur_pts[j];
        if (d > n) continue;
        const double* s_t = tmpl + tmpl_off[j];
        double s_sum = 0.0;
        for (int64_t k = 0; k < d; k++) s_sum += s_t[k];
        const double s_mean = s_sum / (double)d;
        int64_t st = (int64_t)floor((double)d * dt0);
        if (st < 1) st = 1;
        for (int64_t s = 0; s < n; s += st) {
            /* 6. depth from the moving average */
            const double f_avg = (fcum[s + d] - fcum[s]) / (double)d;
            double depth = (1.0 - f_avg) / s_mean;
            if (depth < 0.0) depth = 0.0;
            /* 7. out of transit: before s, after s + D, minus the edge term */
            const double out_a = r2cum[s];
            const double out_b = r2cum[np_] - r2cum[s + d];
            const double c_out = out_a + out_b - chi2_edge;
            /* 8. in transit, point by point */
            double c_in = 0.0;
            for (int64_t k = 0; k < d; k++) {
                const double model = 1.0 - depth * s_t[k];
                const double z = (f[s + k] - model) / e[s + k];
                c_in += z * z;
            }
            const double c = c_out + c_in;
            if (c < best) {
                best = c;
                best_j = j;
                best_s = s;
                best_depth = depth;
            }
        }
    }
    *chi2_out = best;
    *j_out = best_j;
    *s_out = best_s;
    *depth_out = best_depth;
    if (best_j >= 0) {
        const int64_t c = (best_s + dur_pts[best_j] / 2) % n;
        *rho_c_out = keys[c].rho;
    } else {
        *rho_c_out = 0;
    }
}

/*
 * Search the periods listed in sel[0..n_sel).  Per selected period k the
 * outputs are chi2[k], j_best[k] (global duration index), s_best[k] (window
 * start in folded order), depth[k] and rho_c[k] (lattice phase of the
 * window's centre point, for T0).  Returns 0, or -1 on allocation failure.
 */
int tls_oracle_search(int64_t n, const double* y, const double* dy,
                      const int64_t* d_lat, const int64_t* p_int,
                      const int64_t* jlo, const int64_t* jhi,
                      const int64_t* dur_pts, const int64_t* tmpl_off,
                      const double* tmpl, double dt0,
                      int64_t n_sel, const int64_t* sel,
                      double* chi2, int64_t* j_best, int64_t* s_best,
                      double* depth, int64_t* rho_c, int n_threads)
{
    int64_t d_max = 0;
    for (int64_t k = 0; k < n_sel; k++) {
        const int64_t p = sel[k];
        for (int64_t j = jlo[p]; j <= jhi[p]; j++)
            if (dur_pts[j] > d_max) d_max = dur_pts[j];
    }
    if (d_max > n) d_max = n;
    int failed = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        fold_key* keys = (fold_key*)malloc(sizeof(fold_key) * (size_t)n);
        double* f = (double*)malloc(sizeof(double) * (size_t)(n + d_max));
        double* e = (double*)malloc(sizeof(double) * (size_t)(n + d_max));
        double* fcum = (double*)malloc(sizeof(double) * (size_t)(n + d_max + 1));
        double* r2cum = (double*)malloc(sizeof(double) * (size_t)(n + d_max + 1));
        const int ok = keys && f && e && fcum && r2cum;
        if (!ok) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            failed = 1;
        }
        /* every thread reaches the work-sharing loop; one without buffers skips */
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t k = 0; k < n_sel; k++) {
            if (!ok) continue;
            const int64_t p = sel[k];
            search_one_period(n, y, dy, d_lat, p_int[p], jlo[p], jhi[p],
                              dur_pts, tmpl_off, tmpl, dt0, keys, f, e,
                              fcum, r2cum, &chi2[k], &j_best[k], &s_best[k],
                              &depth[k], &rho_c[k]);
        }
        free(keys);
        free(f);
        free(e);
        free(fcum);
        free(r2cum);
    }
    return failed ? -1 : 0;
}

/* Number of threads an OpenMP parallel region gets with n_threads (0 = default). */
int tls_oracle_threads(int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) return n_threads;
    return omp_get_max_threads();
#else
    (void)n_threads;
    return 1;
#endif
}

static int cmp_double(const void* a, const void* b)
{
    const double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/*
 * Running median of v[0..n) with an odd window w = 2h + 1, truncated at the
 * ends, lower median for even counts.  A sorted copy of the window is kept
 * and updated by one insertion and one deletion per step.
 */
int tls_oracle_running_median(int64_t n, const double* v, int64_t w, double* out)
{
    if (n <= 0) return 0;
    const int64_t h = w / 2;
    double* win = (double*)malloc(sizeof(double) * (size_t)(2 * h + 2));
    if (!win) return -1;
    int64_t lo = 0, hi = (h < n - 1) ? h : n - 1; /* window [lo, hi] */
    int64_t cnt = hi - lo + 1;
    for (int64_t k = 0; k < cnt; k++) win[k] = v[lo + k];
    qsort(win, (size_t)cnt, sizeof(double), cmp_double);
    for (int64_t i = 0; i < n; i++) {
        out[i] = win[(cnt - 1) / 2];
        if (i + 1 >= n) break;
        /* next window [max(0, i+1-h), min(n-1, i+1+h)] */
        const int64_t nlo = (i + 1 - h > 0) ? i + 1 - h : 0;
        const int64_t nhi = (i + 1 + h < n - 1) ? i + 1 + h : n - 1;
        if (nlo > lo) { /* remove v[lo] */
            const double x = v[lo];
            int64_t k = 0;
            while (k < cnt && win[k] != x) k++;
            memmove(win + k, win + k + 1, sizeof(double) * (size_t)(cnt - k - 1));
            cnt--;
            lo = nlo;
        }
        if (nhi > hi) { /* insert v[nhi] */
            const double x = v[nhi];
            int64_t k = cnt;
            while (k > 0 && win[k - 1] > x) {
                win[k] = win[k - 1];
                k--;
            }
            win[k] = x;
            cnt++;
            hi = nhi;
        }
    }
    free(win);
    return 0;
}

/* Folded order of one period: order[k] = index of the k-th point by phase. */
int tls_oracle_fold_order(int64_t n, const int64_t* d_lat, int64_t p_int, int64_t* order)
{
    fold_key* keys = (fold_key*)malloc(sizeof(fold_key) * (size_t)n);
    if (!keys) return -1;
    for (int64_t i = 0; i < n; i++) {
        keys[i].rho = d_lat[i] % p_int;
        keys[i].idx = i;
    }
    qsort(keys, (size_t)n, sizeof(fold_key), cmp_fold_key);
    for (int64_t k = 0; k < n; k++) order[k] = keys[k].idx;
    free(keys);
    return 0;
}

/*
 * Every window of one period and one duration D (template s_t[0..D)), by
 * the padded decomposition: chi2[m] and depth[m] for s = m*st, m < ceil(N/st).
 * d_m is the padding length (the period's largest duration).  Used by the
 * brute-force tests to pin the decomposition window by window.
 */
int tls_oracle_period_windows(int64_t n, const double* y, const double* dy,
                              const int64_t* d_lat, int64_t p_int, int64_t d_m,
                              int64_t d, const double* s_t, double dt0,
                              double* chi2, double* depth)
{
    fold_key* keys = (fold_key*)malloc(sizeof(fold_key) * (size_t)n);
    double* f = (double*)malloc(sizeof(double) * (size_t)(n + d_m));
    double* e = (double*)malloc(sizeof(double) * (size_t)(n + d_m));
    double* fcum = (double*)malloc(sizeof(double) * (size_t)(n + d_m + 1));
    double* r2cum = (double*)malloc(sizeof(double) * (size_t)(n + d_m + 1));
    int rc = 0;
    if (!keys || !f || !e || !fcum || !r2cum || d > d_m || d_m > n) {
        rc = -1;
        goto done;
    }
    for (int64_t i = 0; i < n; i++) {
        keys[i].rho = d_lat[i] % p_int;
        keys[i].idx = i;
    }
    qsort(keys, (size_t)n, sizeof(fold_key), cmp_fold_key);
    const int64_t np_ = n + d_m;
    for (int64_t k = 0; k < n; k++) {
        f[k] = y[keys[k].idx];
        e[k] = dy[keys[k].idx];
    }
    for (int64_t k = 0; k < d_m; k++) {
        f[n + k] = f[k];
        e[n + k] = e[k];
    }
    double chi2_edge = 0.0;
    for (int64_t k = 0; k < d_m; k++) {
        const double z = (1.0 - f[k]) / e[k];
        chi2_edge += z * z;
    }
    fcum[0] = 0.0;
    r2cum[0] = 0.0;
    for (int64_t k = 0; k < np_; k++) {
        const double z = (f[k] - 1.0) / e[k];
        fcum[k + 1] = fcum[k] + f[k];
        r2cum[k + 1] = r2cum[k] + z * z;
    }
    double s_sum = 0.0;
    for (int64_t k = 0; k < d; k++) s_sum += s_t[k];
    const double s_mean = s_sum / (double)d;
    int64_t st = (int64_t)floor((double)d * dt0);
    if (st < 1) st = 1;
    int64_t m = 0;
    for (int64_t s = 0; s < n; s += st, m++) {
        const double f_avg = (fcum[s + d] - fcum[s]) / (double)d;
        double dep = (1.0 - f_avg) / s_mean;
        if (dep < 0.0) dep = 0.0;
        const double c_out = r2cum[s] + (r2cum[np_] - r2cum[s + d]) - chi2_edge;
        double c_in = 0.0;
        for (int64_t k = 0; k < d; k++) {
            const double z = (f[s + k] - (1.0 - dep * s_t[k])) / e[s + k];
            c_in += z * z;
        }
        chi2[m] = c_out + c_in;
        depth[m] = dep;
    }
done:
    free(keys);
    free(f);
    free(e);
    free(fcum);
    free(r2cum);
    return rc;
}
