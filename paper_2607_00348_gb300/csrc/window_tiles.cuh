// Tiled window search of one chunk of periods (uniform weights).
//
// This is the hot path of the search: for every period, every duration D of
// the period and every T0 start s = m st (st = max(1, floor(D dt0)),
// Eq. N_skip) it forms C1(m) = sum_k r[s+k] s_k over the folded, padded
// curve (the in-transit sum of Eq. in, expanded) and, with the exact window
// sum S(m) of r from the prefix array (Eq. cumsum), the depth
// delta = max(0, S / sum_k s_k) (Eqs. k, depth) and
// chi2 - chi2_0 = w delta (delta sum_k s_k^2 - 2 C1) (Eqs. out, in).
//
// Work decomposition (one persistent CTA per SM):
//   item  = (period, tile of L window starts); the CTA stages the tile's
//           folded curve [x0, x0 + BUF) in shared memory once and evaluates
//           every duration of the period on it.
//   task  = one warp, one duration, 32 W / nc consecutive windows.
//           Lane (b, c): block b of W consecutive windows, phase class c of
//           the T0 stride (rho = c, c + nc, ...; rows of st points).  For a
//           fixed rho, window w needs rows w .. w+J-1 of column rho, so a
//           register window slides down the rows: one shared load feeds W
//           FMAs.  Pairs of windows (w, w + W/2) share one FFMA2.
//           nc and W are chosen so that the lanes of a warp hit 32 distinct
//           shared-memory banks: W st = nc * odd (mod 32).
//   The nc lanes of a block add their partial sums with a butterfly; each
//   lane then finishes W / nc windows and keeps a packed running minimum
//   (delta-chi2 key, duration index, window index), merged per period
//   with one 64-bit atomicMin.
#pragma once

namespace gtls {
namespace tiles {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxDur = 64;

enum Variant : int { kScalar15 = 0, kPair16 = 1, kPair14 = 2, kPair12 = 3, kPair8 = 4 };

struct DurTask {
    int j, d, st, nc, variant, w, per_task, tasks, first, m_a, m_b, hi_start, m_total;
};

__device__ __forceinline__ int variant_w(int v)
{
    return v == kScalar15 ? 15 : v == kPair16 ? 16 : v == kPair14 ? 14 : v == kPair12 ? 12 : 8;
}

// Pick (variant, nc) for a duration with T0 step st and `nwin` windows in the tile.
__device__ void pick_config(int st, int nwin, int& variant, int& nc)
{
    const int v = min(5, __ffs(st) - 1);
    float best = -1.0f;
    variant = kPair16;
    nc = 32;
    auto consider = [&](int var, int c_nc, float ipc) {
        if (c_nc > 32) return;
        const int w = variant_w(var);
        const int rounds = (st + c_nc - 1) / c_nc;
        const float util = (float)st / (float)(c_nc * rounds);
        const int per = 32 * w / c_nc;
        const int tasks = (nwin + per - 1) / per;
        const float fill = (float)nwin / (float)(tasks * per);
        const float eff = util * fill * ipc;
        if (eff > best) {
            best = eff;
            variant = var;
            nc = c_nc;
        }
    };
    consider(kPair16, 32, 1.0f);
    if (v <= 4) consider(kScalar15, 1 << v, 0.85f);
    if (v + 1 <= 5) consider(kPair14, 1 << (v + 1), 1.0f);
    if (v + 2 <= 5) consider(kPair12, 1 << (v + 2), 1.0f);
    if (v + 3 <= 5) consider(kPair8, 1 << (v + 3), 0.9f);
    if (v + 4 <= 5) consider(kPair16, 1 << (v + 4), 1.0f);
}

struct WinCtx {
    const float* tile;        // shared: folded r at x0 .. x0 + BUF
    int x0;
    int d, st, nc, lg_nc;
    int m_first;              // first window of this warp task
    int m_a, m_b, hi_start, m_total;
    const float* tg;          // template of the duration (global)
    float inv_sum_t, sum_t2, w_uni;
    int j;
    const long long* pf;      // prefix sums of the period (global)
};

__device__ __forceinline__ unsigned long long finish_window(const WinCtx& c, long long m, float c1)
{
    const long long s = m * c.st;
    const long long sfx = c.pf[s + c.d] - c.pf[s];
    const float sum_r = (float)((double)sfx * (1.0 / 1099511627776.0));
    const float depth = fmaxf(0.0f, sum_r * c.inv_sum_t);
    const float dchi = c.w_uni * depth * fmaf(depth, c.sum_t2, -2.0f * c1);
    unsigned int u = __float_as_uint(dchi);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | ((unsigned long long)c.j << 24) | (unsigned long long)m;
}

// Butterfly over the nc lanes of a block, then lane c finishes the windows
// w with w mod nc == c.
template <int W>
__device__ __forceinline__ void reduce_finish(const WinCtx& c, float (&tot)[W], int mb, bool active,
                                              int lane, unsigned long long& best)
{
    for (int o = 1; o < c.nc; o <<= 1) {
#pragma unroll
        for (int w = 0; w < W; ++w) tot[w] += __shfl_xor_sync(0xffffffffu, tot[w], o);
    }
    const int cc = lane & (c.nc - 1);
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int m = mb + w;
        if (active && (w & (c.nc - 1)) == cc && m < c.m_total) {
            const unsigned long long k = finish_window(c, m, tot[w]);
            best = k < best ? k : best;
        }
    }
}

__device__ __forceinline__ int block_start(const WinCtx& c, int b, int w, bool& active)
{
    const int m0 = c.m_first + b * w;
    active = m0 < c.m_b;
    return max(c.m_a, min(m0, c.hi_start));
}

template <int W>
__device__ void warp_task_pair(const WinCtx& c, int lane, unsigned long long& best)
{
    constexpr int H = W / 2;
    const int b = lane >> c.lg_nc;
    const int cl = lane & (c.nc - 1);
    bool active;
    const int mb = block_start(c, b, W, active);
    const int st = c.st;
    float2 acc[H];
#pragma unroll
    for (int w = 0; w < H; ++w) acc[w] = make_float2(0.0f, 0.0f);
    if (active) {
        const float* abase = c.tile + (mb * st - c.x0);
        float tv = __ldg(c.tg + cl);               // template row 0 of the first round
        for (int rho = cl; rho < st; rho += c.nc) {
            const float* a = abase + rho;
            const float* tp = c.tg + rho + st;       // next template row to fetch
            const float t_round = __ldg(c.tg + rho + c.nc);   // row 0 of the next round
            const int jn = (c.d - rho + st - 1) / st;
            float2 p[H];
#pragma unroll
            for (int w = 0; w < H; ++w) {
                p[w].x = a[w * st];
                p[w].y = a[(w + H) * st];
            }
            const float* an = a + W * st;
            int jj = 0;
            for (; jj + H <= jn; jj += H) {
#pragma unroll
                for (int u = 0; u < H; ++u) {
                    const float2 t2 = make_float2(tv, tv);
                    tv = __ldg(tp);                  // one row ahead (table is zero padded)
                    tp += st;
#pragma unroll
                    for (int w = 0; w < H; ++w) acc[w] = __ffma2_rn(p[(w + u) % H], t2, acc[w]);
                    p[u].x = p[u].y;
                    p[u].y = *an;
                    an += st;
                }
            }
#pragma unroll
            for (int u = 0; u < H; ++u) {
                if (jj + u < jn) {
                    const float2 t2 = make_float2(tv, tv);
                    tv = __ldg(tp);
                    tp += st;
#pragma unroll
                    for (int w = 0; w < H; ++w) acc[w] = __ffma2_rn(p[(w + u) % H], t2, acc[w]);
                    p[u].x = p[u].y;
                    p[u].y = *an;
                    an += st;
                }
            }
            tv = t_round;
        }
    }
    float tot[W];
#pragma unroll
    for (int w = 0; w < H; ++w) {
        tot[w] = acc[w].x;
        tot[w + H] = acc[w].y;
    }
    reduce_finish<W>(c, tot, mb, active, lane, best);
}

template <int W>
__device__ void warp_task_scalar(const WinCtx& c, int lane, unsigned long long& best)
{
    const int b = lane >> c.lg_nc;
    const int cl = lane & (c.nc - 1);
    bool active;
    const int mb = block_start(c, b, W, active);
    const int st = c.st;
    float acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = 0.0f;
    if (active) {
        const float* abase = c.tile + (mb * st - c.x0);
        float tv = __ldg(c.tg + cl);
        for (int rho = cl; rho < st; rho += c.nc) {
            const float* a = abase + rho;
            const float* tp = c.tg + rho + st;
            const float t_round = __ldg(c.tg + rho + c.nc);
            const int jn = (c.d - rho + st - 1) / st;
            float p[W];
#pragma unroll
            for (int w = 0; w < W; ++w) p[w] = a[w * st];
            const float* an = a + W * st;
            int jj = 0;
            for (; jj + W <= jn; jj += W) {
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    const float tcur = tv;
                    tv = __ldg(tp);
                    tp += st;
#pragma unroll
                    for (int w = 0; w < W; ++w) acc[w] = fmaf(p[(w + u) % W], tcur, acc[w]);
                    p[u] = *an;
                    an += st;
                }
            }
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if (jj + u < jn) {
                    const float tcur = tv;
                    tv = __ldg(tp);
                    tp += st;
#pragma unroll
                    for (int w = 0; w < W; ++w) acc[w] = fmaf(p[(w + u) % W], tcur, acc[w]);
                    p[u] = *an;
                    an += st;
                }
            }
            tv = t_round;
        }
    }
    reduce_finish<W>(c, acc, mb, active, lane, best);
}

}  // namespace tiles
}  // namespace gtls
