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
//           The folded curve is read as rows of st points: window m covers
//           rows m .. m+J-1 (J = ceil(D / st)) of every phase column rho.
//           Lane (b, c) owns block b of W consecutive windows and the
//           columns rho = c, c + nc, ...; for a fixed column a register
//           ring of W rows slides down the rows, so one shared load feeds W
//           FMAs.  nc and W satisfy W st = nc * odd (mod 32): the 32 lanes
//           then read 32 distinct shared-memory banks.
//   Variants (chosen per duration when the plan is made):
//     colpair<W>  one FFMA2 per window covers the two columns rho, rho + nc
//                 (template pairs come from a per-duration pair table whose
//                 second value is zero where rho + nc >= st);  W = 16, 15, 12
//     colpair_rot<16> the same for even T0 steps with any nc, each block
//                 walking its column rounds from round b on, so that the
//                 blocks (whose rows are 16 st = 0 mod 32 floats apart) read
//                 different banks but in pairs;
//     winpair<16> one FFMA2 covers windows w and w + 8 of one column
//                 (T0 steps that are multiples of 32);
//     scalar<15>  T0 steps 1, 2, 4, 8, 16 (one column per lane): each FFMA2
//                 accumulates (C1, S) of one window from a (s_k, 1) table.
//   Each variant walks the J rows in blocks of W (the unroll period of the
//   data ring): full blocks run without exit tests, the last partial block
//   tests once per row (a uniform test).
//   Templates are followed by zeros, so every lane runs the same J steps
//   and template rows can be fetched R rows ahead into a register ring of
//   R + 1 slots: the load of row u + R goes to the slot that row u - 1 has
//   freed, never to the one row u is multiplied with, so the registers keep
//   their roles from row to row (a ring of R slots makes the compiler rename
//   and copy a slot every row).  R + 1 divides W, so each block of W rows
//   starts with the same slot assignment.
//   The nc lanes of a block combine their partial sums by recursive halving
//   (each exchange halves the values a lane holds), so every lane ends with
//   exactly its W / nc windows, finishes them and keeps a packed running
//   minimum (delta-chi2 key, duration index, window index), merged per
//   period with one 64-bit atomicMin.
#pragma once

namespace gtls {
namespace tiles {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kCtasPerSm = 1;  // persistent window CTAs per SM (each with its own staged tile)
constexpr int kMaxDur = 64;
constexpr int kMaxRing = 7;   // template rows fetched ahead; tables carry (kMaxRing + 2) st + 64 zeros

// Variant codes (also used by the host plan).
enum Variant : int {
    kScalar15 = 0,
    kWin16 = 1,
    kWin14 = 2,
    kWin12 = 3,
    kWin8 = 4,
    kCol16 = 5,
    kCol15 = 6,
    kCol14 = 7,
    kCol12 = 8,
    kCol8 = 9,
    kWeighted15 = 10,   // per-point weights: (w r, w) tile pairs x (s_k, s_k^2) template pairs
    kCol16R = 11,       // column pairs, 16 windows, rounds rotated by block (W st = 0 mod 32)
    kWindowOnly = 12,   // duration too long for a tile: the one-thread-per-window kernel takes it
    kTensor = 13,       // uniform weights: the tensor-core kernel (window_tc.cuh) takes it
};

__host__ __device__ inline int variant_w(int v)
{
    switch (v) {
    case kScalar15: return 15;
    case kWin16: return 16;
    case kWin14: return 14;
    case kWin12: return 12;
    case kWin8: return 8;
    case kCol16: return 16;
    case kCol16R: return 16;
    case kCol15: return 15;
    case kCol14: return 14;
    case kCol12: return 12;
    case kWeighted15: return 15;
    default: return 8;
    }
}

__host__ __device__ inline bool variant_colpair(int v) { return (v >= kCol16 && v <= kCol8) || v == kCol16R; }

struct DurTask {
    int j, d, st, nc, variant, w, per_task, tasks, first, m_a, m_b, hi_start, m_total, jrows;
    const float* tg;          // template of the duration (global, zero padded)
    const float2* tg2;        // its pair table (pair variants)
    float inv_sum_t, sum_t2;  // 2^-40 / sum_k s_k and sum_k s_k^2
    float inv_sum_t_f;        // 1 / sum_k s_k
};

struct WinCtx {
    const float* tile;        // shared: folded r at x0 .. x0 + BUF
    const float2* tile2;      // shared: folded (w r, w) at x0 .. x0 + BUF (per-point weights)
    int x0;
    int d, st, nc, lg_nc, jrows;
    int m_first;              // first window of this warp task
    int m_a, m_b, hi_start, m_total;
    const float* tg;          // template of the duration (global, zero padded)
    const float2* tg2;        // template pairs (colpair variants)
    float inv_sum_t, sum_t2, w_uni;
    float inv_sum_t_f;        // 1 / sum_k s_k (no fixed-point scale)
    int j;
    const long long* pf;      // prefix sums of the period (global)
};

// Exact 64-bit window sum of r (fixed point, 2^40) to float through two
// 32-bit conversions (the FP64 pipe is narrow on this GPU); c.inv_sum_t
// already carries the 2^-40 scale.
__device__ __forceinline__ float fixed_to_float(long long v)
{
    const float hi = (float)(int)(v >> 32);
    const float lo = (float)(unsigned int)(v & 0xffffffffll);
    return fmaf(hi, 4294967296.0f, lo);
}

__device__ __forceinline__ unsigned long long finish_window(const WinCtx& c, long long m, float c1)
{
    const long long s = m * c.st;
    const long long sfx = c.pf[s + c.d] - c.pf[s];
    const float depth = fmaxf(0.0f, fixed_to_float(sfx) * c.inv_sum_t);
    const float dchi = c.w_uni * depth * fmaf(depth, c.sum_t2, -2.0f * c1);
    unsigned int u = __float_as_uint(dchi);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | ((unsigned long long)c.j << 24) | (unsigned long long)m;
}

// One recursive-halving exchange over lane bit `o`: the lane keeps the lower
// (bit clear) or upper (bit set) half of its CNT values, adds the partner's
// copy of that half, and sends the other half.
template <int CNT>
__device__ __forceinline__ void halve(float (&v)[16], int lane, int o, int& base)
{
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < CNT / 2; ++i) {
        const float send = up ? v[i] : v[i + CNT / 2];
        const float keep = up ? v[i + CNT / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    if (up) base += CNT / 2;
}

// Combine the nc = 2^lg_nc partial sums of a block (lanes b*nc .. b*nc+nc-1)
// and finish this lane's windows mb + base .. mb + base + cnt - 1.
template <int W>
__device__ __forceinline__ void reduce_finish(const WinCtx& c, const float (&tot)[W], int mb, bool active,
                                              int lane, unsigned long long& best)
{
    static_assert(W <= 16, "at most 16 windows per block");
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = i < W ? tot[i] : 0.0f;
    const int k = c.lg_nc;
    int base = 0;
    if (k >= 1) halve<16>(v, lane, 1, base);
    if (k >= 2) halve<8>(v, lane, 2, base);
    if (k >= 3) halve<4>(v, lane, 4, base);
    if (k >= 4) halve<2>(v, lane, 8, base);
    if (k >= 5) v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16);   // lanes 16..31 repeat 0..15
    const int cnt = 16 >> min(k, 4);
    if (!active || (k >= 5 && (lane & 16))) return;
    float e[16];   // this lane's window totals, walked with a runtime count
#pragma unroll
    for (int i = 0; i < 16; ++i) e[i] = v[i];
#pragma unroll 4
    for (int i = 0; i < cnt; ++i) {
        const int w = base + i;
        const int m = mb + w;
        if (w < W && m < c.m_total) {
            const unsigned long long key = finish_window(c, m, e[i]);
            best = key < best ? key : best;
        }
    }
}

template <int CNT>
__device__ __forceinline__ void halve2(float2 (&v)[16], int lane, int o, int& base)
{
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < CNT / 2; ++i) {
        const float2 send = up ? v[i] : v[i + CNT / 2];
        const float2 keep = up ? v[i + CNT / 2] : v[i];
        v[i].x = keep.x + __shfl_xor_sync(0xffffffffu, send.x, o);
        v[i].y = keep.y + __shfl_xor_sync(0xffffffffu, send.y, o);
    }
    if (up) base += CNT / 2;
}

// As reduce_finish for (C1, S) pairs: the window sum comes with C1, so the
// epilogue reads no prefix sums.
template <int W>
__device__ __forceinline__ void reduce_pair_finish(const WinCtx& c, const float2 (&tot)[W], int mb, bool active,
                                                   int lane, unsigned long long& best)
{
    static_assert(W <= 16, "at most 16 windows per block");
    float2 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = i < W ? tot[i] : make_float2(0.0f, 0.0f);
    const int k = c.lg_nc;
    int base = 0;
    if (k >= 1) halve2<16>(v, lane, 1, base);
    if (k >= 2) halve2<8>(v, lane, 2, base);
    if (k >= 3) halve2<4>(v, lane, 4, base);
    if (k >= 4) halve2<2>(v, lane, 8, base);
    if (k >= 5) {
        v[0].x += __shfl_xor_sync(0xffffffffu, v[0].x, 16);
        v[0].y += __shfl_xor_sync(0xffffffffu, v[0].y, 16);
    }
    const int cnt = 16 >> min(k, 4);
    if (!active || (k >= 5 && (lane & 16))) return;
    float2 e[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) e[i] = v[i];
    for (int i = 0; i < cnt; ++i) {
        const int w = base + i;
        const int m = mb + w;
        if (w < W && m < c.m_total) {
            const float depth = fmaxf(0.0f, e[i].y * c.inv_sum_t_f);
            const float dchi = c.w_uni * depth * fmaf(depth, c.sum_t2, -2.0f * e[i].x);
            unsigned int u = __float_as_uint(dchi);
            u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
            const unsigned long long key =
                ((unsigned long long)u << 32) | ((unsigned long long)c.j << 24) | (unsigned long long)m;
            best = key < best ? key : best;
        }
    }
}

__device__ __forceinline__ int block_start(const WinCtx& c, int b, int w, bool& active)
{
    const int m0 = c.m_first + b * w;
    active = m0 < c.m_b;
    return max(c.m_a, min(m0, c.hi_start));
}

// Rows jj .. jj + cnt - 1 of one column (cnt = W unless !kFull): row u is
// multiplied into the W window sums (acc[w] += p[(w + u) % W] x template row),
// then its data slot takes row u + W and its template slot row u + R.
template <int W, int R, bool kFull>
__device__ __forceinline__ void colpair_rows(float2 (&acc)[W], float2 (&p)[W], float2 (&ring)[R + 1],
                                             const float2*& tp, const float*& an, int st, int nc, int cnt)
{
#pragma unroll
    for (int u = 0; u < W; ++u) {
        if (!kFull && u >= cnt) break;
        ring[(u + R) % (R + 1)] = __ldg(tp);     // row u + R (zero padded past D)
        tp += st;
        const float2 tcur = ring[u % (R + 1)];
#pragma unroll
        for (int w = 0; w < W; ++w) acc[w] = __ffma2_rn(p[(w + u) % W], tcur, acc[w]);
        p[u].x = an[0];
        p[u].y = an[nc];
        an += st;
    }
}

// Column pairs: acc[w] = (column rho, column rho + nc) partial sums of window w.
template <int W, int R>
__device__ void warp_task_colpair(const WinCtx& c, int lane, unsigned long long& best)
{
    static_assert(W % (R + 1) == 0, "template ring length must divide the unroll period");
    const int b = lane >> c.lg_nc;
    const int cl = lane & (c.nc - 1);
    bool active;
    const int mb = block_start(c, b, W, active);
    const int st = c.st, nc = c.nc, jrows = c.jrows;
    float2 acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = make_float2(0.0f, 0.0f);
    if (active) {
        const float* abase = c.tile + (mb * st - c.x0);
        float2 nxt[R];   // first R template rows of the coming column round
#pragma unroll
        for (int r = 0; r < R; ++r) nxt[r] = __ldg(c.tg2 + cl + r * st);
        for (int rho = cl; rho < st; rho += 2 * nc) {
            const float* a = abase + rho;
            float2 ring[R + 1];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ring[r] = nxt[r];
                nxt[r] = __ldg(c.tg2 + rho + 2 * nc + r * st);   // next round (zero padded)
            }
            const float2* tp = c.tg2 + rho + R * st;
            float2 p[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                p[w].x = a[w * st];
                p[w].y = a[w * st + nc];
            }
            const float* an = a + W * st;
            int jj = 0;
            for (; jj + W <= jrows; jj += W) colpair_rows<W, R, true>(acc, p, ring, tp, an, st, nc, W);
            if (jj < jrows) colpair_rows<W, R, false>(acc, p, ring, tp, an, st, nc, jrows - jj);
        }
    }
    float tot[W];
#pragma unroll
    for (int w = 0; w < W; ++w) tot[w] = acc[w].x + acc[w].y;
    reduce_finish<W>(c, tot, mb, active, lane, best);
}

// Column pairs with rotated rounds (any T0 step with W st = 0 mod 32, where
// every block of W windows would read the same banks): block b walks its
// column rounds starting at round b (mod the round count), so that at a
// given time the blocks read columns 2 nc apart (at most two blocks per
// bank).  Every lane still covers its columns once, in another order.
template <int W, int R>
__device__ void warp_task_colpair_rot(const WinCtx& c, int lane, unsigned long long& best)
{
    static_assert(W % (R + 1) == 0, "template ring length must divide the unroll period");
    const int b = lane >> c.lg_nc;
    const int cl = lane & (c.nc - 1);
    bool active;
    const int mb = block_start(c, b, W, active);
    const int st = c.st, nc = c.nc, jrows = c.jrows;
    float2 acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = make_float2(0.0f, 0.0f);
    if (active) {
        const float* abase = c.tile + (mb * st - c.x0);
        const int rounds = (st + 2 * nc - 1) / (2 * nc);
        int rr = b % rounds;
        float2 nxt[R];   // first R template rows of the coming column round
#pragma unroll
        for (int r = 0; r < R; ++r) nxt[r] = __ldg(c.tg2 + cl + 2 * nc * rr + r * st);
        for (int k = 0; k < rounds; ++k) {
            const int rho = cl + 2 * nc * rr;
            rr = rr + 1 == rounds ? 0 : rr + 1;
            float2 ring[R + 1];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ring[r] = nxt[r];
                nxt[r] = __ldg(c.tg2 + cl + 2 * nc * rr + r * st);   // next round (zero padded)
            }
            if (rho >= st) continue;
            const float* a = abase + rho;
            const float2* tp = c.tg2 + rho + R * st;
            float2 p[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                p[w].x = a[w * st];
                p[w].y = a[w * st + nc];
            }
            const float* an = a + W * st;
            int jj = 0;
            for (; jj + W <= jrows; jj += W) colpair_rows<W, R, true>(acc, p, ring, tp, an, st, nc, W);
            if (jj < jrows) colpair_rows<W, R, false>(acc, p, ring, tp, an, st, nc, jrows - jj);
        }
    }
    float tot[W];
#pragma unroll
    for (int w = 0; w < W; ++w) tot[w] = acc[w].x + acc[w].y;
    reduce_finish<W>(c, tot, mb, active, lane, best);
}

// Rows of one column for window pairs (H = W / 2 rows per block): acc[w]
// holds windows w and w + H, p[w] the rows w and w + H ahead.
template <int H, int R, bool kFull>
__device__ __forceinline__ void winpair_rows(float2 (&acc)[H], float2 (&p)[H], float (&ring)[R + 1],
                                             const float*& tp, const float*& an, int st, int cnt)
{
#pragma unroll
    for (int u = 0; u < H; ++u) {
        if (!kFull && u >= cnt) break;
        ring[(u + R) % (R + 1)] = __ldg(tp);
        tp += st;
        const float tv = ring[u % (R + 1)];
        const float2 t2 = make_float2(tv, tv);
#pragma unroll
        for (int w = 0; w < H; ++w) acc[w] = __ffma2_rn(p[(w + u) % H], t2, acc[w]);
        p[u].x = p[u].y;
        p[u].y = *an;
        an += st;
    }
}

// Window pairs: acc[w] = (window w, window w + W/2) partial sums of one column.
template <int W, int R>
__device__ void warp_task_winpair(const WinCtx& c, int lane, unsigned long long& best)
{
    constexpr int H = W / 2;
    static_assert(H % (R + 1) == 0, "template ring length must divide the unroll period");
    const int b = lane >> c.lg_nc;
    const int cl = lane & (c.nc - 1);
    bool active;
    const int mb = block_start(c, b, W, active);
    const int st = c.st, jrows = c.jrows;
    float2 acc[H];
#pragma unroll
    for (int w = 0; w < H; ++w) acc[w] = make_float2(0.0f, 0.0f);
    if (active) {
        const float* abase = c.tile + (mb * st - c.x0);
        float nxt[R];
#pragma unroll
        for (int r = 0; r < R; ++r) nxt[r] = __ldg(c.tg + cl + r * st);
        for (int rho = cl; rho < st; rho += c.nc) {
            const float* a = abase + rho;
            float ring[R + 1];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ring[r] = nxt[r];
                nxt[r] = __ldg(c.tg + rho + c.nc + r * st);
            }
            const float* tp = c.tg + rho + R * st;
            float2 p[H];
#pragma unroll
            for (int w = 0; w < H; ++w) {
                p[w].x = a[w * st];
                p[w].y = a[(w + H) * st];
            }
            const float* an = a + W * st;
            int jj = 0;
            for (; jj + H <= jrows; jj += H) winpair_rows<H, R, true>(acc, p, ring, tp, an, st, H);
            if (jj < jrows) winpair_rows<H, R, false>(acc, p, ring, tp, an, st, jrows - jj);
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

// Rows of one column for the (C1, S) pairs: the data value is duplicated
// into both halves of its slot.
template <int W, int R, bool kFull>
__device__ __forceinline__ void scalar_rows(float2 (&acc)[W], float2 (&p)[W], float2 (&ring)[R + 1],
                                            const float2*& tp, const float*& an, int st, int cnt)
{
#pragma unroll
    for (int u = 0; u < W; ++u) {
        if (!kFull && u >= cnt) break;
        ring[(u + R) % (R + 1)] = __ldg(tp);
        tp += st;
        const float2 tcur = ring[u % (R + 1)];
#pragma unroll
        for (int w = 0; w < W; ++w) acc[w] = __ffma2_rn(p[(w + u) % W], tcur, acc[w]);
        const float v = *an;
        p[u] = make_float2(v, v);
        an += st;
    }
}

// Small T0 steps (st = nc = 1, 2, 4, 8, 16): one column per lane.  Each
// FFMA2 accumulates (C1, S) = (sum r s_k, sum r) of one window and column
// from the pair table (s_k, 1); the nc columns are then combined, so the
// window sum needs no prefix-sum reads.
template <int W, int R>
__device__ void warp_task_scalar(const WinCtx& c, int lane, unsigned long long& best)
{
    static_assert(W % (R + 1) == 0, "template ring length must divide the unroll period");
    const int b = lane >> c.lg_nc;
    const int cl = lane & (c.nc - 1);
    bool active;
    const int mb = block_start(c, b, W, active);
    const int st = c.st, jrows = c.jrows;
    float2 acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = make_float2(0.0f, 0.0f);
    if (active) {
        const float* abase = c.tile + (mb * st - c.x0);
        for (int rho = cl; rho < st; rho += c.nc) {
            const float* a = abase + rho;
            const float2* tp = c.tg2 + rho;
            float2 ring[R + 1];
#pragma unroll
            for (int r = 0; r < R; ++r) ring[r] = __ldg(tp + r * st);
            tp += R * st;
            float2 p[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const float v = a[w * st];
                p[w] = make_float2(v, v);
            }
            const float* an = a + W * st;
            int jj = 0;
            for (; jj + W <= jrows; jj += W) scalar_rows<W, R, true>(acc, p, ring, tp, an, st, W);
            if (jj < jrows) scalar_rows<W, R, false>(acc, p, ring, tp, an, st, jrows - jj);
        }
    }
    reduce_pair_finish<W>(c, acc, mb, active, lane, best);
}

// Per-point weights: every lane ends with (C1w, C2w) = (sum w r s_k,
// sum w s_k^2) of its windows; S comes from the exact prefix sums and
// delta-chi2 = delta (delta C2w - 2 C1w) (Eqs. out, in with weights;
// depth = max(0, S / sum s_k), the unweighted moving average).
template <int W>
__device__ __forceinline__ void reduce_weighted_finish(const WinCtx& c, const float2 (&tot)[W], int mb,
                                                       bool active, int lane, unsigned long long& best)
{
    static_assert(W <= 16, "at most 16 windows per block");
    float2 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = i < W ? tot[i] : make_float2(0.0f, 0.0f);
    const int k = c.lg_nc;
    int base = 0;
    if (k >= 1) halve2<16>(v, lane, 1, base);
    if (k >= 2) halve2<8>(v, lane, 2, base);
    if (k >= 3) halve2<4>(v, lane, 4, base);
    if (k >= 4) halve2<2>(v, lane, 8, base);
    if (k >= 5) {
        v[0].x += __shfl_xor_sync(0xffffffffu, v[0].x, 16);
        v[0].y += __shfl_xor_sync(0xffffffffu, v[0].y, 16);
    }
    const int cnt = 16 >> min(k, 4);
    if (!active || (k >= 5 && (lane & 16))) return;
    float2 e[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) e[i] = v[i];
    for (int i = 0; i < cnt; ++i) {
        const int w = base + i;
        const long long m = mb + w;
        if (w < W && m < c.m_total) {
            const long long s0 = m * c.st;
            const long long sfx = c.pf[s0 + c.d] - c.pf[s0];
            const float depth = fmaxf(0.0f, fixed_to_float(sfx) * c.inv_sum_t);
            const float dchi = depth * fmaf(depth, e[i].y, -2.0f * e[i].x);
            unsigned int u = __float_as_uint(dchi);
            u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
            const unsigned long long key =
                ((unsigned long long)u << 32) | ((unsigned long long)c.j << 24) | (unsigned long long)m;
            best = key < best ? key : best;
        }
    }
}

// Rows of one column of (w r, w) pairs.
template <int W, int R, bool kFull>
__device__ __forceinline__ void weighted_rows(float2 (&acc)[W], float2 (&p)[W], float2 (&ring)[R + 1],
                                              const float2*& tp, const float2*& an, int st, int cnt)
{
#pragma unroll
    for (int u = 0; u < W; ++u) {
        if (!kFull && u >= cnt) break;
        ring[(u + R) % (R + 1)] = __ldg(tp);
        tp += st;
        const float2 tcur = ring[u % (R + 1)];
#pragma unroll
        for (int w = 0; w < W; ++w) acc[w] = __ffma2_rn(p[(w + u) % W], tcur, acc[w]);
        p[u] = *an;
        an += st;
    }
}

// Per-point weights: nc lanes per window block (2^v for st = 2^v odd, or 16 /
// 32: one block per half-warp / warp), each lane one column at a time; each
// FFMA2 multiplies the staged pair (w r, w) of a point by the template pair
// (s_k, s_k^2), i.e. one FFMA2 per window-point evaluation.  Pairs are 8-byte
// shared loads: the 16 lanes of a half-warp read 16 distinct bank pairs.
template <int W, int R>
__device__ void warp_task_weighted(const WinCtx& c, int lane, unsigned long long& best)
{
    static_assert(W % (R + 1) == 0, "template ring length must divide the unroll period");
    const int b = lane >> c.lg_nc;
    const int cl = lane & (c.nc - 1);
    bool active;
    const int mb = block_start(c, b, W, active);
    const int st = c.st, jrows = c.jrows;
    float2 acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = make_float2(0.0f, 0.0f);
    if (active) {
        const float2* abase = c.tile2 + (mb * st - c.x0);
        for (int rho = cl; rho < st; rho += c.nc) {
            const float2* a = abase + rho;
            const float2* tp = c.tg2 + rho;
            float2 ring[R + 1];
#pragma unroll
            for (int r = 0; r < R; ++r) ring[r] = __ldg(tp + r * st);
            tp += R * st;
            float2 p[W];
#pragma unroll
            for (int w = 0; w < W; ++w) p[w] = a[w * st];
            const float2* an = a + W * st;
            int jj = 0;
            for (; jj + W <= jrows; jj += W) weighted_rows<W, R, true>(acc, p, ring, tp, an, st, W);
            if (jj < jrows) weighted_rows<W, R, false>(acc, p, ring, tp, an, st, jrows - jj);
        }
    }
    reduce_weighted_finish<W>(c, acc, mb, active, lane, best);
}

}  // namespace tiles
}  // namespace gtls
