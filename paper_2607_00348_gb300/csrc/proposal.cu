// Learned period proposal: a small 1D CNN over the time-binned light curve
// that predicts, per log-spaced region of trial periods, the largest signal
// residue SR(P) the TLS search finds there (the paper has no such stage; it
// is trained on spectra that the search itself produces).
//
// Network (fixed): input [B][4096][1]; six 'same' convolutions (taps 7, 5,
// 5, 5, 5, 5, dilated 1, 2, 2, 4, 4, 8 bins of their own input; 64
// channels) each followed by ReLU and max-pooling by 2; linear head 4096 ->
// 128 regions; logistic loss with soft targets; Adam.  The dilations give
// a last-layer unit a receptive field of about 1530 input bins (taps and
// pooling windows; more than a third of the curve) instead of about 320.
//
// Every contraction (convolution forward, data and weight gradients, head
// forward and its two gradients) runs through one BF16 tensor-core tile GEMM
// (mma.sync m16n8k16, FP32 accumulation) whose operand tiles are gathered
// into shared memory by small loader functors (implicit im2col for the
// convolutions, transposed views for the gradients).  Activations are BF16
// [batch][length][channel]; gradients and master parameters are FP32.  The
// whole network costs about 0.2 GFLOP per light curve for inference, so the
// kernels favour simplicity over peak tensor throughput.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gtls_internal.h"

namespace {

using gtls::set_error;
using bf16 = __nv_bfloat16;

#define PROP_CUDA(call)                                                                         \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return set_error(e_ == cudaErrorMemoryAllocation ? GTLS_ERR_OOM : GTLS_ERR_CUDA,    \
                             std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

#define PROP_TRY(x)                   \
    do {                              \
        gtls_status s_ = (x);         \
        if (s_ != GTLS_OK) return s_; \
    } while (0)

constexpr int kBins = 4096;
constexpr int kCh = 64;
constexpr int kConv = 6;
constexpr int kReg = 128;
constexpr int kFeat = (kBins >> kConv) * kCh;
constexpr int kTaps[kConv] = {7, 5, 5, 5, 5, 5};
constexpr int kDil[kConv] = {1, 2, 2, 4, 4, 8};   // tap spacing of each convolution (its input's bins)
constexpr double kRegionLo = 0.5, kRegionHi = 1024.0;   // days: regions split this range evenly in log P

// offsets of the flat parameter vector (order: w0 b0 ... w5 b5 wh bh)
struct Layout {
    int64_t w[kConv], b[kConv], wh, bh, total;
    Layout()
    {
        int64_t pos = 0;
        int cin = 1;
        for (int i = 0; i < kConv; ++i) {
            w[i] = pos;
            pos += (int64_t)kCh * kTaps[i] * cin;
            b[i] = pos;
            pos += kCh;
            cin = kCh;
        }
        wh = pos;
        pos += (int64_t)kReg * kFeat;
        bh = pos;
        pos += kReg;
        total = pos;
    }
};

// ---------------------------------------------------------------------------
// tile GEMM: C[m][n] = sum_k A(m, k) B(n, k), 64 x 64 tiles, K steps of 32,
// four warps of 32 x 32 (2 x 4 mma tiles of 16 x 8)
// ---------------------------------------------------------------------------

constexpr int kBM = 64, kBN = 64, kBK = 32, kLd = kBK + 8;   // +8: conflict-free fragment loads

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Operand views (value at (row, k); callers guarantee row and k in range)
struct ConvIn {        // implicit im2col of x[B][L][C]: row = b L + l, k = tap C + c
    const bf16* x;
    int L, C, half, dil;   // taps at l + (tap - half) dil
    __device__ bf16 operator()(int row, int k) const
    {
        const int b = row / L, l = row - b * L;
        const int tap = k / C, c = k - tap * C;
        const int src = l + (tap - half) * dil;
        return (src >= 0 && src < L) ? x[((int64_t)b * L + src) * C + c] : __float2bfloat16(0.0f);
    }
};
struct ConvInT {       // the same view with the roles swapped: row = tap C + c, k = b L + l
    ConvIn in;
    __device__ bf16 operator()(int row, int k) const { return in(k, row); }
};
struct RowMajor {      // m[row][k], leading dimension ld
    const bf16* m;
    int ld;
    __device__ bf16 operator()(int row, int k) const { return m[(int64_t)row * ld + k]; }
};
struct ColMajor {      // m[k][row], leading dimension ld
    const bf16* m;
    int ld;
    __device__ bf16 operator()(int row, int k) const { return m[(int64_t)k * ld + row]; }
};
struct FlippedW {      // data gradient: row = input channel ci, k = tap' C + co -> w[co][T-1-tap'][ci]
    const bf16* w;
    int taps, cin, cout;
    __device__ bf16 operator()(int row, int k) const
    {
        const int tp = k / cout, co = k - tp * cout;
        return w[((int64_t)co * taps + (taps - 1 - tp)) * cin + row];
    }
};

enum EpiKind { kEpiPoolRelu = 0, kEpiStore = 1, kEpiAtomic = 2 };

struct Epi {
    int kind;
    float* out;            // kEpiStore / kEpiAtomic: out[row * ld + col]
    int ld;
    const float* bias;     // per column, nullable
    bf16* pooled;          // kEpiPoolRelu: pooled[(row / 2) * ld + col]
    uint8_t* arg;          // 1 where the odd row of a pair won
};

template <class LA, class LB>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, int k_chunk, LA la, LB lb, Epi ep)
{
    __shared__ __align__(16) bf16 As[kBM][kLd];
    __shared__ __align__(16) bf16 Bs[kBN][kLd];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int kbeg = blockIdx.z * k_chunk;
    const int kend = min(K, kbeg + k_chunk);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[i][j][u] = 0.0f;
    const bf16 zero = __float2bfloat16(0.0f);
    for (int k0 = kbeg; k0 < kend; k0 += kBK) {
        for (int e = tid; e < kBM * kBK; e += 128) {
            const int r = e / kBK, c = e - (e / kBK) * kBK;
            const int k = k0 + c;
            const bool kin = k < kend;
            As[r][c] = (kin && m0 + r < M) ? la(m0 + r, k) : zero;
            Bs[r][c] = (kin && n0 + r < N) ? lb(n0 + r, k) : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int row = wm + i * 16 + g;
                a[i][0] = *reinterpret_cast<const uint32_t*>(&As[row][kk + 2 * t]);
                a[i][1] = *reinterpret_cast<const uint32_t*>(&As[row + 8][kk + 2 * t]);
                a[i][2] = *reinterpret_cast<const uint32_t*>(&As[row][kk + 2 * t + 8]);
                a[i][3] = *reinterpret_cast<const uint32_t*>(&As[row + 8][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int col = wn + j * 8 + g;
                b[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[col][kk + 2 * t]);
                b[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[col][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    // accumulator (i, j, u): row m0 + wm + 16 i + g + 8 (u >> 1), column
    // n0 + wn + 8 j + 2 t + (u & 1)
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int row = m0 + wm + i * 16 + g + 8 * (u >> 1);
                const int col = n0 + wn + j * 8 + 2 * t + (u & 1);
                float v = acc[i][j][u];
                if (ep.kind == kEpiPoolRelu) {
                    // rows 2q and 2q+1 sit in lanes g and g ^ 1 (lane ^ 4)
                    v = fmaxf(v + (col < N ? ep.bias[col] : 0.0f), 0.0f);
                    const float other = __shfl_xor_sync(0xffffffffu, v, 4);
                    if ((g & 1) == 0 && row < M && col < N) {
                        const bool odd_wins = other > v;
                        ep.pooled[(int64_t)(row >> 1) * ep.ld + col] = __float2bfloat16(odd_wins ? other : v);
                        ep.arg[(int64_t)(row >> 1) * ep.ld + col] = odd_wins ? 1 : 0;
                    }
                } else if (row < M && col < N) {
                    if (ep.bias) v += ep.bias[col];
                    if (ep.kind == kEpiStore) ep.out[(int64_t)row * ep.ld + col] = v;
                    else atomicAdd(&ep.out[(int64_t)row * ep.ld + col], v);
                }
            }
        }
    }
}

template <class LA, class LB>
gtls_status gemm(int M, int N, int K, int k_chunk, LA la, LB lb, Epi ep, cudaStream_t st)
{
    if (k_chunk <= 0) k_chunk = K;
    k_chunk = (k_chunk + kBK - 1) / kBK * kBK;
    const dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + kBN - 1) / kBN),
                    (unsigned)((K + k_chunk - 1) / k_chunk));
    k_gemm<LA, LB><<<grid, 128, 0, st>>>(M, N, K, k_chunk, la, lb, ep);
    PROP_CUDA(cudaGetLastError());
    return GTLS_OK;
}

// ---------------------------------------------------------------------------
// element-wise and reduction kernels
// ---------------------------------------------------------------------------

__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

// d pre-activation of a ReLU + max-pool layer: the pooled gradient goes to
// the winning row of each pair when the pooled value is positive.
__global__ void k_pool_back(const float* __restrict__ dpool, const bf16* __restrict__ pooled,
                            const uint8_t* __restrict__ arg, bf16* __restrict__ dpre, int64_t n_pooled)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_pooled;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pos = q / kCh, c = q - pos * kCh;
        const float gsum = __bfloat162float(pooled[q]) > 0.0f ? dpool[q] : 0.0f;
        const int a = arg[q];
        dpre[(2 * pos + a) * kCh + c] = __float2bfloat16(gsum);
        dpre[(2 * pos + 1 - a) * kCh + c] = __float2bfloat16(0.0f);
    }
}

// Column sums of a [rows][cols] matrix (bf16 or f32) into g[cols] (+=).
template <class T>
__global__ void k_col_sum(const T* __restrict__ m, int64_t rows, int cols, float* __restrict__ g)
{
    const int c = threadIdx.x % cols;
    const int lanes = blockDim.x / cols;
    const int r0 = threadIdx.x / cols;
    float s = 0.0f;
    for (int64_t r = blockIdx.x * (int64_t)lanes + r0; r < rows; r += (int64_t)gridDim.x * lanes) {
        if constexpr (sizeof(T) == 2) s += __bfloat162float(m[r * cols + c]);
        else s += m[r * cols + c];
    }
    if (r0 < lanes) atomicAdd(&g[c], s);
}

// Masked logistic loss with soft targets (one block): loss = sum mask
// (softplus(z) - t z) / sum mask; dz = mask (sigmoid(z) - t) / sum mask.
__global__ void __launch_bounds__(1024) k_loss(const float* __restrict__ z, const float* __restrict__ tgt,
                                               const float* __restrict__ mask, int n, float* __restrict__ dz,
                                               double* __restrict__ loss)
{
    __shared__ double sh[1024];
    double cnt = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) cnt += mask[i];
    sh[threadIdx.x] = cnt;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double total = fmax(sh[0], 1.0);
    __syncthreads();
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double zi = z[i], m = mask[i], ti = tgt[i];
        const double sp = zi > 0.0 ? zi + log1p(exp(-zi)) : log1p(exp(zi));
        acc += m * (sp - ti * zi);
        const double sg = 1.0 / (1.0 + exp(-zi));
        dz[i] = (float)(m * (sg - ti) / total);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = sh[0] / total;
}

__global__ void k_sigmoid(const float* __restrict__ z, float* __restrict__ s, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) s[i] = 1.0f / (1.0f + expf(-z[i]));
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters, then their BF16 copy.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, bf16* __restrict__ pb, int64_t n, float lr, float c1, float c2)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        pb[i] = __float2bfloat16(pi);
    }
}

// Time binning, one block per light curve: bin b of curve i holds its points
// with floor((t - t_min) / (t_max - t_min) * 4096) = b (the last point in the
// last bin); value sum(w r) / sqrt(sum w), r = 1 - y, w = 1/dy^2; empty
// bins 0.  Accumulated in FP64 in shared memory.
__global__ void __launch_bounds__(1024) k_bin(const double* __restrict__ t, const double* __restrict__ y,
                                              const double* __restrict__ dy, const int64_t* __restrict__ off,
                                              float* __restrict__ x, float* __restrict__ mean,
                                              float* __restrict__ wsum)
{
    extern __shared__ double sb[];   // [kBins] sum w r, [kBins] sum w
    __shared__ double mn[32], mx[32];
    const int lc = blockIdx.x;
    const int64_t o = off[lc], n = off[lc + 1] - o;
    for (int b = threadIdx.x; b < 2 * kBins; b += blockDim.x) sb[b] = 0.0;
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        lo = fmin(lo, t[o + i]);
        hi = fmax(hi, t[o + i]);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, s));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, s));
    }
    if ((threadIdx.x & 31) == 0) {
        mn[threadIdx.x >> 5] = lo;
        mx[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    lo = mn[0];
    hi = mx[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        lo = fmin(lo, mn[w]);
        hi = fmax(hi, mx[w]);
    }
    const double span = __dsub_rn(hi, lo);
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        int b = 0;
        if (span > 0.0) {
            const double f = __dmul_rn(__ddiv_rn(__dsub_rn(t[o + i], lo), span), (double)kBins);
            b = (int)fmin(floor(f), (double)(kBins - 1));
            b = max(b, 0);
        }
        const double w = __ddiv_rn(1.0, __dmul_rn(dy[o + i], dy[o + i]));
        atomicAdd(&sb[b], __dmul_rn(w, __dsub_rn(1.0, y[o + i])));
        atomicAdd(&sb[kBins + b], w);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) {
        const double sw = sb[kBins + b];
        x[(int64_t)lc * kBins + b] = sw > 0.0 ? (float)(sb[b] / sqrt(sw)) : 0.0f;
        if (mean) mean[(int64_t)lc * kBins + b] = sw > 0.0 ? (float)(sb[b] / sw) : 0.0f;
        if (wsum) wsum[(int64_t)lc * kBins + b] = (float)sw;
    }
}

int grid_for(int64_t n)
{
    return (int)std::min<int64_t>(4096, std::max<int64_t>(1, (n + 255) / 256));
}

}  // namespace

struct gtls_cnn {
    int device = -1;
    int max_batch = 0;
    Layout lay;
    float* p = nullptr;       // FP32 master parameters
    bf16* pb = nullptr;       // BF16 copy used by the GEMMs
    float* g = nullptr;       // gradients
    float* m = nullptr;       // Adam moments
    float* v = nullptr;
    int64_t step = 0;
    bf16* act[kConv + 1] = {};   // act[0] input, act[i+1] pooled output of conv i
    uint8_t* arg[kConv] = {};
    float* z = nullptr;
    float* dz = nullptr;
    bf16* dz_b = nullptr;
    float* da[2] = {};        // FP32 gradient of a pooled output (ping-pong)
    bf16* dpre = nullptr;     // BF16 gradient of a pre-activation
    double* loss = nullptr;
    int64_t* off = nullptr;   // binning offsets (max_batch + 1)
    std::vector<void*> allocs;
};

namespace {

template <class T>
gtls_status cnn_alloc(gtls_cnn* c, T** ptr, int64_t count)
{
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, std::max<int64_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return set_error(GTLS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    *ptr = static_cast<T*>(q);
    return GTLS_OK;
}

int conv_len(int i) { return kBins >> i; }      // input length of conv i
int conv_cin(int i) { return i == 0 ? 1 : kCh; }

gtls_status cnn_forward(gtls_cnn* c, const float* x, int B, cudaStream_t st)
{
    const int64_t nin = (int64_t)B * kBins;
    k_to_bf16<<<grid_for(nin), 256, 0, st>>>(x, c->act[0], nin);
    PROP_CUDA(cudaGetLastError());
    for (int i = 0; i < kConv; ++i) {
        const int L = conv_len(i), cin = conv_cin(i), taps = kTaps[i];
        ConvIn a{c->act[i], L, cin, (taps - 1) / 2, kDil[i]};
        RowMajor w{c->pb + c->lay.w[i], taps * cin};
        Epi ep{kEpiPoolRelu, nullptr, kCh, c->p + c->lay.b[i], c->act[i + 1], c->arg[i]};
        PROP_TRY(gemm(B * L, kCh, taps * cin, 0, a, w, ep, st));
    }
    RowMajor f{c->act[kConv], kFeat};
    RowMajor wh{c->pb + c->lay.wh, kFeat};
    Epi ep{kEpiStore, c->z, kReg, c->p + c->lay.bh, nullptr, nullptr};
    return gemm(B, kReg, kFeat, 0, f, wh, ep, st);
}

gtls_status cnn_backward(gtls_cnn* c, const float* tgt, const float* mask, int B, cudaStream_t st)
{
    const int nz = B * kReg;
    k_loss<<<1, 1024, 0, st>>>(c->z, tgt, mask, nz, c->dz, c->loss);
    PROP_CUDA(cudaGetLastError());
    PROP_CUDA(cudaMemsetAsync(c->g, 0, c->lay.total * sizeof(float), st));
    k_to_bf16<<<grid_for(nz), 256, 0, st>>>(c->dz, c->dz_b, nz);
    PROP_CUDA(cudaGetLastError());
    // head: dWh[r][f] = sum_b dz[b][r] feat[b][f]; dbh = sum_b dz; dfeat = dz Wh
    {
        ColMajor a{c->dz_b, kReg};
        ColMajor b{c->act[kConv], kFeat};
        Epi ep{kEpiAtomic, c->g + c->lay.wh, kFeat, nullptr, nullptr, nullptr};
        PROP_TRY(gemm(kReg, kFeat, B, 0, a, b, ep, st));
        k_col_sum<float><<<1, 1024, 0, st>>>(c->dz, B, kReg, c->g + c->lay.bh);
        PROP_CUDA(cudaGetLastError());
        RowMajor a2{c->dz_b, kReg};
        ColMajor b2{c->pb + c->lay.wh, kFeat};
        Epi ep2{kEpiStore, c->da[0], kFeat, nullptr, nullptr, nullptr};
        PROP_TRY(gemm(B, kFeat, kReg, 0, a2, b2, ep2, st));
    }
    int cur = 0;
    for (int i = kConv - 1; i >= 0; --i) {
        const int L = conv_len(i), cin = conv_cin(i), taps = kTaps[i];
        const int64_t npool = (int64_t)B * (L / 2) * kCh;
        k_pool_back<<<grid_for(npool), 256, 0, st>>>(c->da[cur], c->act[i + 1], c->arg[i], c->dpre, npool);
        PROP_CUDA(cudaGetLastError());
        const int64_t rows = (int64_t)B * L;
        // dW[co][tap ci] = sum over positions of dpre[pos][co] x(pos, tap ci)
        {
            ColMajor a{c->dpre, kCh};
            ConvInT b{ConvIn{c->act[i], L, cin, (taps - 1) / 2, kDil[i]}};
            Epi ep{kEpiAtomic, c->g + c->lay.w[i], taps * cin, nullptr, nullptr, nullptr};
            PROP_TRY(gemm(kCh, taps * cin, (int)rows, 8192, a, b, ep, st));
        }
        k_col_sum<bf16><<<256, 1024, 0, st>>>(c->dpre, rows, kCh, c->g + c->lay.b[i]);
        PROP_CUDA(cudaGetLastError());
        if (i > 0) {
            // data gradient: 'same' convolution of dpre with the flipped,
            // transposed taps -> gradient of conv i-1's pooled output
            ConvIn a{c->dpre, L, kCh, (taps - 1) / 2, kDil[i]};
            FlippedW b{c->pb + c->lay.w[i], taps, cin, kCh};
            Epi ep{kEpiStore, c->da[cur ^ 1], cin, nullptr, nullptr, nullptr};
            PROP_TRY(gemm((int)rows, cin, taps * kCh, 0, a, b, ep, st));
            cur ^= 1;
        }
    }
    return GTLS_OK;
}

gtls_status check_batch(const gtls_cnn* c, int B)
{
    if (!c) return set_error(GTLS_ERR_INVALID_ARG, "null network");
    if (B < 1 || B > c->max_batch)
        return set_error(GTLS_ERR_INVALID_ARG, "batch must be in [1, max_batch]");
    int dev = -1;
    PROP_CUDA(cudaGetDevice(&dev));
    if (dev != c->device) return set_error(GTLS_ERR_INVALID_ARG, "current device differs from the network's");
    return GTLS_OK;
}

}  // namespace

extern "C" {

int64_t gtls_cnn_param_count(void)
{
    return Layout().total;
}

gtls_status gtls_cnn_create(int32_t max_batch, const float* params, gtls_cnn** out)
{
    if (!out) return set_error(GTLS_ERR_INVALID_ARG, "null pointer argument");
    *out = nullptr;
    if (max_batch < 1 || max_batch > 4096) return set_error(GTLS_ERR_INVALID_ARG, "max_batch must be in [1, 4096]");
    gtls_cnn* c = new (std::nothrow) gtls_cnn();
    if (!c) return set_error(GTLS_ERR_OOM, "host allocation of the network failed");
    auto bail = [&](gtls_status s) {
        for (void* q : c->allocs) cudaFree(q);
        delete c;
        return s;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return bail(set_error(GTLS_ERR_CUDA, cudaGetErrorString(e)));
    c->max_batch = max_batch;
    const int64_t np = c->lay.total, B = max_batch;
    gtls_status s = GTLS_OK;
    auto A = [&](auto** ptr, int64_t cnt) {
        if (s == GTLS_OK) s = cnn_alloc(c, ptr, cnt);
    };
    A(&c->p, np);
    A(&c->pb, np);
    A(&c->g, np);
    A(&c->m, np);
    A(&c->v, np);
    A(&c->act[0], B * kBins);
    for (int i = 0; i < kConv; ++i) {
        A(&c->act[i + 1], B * (conv_len(i) / 2) * kCh);
        A(&c->arg[i], B * (conv_len(i) / 2) * kCh);
    }
    A(&c->z, B * kReg);
    A(&c->dz, B * kReg);
    A(&c->dz_b, B * kReg);
    A(&c->da[0], B * (kBins / 2) * kCh);
    A(&c->da[1], B * (kBins / 2) * kCh);
    A(&c->dpre, B * kBins * kCh);
    A(&c->loss, 1);
    A(&c->off, B + 1);
    if (s != GTLS_OK) return bail(s);
    std::vector<float> h(np, 0.0f);
    if (params) std::memcpy(h.data(), params, np * sizeof(float));
    if ((e = cudaMemcpy(c->p, h.data(), np * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(c->m, 0, np * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(c->v, 0, np * sizeof(float))) != cudaSuccess)
        return bail(set_error(GTLS_ERR_CUDA, cudaGetErrorString(e)));
    k_to_bf16<<<grid_for(np), 256>>>(c->p, c->pb, np);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(set_error(GTLS_ERR_CUDA, cudaGetErrorString(e)));
    if ((e = cudaFuncSetAttribute(k_bin, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  2 * kBins * (int)sizeof(double))) != cudaSuccess)
        return bail(set_error(GTLS_ERR_CUDA, cudaGetErrorString(e)));
    *out = c;
    return GTLS_OK;
}

gtls_status gtls_cnn_get_params(const gtls_cnn* c, float* params)
{
    if (!c || !params) return set_error(GTLS_ERR_INVALID_ARG, "null pointer argument");
    PROP_CUDA(cudaMemcpy(params, c->p, c->lay.total * sizeof(float), cudaMemcpyDeviceToHost));
    return GTLS_OK;
}

gtls_status gtls_cnn_set_params(gtls_cnn* c, const float* params)
{
    if (!c || !params) return set_error(GTLS_ERR_INVALID_ARG, "null pointer argument");
    PROP_CUDA(cudaMemcpy(c->p, params, c->lay.total * sizeof(float), cudaMemcpyHostToDevice));
    k_to_bf16<<<grid_for(c->lay.total), 256>>>(c->p, c->pb, c->lay.total);
    PROP_CUDA(cudaGetLastError());
    PROP_CUDA(cudaMemset(c->m, 0, c->lay.total * sizeof(float)));
    PROP_CUDA(cudaMemset(c->v, 0, c->lay.total * sizeof(float)));
    PROP_CUDA(cudaDeviceSynchronize());
    c->step = 0;
    return GTLS_OK;
}

gtls_status gtls_cnn_bin(gtls_cnn* c, const double* t, const double* y, const double* dy,
                         const int64_t* offsets, int64_t n_lc, float* x, float* mean, float* wsum,
                         void* stream)
{
    PROP_TRY(check_batch(c, (int)std::min<int64_t>(n_lc, 1 << 30)));
    if (!t || !y || !dy || !offsets || !x) return set_error(GTLS_ERR_INVALID_ARG, "null pointer argument");
    const int64_t o0 = offsets[0];
    std::vector<int64_t> off(n_lc + 1);
    for (int64_t i = 0; i <= n_lc; ++i) off[i] = offsets[i] - o0;
    for (int64_t i = 0; i < n_lc; ++i)
        if (off[i + 1] - off[i] < 1) return set_error(GTLS_ERR_INVALID_ARG, "every light curve needs a point");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PROP_CUDA(cudaMemcpyAsync(c->off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    k_bin<<<(unsigned)n_lc, 1024, 2 * kBins * sizeof(double), st>>>(t + o0, y + o0, dy + o0, c->off, x, mean, wsum);
    PROP_CUDA(cudaGetLastError());
    PROP_CUDA(cudaStreamSynchronize(st));   // the offsets live in host memory of this call
    return GTLS_OK;
}

gtls_status gtls_cnn_forward(gtls_cnn* c, const float* x, int32_t batch, float* logits, float* scores,
                             void* stream)
{
    PROP_TRY(check_batch(c, batch));
    if (!x) return set_error(GTLS_ERR_INVALID_ARG, "null input");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PROP_TRY(cnn_forward(c, x, batch, st));
    const int nz = batch * kReg;
    if (logits) PROP_CUDA(cudaMemcpyAsync(logits, c->z, nz * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (scores) {
        k_sigmoid<<<(nz + 255) / 256, 256, 0, st>>>(c->z, scores, nz);
        PROP_CUDA(cudaGetLastError());
    }
    return GTLS_OK;
}

gtls_status gtls_cnn_gradient(gtls_cnn* c, const float* x, const float* target, const float* mask,
                              int32_t batch, float* grad, double* loss, void* stream)
{
    PROP_TRY(check_batch(c, batch));
    if (!x || !target || !mask) return set_error(GTLS_ERR_INVALID_ARG, "null pointer argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PROP_TRY(cnn_forward(c, x, batch, st));
    PROP_TRY(cnn_backward(c, target, mask, batch, st));
    if (grad) PROP_CUDA(cudaMemcpyAsync(grad, c->g, c->lay.total * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (loss) PROP_CUDA(cudaMemcpyAsync(loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    PROP_CUDA(cudaStreamSynchronize(st));
    return GTLS_OK;
}

gtls_status gtls_cnn_train_step(gtls_cnn* c, const float* x, const float* target, const float* mask,
                                int32_t batch, float lr, double* loss, void* stream)
{
    PROP_TRY(check_batch(c, batch));
    if (!x || !target || !mask) return set_error(GTLS_ERR_INVALID_ARG, "null pointer argument");
    if (!(lr > 0.0f)) return set_error(GTLS_ERR_INVALID_ARG, "lr must be > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PROP_TRY(cnn_forward(c, x, batch, st));
    PROP_TRY(cnn_backward(c, target, mask, batch, st));
    c->step += 1;
    const float c1 = 1.0f - (float)std::pow(0.9, (double)c->step);
    const float c2 = 1.0f - (float)std::pow(0.999, (double)c->step);
    k_adam<<<grid_for(c->lay.total), 256, 0, st>>>(c->p, c->g, c->m, c->v, c->pb, c->lay.total, lr, c1, c2);
    PROP_CUDA(cudaGetLastError());
    if (loss) {
        PROP_CUDA(cudaMemcpyAsync(loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        PROP_CUDA(cudaStreamSynchronize(st));
    }
    return GTLS_OK;
}

gtls_status gtls_region_targets(const double* periods, const double* sr, int64_t n_periods, float* target,
                                float* mask)
{
    if (!periods || !sr || !target || !mask || n_periods < 0)
        return set_error(GTLS_ERR_INVALID_ARG, "null pointer argument");
    const double scale = kReg / std::log(kRegionHi / kRegionLo);
    std::fill(target, target + kReg, 0.0f);
    std::fill(mask, mask + kReg, 0.0f);
    std::vector<double> best(kReg, 0.0);
    for (int64_t i = 0; i < n_periods; ++i) {
        const int64_t r = (int64_t)std::floor(scale * std::log(periods[i] / kRegionLo));
        if (r < 0 || r >= kReg) continue;
        best[r] = std::max(best[r], sr[i]);
        mask[r] = 1.0f;
    }
    for (int r = 0; r < kReg; ++r) target[r] = (float)best[r];
    return GTLS_OK;
}

gtls_status gtls_proposal_periods(const double* periods, int64_t n_periods, const float* scores, double frac,
                                  int64_t* idx, int64_t* n_idx)
{
    if (!periods || !scores || !idx || !n_idx || n_periods < 0)
        return set_error(GTLS_ERR_INVALID_ARG, "null pointer argument");
    if (!(frac > 0.0 && frac <= 1.0)) return set_error(GTLS_ERR_INVALID_ARG, "frac must be in (0, 1]");
    const double scale = kReg / std::log(kRegionHi / kRegionLo);
    std::vector<int> reg(n_periods);
    std::vector<char> valid(kReg, 0);
    for (int64_t i = 0; i < n_periods; ++i) {
        const int64_t r = (int64_t)std::floor(scale * std::log(periods[i] / kRegionLo));
        reg[i] = (r < 0 || r >= kReg) ? -1 : (int)r;
        if (reg[i] >= 0) valid[reg[i]] = 1;
    }
    std::vector<int> cand;
    for (int r = 0; r < kReg; ++r)
        if (valid[r]) cand.push_back(r);
    const int k = std::max(1, (int)std::ceil(frac * (double)cand.size()));
    std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) { return scores[a] > scores[b]; });
    std::vector<char> keep(kReg, 0);
    for (int i = 0; i < k && i < (int)cand.size(); ++i) keep[cand[i]] = 1;
    int64_t n = 0;
    for (int64_t i = 0; i < n_periods; ++i)
        if (reg[i] >= 0 && keep[reg[i]]) idx[n++] = i;
    *n_idx = n;
    return GTLS_OK;
}

void gtls_cnn_destroy(gtls_cnn* c)
{
    if (!c) return;
    int cur = -1;
    const bool sw = cudaGetDevice(&cur) == cudaSuccess && cur != c->device && c->device >= 0;
    if (sw) cudaSetDevice(c->device);
    for (void* q : c->allocs) cudaFree(q);
    if (sw) cudaSetDevice(cur);
    delete c;
}

}  // extern "C"
