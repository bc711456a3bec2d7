// The learned form: a small multilayer perceptron that stands in for the
// coarsest-level solve of the V-cycle and predicts a warm-start guess.
//
// Network: four affine layers 2 n_r -> h -> h -> h -> n_r, ReLU after the
// first three, evaluated per column.  Weights are used in bfloat16 (rounded
// from FP32 masters after every update), activations and accumulation are
// FP32, biases FP32.  Training minimises the mean squared error with Adam
// (Kingma & Ba, 2015); every step -- forward, loss, backward, update -- runs
// in the kernels below.
//
// Features of a column T (on one multigrid level, vertical index k), in FP32:
//   x_T[k]       = f_Tk / (|T| v_k) / s,
//   x_T[n_r + k] = sum_e g_e f_{n_e k} / (|n_e| v_k) / (s sum_e g_e),
// i.e. the right-hand side as point values (cell integral over cell volume)
// of the column and the flux-weighted mean over its three edge neighbours
// (a symmetric function of the 1-ring, whose order is arbitrary on a
// triangle), scaled by the root mean square s of the point values over the
// whole level.  The network predicts u_T / s, so the map f -> u is equivariant
// under scaling of f, as the operator's inverse is.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tpmg_internal.h"
#include "../../include/tpmg_learned.h"

struct tpmg_net {
    int sizes[5] = {};            // layer widths: in, h, h, h, out
    size_t off_w[4] = {}, off_b[4] = {}, n_params = 0;
    float *master = nullptr;      // FP32 parameters: W_1 [h][in] row-major, b_1, W_2, b_2, ...
    float *grad = nullptr;        // gradient, same layout
    float *adam_m = nullptr, *adam_v = nullptr;
    uint16_t *wbf = nullptr;      // bfloat16 copy of master (the weights every pass uses)
    long step = 0;                // Adam steps taken
    cudaStream_t stream = nullptr;
    // training workspace: activations a_1..a_3, output y, two gradient
    // buffers, split-K partials of the weight gradients
    long ws_rows = 0;
    float *ws = nullptr;
    float *split = nullptr;
    size_t split_cap = 0;
    double *d_part = nullptr, *d_loss = nullptr, *h_loss = nullptr;
    std::string err;
};

namespace tpmg {

namespace {

constexpr int GBM = 64, GBN = 64, GBK = 16, GNT = 256;
constexpr int kLossBlocks = 256;

enum { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_RELU = 2, EPI_MASK = 3 };

__device__ __forceinline__ float ldf(float x) { return x; }
__device__ __forceinline__ float ldf(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// bfloat16 nearest, ties to even, of an FP32 value (NaN stays NaN)
__device__ __forceinline__ uint16_t to_bf16(float x)
{
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

template <int NT>
__device__ __forceinline__ double block_sum_d(double v)
{
    __shared__ double red[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < NT / 32 ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;   // valid in thread 0
}

// C[m][n] = epi(sum_{k in chunk z} A(m, k) B(k, n)), FP32 accumulation in
// ascending k.  A(m, k) = A[m lda + k], or A[k lda + m] if AT; B(k, n) =
// B[n ldb + k] if BT (a weight matrix [out][in]), else B[k ldb + n].  Split-K:
// block z covers k in [z k_chunk, (z+1) k_chunk) and writes slice z of C
// (C + z M ldc).  64 x 64 tile per CTA, 4 x 4 outputs per thread at rows
// ty + 16 i and columns tx + 16 j.
template <bool AT, bool BT, typename TB, int EPI>
__global__ void __launch_bounds__(GNT) k_gemm(int M, int N, int K, int k_chunk, const float *__restrict__ A, int lda,
                                              const TB *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                                              const float *__restrict__ bias, const float *__restrict__ mask, int ldm)
{
    __shared__ float As[GBK][GBM + 4];
    __shared__ float Bs[GBK][GBN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int kb = blockIdx.z * k_chunk, ke = min(K, kb + k_chunk);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += GBK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + GNT * q;   // 0 .. 1023: one element of each 64 x 16 tile
            const int am = AT ? e % GBM : e / GBK, ak = AT ? e / GBM : e % GBK;
            const int gm = m0 + am, gk = k0 + ak;
            As[ak][am] = (gm < M && gk < ke) ? (AT ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : 0.f;
            const int bn = BT ? e / GBK : e % GBN, bk = BT ? e % GBK : e / GBN;
            const int gn = n0 + bn, gk2 = k0 + bk;
            Bs[bk][bn] = (gn < N && gk2 < ke) ? ldf(BT ? B[(size_t)gn * ldb + gk2] : B[(size_t)gk2 * ldb + gn]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GBK; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float *Cz = C + (size_t)blockIdx.z * M * ldc;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            float v = acc[i][j];
            if (EPI == EPI_BIAS || EPI == EPI_BIAS_RELU) v += bias[n];
            if (EPI == EPI_BIAS_RELU) v = v > 0.f ? v : 0.f;
            if (EPI == EPI_MASK) v = mask[(size_t)m * ldm + n] > 0.f ? v : 0.f;
            Cz[(size_t)m * ldc + n] = v;
        }
    }
}

// out[z][c] = sum over rows r in chunk z (ascending) of G[r][c]
__global__ void __launch_bounds__(256) k_colsum(const float *__restrict__ G, int rows, int n, int k_chunk,
                                                float *__restrict__ out)
{
    __shared__ float part[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + tx;
    const int rb = blockIdx.y * k_chunk, re = min(rows, rb + k_chunk);
    float acc = 0.f;
    if (c < n)
        for (int r = rb + ty; r < re; r += 8) acc += G[(size_t)r * n + c];
    part[ty][tx] = acc;
    __syncthreads();
    if (ty == 0 && c < n) {
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) s += part[q][tx];
        out[(size_t)blockIdx.y * n + c] = s;
    }
}

// out[i] = sum_{z = 0 .. S-1} parts[z count + i]
__global__ void k_sum_slices(const float *__restrict__ parts, int S, long count, float *__restrict__ out)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < S; ++z) s += parts[(size_t)z * count + i];
        out[i] = s;
    }
}

// G = 2 (y - t) / n and per-block partial sums of (y - t)^2 (double)
__global__ void __launch_bounds__(256) k_mse(const float *__restrict__ y, const float *__restrict__ t, long n,
                                             float *__restrict__ g, double *__restrict__ partials)
{
    const float scale = (float)(2.0 / (double)n);
    double acc = 0.0;
    for (long i = blockIdx.x * 256L + threadIdx.x; i < n; i += (long)gridDim.x * 256) {
        const float d = y[i] - t[i];
        g[i] = scale * d;
        acc += (double)d * (double)d;
    }
    acc = block_sum_d<256>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// one block of 256 threads: a fixed-order tree sum of the partials
__global__ void __launch_bounds__(256) k_loss_finish(const double *__restrict__ partials, int np, long n,
                                                     double *__restrict__ loss)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += 256) v += partials[i];
    v = block_sum_d<256>(v);
    if (threadIdx.x == 0) *loss = v / (double)n;
}

// Adam with bias correction (c1 = 1 - b1^t, c2 = 1 - b2^t); refreshes the bfloat16 copy
__global__ void k_adam(long n, float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, uint16_t *__restrict__ wbf, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wbf[i] = to_bf16(wi);
    }
}

__global__ void k_round_bf16(long n, const float *__restrict__ w, uint16_t *__restrict__ wbf)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        wbf[i] = to_bf16(w[i]);
}

// ---- features -------------------------------------------------------------

// point values p = f / (|T| v_k) in FP32 -- each double converted once -- and
// per-block partial sums of p^2 (each thread's sum in FP32, the block's in double)
template <typename TF>
__global__ void __launch_bounds__(256) k_net_prepare(const TF *__restrict__ f, const float *__restrict__ iarea,
                                                     const float *__restrict__ ivol, long N, int n_r,
                                                     float *__restrict__ p, double *__restrict__ partials,
                                                     float *__restrict__ f32)
{
    float acc = 0.f;
    // 32-bit indices: a level holds fewer than 2^31 unknowns (checked at set-up)
    for (int i = blockIdx.x * 256 + threadIdx.x; i < (int)N; i += gridDim.x * 256) {
        const int T = i / n_r;
        const int k = i - T * n_r;
        const float fi = (float)f[i];
        if (f32) f32[i] = fi;
        const float v = fi * iarea[T] * ivol[k];
        p[i] = v;
        acc = fmaf(v, v, acc);
    }
    const double tot = block_sum_d<256>((double)acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// s = sqrt(sum / N) (0 for a zero field); one block of 256 threads, fixed-order tree sum
__global__ void __launch_bounds__(256) k_net_scale_finish(const double *__restrict__ partials, int np, long N,
                                                          double *__restrict__ s)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += 256) v += partials[i];
    v = block_sum_d<256>(v);
    if (threadIdx.x == 0) *s = sqrt(v / (double)N);
}

// inputs from the FP32 point values: the column and the flux-weighted mean over
// its edge neighbours, times 1 / s
__global__ void k_net_features(const float *__restrict__ p, const int4 *__restrict__ nbr,
                               const float4 *__restrict__ wnb, const int *__restrict__ cells, long rows, int n_r,
                               const double *__restrict__ s, float *__restrict__ X)
{
    const double sv = *s;
    const float inv = sv > 0.0 ? (float)(1.0 / sv) : 0.f;
    const int n = (int)(rows * n_r);   // < 2^31: rows * 2 n_r floats are addressed in 64 bits below
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = i / n_r;
        const int k = i - j * n_r;
        const int T = cells ? cells[j] : j;
        const int4 nb = nbr[T];
        const float4 w = wnb[T];
        const float mean = fmaf(w.z, p[nb.z * n_r + k], fmaf(w.y, p[nb.y * n_r + k], w.x * p[nb.x * n_r + k]));
        float *xr = X + (size_t)j * 2 * n_r;
        xr[k] = p[T * n_r + k] * inv;
        xr[n_r + k] = mean * inv;
    }
}

__global__ void k_net_targets(const double *__restrict__ u, const int *__restrict__ cells, long rows, int n_r,
                              const double *__restrict__ s, float *__restrict__ t)
{
    const double sv = *s;
    const double inv = sv > 0.0 ? 1.0 / sv : 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < rows * n_r; i += (long)gridDim.x * blockDim.x) {
        const long j = i / n_r;
        const int k = (int)(i - j * n_r);
        const long T = cells ? cells[j] : j;
        t[i] = (float)(u[T * n_r + k] * inv);
    }
}

template <typename TO>
__global__ void k_net_output(const float *__restrict__ y, long n, const double *__restrict__ s, TO *__restrict__ u)
{
    const float sv = (float)*s;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        u[i] = (TO)(sv * y[i]);
}

// judge of the initial guess: if the finish kernel rejected it, u = 0 and r = f
__global__ void k_judge_reset(const Scalars *__restrict__ sc, long n, const double *__restrict__ f,
                              double *__restrict__ u, double *__restrict__ r, float *__restrict__ r32)
{
    if (!(sc->info & 2)) return;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        u[i] = 0.0;
        r[i] = f[i];
        if (r32) r32[i] = (float)f[i];
    }
}

__global__ void k_to_f32(long n, const double *__restrict__ x, float *__restrict__ y)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

// ---- fused inference on the tensor cores ------------------------------------
//
// The whole network for 16 columns per warp with mma.sync m16n8k16 (bfloat16
// operands, FP32 accumulation): every weight matrix is staged once per CTA in
// shared memory ([out][in] rows padded by 8 bfloat16, so that the B fragments
// of the 8 row groups fall in distinct banks), and the activations never leave
// the registers: the accumulator fragments of two adjacent 8-column tiles are,
// after bias, ReLU and rounding to bfloat16, exactly the A fragment of one
// 16-wide k-step of the next layer.  Inputs are rounded to bfloat16 as they
// are loaded.  Hidden width 64; n_r a multiple of 8.
constexpr int kFusedH = 64;
constexpr int kFusedWarps = 8;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    return (uint32_t)to_bf16(lo) | ((uint32_t)to_bf16(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// accumulators of 8 n-tiles (64 columns) -> A fragments of the next layer's 4 k-steps
__device__ __forceinline__ void to_fragments(const float acc[8][4], const float *bias, int t, uint32_t h[4][4])
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c0 = 16 * j + 2 * t, c1 = c0 + 8;
        const float p0 = bias[c0], p1 = bias[c0 + 1], q0 = bias[c1], q1 = bias[c1 + 1];
        h[j][0] = pack_bf16(fmaxf(acc[2 * j][0] + p0, 0.f), fmaxf(acc[2 * j][1] + p1, 0.f));
        h[j][1] = pack_bf16(fmaxf(acc[2 * j][2] + p0, 0.f), fmaxf(acc[2 * j][3] + p1, 0.f));
        h[j][2] = pack_bf16(fmaxf(acc[2 * j + 1][0] + q0, 0.f), fmaxf(acc[2 * j + 1][1] + q1, 0.f));
        h[j][3] = pack_bf16(fmaxf(acc[2 * j + 1][2] + q0, 0.f), fmaxf(acc[2 * j + 1][3] + q1, 0.f));
    }
}

// one hidden layer (64 -> 64) on the fragments h, in place
__device__ __forceinline__ void hidden_layer(uint32_t h[4][4], const uint32_t *w, int ldw, const float *bias, int g,
                                             int t)
{
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const uint32_t *wr = w + (nt * 8 + g) * ldw + 8 * j + t;
            mma_bf16(acc[nt], h[j], wr[0], wr[4]);
        }
    to_fragments(acc, bias, t, h);
}

template <typename TO>
__global__ void __launch_bounds__(32 * kFusedWarps) k_mlp_fused(const float *__restrict__ X, long rows, int n_r,
                                                                 NetView v, const double *__restrict__ s,
                                                                 TO *__restrict__ out)
{
    extern __shared__ uint32_t sm[];
    const int K1 = 2 * n_r;
    const int ld1 = K1 / 2 + 4, ldh = kFusedH / 2 + 4;   // words per padded row
    uint32_t *s1 = sm, *s2 = s1 + kFusedH * ld1, *s3 = s2 + kFusedH * ldh, *s4 = s3 + kFusedH * ldh;
    float *sb = reinterpret_cast<float *>(s4 + n_r * ldh);   // b_1 | b_2 | b_3 | b_4
    {
        const uint32_t *g1 = reinterpret_cast<const uint32_t *>(v.w[0]);
        for (int i = threadIdx.x; i < kFusedH * (K1 / 2); i += blockDim.x)
            s1[(i / (K1 / 2)) * ld1 + i % (K1 / 2)] = g1[i];
        const uint32_t *g2 = reinterpret_cast<const uint32_t *>(v.w[1]);
        const uint32_t *g3 = reinterpret_cast<const uint32_t *>(v.w[2]);
        for (int i = threadIdx.x; i < kFusedH * (kFusedH / 2); i += blockDim.x) {
            s2[(i / (kFusedH / 2)) * ldh + i % (kFusedH / 2)] = g2[i];
            s3[(i / (kFusedH / 2)) * ldh + i % (kFusedH / 2)] = g3[i];
        }
        const uint32_t *g4 = reinterpret_cast<const uint32_t *>(v.w[3]);
        for (int i = threadIdx.x; i < n_r * (kFusedH / 2); i += blockDim.x)
            s4[(i / (kFusedH / 2)) * ldh + i % (kFusedH / 2)] = g4[i];
        for (int i = threadIdx.x; i < kFusedH; i += blockDim.x) {
            sb[i] = v.b[0][i];
            sb[kFusedH + i] = v.b[1][i];
            sb[2 * kFusedH + i] = v.b[2][i];
        }
        for (int i = threadIdx.x; i < n_r; i += blockDim.x) sb[3 * kFusedH + i] = v.b[3][i];
    }
    __syncthreads();
    const float sv = (float)*s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long n_tiles = (rows + 15) / 16;
    for (long tile = (long)blockIdx.x * kFusedWarps + warp; tile < n_tiles; tile += (long)gridDim.x * kFusedWarps) {
        const long r0 = tile * 16 + g, r1 = r0 + 8;
        const bool v0 = r0 < rows, v1 = r1 < rows;
        const float *x0 = X + r0 * K1 + 2 * t, *x1 = X + r1 * K1 + 2 * t;
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
        for (int kk = 0; kk < K1; kk += 16) {
            const float2 z = make_float2(0.f, 0.f);
            const float2 a00 = v0 ? __ldg(reinterpret_cast<const float2 *>(x0 + kk)) : z;
            const float2 a10 = v1 ? __ldg(reinterpret_cast<const float2 *>(x1 + kk)) : z;
            const float2 a01 = v0 ? __ldg(reinterpret_cast<const float2 *>(x0 + kk + 8)) : z;
            const float2 a11 = v1 ? __ldg(reinterpret_cast<const float2 *>(x1 + kk + 8)) : z;
            const uint32_t a[4] = {pack_bf16(a00.x, a00.y), pack_bf16(a10.x, a10.y), pack_bf16(a01.x, a01.y),
                                   pack_bf16(a11.x, a11.y)};
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const uint32_t *wr = s1 + (nt * 8 + g) * ld1 + kk / 2 + t;
                mma_bf16(acc[nt], a, wr[0], wr[4]);
            }
        }
        uint32_t h[4][4];
        to_fragments(acc, sb, t, h);
        hidden_layer(h, s2, ldh, sb + kFusedH, g, t);
        hidden_layer(h, s3, ldh, sb + 2 * kFusedH, g, t);
        const float *b4 = sb + 3 * kFusedH;
        for (int n0 = 0; n0 < n_r; n0 += 64) {
            const int ntn = min(8, (n_r - n0) / 8);
            float o[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) o[nt][0] = o[nt][1] = o[nt][2] = o[nt][3] = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int nt = 0; nt < 8; ++nt)
                    if (nt < ntn) {
                        const uint32_t *wr = s4 + (n0 + nt * 8 + g) * ldh + 8 * j + t;
                        mma_bf16(o[nt], h[j], wr[0], wr[4]);
                    }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
                if (nt < ntn) {
                    const int c = n0 + nt * 8 + 2 * t;
                    if (v0) {
                        out[r0 * n_r + c] = (TO)(sv * (o[nt][0] + b4[c]));
                        out[r0 * n_r + c + 1] = (TO)(sv * (o[nt][1] + b4[c + 1]));
                    }
                    if (v1) {
                        out[r1 * n_r + c] = (TO)(sv * (o[nt][2] + b4[c]));
                        out[r1 * n_r + c + 1] = (TO)(sv * (o[nt][3] + b4[c + 1]));
                    }
                }
        }
    }
}

// ---- fused inference on the 5th-generation tensor cores (tcgen05) ----------
//
// The network for tiles of 128 columns per CTA on tcgen05.mma (kind::f16:
// bfloat16 operands in shared memory, FP32 accumulators in tensor memory).
// Per layer one thread issues the chain of MMAs D[128 x N] = A[128 x K] W^T
// (K / 16 instructions) and tcgen05.commit signals their completion on an
// mbarrier; then every warp reads 32 rows of D from tensor memory
// (tcgen05.ld), adds the bias, applies ReLU and rounds to bfloat16 into the
// next layer's A tile in shared memory, and the last layer scales its D and
// writes the output.  The operands use the K-major layout without swizzle:
// core matrices of 8 rows x 16 bytes (row stride 16 B), adjacent along K at
// 128 bytes (the descriptor's leading byte offset) and 8-row groups at
// K * 16 bytes (its stride byte offset).  The rounding is that of
// k_mlp_fused: inputs and hidden activations in bfloat16, FP32 accumulation
// (in the tensor cores' order).  Every mbarrier wait is bounded: a CTA that
// gives up writes NaN over the outputs it has not written, sets *err, frees
// its tensor memory and returns.
constexpr int kTcRows = 128;        // rows (grid columns) per tile = the MMA's M
constexpr int kTcThreads = 256;     // 8 warps: warp w reads TMEM lanes 32 (w % 4) + 0..31, column half w / 4
constexpr uint32_t kTcCols = 128;   // tensor-memory columns allocated (>= 64 and >= n_r)
constexpr long kTcSpin = 1L << 22;  // mbarrier polls before a CTA gives up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a K-major tile with K columns (no swizzle)
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int K)
{
    return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading and stride byte
// offsets (in 16-byte units), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D in FP32, A and B bfloat16, both K-major, N x M = n x 128
__device__ __forceinline__ uint32_t umma_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// generic-proxy writes of shared memory made visible to the tensor cores' (async proxy) reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// wait until the phase with the given parity has completed; false after kTcSpin polls
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (long i = 0; i < kTcSpin; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 8 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// weights W [N][K] (bfloat16, row-major) into the K-major tile
__device__ __forceinline__ void tc_stage_w(const uint16_t *__restrict__ g, uint8_t *dst, int N, int K)
{
    const int cpr = K / 8;
    for (int i = threadIdx.x; i < N * cpr; i += kTcThreads) {
        const int n = i / cpr, c = i - n * cpr;
        const uint4 val = __ldg(reinterpret_cast<const uint4 *>(g + (size_t)n * K + c * 8));
        *reinterpret_cast<uint4 *>(dst + kmajor_off(n, c * 8, K)) = val;
    }
}

// one layer's MMA chain D = A W^T over K (issued by one thread) and its commit
__device__ __forceinline__ void tc_layer(uint32_t d_tmem, uint32_t a_s, uint32_t w_s, int K, int N, uint32_t mbar)
{
    const uint32_t idesc = umma_idesc(N);
    for (int k = 0; k < K; k += 16)
        umma_bf16(d_tmem, umma_desc(a_s + k * 16, 128, K * 16), umma_desc(w_s + k * 16, 128, K * 16), idesc, k > 0);
    umma_commit(mbar);
}

// hidden epilogue: this thread's row, its 32 of the 64 columns: bias, ReLU, bfloat16 into H
__device__ __forceinline__ void tc_epi_hidden(uint32_t t_row, int row, int half, const float *bias, uint8_t *ht)
{
#pragma unroll
    for (int c0 = 0; c0 < 32; c0 += 8) {
        const int col = half * 32 + c0;
        float d[8];
        tmem_ld8(t_row + col, d);
        uint4 p;
        p.x = pack_bf16(fmaxf(d[0] + bias[col + 0], 0.f), fmaxf(d[1] + bias[col + 1], 0.f));
        p.y = pack_bf16(fmaxf(d[2] + bias[col + 2], 0.f), fmaxf(d[3] + bias[col + 3], 0.f));
        p.z = pack_bf16(fmaxf(d[4] + bias[col + 4], 0.f), fmaxf(d[5] + bias[col + 5], 0.f));
        p.w = pack_bf16(fmaxf(d[6] + bias[col + 6], 0.f), fmaxf(d[7] + bias[col + 7], 0.f));
        *reinterpret_cast<uint4 *>(ht + kmajor_off(row, col, kFusedH)) = p;
    }
}

__device__ __forceinline__ void tc_store8(float *o, const float v[8])
{
    reinterpret_cast<float4 *>(o)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4 *>(o)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void tc_store8(double *o, const float v[8])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) reinterpret_cast<double2 *>(o)[i] = make_double2(v[2 * i], v[2 * i + 1]);
}

// mbarrier arrival that also expects `bytes` of asynchronous copies in this phase
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

// one bulk copy global -> shared memory, completed on the mbarrier (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// The network's inputs (those of k_net_features, over every column of the level)
// rounded to bfloat16 and written in the A-tile layout of k_mlp_tc: tile t of 128
// rows at t * 128 * 2 n_r elements, K-major without swizzle; rows past `rows` are
// zero.  A warp's 32 chunks of 8 inputs are 8 rows x 4 chunks, so that each row's
// loads are 128 contiguous bytes and each 8 lanes store 128 contiguous bytes.
__global__ void __launch_bounds__(256) k_net_features_tiled(const float *__restrict__ p, const int4 *__restrict__ nbr,
                                                            const float4 *__restrict__ wnb, long rows, int n_r,
                                                            const double *__restrict__ s, uint16_t *__restrict__ Xt)
{
    const double sv = *s;
    const float inv = sv > 0.0 ? (float)(1.0 / sv) : 0.f;
    const int K1 = 2 * n_r, cpr = K1 / 8, nb = cpr / 4, half = n_r / 8;
    const long per_tile = (long)kTcRows * cpr, n_tiles = (rows + kTcRows - 1) / kTcRows;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n_tiles * per_tile;
         i += (long)gridDim.x * blockDim.x) {
        const long t = i / per_tile;
        const int w = (int)(i - t * per_tile), l = w & 31, blk = w >> 5, g = blk / nb, cb = blk - g * nb;
        const int r = g * 8 + (l & 7), c = cb * 4 + (l >> 3);
        const long j = t * kTcRows + r;
        float x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = 0.f;
        if (j < rows) {
            const int T = (int)j;
            if (c < half) {
                const float *src = p + (size_t)T * n_r + 8 * c;
#pragma unroll
                for (int q = 0; q < 8; ++q) x[q] = src[q] * inv;
            } else {
                const int k0 = 8 * (c - half);
                const int4 nb4 = nbr[T];
                const float4 wv = wnb[T];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = k0 + q;
                    const float mean = fmaf(wv.z, p[nb4.z * n_r + k], fmaf(wv.y, p[nb4.y * n_r + k], wv.x * p[nb4.x * n_r + k]));
                    x[q] = mean * inv;
                }
            }
        }
        uint4 o;
        o.x = pack_bf16(x[0], x[1]);
        o.y = pack_bf16(x[2], x[3]);
        o.z = pack_bf16(x[4], x[5]);
        o.w = pack_bf16(x[6], x[7]);
        *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(Xt) + t * ((long)kTcRows * K1 * 2) +
                                   kmajor_off(r, 8 * c, K1)) = o;
    }
}

// The network on tcgen05 for the A tiles of k_net_features_tiled.  Each CTA walks its
// tiles with two A buffers: while one tile's four layers run, one thread's bulk copy
// brings the next tile's inputs into the other buffer (completion on that buffer's
// mbarrier).
template <typename TO>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_mlp_tc(const uint16_t *__restrict__ Xt, long rows, int n_r, NetView v, const double *__restrict__ s,
             TO *__restrict__ out, int *__restrict__ err)
{
    extern __shared__ __align__(128) uint8_t tsm[];
    const int K1 = 2 * n_r, H = kFusedH;
    const uint32_t a_bytes = (uint32_t)kTcRows * K1 * 2;
    uint8_t *w1 = tsm;                      // [H][K1]
    uint8_t *w2 = w1 + H * K1 * 2;          // [H][H]
    uint8_t *w3 = w2 + H * H * 2;           // [H][H]
    uint8_t *w4 = w3 + H * H * 2;           // [n_r][H]
    uint8_t *at = w4 + n_r * H * 2;         // two A tiles [128][K1]
    uint8_t *ht = at + 2 * a_bytes;         // hidden tile [128][H]
    float *sb = reinterpret_cast<float *>(ht + kTcRows * H * 2);   // b_1 | b_2 | b_3 | b_4
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sb + 3 * H + n_r);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(tslot + 2);      // [0] MMAs, [1], [2] the A buffers' loads
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t mb = smem_u32(mbar), mb_ld0 = smem_u32(mbar + 1), mb_ld1 = smem_u32(mbar + 2);
    const uint32_t a_s0 = smem_u32(at), a_s1 = smem_u32(at + a_bytes);
    const long n_tiles = (rows + kTcRows - 1) / kTcRows;
    if (tid == 0) {
        mbar_init(mb, 1);
        mbar_init(mb_ld0, 1);
        mbar_init(mb_ld1, 1);
    }
    __syncthreads();
    long tile = blockIdx.x;
    if (tid == 0 && tile < n_tiles) {   // the first tile's inputs, while the weights are staged
        mbar_expect_tx(mb_ld0, a_bytes);
        bulk_g2s(a_s0, reinterpret_cast<const uint8_t *>(Xt) + tile * a_bytes, a_bytes, mb_ld0);
    }
    tc_stage_w(v.w[0], w1, H, K1);
    tc_stage_w(v.w[1], w2, H, H);
    tc_stage_w(v.w[2], w3, H, H);
    tc_stage_w(v.w[3], w4, n_r, H);
    for (int i = tid; i < H; i += kTcThreads) {
        sb[i] = v.b[0][i];
        sb[H + i] = v.b[1][i];
        sb[2 * H + i] = v.b[2][i];
    }
    for (int i = tid; i < n_r; i += kTcThreads) sb[3 * H + i] = v.b[3][i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const int q = warp & 3, half = warp >> 2, row = q * 32 + lane;
    const uint32_t t_row = tmem + ((uint32_t)(q * 32) << 16);   // this warp's lane quarter
    const uint32_t h_s = smem_u32(ht);
    const uint32_t w1_s = smem_u32(w1), w2_s = smem_u32(w2), w3_s = smem_u32(w3), w4_s = smem_u32(w4);
    const float sv = (float)*s;
    // per A buffer: its load phase parity and whether a copy into it is in flight (bits 0, 1)
    uint32_t phase = 0, ld_phase = 0, pending = tile < n_tiles ? 1u : 0u;
    bool failed = false;
    for (int it = 0; tile < n_tiles; ++it, tile += gridDim.x) {
        const int b = it & 1;
        const uint32_t mb_cur = b ? mb_ld1 : mb_ld0, mb_oth = b ? mb_ld0 : mb_ld1;
        const long next = tile + gridDim.x;
        if (tid == 0 && next < n_tiles) {   // the next tile's inputs into the other buffer (its MMAs are done)
            mbar_expect_tx(mb_oth, a_bytes);
            bulk_g2s(b ? a_s0 : a_s1, reinterpret_cast<const uint8_t *>(Xt) + next * a_bytes, a_bytes, mb_oth);
        }
        if (next < n_tiles) pending |= 1u << (b ^ 1);
        bool ok = __syncthreads_and(mbar_wait(mb_cur, (ld_phase >> b) & 1u)) != 0;
        if (ok) {
            ld_phase ^= 1u << b;
            pending &= ~(1u << b);
        }
        const long r0 = tile * kTcRows;
#pragma unroll 1
        for (int l = 0; l < 4 && ok; ++l) {
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                if (l == 0) tc_layer(tmem, b ? a_s1 : a_s0, w1_s, K1, H, mb);
                else tc_layer(tmem, h_s, l == 1 ? w2_s : (l == 2 ? w3_s : w4_s), H, l == 3 ? n_r : H, mb);
            }
            ok = __syncthreads_and(mbar_wait(mb, phase)) != 0;
            if (!ok) break;
            phase ^= 1;
            tc_fence_after();
            if (l < 3) {
                tc_epi_hidden(t_row, row, half, sb + l * H, ht);
            } else {
                const long gr = r0 + row;
                const int per = n_r / 2;
                for (int c0 = 0; c0 < per; c0 += 8) {
                    const int col = half * per + c0;
                    float d[8];
                    tmem_ld8(t_row + col, d);
#pragma unroll
                    for (int i = 0; i < 8; ++i) d[i] = sv * (d[i] + sb[3 * H + col + i]);
                    if (gr < rows) tc_store8(out + gr * n_r + col, d);
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        if (!ok) {
            failed = true;
            break;
        }
    }
    if (failed) {   // the outputs of this CTA's remaining tiles are not valid
        for (; tile < n_tiles; tile += gridDim.x)
            for (long i = tid; i < (long)kTcRows * n_r; i += kTcThreads) {
                const long gr = tile * kTcRows + i / n_r;
                if (gr < rows) out[gr * n_r + i % n_r] = (TO)NAN;
            }
        if (tid == 0) {
            atomicExch(err, 1);
            // let the copies and MMAs still in flight finish (bounded) before the memory is released
            if (pending & 1u) (void)mbar_wait(mb_ld0, ld_phase & 1u);
            if (pending & 2u) (void)mbar_wait(mb_ld1, (ld_phase >> 1) & 1u);
            (void)mbar_wait(mb, phase);
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcCols) : "memory");
    }
}

size_t tc_smem_bytes(int n_r)
{
    const size_t K1 = 2 * (size_t)n_r, H = kFusedH;
    const size_t b = H * K1 * 2 + 2 * H * H * 2 + (size_t)n_r * H * 2 + 2 * kTcRows * K1 * 2 + kTcRows * H * 2 +
                     (3 * H + (size_t)n_r) * 4 + 32;
    // at least 116 KB: one CTA per SM, so that its tensor-memory allocation never waits for another's
    return std::max<size_t>(b, 116 * 1024);
}

size_t fused_smem_bytes(int n_r)
{
    const size_t ld1 = (size_t)n_r + 4, ldh = kFusedH / 2 + 4;
    return 4 * (kFusedH * ld1 + 2 * kFusedH * ldh + (size_t)n_r * ldh + 3 * kFusedH + (size_t)n_r);
}

inline int grid_1d(long work, int nt, int sm_count)
{
    long b = (work + nt - 1) / nt;
    const long cap = (long)std::max(sm_count, 1) * 8;
    return (int)std::max(1L, std::min(b, cap));
}

template <bool AT, bool BT, typename TB, int EPI>
cudaError_t gemm(cudaStream_t s, int M, int N, int K, int splits, const float *A, int lda, const TB *B, int ldb,
                 float *C, int ldc, const float *bias = nullptr, const float *mask = nullptr, int ldm = 0)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    splits = std::max(1, splits);
    int chunk = (K + splits - 1) / splits;
    chunk = std::max(GBK, (chunk + GBK - 1) / GBK * GBK);
    splits = std::max(1, (K + chunk - 1) / chunk);
    const dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM, splits);
    k_gemm<AT, BT, TB, EPI><<<grid, GNT, 0, s>>>(M, N, K, chunk, A, lda, B, ldb, C, ldc, bias, mask, ldm);
    return cudaGetLastError();
}

int sm_count_of_current()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return std::max(n, 1);
}

}  // namespace

// ---- launchers shared with api.cu ------------------------------------------

NetView net_view(const tpmg_net *net)
{
    NetView v{};
    for (int i = 0; i < 5; ++i) v.sizes[i] = net->sizes[i];
    for (int l = 0; l < 4; ++l) {
        v.w[l] = net->wbf + net->off_w[l];
        v.b[l] = net->master + net->off_b[l];
    }
    return v;
}

cudaError_t launch_net_layer(cudaStream_t s, const NetView &v, int l, const float *x, long rows, float *y)
{
    const int in = v.sizes[l], out = v.sizes[l + 1];
    if (l < 3)
        return gemm<false, true, uint16_t, EPI_BIAS_RELU>(s, (int)rows, out, in, 1, x, in, v.w[l], in, y, out, v.b[l]);
    return gemm<false, true, uint16_t, EPI_BIAS>(s, (int)rows, out, in, 1, x, in, v.w[l], in, y, out, v.b[l]);
}

bool net_tc_ok(const NetView &v)
{
    const int n_r = v.sizes[4];
    return v.sizes[1] == kFusedH && v.sizes[2] == kFusedH && v.sizes[3] == kFusedH && v.sizes[0] == 2 * n_r &&
           n_r % 16 == 0 && n_r >= 16 && n_r <= (int)kTcCols && tc_smem_bytes(n_r) <= 227 * 1024;
}

size_t net_tc_input_elems(long rows, int n_r) { return (size_t)((rows + kTcRows - 1) / kTcRows) * kTcRows * 2 * n_r; }

cudaError_t launch_net_features_tiled(const Launch &L, const LevelDev &lv, const float *p, long rows,
                                      const double *s, uint16_t *Xt)
{
    const long chunks = (long)net_tc_input_elems(rows, L.n_r) / 8;
    k_net_features_tiled<<<grid_1d(chunks, 256, L.sm_count), 256, 0, L.s>>>(p, lv.nbr, lv.wnb32, rows, L.n_r, s, Xt);
    return cudaGetLastError();
}

template <typename TO>
cudaError_t launch_net_tc(const Launch &L, const NetView &v, const uint16_t *Xt, long rows, const double *s, TO *out,
                          int *err)
{
    const int n_r = v.sizes[4];
    const size_t smem = tc_smem_bytes(n_r);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_tc<TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long tiles = (rows + kTcRows - 1) / kTcRows;
    const int grid = (int)std::max<long>(1, std::min<long>(tiles, (long)std::max(L.sm_count, 1)));
    k_mlp_tc<TO><<<grid, kTcThreads, smem, L.s>>>(Xt, rows, n_r, v, s, out, err);
    return cudaGetLastError();
}

bool net_fused_ok(const NetView &v)
{
    const int n_r = v.sizes[4];
    return v.sizes[1] == kFusedH && v.sizes[2] == kFusedH && v.sizes[3] == kFusedH && v.sizes[0] == 2 * n_r &&
           n_r % 8 == 0 && fused_smem_bytes(n_r) <= 200 * 1024;
}

template <typename TO>
cudaError_t launch_net_fused(const Launch &L, const NetView &v, const float *X, long rows, const double *s, TO *out)
{
    const int n_r = v.sizes[4];
    const size_t smem = fused_smem_bytes(n_r);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_fused<TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long tiles = (rows + 15) / 16;
    const long per_sm = std::max<long>(1, (long)(220 * 1024 / std::max<size_t>(smem, 1)));
    const long grid = std::max<long>(1, std::min<long>((tiles + kFusedWarps - 1) / kFusedWarps,
                                                       (long)std::max(L.sm_count, 1) * std::min<long>(per_sm, 4)));
    k_mlp_fused<TO><<<(int)grid, 32 * kFusedWarps, smem, L.s>>>(X, rows, n_r, v, s, out);
    return cudaGetLastError();
}

template <typename TF>
cudaError_t launch_net_prepare(const Launch &L, const LevelDev &lv, const VertDev &vert, const TF *f, float *p,
                               double *partials, int n_part, float *f32)
{
    const long N = (long)lv.n * L.n_r;
    k_net_prepare<TF><<<n_part, 256, 0, L.s>>>(f, lv.iarea32, vert.ivol32, N, L.n_r, p, partials, f32);
    return cudaGetLastError();
}

cudaError_t launch_net_scale_finish(const Launch &L, const LevelDev &lv, const double *partials, int n_part, double *s)
{
    k_net_scale_finish<<<1, 256, 0, L.s>>>(partials, n_part, (long)lv.n * L.n_r, s);
    return cudaGetLastError();
}

cudaError_t launch_net_features(const Launch &L, const LevelDev &lv, const float *p, const int *cells, long rows,
                                const double *s, float *X)
{
    if (rows <= 0) return cudaSuccess;
    k_net_features<<<grid_1d(rows * L.n_r, 256, L.sm_count), 256, 0, L.s>>>(p, lv.nbr, lv.wnb32, cells, rows, L.n_r,
                                                                          s, X);
    return cudaGetLastError();
}

cudaError_t launch_net_targets(const Launch &L, const double *u, const int *cells, long rows, const double *s, float *t)
{
    if (rows <= 0) return cudaSuccess;
    k_net_targets<<<grid_1d(rows * L.n_r, 256, L.sm_count), 256, 0, L.s>>>(u, cells, rows, L.n_r, s, t);
    return cudaGetLastError();
}

template <typename TO>
cudaError_t launch_net_output(const Launch &L, const float *y, long n, const double *s, TO *u)
{
    k_net_output<TO><<<grid_1d(n, 256, L.sm_count), 256, 0, L.s>>>(y, n, s, u);
    return cudaGetLastError();
}

cudaError_t launch_judge_reset(const Launch &L, const Scalars *sc, long n, const double *f, double *u, double *r,
                               float *r32)
{
    k_judge_reset<<<grid_1d(n, 256, L.sm_count), 256, 0, L.s>>>(sc, n, f, u, r, r32);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const Launch &L, long n, const double *x, float *y)
{
    k_to_f32<<<grid_1d(n, 256, L.sm_count), 256, 0, L.s>>>(n, x, y);
    return cudaGetLastError();
}

template cudaError_t launch_net_prepare<float>(const Launch &, const LevelDev &, const VertDev &, const float *, float *,
                                               double *, int, float *);
template cudaError_t launch_net_prepare<double>(const Launch &, const LevelDev &, const VertDev &, const double *,
                                                float *, double *, int, float *);
template cudaError_t launch_net_tc<float>(const Launch &, const NetView &, const uint16_t *, long, const double *,
                                          float *, int *);
template cudaError_t launch_net_tc<double>(const Launch &, const NetView &, const uint16_t *, long, const double *,
                                           double *, int *);
template cudaError_t launch_net_fused<float>(const Launch &, const NetView &, const float *, long, const double *, float *);
template cudaError_t launch_net_fused<double>(const Launch &, const NetView &, const float *, long, const double *,
                                              double *);
template cudaError_t launch_net_output<float>(const Launch &, const float *, long, const double *, float *);
template cudaError_t launch_net_output<double>(const Launch &, const float *, long, const double *, double *);

}  // namespace tpmg

// ---- C ABI: the network -----------------------------------------------------

using namespace tpmg;

namespace {

tpmg_status net_fail(tpmg_net *net, tpmg_status s, const std::string &msg)
{
    if (net) net->err = msg;
    return s;
}

#define NCU(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return net_fail(net, e_ == cudaErrorMemoryAllocation ? TPMG_ERR_OOM : TPMG_ERR_CUDA,  \
                            std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

constexpr long kMaxRows = 64L * 65535L;   // rows of one pass (grid.y limit of the GEMM)

// workspace floats per row: a_1..a_3 (3 h), y (out), two gradient buffers (2 max(h, out))
long ws_per_row(const tpmg_net *net)
{
    const long h = net->sizes[1], out = net->sizes[4];
    return 3 * h + out + 2 * std::max(h, out);
}

tpmg_status ensure_ws(tpmg_net *net, long rows, bool training)
{
    if (rows > net->ws_rows) {
        if (net->ws) cudaFree(net->ws);
        net->ws = nullptr;
        net->ws_rows = 0;
        NCU(cudaMalloc(&net->ws, sizeof(float) * (size_t)rows * ws_per_row(net)));
        net->ws_rows = rows;
    }
    if (training) {
        // split-K slices of the largest weight gradient; chunks of >= 256 rows
        const int splits = (int)std::min<long>(64, std::max<long>(1, rows / 256));
        size_t need = 0;
        for (int l = 0; l < 4; ++l) need = std::max(need, (size_t)net->sizes[l] * net->sizes[l + 1]);
        need = need * splits + (size_t)splits * std::max(net->sizes[1], net->sizes[4]);
        if (need > net->split_cap) {
            if (net->split) cudaFree(net->split);
            net->split = nullptr;
            net->split_cap = 0;
            NCU(cudaMalloc(&net->split, sizeof(float) * need));
            net->split_cap = need;
        }
    }
    return TPMG_OK;
}

// forward pass into the workspace: a_l at ws + (l-1) rows h (l = 1..3), y after them
tpmg_status forward_ws(tpmg_net *net, const float *x, long rows, float **acts, float **y)
{
    const long h = net->sizes[1];
    float *a = net->ws;
    acts[0] = const_cast<float *>(x);
    for (int l = 1; l < 4; ++l) acts[l] = a + (size_t)(l - 1) * rows * h;
    *y = a + (size_t)3 * rows * h;
    const NetView v = net_view(net);
    for (int l = 0; l < 4; ++l) NCU(launch_net_layer(net->stream, v, l, acts[l], rows, l < 3 ? acts[l + 1] : *y));
    return TPMG_OK;
}

// loss and gradient (parameter layout) into net->grad / out; the loss stays on the device
tpmg_status backward_ws(tpmg_net *net, const float *x, const float *t, long rows, float *gout)
{
    float *acts[4], *y;
    tpmg_status st = forward_ws(net, x, rows, acts, &y);
    if (st != TPMG_OK) return st;
    const long h = net->sizes[1], out = net->sizes[4];
    float *g0 = y + (size_t)rows * out, *g1 = g0 + (size_t)rows * std::max(h, out);
    const long n = rows * out;
    k_mse<<<kLossBlocks, 256, 0, net->stream>>>(y, t, n, g0, net->d_part);
    NCU(cudaGetLastError());
    k_loss_finish<<<1, 256, 0, net->stream>>>(net->d_part, kLossBlocks, n, net->d_loss);
    NCU(cudaGetLastError());
    const int splits = (int)std::min<long>(64, std::max<long>(1, rows / 256));
    const NetView v = net_view(net);
    float *g = g0, *gn = g1;
    for (int l = 3; l >= 0; --l) {
        const int in = net->sizes[l], o = net->sizes[l + 1];
        // dW_l = G_l^T a_{l-1}: split-K over the rows, then the slices summed in order
        NCU((gemm<true, false, float, EPI_NONE>(net->stream, o, in, (int)rows, splits, g, o, acts[l], in, net->split, in)));
        int chunk = (int)((rows + splits - 1) / splits);
        chunk = std::max(GBK, (chunk + GBK - 1) / GBK * GBK);
        const int S = (int)((rows + chunk - 1) / chunk);
        const long nw = (long)o * in;
        k_sum_slices<<<grid_1d(nw, 256, sm_count_of_current()), 256, 0, net->stream>>>(net->split, S, nw,
                                                                                     gout + net->off_w[l]);
        NCU(cudaGetLastError());
        // db_l = column sums of G_l (same row chunks)
        float *cs = net->split + (size_t)S * nw;
        k_colsum<<<dim3((o + 31) / 32, S), 256, 0, net->stream>>>(g, (int)rows, o, chunk, cs);
        NCU(cudaGetLastError());
        k_sum_slices<<<1, 256, 0, net->stream>>>(cs, S, o, gout + net->off_b[l]);
        NCU(cudaGetLastError());
        if (l > 0) {
            // G_{l-1} = (G_l W_l) * [a_{l-1} > 0]
            NCU((gemm<false, false, uint16_t, EPI_MASK>(net->stream, (int)rows, in, o, 1, g, o, v.w[l], in, gn, in,
                                                          nullptr, acts[l], in)));
            std::swap(g, gn);
        }
    }
    return TPMG_OK;
}

tpmg_status check_rows(tpmg_net *net, const void *x, const void *p2, long rows)
{
    if (!x || !p2) return net_fail(net, TPMG_ERR_INVALID_ARG, "NULL pointer");
    if (rows < 1 || rows > kMaxRows) return net_fail(net, TPMG_ERR_INVALID_ARG, "rows must be in 1..4194240");
    return TPMG_OK;
}

tpmg_status read_loss(tpmg_net *net, double *h_loss)
{
    if (!h_loss) return TPMG_OK;
    NCU(cudaMemcpyAsync(net->h_loss, net->d_loss, sizeof(double), cudaMemcpyDeviceToHost, net->stream));
    NCU(cudaStreamSynchronize(net->stream));
    *h_loss = *net->h_loss;
    return TPMG_OK;
}

}  // namespace

extern "C" {

tpmg_status tpmg_net_create(int n_r, int hidden, void *cuda_stream, tpmg_net **out)
{
    if (!out || n_r < 1 || n_r > 1024 || hidden < 1 || hidden > 1024) return TPMG_ERR_INVALID_ARG;
    tpmg_net *net = new (std::nothrow) tpmg_net();
    if (!net) return TPMG_ERR_OOM;
    net->stream = static_cast<cudaStream_t>(cuda_stream);
    const int sz[5] = {2 * n_r, hidden, hidden, hidden, n_r};
    size_t off = 0;
    for (int l = 0; l < 5; ++l) net->sizes[l] = sz[l];
    for (int l = 0; l < 4; ++l) {
        net->off_w[l] = off;
        off += (size_t)sz[l] * sz[l + 1];
        net->off_b[l] = off;
        off += sz[l + 1];
    }
    net->n_params = off;
    const size_t n = off;
    cudaError_t e = cudaMalloc(&net->master, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&net->grad, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&net->adam_m, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&net->adam_v, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&net->wbf, n * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(&net->d_part, kLossBlocks * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&net->d_loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&net->h_loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(net->master, 0, n * sizeof(float), net->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(net->grad, 0, n * sizeof(float), net->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(net->adam_m, 0, n * sizeof(float), net->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(net->adam_v, 0, n * sizeof(float), net->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(net->wbf, 0, n * sizeof(uint16_t), net->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) {
        tpmg_net_destroy(net);
        return e == cudaErrorMemoryAllocation ? TPMG_ERR_OOM : TPMG_ERR_CUDA;
    }
    *out = net;
    return TPMG_OK;
}

size_t tpmg_net_n_params(const tpmg_net *net) { return net ? net->n_params : 0; }

tpmg_status tpmg_net_set_params(tpmg_net *net, const float *h_params)
{
    if (!net || !h_params) return net_fail(net, TPMG_ERR_INVALID_ARG, "NULL pointer");
    const size_t n = net->n_params;
    NCU(cudaMemcpyAsync(net->master, h_params, n * sizeof(float), cudaMemcpyHostToDevice, net->stream));
    NCU(cudaMemsetAsync(net->adam_m, 0, n * sizeof(float), net->stream));
    NCU(cudaMemsetAsync(net->adam_v, 0, n * sizeof(float), net->stream));
    k_round_bf16<<<grid_1d((long)n, 256, sm_count_of_current()), 256, 0, net->stream>>>((long)n, net->master, net->wbf);
    NCU(cudaGetLastError());
    NCU(cudaStreamSynchronize(net->stream));
    net->step = 0;
    return TPMG_OK;
}

tpmg_status tpmg_net_get_params(tpmg_net *net, float *h_params)
{
    if (!net || !h_params) return net_fail(net, TPMG_ERR_INVALID_ARG, "NULL pointer");
    NCU(cudaMemcpyAsync(h_params, net->master, net->n_params * sizeof(float), cudaMemcpyDeviceToHost, net->stream));
    NCU(cudaStreamSynchronize(net->stream));
    return TPMG_OK;
}

tpmg_status tpmg_net_forward(tpmg_net *net, const float *d_x, long rows, float *d_y)
{
    if (!net) return TPMG_ERR_INVALID_ARG;
    tpmg_status st = check_rows(net, d_x, d_y, rows);
    if (st != TPMG_OK || (st = ensure_ws(net, rows, false)) != TPMG_OK) return st;
    float *acts[4], *y;
    if ((st = forward_ws(net, d_x, rows, acts, &y)) != TPMG_OK) return st;
    NCU(cudaMemcpyAsync(d_y, y, sizeof(float) * rows * net->sizes[4], cudaMemcpyDeviceToDevice, net->stream));
    return TPMG_OK;
}

tpmg_status tpmg_net_gradients(tpmg_net *net, const float *d_x, const float *d_t, long rows, float *d_grad,
                               double *h_loss)
{
    if (!net) return TPMG_ERR_INVALID_ARG;
    tpmg_status st = check_rows(net, d_x, d_t, rows);
    if (st == TPMG_OK && !d_grad) st = net_fail(net, TPMG_ERR_INVALID_ARG, "NULL pointer");
    if (st != TPMG_OK || (st = ensure_ws(net, rows, true)) != TPMG_OK) return st;
    if ((st = backward_ws(net, d_x, d_t, rows, d_grad)) != TPMG_OK) return st;
    return read_loss(net, h_loss);
}

tpmg_status tpmg_net_train_step(tpmg_net *net, const float *d_x, const float *d_t, long rows, float lr,
                                double *h_loss)
{
    if (!net) return TPMG_ERR_INVALID_ARG;
    if (!(lr >= 0.f) || !std::isfinite(lr)) return net_fail(net, TPMG_ERR_INVALID_ARG, "lr must be finite and >= 0");
    tpmg_status st = check_rows(net, d_x, d_t, rows);
    if (st != TPMG_OK || (st = ensure_ws(net, rows, true)) != TPMG_OK) return st;
    if ((st = backward_ws(net, d_x, d_t, rows, net->grad)) != TPMG_OK) return st;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    ++net->step;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)net->step));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)net->step));
    const long n = (long)net->n_params;
    k_adam<<<grid_1d(n, 256, sm_count_of_current()), 256, 0, net->stream>>>(n, net->master, net->adam_m, net->adam_v,
                                                                          net->grad, net->wbf, lr, b1, b2, eps, c1, c2);
    NCU(cudaGetLastError());
    return read_loss(net, h_loss);
}

const char *tpmg_net_last_error(const tpmg_net *net) { return net ? net->err.c_str() : ""; }

void tpmg_net_destroy(tpmg_net *net)
{
    if (!net) return;
    if (net->stream) cudaStreamSynchronize(net->stream);
    else cudaDeviceSynchronize();
    cudaFree(net->master);
    cudaFree(net->grad);
    cudaFree(net->adam_m);
    cudaFree(net->adam_v);
    cudaFree(net->wbf);
    cudaFree(net->ws);
    cudaFree(net->split);
    cudaFree(net->d_part);
    cudaFree(net->d_loss);
    if (net->h_loss) cudaFreeHost(net->h_loss);
    delete net;
}

}  // extern "C"
