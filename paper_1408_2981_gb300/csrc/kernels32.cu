// FP32 kernels of the mixed-precision TPMG V-cycle for sm_103a.
//
// The V-cycle (Algorithm 1: line relaxation, residual, restriction,
// prolongation) runs in FP32 on every level.  The stencil is stored per
// unknown in BF16 (full storage of Sec. 4.2): per (cell, k) the three
// horizontal couplings alphaS_hat and the mass term beta_hat in one 8-byte
// bf16x4, and the vertical coupling alphar_hat of the lower face k in a
// 2-byte array (the upper face of k is the lower face of k+1).  Each edge
// coupling is rounded once and used by both of its cells, so the BF16
// operator is symmetric and still maps constants to beta_hat.  The column
// blocks are factorised on the fly in FP32 from those coefficients, with the
// excess-carried twisted elimination of the FP64 path; nothing else about
// the operator is stored.  The outer Krylov vectors stay in FP64: the finest
// level reads its right-hand side as double and writes its result as double.
#include <cuda_runtime.h>

#include "tpmg_internal.h"

namespace tpmg {

namespace {

constexpr int kThreads32 = 256;

__device__ __forceinline__ float bf(unsigned short h) { return __uint_as_float((unsigned)h << 16); }

// Twisted Thomas factors of the BF16 column blocks (set-up, one thread per
// column of a task): the recurrences of the FP64 path (excess-carried pivots,
// elimination from both ends towards the meeting row j) evaluated in FP64 on
// the BF16 coefficients -- diagonal excess m_k = beta_hat + sum_e alphaS_hat_e,
// couplings c_k = alphar_hat of face k -- and stored in FP32: rinv [cell][k],
// multipliers fb, fc [task][step][lane], meeting row fm [task][2][16].
__global__ void k_twisted_factors32(int n_tasks, const int *__restrict__ cells, const bf16x4 *__restrict__ cpack,
                                    const unsigned short *__restrict__ cvert, int n, int S, int j,
                                    float *__restrict__ rinv, float *__restrict__ fb, float *__restrict__ fc,
                                    float *__restrict__ fm)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n_tasks * kRelaxCols) return;
    const int t = gid / kRelaxCols, col = gid - t * kRelaxCols;
    const int T = cells[gid];
    const size_t base = (size_t)t * S * 32;
    for (int s = 0; s < S; ++s) {
        fb[base + s * 32 + col] = fc[base + s * 32 + col] = 0.f;
        fb[base + s * 32 + col + 16] = fc[base + s * 32 + col + 16] = 0.f;
    }
    float *M = fm + (size_t)t * 2 * kRelaxCols;
    M[col] = M[kRelaxCols + col] = 0.f;
    if (T < 0) return;
    const size_t row0 = (size_t)T * n;
    auto m_of = [&](int k) {
        const bf16x4 c = cpack[row0 + k];
        return (double)bf(c.w) + (double)bf(c.x) + (double)bf(c.y) + (double)bf(c.z);
    };
    auto c_of = [&](int k) { return k < n ? (double)bf(cvert[row0 + k]) : 0.0; };
    double e = 0.0, p = 1.0;
    for (int k = 0; k < j; ++k) {
        const double m = m_of(k), c = c_of(k), cu = c_of(k + 1);
        e = k == 0 ? m : m + c * e / p;
        p = e + cu;
        rinv[row0 + k] = (float)(1.0 / p);
        fb[base + k * 32 + col] = (float)(c / p);
        fc[base + k * 32 + col] = (float)(cu / p);
    }
    double eb = 0.0, q = 1.0;
    for (int k = n - 1, s = 0; k > j; --k, ++s) {
        const double m = m_of(k), cd = c_of(k), cu = c_of(k + 1);
        eb = k == n - 1 ? m : m + cu * eb / q;
        q = eb + cd;
        rinv[row0 + k] = (float)(1.0 / q);
        fb[base + s * 32 + col + 16] = (float)(cu / q);
        fc[base + s * 32 + col + 16] = (float)(cd / q);
    }
    const double cj = c_of(j), cj1 = c_of(j + 1);
    double gam = m_of(j);
    if (j > 0) gam += cj * e / p;
    if (j < n - 1) gam += cj1 * eb / q;
    rinv[row0 + j] = (float)(1.0 / gam);
    M[col] = (float)(cj / gam);
    M[kRelaxCols + col] = (float)(cj1 / gam);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Twisted Thomas solve of one column pair in FP32 (lane = column + 16 * half)
// with precomputed factors: tc holds t = d / pivot on entry and x on exit;
// B, C point at the task's [step][32] multiplier blocks.  The loads of the
// next P steps are issued while the current P are computed.
template <int P>
__device__ __forceinline__ void twisted_solve32(const float *B, const float *C, const float *M, float *tc, int n_r,
                                                int j, int lane)
{
    const int c = lane & (kRelaxCols - 1), half = lane >> 4;
    const int rows = half ? n_r - 1 - j : j;
    auto row_of = [&](int s) { return half ? n_r - 1 - s : s; };
    float y = 0.f;
    {
        float b[P], d[P];
#pragma unroll
        for (int q = 0; q < P; ++q)
            if (q < rows) { b[q] = B[q * 32]; d[q] = tc[row_of(q)]; }
        for (int s0 = 0; s0 < rows; s0 += P) {
            float bn[P], dn[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int s = s0 + P + q;
                if (s < rows) { bn[q] = B[s * 32]; dn[q] = tc[row_of(s)]; }
            }
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int s = s0 + q;
                if (s < rows) {
                    y = fmaf(b[q], y, d[q]);
                    tc[row_of(s)] = y;
                }
            }
#pragma unroll
            for (int q = 0; q < P; ++q) { b[q] = bn[q]; d[q] = dn[q]; }
        }
    }
    __syncwarp();
    const float other = __shfl_xor_sync(0xffffffffu, y, 16);
    const float ytop = half ? other : y, zbot = half ? y : other;
    const float xj = fmaf(M[kRelaxCols + c], zbot, fmaf(M[c], ytop, tc[j]));
    __syncwarp();
    if (half == 0) tc[j] = xj;
    float x = xj;
    {
        float cc[P], yy[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int s = rows - 1 - q;
            if (s >= 0) { cc[q] = C[s * 32]; yy[q] = tc[row_of(s)]; }
        }
        for (int s0 = rows - 1; s0 >= 0; s0 -= P) {
            float cn[P], yn[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int s = s0 - P - q;
                if (s >= 0) { cn[q] = C[s * 32]; yn[q] = tc[row_of(s)]; }
            }
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int s = s0 - q;
                if (s >= 0) {
                    x = fmaf(cc[q], x, yy[q]);
                    tc[row_of(s)] = x;
                }
            }
#pragma unroll
            for (int q = 0; q < P; ++q) { cc[q] = cn[q]; yy[q] = yn[q]; }
        }
    }
}

// Gather of one relaxation task (shared by both kernels): t = (f + sum_e
// alphaS_hat_e u_{T_e}) / pivot into tile[c * ld + k] for elements
// e = first, first + stride, ...; U elements' loads in flight per thread.
template <int MODE, typename TF, int U>
__device__ __forceinline__ void gather32(const int *s_cell, const int4 *s_nb, const bf16x4 *__restrict__ cpack,
                                         const float *__restrict__ rinv, const TF *__restrict__ f, const float *u_in,
                                         int n_r, int ld, int first, int stride, float *tile)
{
    const int ne = kRelaxCols * n_r;
    for (int e0 = first; e0 < ne; e0 += stride * U) {
        float fv[U], iv[U], v0[U], v1[U], v2[U];
        bf16x4 cp[U];
        int o[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int e = e0 + stride * q;
            o[q] = -1;
            fv[q] = iv[q] = v0[q] = v1[q] = v2[q] = 0.f;
            cp[q] = bf16x4{0, 0, 0, 0};
            if (e < ne) {
                const int c = e / n_r, k = e - c * n_r;
                o[q] = c * ld + k;
                const int T = s_cell[c];
                if (T >= 0) {
                    const int i = T * n_r + k;
                    fv[q] = (float)f[i];
                    iv[q] = __ldg(&rinv[i]);
                    if (MODE != PASS_RHS_ONLY) {
                        cp[q] = cpack[i];
                        const int4 nb = s_nb[c];
                        if (MODE == PASS_NORMAL || (nb.w & 1)) v0[q] = u_in[nb.x * n_r + k];
                        if (MODE == PASS_NORMAL || (nb.w & 2)) v1[q] = u_in[nb.y * n_r + k];
                        if (MODE == PASS_NORMAL || (nb.w & 4)) v2[q] = u_in[nb.z * n_r + k];
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (o[q] < 0) continue;
            float d = fv[q];
            if (MODE != PASS_RHS_ONLY)
                d = fmaf(bf(cp[q].z), v2[q], fmaf(bf(cp[q].y), v1[q], fmaf(bf(cp[q].x), v0[q], d)));
            tile[o[q]] = d * iv[q];
        }
    }
}

// Write-back of one relaxation task (shared by both kernels): u_out, the
// optional relaxation weight, the double copy out64 (the finest level's
// result) and the prolongation into the 4 children in u_fine; the loads of W
// elements are issued before their stores.
template <int MODE, int W>
__device__ __forceinline__ void write_back32(const int *s_cell, const float *tile, int n_r, int ld, int first,
                                             int stride, const float *u_in, float *u_out, float *__restrict__ u_fine,
                                             double *__restrict__ out64, float relax)
{
    const int ne = kRelaxCols * n_r;
    for (int e0 = first; e0 < ne; e0 += stride * W) {
        float x[W], uo[W], uf[W][4];
        int idx[W], fi[W];
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const int e = e0 + stride * q;
            idx[q] = -1;
            if (e >= ne) continue;
            const int c = e / n_r, k = e - c * n_r;
            const int T = s_cell[c];
            if (T < 0) continue;
            idx[q] = T * n_r + k;
            fi[q] = 4 * T * n_r + k;
            x[q] = tile[c * ld + k];
            uo[q] = (MODE == PASS_NORMAL && relax != 1.f) ? u_in[idx[q]] : 0.f;
            if (u_fine) {
#pragma unroll
                for (int h = 0; h < 4; ++h) uf[q][h] = u_fine[fi[q] + h * n_r];
            }
        }
#pragma unroll
        for (int q = 0; q < W; ++q) {
            if (idx[q] < 0) continue;
            float v = x[q];
            if (relax != 1.f) v = fmaf(relax, v - uo[q], uo[q]);
            u_out[idx[q]] = v;
            if (out64) out64[idx[q]] = (double)v;
            if (u_fine) {
#pragma unroll
                for (int h = 0; h < 4; ++h) u_fine[fi[q] + h * n_r] = uf[q][h] + v;
            }
        }
    }
}

// One relaxation pass (eq. BlockJacobi) in FP32 over whole tasks of 16 columns,
// one task per CTA of NT threads (64, 128 or 256; chosen per level by the autotuner):
//   u_T <- (1 - relax) u_T + relax A_T^{-1} (f_T + sum_e alphaS_hat_e u_{T_e}).
// The task's multiplier blocks are copied to shared memory by cp.async during
// the gather; one warp (rotating over the sub-partitions) solves.
template <int MODE, typename TF, int NT>
__global__ void __launch_bounds__(NT)
    k_relax32(const int *__restrict__ cells, const int4 *__restrict__ tnb, const bf16x4 *__restrict__ cpack,
              const float *__restrict__ rinv, const float *__restrict__ fb, const float *__restrict__ fcf,
              const float *__restrict__ fm, int n_r, int S, int j, int task0, const TF *__restrict__ f,
              const float *u_in, float *u_out, float *__restrict__ u_fine, double *__restrict__ out64, float relax)
{
    extern __shared__ float sm32[];
    __shared__ int s_cell[kRelaxCols];
    __shared__ int4 s_nb[kRelaxCols];
    __shared__ float s_m[2 * kRelaxCols];
    const int ld = n_r + 1;
    float *tile = sm32;
    float *sf = sm32 + ((kRelaxCols * ld + 3) & ~3);   // staged multipliers, 16-byte aligned
    const int t = task0 + blockIdx.x;
    const size_t fbase = (size_t)t * S * 32;
    {
        const int chunks = S * 8;   // 16-byte chunks per multiplier block
        for (int q = threadIdx.x; q < 2 * chunks; q += NT) {
            const int a = q >= chunks, r = q - a * chunks;
            cp_async16(sf + (size_t)a * S * 32 + 4 * r, (a ? fcf : fb) + fbase + 4 * r);
        }
    }
    if (threadIdx.x < kRelaxCols) {
        const int q = t * kRelaxCols + threadIdx.x;
        s_cell[threadIdx.x] = __ldg(&cells[q]);
        s_nb[threadIdx.x] = __ldg(&tnb[q]);
    } else if (threadIdx.x < 3 * kRelaxCols) {
        const int q = threadIdx.x - kRelaxCols;
        s_m[q] = __ldg(&fm[(size_t)t * 2 * kRelaxCols + q]);
    }
    __syncthreads();
    gather32<MODE, TF, 8>(s_cell, s_nb, cpack, rinv, f, u_in, n_r, ld, threadIdx.x, NT, tile);
    cp_async_wait_all();
    __syncthreads();
    if ((threadIdx.x >> 5) == (int)(blockIdx.x % (NT / 32))) {
        const int lane = threadIdx.x & 31;
        twisted_solve32<8>(sf + lane, sf + (size_t)S * 32 + lane, s_m, tile + (lane & (kRelaxCols - 1)) * ld, n_r, j,
                           lane);
    }
    __syncthreads();
    write_back32<MODE, 4>(s_cell, tile, n_r, ld, threadIdx.x, NT, u_in, u_out, u_fine, out64, relax);
}

// The same pass with one warp per task and no block barrier (passes with many
// tasks): the serial phases of the tasks resident on an SM overlap with the
// gathers and write-backs of others.
template <int MODE, typename TF>
__global__ void __launch_bounds__(32, 16)
    k_relax32_warp(const int *__restrict__ cells, const int4 *__restrict__ tnb, const bf16x4 *__restrict__ cpack,
                   const float *__restrict__ rinv, const float *__restrict__ fb, const float *__restrict__ fcf,
                   const float *__restrict__ fm, int n_r, int S, int j, int task0, const TF *__restrict__ f,
                   const float *u_in, float *u_out, float *__restrict__ u_fine, double *__restrict__ out64,
                   float relax)
{
    extern __shared__ float tile32[];
    __shared__ int s_cell[kRelaxCols];
    __shared__ int4 s_nb[kRelaxCols];
    __shared__ float s_m[2 * kRelaxCols];
    const int t = task0 + blockIdx.x, lane = threadIdx.x, ld = n_r + 1;
    s_m[lane] = __ldg(&fm[(size_t)t * 2 * kRelaxCols + lane]);
    if (lane < kRelaxCols) {
        const int q = t * kRelaxCols + lane;
        s_cell[lane] = __ldg(&cells[q]);
        s_nb[lane] = __ldg(&tnb[q]);
    }
    __syncwarp();
    gather32<MODE, TF, 8>(s_cell, s_nb, cpack, rinv, f, u_in, n_r, ld, lane, 32, tile32);
    __syncwarp();
    const size_t fbase = (size_t)t * S * 32 + lane;
    twisted_solve32<8>(fb + fbase, fcf + fbase, s_m, tile32 + (lane & (kRelaxCols - 1)) * ld, n_r, j, lane);
    __syncwarp();
    write_back32<MODE, 4>(s_cell, tile32, n_r, ld, lane, 32, u_in, u_out, u_fine, out64, relax);
}

// f_c[T][k] = sum_j (f - A u)[4T + j][k] in FP32 with the BF16 stencil, the row
// in the flux form of Appendix A (Algorithm 1 residual + restriction).
template <typename TF>
__global__ void __launch_bounds__(kThreads32)
    k_resid_restrict32(const int4 *__restrict__ nbr, const bf16x4 *__restrict__ cpack,
                       const unsigned short *__restrict__ cvert, int n_r, const TF *__restrict__ f,
                       const float *__restrict__ u, float *__restrict__ fc, int Nc)
{
    for (int ic = blockIdx.x * kThreads32 + threadIdx.x; ic < Nc; ic += gridDim.x * kThreads32) {
        const int Tc = ic / n_r, k = ic - Tc * n_r;
        float s = 0.f;
#pragma unroll
        for (int jc = 0; jc < 4; ++jc) {
            const int T = 4 * Tc + jc, i = T * n_r + k;
            const int4 nb = __ldg(&nbr[T]);
            const bf16x4 cp = cpack[i];
            const float uc = u[i];
            const float um = k > 0 ? u[i - 1] : uc, up = k < n_r - 1 ? u[i + 1] : uc;
            const float cl = bf(__ldg(&cvert[i])), cu = k < n_r - 1 ? bf(__ldg(&cvert[i + 1])) : 0.f;
            float a = bf(cp.w) * uc;
            a = fmaf(cl, uc - um, a);
            a = fmaf(cu, uc - up, a);
            a = fmaf(bf(cp.x), uc - u[nb.x * n_r + k], a);
            a = fmaf(bf(cp.y), uc - u[nb.y * n_r + k], a);
            a = fmaf(bf(cp.z), uc - u[nb.z * n_r + k], a);
            s += (float)f[i] - a;
        }
        fc[ic] = s;
    }
}

__global__ void __launch_bounds__(kThreads32) k_prolong_add32(const float *__restrict__ uc, float *__restrict__ u,
                                                              int n_r, int N)
{
    for (int i = blockIdx.x * kThreads32 + threadIdx.x; i < N; i += gridDim.x * kThreads32) {
        const int T = i / n_r, k = i - T * n_r;
        u[i] += uc[(T >> 2) * n_r + k];
    }
}

__global__ void __launch_bounds__(kThreads32) k_to_f64(const float *__restrict__ x, double *__restrict__ y, int N)
{
    for (int i = blockIdx.x * kThreads32 + threadIdx.x; i < N; i += gridDim.x * kThreads32) y[i] = (double)x[i];
}

inline int grid32(long work, int sm_count)
{
    long b = (work + kThreads32 - 1) / kThreads32;
    const long cap = (long)sm_count * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <int MODE, typename TF, int NT>
cudaError_t relax32_cta(const Launch &L, const LevelDev &lv, int task0, int n_tasks, float relax, const TF *f,
                        const float *u_in, float *u_out, float *u_fine, double *out64, size_t smem)
{
    auto kern = k_relax32<MODE, TF, NT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<n_tasks, NT, smem, L.s>>>(lv.task_cells, lv.task_nbr, lv.cpack, lv.rinv32, lv.fb32, lv.fc32, lv.fm32, L.n_r,
                                     lv.steps, lv.jmid, task0, f, u_in, u_out, u_fine, out64, relax);
    return cudaGetLastError();
}

// Kernel choice (RELAX_*): the level's autotuned variant; without one a
// 128-thread CTA per task (measured faster than one warp per task at every
// FP32 pass size tried, e.g. 313 against 352 us for 10k tasks of 128 levels).
template <int MODE, typename TF>
cudaError_t relax32_t(const Launch &L, const LevelDev &lv, int task0, int n_tasks, float relax, const TF *f,
                      const float *u_in, float *u_out, float *u_fine, double *out64)
{
    const size_t tile = (((size_t)kRelaxCols * (L.n_r + 1) + 3) & ~(size_t)3) * sizeof(float);
    const int var = lv.relax_variant < 0 ? RELAX_CTA128 : lv.relax_variant;
    if (var == RELAX_WARP && tile <= 32 * 1024) {
        k_relax32_warp<MODE, TF><<<n_tasks, 32, tile, L.s>>>(lv.task_cells, lv.task_nbr, lv.cpack, lv.rinv32,
                                                             lv.fb32, lv.fc32, lv.fm32, L.n_r, lv.steps, lv.jmid,
                                                             task0, f, u_in, u_out, u_fine, out64, relax);
        return cudaGetLastError();
    }
    const size_t smem = tile + (size_t)2 * lv.steps * 32 * sizeof(float);
    if (var == RELAX_CTA64) return relax32_cta<MODE, TF, 64>(L, lv, task0, n_tasks, relax, f, u_in, u_out, u_fine, out64, smem);
    if (var == RELAX_CTA256) return relax32_cta<MODE, TF, 256>(L, lv, task0, n_tasks, relax, f, u_in, u_out, u_fine, out64, smem);
    return relax32_cta<MODE, TF, 128>(L, lv, task0, n_tasks, relax, f, u_in, u_out, u_fine, out64, smem);
}

}  // namespace

template <typename TF>
cudaError_t launch_relax32(const Launch &L, const LevelDev &lv, int mode, int task0, int n_tasks, float relax,
                           const TF *f, const float *u_in, float *u_out, float *u_fine, double *out64)
{
    if (n_tasks <= 0) return cudaSuccess;
    switch (mode) {
    case PASS_ZERO: return relax32_t<PASS_ZERO>(L, lv, task0, n_tasks, relax, f, u_in, u_out, u_fine, out64);
    case PASS_RHS_ONLY: return relax32_t<PASS_RHS_ONLY>(L, lv, task0, n_tasks, relax, f, u_in, u_out, u_fine, out64);
    default: return relax32_t<PASS_NORMAL>(L, lv, task0, n_tasks, relax, f, u_in, u_out, u_fine, out64);
    }
}

template <typename TF>
cudaError_t launch_resid_restrict32(const Launch &L, const LevelDev &fine, const LevelDev &coarse, const TF *f,
                                    const float *u, float *fc)
{
    const int Nc = coarse.n * L.n_r;
    k_resid_restrict32<TF><<<grid32(Nc, L.sm_count), kThreads32, 0, L.s>>>(fine.nbr, fine.cpack, fine.cvert, L.n_r, f,
                                                                           u, fc, Nc);
    return cudaGetLastError();
}

cudaError_t launch_prolong_add32(const Launch &L, const LevelDev &fine, const float *uc, float *u)
{
    const int N = fine.n * L.n_r;
    k_prolong_add32<<<grid32(N, L.sm_count), kThreads32, 0, L.s>>>(uc, u, L.n_r, N);
    return cudaGetLastError();
}

cudaError_t launch_twisted_factors32(const Launch &L, const LevelDev &lv)
{
    const int n = lv.n_tasks * kRelaxCols;
    k_twisted_factors32<<<(n + 127) / 128, 128, 0, L.s>>>(lv.n_tasks, lv.task_cells, lv.cpack, lv.cvert, L.n_r,
                                                          lv.steps, lv.jmid, lv.rinv32, lv.fb32, lv.fc32, lv.fm32);
    return cudaGetLastError();
}

cudaError_t launch_to_f64(const Launch &L, long n, const float *x, double *y)
{
    k_to_f64<<<grid32(n, L.sm_count), kThreads32, 0, L.s>>>(x, y, (int)n);
    return cudaGetLastError();
}

template cudaError_t launch_relax32<double>(const Launch &, const LevelDev &, int, int, int, float, const double *,
                                            const float *, float *, float *, double *);
template cudaError_t launch_relax32<float>(const Launch &, const LevelDev &, int, int, int, float, const float *,
                                           const float *, float *, float *, double *);
template cudaError_t launch_resid_restrict32<double>(const Launch &, const LevelDev &, const LevelDev &,
                                                     const double *, const float *, float *);
template cudaError_t launch_resid_restrict32<float>(const Launch &, const LevelDev &, const LevelDev &, const float *,
                                                    const float *, float *);

}  // namespace tpmg
