// FP64 kernels of the TPMG-preconditioned CG path for sm_103a.
//
// Layout: a field is [cell][k] with the vertical index fastest (Sec. 4.1: the
// column of a horizontal cell is stored contiguously).  Per cell: int4
// {nbr0, nbr1, nbr2, mask}, mask bit e set when neighbour e has a smaller
// colour; double4 {g0, g1, g2, g0+g1+g2}; area |T|.  Vertical factors are
// shared by all levels (no vertical coarsening, Sec. 3.3).
//
// The operator in the flux form of Appendix A (constant profiles, factorised
// storage: per-level vertical vectors times per-cell scalars, Sec. 3.2):
//   (A x)_{T,k} = |T| (v_k x_k + w_k (x_k - x_{k-1}) + w_{k+1} (x_k - x_{k+1}))
//               + hr_k sum_e g_e (x_k - x_{T_e,k}),
// w_k = omega^2 sigma_k 2 r_k^2/(r_{k+1}-r_{k-1}), hr_k = omega^2 (r_{k+1}-r_k).
// Every coupling multiplies a difference, so the large vertical couplings never
// round the nearly singular vertically constant mode of a column.
//
// On GB300 the FP64 pipe, not HBM, bounds this arithmetic (a warp-wide FP64
// instruction holds an SM sub-partition's FP64 unit for ~64 cycles whatever
// the number of active lanes), so every kernel counts its FP64 instructions:
// address arithmetic is 32-bit integer, the Thomas pivots are precomputed once
// per level, and the line relaxation forms u_T = A_T^{-1} (f_T - sum_T' A_TT'
// u_T') directly (no residual, no cancellation).
#include <cuda_runtime.h>

#include "tpmg_internal.h"

namespace tpmg {

namespace {

constexpr int kThreads = 256;   // element-wise kernels
constexpr int kSmooth = 128;    // line-relaxation kernels

template <int NT>
__device__ __forceinline__ double block_sum(double v)
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

struct OpView {
    const int4 *__restrict__ nbr;
    const dbl4 *__restrict__ g;
    const double *__restrict__ area;
    const double *__restrict__ vol;
    const double *__restrict__ w;
    const double *__restrict__ hr;
    int n_r;
};

inline OpView make_view(const LevelDev &lv, const VertDev &v, int n_r)
{
    return OpView{lv.nbr, lv.g, lv.area, v.vol, v.w, v.hr, n_r};
}

// (A x)_{T,k} in flux form: 13 FP64 instructions.
__device__ __forceinline__ double apply_at(const OpView &o, const double *__restrict__ x, int T, int k, int i)
{
    const int n_r = o.n_r;
    const int4 nb = __ldg(&o.nbr[T]);
    const dbl4 g = o.g[T];
    const double xc = x[i];
    const double dm = k > 0 ? xc - x[i - 1] : 0.0;
    const double dp = k < n_r - 1 ? xc - x[i + 1] : 0.0;
    const double vert = fma(__ldg(&o.w[k + 1]), dp, fma(__ldg(&o.w[k]), dm, __ldg(&o.vol[k]) * xc));
    const double hor = fma(g.z, xc - x[nb.z * n_r + k], fma(g.y, xc - x[nb.y * n_r + k], g.x * (xc - x[nb.x * n_r + k])));
    return fma(__ldg(&o.area[T]), vert, __ldg(&o.hr[k]) * hor);
}

template <int NT>
__global__ void __launch_bounds__(NT) k_apply(OpView o, const double *__restrict__ x, double *__restrict__ y,
                                              int N, double *__restrict__ partials)
{
    double acc = 0.0;
    for (int i = blockIdx.x * NT + threadIdx.x; i < N; i += gridDim.x * NT) {
        const int T = i / o.n_r, k = i - T * o.n_r;
        const double v = apply_at(o, x, T, k, i);
        y[i] = v;
        acc = fma(x[i], v, acc);
    }
    if (partials) {
        acc = block_sum<NT>(acc);
        if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_residual(OpView o, const double *__restrict__ f, const double *__restrict__ u,
                                                 double *__restrict__ r, int N, double *__restrict__ partials)
{
    double acc = 0.0;
    for (int i = blockIdx.x * NT + threadIdx.x; i < N; i += gridDim.x * NT) {
        const int T = i / o.n_r, k = i - T * o.n_r;
        const double v = f[i] - apply_at(o, u, T, k, i);
        r[i] = v;
        acc = fma(v, v, acc);
    }
    if (partials) {
        acc = block_sum<NT>(acc);
        if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    }
}

// f_c[T][k] = sum_j (f - A u)[4T + j][k]  (Algorithm 1 residual + restriction, Sec. 5)
template <int NT>
__global__ void __launch_bounds__(NT) k_resid_restrict(OpView o, const double *__restrict__ f,
                                                       const double *__restrict__ u, double *__restrict__ fc, int Nc)
{
    for (int ic = blockIdx.x * NT + threadIdx.x; ic < Nc; ic += gridDim.x * NT) {
        const int Tc = ic / o.n_r, k = ic - Tc * o.n_r;
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int T = 4 * Tc + j, i = T * o.n_r + k;
            s += f[i] - apply_at(o, u, T, k, i);
        }
        fc[ic] = s;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_prolong_add(const double *__restrict__ uc, double *__restrict__ u, int n_r, int N)
{
    for (int i = blockIdx.x * NT + threadIdx.x; i < N; i += gridDim.x * NT) {
        const int T = i / n_r, k = i - T * n_r;
        u[i] += uc[(T >> 2) * n_r + k];
    }
}

// Thomas pivots of the column block A_T (one thread per column).  A_T has
// couplings c_k = |T| w_k to the level below, c_{k+1} above, and diagonal
// c_k + c_{k+1} + m_k with excess m_k = |T| v_k + hr_k G_T.  The pivots are
// carried through their excess, e_0 = m_0, e_k = m_k + c_k e_{k-1} / p_{k-1},
// p_k = e_k + c_{k+1}: only sums of non-negative terms, so they keep full
// relative precision although c_k / m_k reaches 1e6-1e9 in a thin shell.
// Stored: inv = 1/p_k, ef = c_k/p_k, cpf = c_{k+1}/p_k, so that the solve is
//   y_k = rhs_k inv_k + ef_k y_{k-1};   x_k = y_k + cpf_k x_{k+1}.
__global__ void k_factors(int n, OpView o, double *__restrict__ inv, double *__restrict__ ef, double *__restrict__ cpf)
{
    const int T = blockIdx.x * blockDim.x + threadIdx.x;
    if (T >= n) return;
    const int n_r = o.n_r;
    const double A = o.area[T], Gs = o.g[T].w;
    double e = 0.0, p = 1.0;
    for (int k = 0; k < n_r; ++k) {
        const double m = A * o.vol[k] + o.hr[k] * Gs;
        const double c = A * o.w[k], cu = A * o.w[k + 1];
        e = k == 0 ? m : m + c * e / p;
        p = e + cu;
        const double iv = 1.0 / p;
        inv[T * n_r + k] = iv;
        ef[T * n_r + k] = c * iv;
        cpf[T * n_r + k] = cu * iv;
    }
}

// One colour pass of multicolour block-SOR (eq. BlockJacobi) over a tile of
// CT columns of colour c:
//   u_T <- (1 - relax) u_T + relax A_T^{-1} (f_T + hr sum_e g_e u_{T_e}).
// MODE PASS_ZERO: first forward sweep from a zero guess (neighbours of a larger
// colour and the old u_T are zero).  MODE PASS_PROLONG: first reverse sweep after
// the coarse-grid correction u += P u_c, applied on the fly to every value not
// yet overwritten in this sweep (neighbours of a smaller colour, the old u_T).
// Phase 1 (all threads, coalesced along k): t = rhs * inv into shared memory;
// phase 2 (one thread per column): the two Thomas recurrences, 2 FP64 each;
// phase 3 (all threads): write back.  u_in and u_out are the same array in
// the multicolour passes (in-place; a pass reads only other colours'
// columns and its own column before writing it), distinct for block Jacobi.
template <int MODE, bool JACOBI>
__global__ void __launch_bounds__(kSmooth)
    k_relax(OpView o, const int *__restrict__ cells, int nc, int CT, const double *__restrict__ f,
            const double *u_in, double *u_out, const double *__restrict__ uc,
            const double *__restrict__ inv, const double *__restrict__ ef, const double *__restrict__ cpf, double relax)
{
    extern __shared__ double sm[];
    const int n_r = o.n_r, ld = n_r + 1;
    double *st = sm, *se = sm + CT * ld, *sc = sm + 2 * CT * ld;
    const int c0 = blockIdx.x * CT;
    const int nt = min(CT, nc - c0);
    const int ne = nt * n_r;
    for (int idx = threadIdx.x; idx < ne; idx += kSmooth) {
        const int j = idx / n_r, k = idx - j * n_r;
        const int T = JACOBI ? c0 + j : __ldg(&cells[c0 + j]);
        const int i = T * n_r + k;
        const int4 nb = __ldg(&o.nbr[T]);
        const dbl4 g = o.g[T];
        double v0, v1, v2;
        if (MODE == PASS_NORMAL) {
            v0 = u_in[nb.x * n_r + k]; v1 = u_in[nb.y * n_r + k]; v2 = u_in[nb.z * n_r + k];
        } else if (MODE == PASS_ZERO) {
            if (JACOBI) {
                v0 = v1 = v2 = 0.0;
            } else {
                v0 = (nb.w & 1) ? u_in[nb.x * n_r + k] : 0.0;
                v1 = (nb.w & 2) ? u_in[nb.y * n_r + k] : 0.0;
                v2 = (nb.w & 4) ? u_in[nb.z * n_r + k] : 0.0;
            }
        } else {
            const bool a0 = JACOBI || (nb.w & 1), a1 = JACOBI || (nb.w & 2), a2 = JACOBI || (nb.w & 4);
            v0 = u_in[nb.x * n_r + k] + (a0 ? uc[(nb.x >> 2) * n_r + k] : 0.0);
            v1 = u_in[nb.y * n_r + k] + (a1 ? uc[(nb.y >> 2) * n_r + k] : 0.0);
            v2 = u_in[nb.z * n_r + k] + (a2 ? uc[(nb.z >> 2) * n_r + k] : 0.0);
        }
        const double h = fma(g.z, v2, fma(g.y, v1, g.x * v0));
        const double rhs = fma(__ldg(&o.hr[k]), h, f[i]);
        st[j * ld + k] = rhs * inv[i];
        se[j * ld + k] = ef[i];
        sc[j * ld + k] = cpf[i];
    }
    __syncthreads();
    if (threadIdx.x < nt) {
        double *t = st + threadIdx.x * ld;
        const double *e = se + threadIdx.x * ld, *c = sc + threadIdx.x * ld;
        double y = t[0];
        for (int k = 1; k < n_r; ++k) {
            y = fma(e[k], y, t[k]);
            t[k] = y;
        }
        double x = y;
        for (int k = n_r - 2; k >= 0; --k) {
            x = fma(c[k], x, t[k]);
            t[k] = x;
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ne; idx += kSmooth) {
        const int j = idx / n_r, k = idx - j * n_r;
        const int T = JACOBI ? c0 + j : __ldg(&cells[c0 + j]);
        const int i = T * n_r + k;
        double x = st[j * ld + k];
        if (relax != 1.0) {
            double uo = 0.0;
            if (MODE == PASS_NORMAL) uo = u_in[i];
            if (MODE == PASS_PROLONG) uo = u_in[i] + uc[(T >> 2) * n_r + k];
            x = fma(relax, x - uo, uo);
        }
        u_out[i] = x;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_dot(const double *__restrict__ a, const double *__restrict__ b, int N,
                                            double *__restrict__ partials)
{
    double acc = 0.0;
    for (int i = blockIdx.x * NT + threadIdx.x; i < N; i += gridDim.x * NT) acc = fma(a[i], b[i], acc);
    acc = block_sum<NT>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// u += alpha p; r -= alpha q; partial ||r||^2
template <int NT>
__global__ void __launch_bounds__(NT) k_axpy_pair(const Scalars *__restrict__ sc, const double *__restrict__ p,
                                                  const double *__restrict__ q, double *__restrict__ u,
                                                  double *__restrict__ r, int N, double *__restrict__ partials)
{
    const double alpha = sc->alpha;
    double acc = 0.0;
    for (int i = blockIdx.x * NT + threadIdx.x; i < N; i += gridDim.x * NT) {
        u[i] = fma(alpha, p[i], u[i]);
        const double rv = fma(-alpha, q[i], r[i]);
        r[i] = rv;
        acc = fma(rv, rv, acc);
    }
    acc = block_sum<NT>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// p = z + beta p
template <int NT>
__global__ void __launch_bounds__(NT) k_xpby(const Scalars *__restrict__ sc, const double *__restrict__ z,
                                             double *__restrict__ p, int N)
{
    const double beta = sc->beta;
    for (int i = blockIdx.x * NT + threadIdx.x; i < N; i += gridDim.x * NT) p[i] = fma(beta, p[i], z[i]);
}

// Deterministic reduction of the block partials (fixed order) and the PCG scalar step.
__global__ void __launch_bounds__(256) k_finish(int what, const double *__restrict__ partials, int n, Scalars *sc)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) v += partials[i];
    v = block_sum<256>(v);
    if (threadIdx.x != 0) return;
    switch (what) {
    case FIN_RR0:
        sc->rr0 = v;
        sc->rr = v;
        sc->flag = isfinite(v) ? 0 : 2;
        break;
    case FIN_RZ0:
        sc->rz = v;
        if (!isfinite(v)) sc->flag |= 2;
        break;
    case FIN_ALPHA:
        sc->pq = v;
        if (!(v > 0.0) || !isfinite(v)) {
            sc->flag |= 1;
            sc->alpha = 0.0;
        } else {
            sc->alpha = sc->rz / v;
        }
        break;
    case FIN_RR:
        sc->rr = v;
        if (!isfinite(v)) sc->flag |= 2;
        break;
    case FIN_BETA:
        sc->rz_new = v;
        sc->beta = v / sc->rz;
        sc->rz = v;
        if (!isfinite(v)) sc->flag |= 2;
        break;
    default:
        break;
    }
}

inline int grid_for(long work, int nt, int sm_count)
{
    long b = (work + nt - 1) / nt;
    const long cap = (long)sm_count * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// Columns per tile of the line-relaxation kernels: three [CT][n_r+1] FP64
// tiles in shared memory, at most 96 KB, at least one column.
inline int relax_tile(int n_r)
{
    int ct = 32;
    while (ct > 1 && 3 * ct * (n_r + 1) * (int)sizeof(double) > 96 * 1024) ct >>= 1;
    return ct;
}

}  // namespace

cudaError_t launch_apply(const Launch &L, const LevelDev &lv, const VertDev &v, const double *x, double *y,
                         double *partials, int n_part)
{
    const int N = lv.n * L.n_r;
    const int grid = partials ? n_part : grid_for(N, kThreads, L.sm_count);
    k_apply<kThreads><<<grid, kThreads, 0, L.s>>>(make_view(lv, v, L.n_r), x, y, N, partials);
    return cudaGetLastError();
}

cudaError_t launch_residual(const Launch &L, const LevelDev &lv, const VertDev &v, const double *f, const double *u,
                            double *r, double *partials, int n_part)
{
    const int N = lv.n * L.n_r;
    const int grid = partials ? n_part : grid_for(N, kThreads, L.sm_count);
    k_residual<kThreads><<<grid, kThreads, 0, L.s>>>(make_view(lv, v, L.n_r), f, u, r, N, partials);
    return cudaGetLastError();
}

cudaError_t launch_resid_restrict(const Launch &L, const LevelDev &fine, const LevelDev &coarse, const VertDev &v,
                                  const double *f, const double *u, double *fc)
{
    const int Nc = coarse.n * L.n_r;
    k_resid_restrict<kThreads><<<grid_for(Nc, kThreads, L.sm_count), kThreads, 0, L.s>>>(make_view(fine, v, L.n_r), f,
                                                                                          u, fc, Nc);
    return cudaGetLastError();
}

cudaError_t launch_prolong_add(const Launch &L, const LevelDev &fine, const double *uc, double *u)
{
    const int N = fine.n * L.n_r;
    k_prolong_add<kThreads><<<grid_for(N, kThreads, L.sm_count), kThreads, 0, L.s>>>(uc, u, L.n_r, N);
    return cudaGetLastError();
}

cudaError_t launch_thomas_factors(const Launch &L, const LevelDev &lv, const VertDev &v)
{
    k_factors<<<(lv.n + 127) / 128, 128, 0, L.s>>>(lv.n, make_view(lv, v, L.n_r), lv.inv, lv.ef, lv.cpf);
    return cudaGetLastError();
}

template <int MODE, bool JACOBI>
static cudaError_t relax_launch(const Launch &L, const LevelDev &lv, const VertDev &v, const int *cells, int nc,
                                const double *f, const double *u_in, double *u_out, const double *uc, double relax)
{
    if (nc <= 0) return cudaSuccess;
    const int ct = relax_tile(L.n_r);
    const size_t smem = (size_t)3 * ct * (L.n_r + 1) * sizeof(double);
    auto kern = k_relax<MODE, JACOBI>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(nc + ct - 1) / ct, kSmooth, smem, L.s>>>(make_view(lv, v, L.n_r), cells, nc, ct, f, u_in, u_out, uc,
                                                      lv.inv, lv.ef, lv.cpf, relax);
    return cudaGetLastError();
}

cudaError_t launch_mcsor_pass(const Launch &L, const LevelDev &lv, const VertDev &v, int colour, int mode, double relax,
                              const double *f, double *u, const double *uc)
{
    const int off = lv.colour_off[colour], nc = lv.colour_off[colour + 1] - off;
    const int *cells = lv.cells_by_colour + off;
    switch (mode) {
    case PASS_ZERO: return relax_launch<PASS_ZERO, false>(L, lv, v, cells, nc, f, u, u, uc, relax);
    case PASS_PROLONG: return relax_launch<PASS_PROLONG, false>(L, lv, v, cells, nc, f, u, u, uc, relax);
    default: return relax_launch<PASS_NORMAL, false>(L, lv, v, cells, nc, f, u, u, uc, relax);
    }
}

cudaError_t launch_jacobi(const Launch &L, const LevelDev &lv, const VertDev &v, int mode, double relax,
                          const double *f, const double *u_in, double *u_out, const double *uc)
{
    switch (mode) {
    case PASS_ZERO: return relax_launch<PASS_ZERO, true>(L, lv, v, nullptr, lv.n, f, u_in, u_out, uc, relax);
    case PASS_PROLONG: return relax_launch<PASS_PROLONG, true>(L, lv, v, nullptr, lv.n, f, u_in, u_out, uc, relax);
    default: return relax_launch<PASS_NORMAL, true>(L, lv, v, nullptr, lv.n, f, u_in, u_out, uc, relax);
    }
}

cudaError_t launch_dot(const Launch &L, long n, const double *a, const double *b, double *partials, int n_part)
{
    k_dot<kThreads><<<n_part, kThreads, 0, L.s>>>(a, b, (int)n, partials);
    return cudaGetLastError();
}

cudaError_t launch_finish(const Launch &L, int what, const double *partials, int n_part, Scalars *sc)
{
    k_finish<<<1, 256, 0, L.s>>>(what, partials, n_part, sc);
    return cudaGetLastError();
}

cudaError_t launch_axpy_pair(const Launch &L, long n, const Scalars *sc, const double *p, const double *q, double *u,
                             double *r, double *partials, int n_part)
{
    k_axpy_pair<kThreads><<<n_part, kThreads, 0, L.s>>>(sc, p, q, u, r, (int)n, partials);
    return cudaGetLastError();
}

cudaError_t launch_xpby(const Launch &L, long n, const Scalars *sc, const double *z, double *p)
{
    k_xpby<kThreads><<<grid_for(n, kThreads, L.sm_count), kThreads, 0, L.s>>>(sc, z, p, (int)n);
    return cudaGetLastError();
}

}  // namespace tpmg
