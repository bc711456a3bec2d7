// FP64 kernels of the TPMG-preconditioned CG path for sm_103a.
//
// Layout: a field is [cell][k] with the vertical index fastest (Sec. 4.1: the
// column of a horizontal cell is stored contiguously).  Per cell: int4
// {nbr0, nbr1, nbr2, mask}, mask bit e set when neighbour e has a smaller
// colour; double4 {g0, g1, g2, g0+g1+g2}; area |T|.  Vertical factors are
// shared by all levels (no vertical coarsening, Sec. 3).
//
// The operator in the flux form of Appendix A (constant profiles, factorised
// storage: per-level vertical vectors times per-cell scalars, Sec. 3.1):
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

#include <algorithm>

#include "tpmg_internal.h"

namespace tpmg {

namespace {

constexpr int kThreads = 256;   // element-wise kernels

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
    const double *__restrict__ area;     // |T| beta^S_T
    const double *__restrict__ area_r;   // |T| alpha_r^S_T
    const double *__restrict__ vol;
    const double *__restrict__ w;
    const double *__restrict__ hr;
    int n_r;
    // the V-cycle's stencil stored per unknown (Sec. 4.2), or NULL for the factorised form:
    // c [n][n_r] {alphaS_hat e = 0, 1, 2, beta_hat} (TPMG^full), cr [n][n_r + 1]
    // alphar_hat of face k (TPMG^full and TPMG^partial)
    const dbl4 *__restrict__ c;
    const double *__restrict__ cr;
    // vertical advection (null without): area_x [n] |T| xi^S_T with the row vectors
    // xm, xp (factorised form), or cx [n][n_r + 1] X per face (stored, TPMG^full) with
    // the row thickness dr
    const double *__restrict__ area_x;
    const double *__restrict__ xm;
    const double *__restrict__ xp;
    const double *__restrict__ cx;
    const double *__restrict__ dr;
    // per-row products of the factorised coefficients (LevelDev::om, oc), or null
    const double *__restrict__ om;
    const double *__restrict__ oc;
    // with them, the horizontal couplings per unknown, three planes [3][n n_r] hr_k g_e
    // (LevelDev::ocs), or null
    const double *__restrict__ ocs;
};

inline OpView make_view(const LevelDev &lv, const VertDev &v, int n_r)
{
    return OpView{lv.nbr, lv.g, lv.area, lv.area_r, v.vol, v.w, v.hr, n_r, lv.vc, lv.vcr,
                  lv.area_x, v.xm, v.xp, lv.vcx_on ? lv.vcx : nullptr, v.dr, lv.om, lv.oc, lv.ocs};
}

// Stencil form of a level's V-cycle operator: factorised profiles (TPMG^fac), alpha_r
// per face (TPMG^partial), or everything per unknown (TPMG^full).
enum { CM_FAC = 0, CM_PARTIAL = 1, CM_FULL = 2 };
inline int stencil_form(const LevelDev &lv) { return lv.vc ? CM_FULL : (lv.vcr ? CM_PARTIAL : CM_FAC); }

// Column block A_T of a level (set-up kernels): the excess m_k of row k (its diagonal
// minus its vertical couplings) and the couplings of row k to the rows below and above,
//   down_k = alphar_hat_k - dr_k X_k,   up_k = alphar_hat_{k+1} + dr_k X_{k+1}
// (diffusion through the face minus / plus the centred vertical advection across it;
// without advection both are the symmetric alphar_hat of the face).
// A = |T| beta^S_T, G = sum of the edge weights g_e, Ar = |T| alpha_r^S_T, Ax = |T| xi^S_T.
__device__ __forceinline__ double col_excess(const OpView &o, int T, int k, double A, double G)
{
    if (o.c) {
        const dbl4 c = o.c[(size_t)T * o.n_r + k];
        return c.w + ((c.x + c.y) + c.z);
    }
    return fma(A, o.vol[k], o.hr[k] * G);
}
__device__ __forceinline__ double col_face(const OpView &o, int T, int k, double Ar)
{
    if (o.cr) return o.cr[(size_t)T * (o.n_r + 1) + k];
    return Ar * o.w[k];
}
__device__ __forceinline__ double col_down(const OpView &o, int T, int k, double Ar, double Ax)
{
    const double a = col_face(o, T, k, Ar);
    if (o.cx) return a - o.dr[k] * o.cx[(size_t)T * (o.n_r + 1) + k];
    if (o.area_x) return a - Ax * o.xm[k];
    return a;
}
__device__ __forceinline__ double col_up(const OpView &o, int T, int k, double Ar, double Ax)
{
    const double a = col_face(o, T, k + 1, Ar);
    if (o.cx) return a + o.dr[k] * o.cx[(size_t)T * (o.n_r + 1) + k + 1];
    if (o.area_x) return a + Ax * o.xp[k];
    return a;
}

// (A x)_{T,k} in flux form: 13 FP64 instructions.
template <bool ADV = false>
__device__ __forceinline__ double apply_at(const OpView &o, const double *__restrict__ x, int T, int k, int i)
{
    const int n_r = o.n_r;
    const int4 nb = __ldg(&o.nbr[T]);
    const dbl4 g = o.g[T];
    const double xc = x[i];
    const double dm = k > 0 ? xc - x[i - 1] : 0.0;
    const double dp = k < n_r - 1 ? xc - x[i + 1] : 0.0;
    const double vert = fma(__ldg(&o.w[k + 1]), dp, __ldg(&o.w[k]) * dm);
    const double hor = fma(g.z, xc - x[nb.z * n_r + k], fma(g.y, xc - x[nb.y * n_r + k], g.x * (xc - x[nb.x * n_r + k])));
    const double v = fma(__ldg(&o.area_r[T]), vert, fma(__ldg(&o.area[T]) * __ldg(&o.vol[k]), xc, __ldg(&o.hr[k]) * hor));
    if (!ADV) return v;
    // centred vertical advection: + Ax (xp_k (u_k - u_{k+1}) - xm_k (u_k - u_{k-1}))
    return fma(__ldg(&o.area_x[T]), fma(__ldg(&o.xp[k]), dp, -__ldg(&o.xm[k]) * dm), v);
}

// Row (T, k) of the problem's operator from its per-unknown coefficients (general,
// non-factorising profiles; the same flux form as apply_at).
struct FullView {
    const dbl4 *__restrict__ c;       // [n][n_r] {alphaS_hat 0, 1, 2, beta_hat}
    const double *__restrict__ cr;    // [n][n_r + 1] alphar_hat of face k
    const double *__restrict__ cx;    // [n][n_r + 1] advection X of face k, or null
};

__device__ __forceinline__ double apply_full_at(const OpView &o, const FullView &fv, const double *__restrict__ x,
                                                int T, int k, int i)
{
    const int n_r = o.n_r;
    const int4 nb = __ldg(&o.nbr[T]);
    const dbl4 c = fv.c[i];
    const double xc = x[i];
    const double dm = k > 0 ? xc - x[i - 1] : 0.0;
    const double dp = k < n_r - 1 ? xc - x[i + 1] : 0.0;
    const double *cr = fv.cr + (size_t)T * (n_r + 1) + k;
    double vert = fma(__ldg(&cr[1]), dp, __ldg(&cr[0]) * dm);
    if (fv.cx) {   // centred vertical advection: dr_k (X_{k+1} (u_k - u_{k+1}) - X_k (u_k - u_{k-1}))
        const double *cx = fv.cx + (size_t)T * (n_r + 1) + k;
        vert = fma(__ldg(&o.dr[k]), fma(__ldg(&cx[1]), dp, -__ldg(&cx[0]) * dm), vert);
    }
    const double hor = fma(c.z, xc - x[nb.z * n_r + k], fma(c.y, xc - x[nb.y * n_r + k], c.x * (xc - x[nb.x * n_r + k])));
    return fma(c.w, xc, vert + hor);
}

template <int NT, bool FULL, bool ADV>
__device__ __forceinline__ double apply_any(const OpView &o, const FullView &fv, const double *__restrict__ x, int T,
                                            int k, int i)
{
    if (FULL) return apply_full_at(o, fv, x, T, k, i);
    return apply_at<ADV>(o, x, T, k, i);
}

// Row (T, k) of the factorised operator for kernels whose warps hold consecutive rows:
// lane l has row i and lane l + 1 row i + 1 (of the same column, or row 0 of the next,
// whose lower difference is 0).  d = x_k - x_{k-1} is this row's lower-face difference
// (0 for k = 0) and du = x_{k+1} - x_k, from the next lane, the upper one, so the
// vertical fluxes stay differences of neighbouring values (the nearly singular vertical
// mode of a column needs them) while each difference is formed once:
//   vertical = w_k d - w_{k+1} du.
// The horizontal part, whose couplings are only omega^2/h^2 times the mass term, is
// summed directly: m x_k - hr_k sum_e g_e x_e with the diagonal excess
// m = |T| v_k + hr_k G.  11 FP64 operations where apply_at takes 14.
template <bool ADV>
__device__ __forceinline__ double apply_at_lanes(const OpView &o, const double *__restrict__ x, int T, int k,
                                                 double xc, double d, double du)
{
    const int n_r = o.n_r;
    const int4 nb = __ldg(&o.nbr[T]);
    const dbl4 g = o.g[T];
    const double S = fma(g.z, x[nb.z * n_r + k], fma(g.y, x[nb.y * n_r + k], g.x * x[nb.x * n_r + k]));
    const double hrk = __ldg(&o.hr[k]);
    const double m = fma(__ldg(&o.area[T]), __ldg(&o.vol[k]), hrk * g.w);
    const double vert = fma(__ldg(&o.w[k]), d, -__ldg(&o.w[k + 1]) * du);
    const double v = fma(__ldg(&o.area_r[T]), vert, fma(m, xc, -hrk * S));
    if (!ADV) return v;
    // centred vertical advection: Ax (xp_k (x_k - x_{k+1}) - xm_k (x_k - x_{k-1}))
    return fma(__ldg(&o.area_x[T]), fma(-__ldg(&o.xp[k]), du, -__ldg(&o.xm[k]) * d), v);
}

// Row (T, k) with the vertical couplings per face (TPMG^partial): apply_at with
// area_r w_k replaced by the stored alphar_hat of face k.
template <bool ADV>
__device__ __forceinline__ double apply_partial_at(const OpView &o, const double *__restrict__ x, int T, int k, int i)
{
    const int n_r = o.n_r;
    const int4 nb = __ldg(&o.nbr[T]);
    const dbl4 g = o.g[T];
    const double xc = x[i];
    const double dm = k > 0 ? xc - x[i - 1] : 0.0;
    const double dp = k < n_r - 1 ? xc - x[i + 1] : 0.0;
    const double *cr = o.cr + (size_t)T * (n_r + 1) + k;
    double vert = fma(__ldg(&cr[1]), dp, __ldg(&cr[0]) * dm);
    if (ADV) vert = fma(__ldg(&o.area_x[T]), fma(__ldg(&o.xp[k]), dp, -__ldg(&o.xm[k]) * dm), vert);
    const double hor = fma(g.z, xc - x[nb.z * n_r + k], fma(g.y, xc - x[nb.y * n_r + k], g.x * (xc - x[nb.x * n_r + k])));
    return vert + fma(__ldg(&o.area[T]) * __ldg(&o.vol[k]), xc, __ldg(&o.hr[k]) * hor);
}

// Row (T, k) of a level's V-cycle operator in stencil form CM.
template <int CM, bool ADV>
__device__ __forceinline__ double apply_vc(const OpView &o, const double *__restrict__ x, int T, int k, int i)
{
    if (CM == CM_FULL) return apply_full_at(o, FullView{o.c, o.cr, o.cx}, x, T, k, i);
    if (CM == CM_PARTIAL) return apply_partial_at<ADV>(o, x, T, k, i);
    return apply_at<ADV>(o, x, T, k, i);
}

// -hr_k sum_e g_e x_e + rest for row (T, k) = i of the finest level's outer operator:
// from the couplings per unknown, three FMAs (hr_k g_e stored: LevelDev::ocs), else
// from the factorised couplings, four operations.
__device__ __forceinline__ double outer_horizontal(const OpView &o, const double *__restrict__ x, int T, int k, int i,
                                                   int N, double rest)
{
    const int n_r = o.n_r;
    const int4 nb = __ldg(&o.nbr[T]);
    if (o.ocs) {
        const double c0 = __ldg(&o.ocs[i]), c1 = __ldg(&o.ocs[(size_t)N + i]), c2 = __ldg(&o.ocs[2 * (size_t)N + i]);
        return fma(-c2, x[nb.z * n_r + k], fma(-c1, x[nb.y * n_r + k], fma(-c0, x[nb.x * n_r + k], rest)));
    }
    const dbl4 g = o.g[T];
    const double S = fma(g.z, x[nb.z * n_r + k], fma(g.y, x[nb.y * n_r + k], g.x * x[nb.x * n_r + k]));
    return fma(-__ldg(&o.hr[k]), S, rest);
}

// The kernels below take the block index and the grid size as arguments of their
// bodies (bid, nblk), so that the batched form runs the same code as block bid of
// a launch of nblk blocks for each member: same partition, same partial sums.
template <int NT, bool FULL, bool ADV>
__device__ __forceinline__ void apply_body(const OpView &o, const FullView &fv, const double *__restrict__ x,
                                           double *__restrict__ y, int N, double *__restrict__ partials, int bid,
                                           int nblk)
{
    double acc = 0.0;
    if (FULL) {
        for (int i = bid * NT + threadIdx.x; i < N; i += nblk * NT) {
            const int T = i / o.n_r, k = i - T * o.n_r;
            const double v = apply_any<NT, FULL, ADV>(o, fv, x, T, k, i);
            y[i] = v;
            acc = fma(x[i], v, acc);
        }
    } else if (!ADV && o.om) {
        // stored row products: the flux through the row's lower face, F_k = oc_k (x_k - x_{k-1}),
        // is formed once and handed to the row below by a shuffle, so the vertical part is
        // F_k - F_{k+1}; the row is om x_k - hr_k sum_e g_e x_e + F_k - F_{k+1} (8 FP64 operations)
        const int lane = threadIdx.x & 31;
        const int stride = nblk * (NT / 32) * 31;
        for (int base = (bid * (NT / 32) + (threadIdx.x >> 5)) * 31; base < N; base += stride) {
            const int i = base + lane;
            int T = 0, k = 0;
            double xc = 0.0, F = 0.0;
            if (i < N) {
                T = i / o.n_r;
                k = i - T * o.n_r;
                xc = x[i];
                if (k > 0) F = __ldg(&o.oc[i]) * (xc - x[i - 1]);
            }
            const double Fu = __shfl_down_sync(0xffffffffu, F, 1);
            if (lane < 31 && i < N) {
                const double v = fma(__ldg(&o.om[i]), xc, outer_horizontal(o, x, T, k, i, N, F - Fu));
                y[i] = v;
                acc = fma(xc, v, acc);
            }
        }
    } else {
        // each warp takes 32 consecutive rows and writes the first 31; lane 31 only hands its
        // lower difference to lane 30 (apply_at_lanes)
        const int lane = threadIdx.x & 31;
        const int stride = nblk * (NT / 32) * 31;
        for (int base = (bid * (NT / 32) + (threadIdx.x >> 5)) * 31; base < N; base += stride) {
            const int i = base + lane;
            int T = 0, k = 0;
            double xc = 0.0, d = 0.0;
            if (i < N) {
                T = i / o.n_r;
                k = i - T * o.n_r;
                xc = x[i];
                if (k > 0) d = xc - x[i - 1];
            }
            const double du = __shfl_down_sync(0xffffffffu, d, 1);
            if (lane < 31 && i < N) {
                const double v = apply_at_lanes<ADV>(o, x, T, k, xc, d, du);
                y[i] = v;
                acc = fma(xc, v, acc);
            }
        }
    }
    if (partials) {
        acc = block_sum<NT>(acc);
        if (threadIdx.x == 0) partials[bid] = acc;
    }
}

template <int NT, bool FULL, bool ADV>
__global__ void __launch_bounds__(NT) k_apply(OpView o, FullView fv, const double *__restrict__ x,
                                              double *__restrict__ y, int N, double *__restrict__ partials)
{
    pdl_wait();
    pdl_trigger();
    apply_body<NT, FULL, ADV>(o, fv, x, y, N, partials, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ bool is_zero(double v) { return (__double_as_longlong(v) << 1) == 0; }

// The per-row products of the factorised coefficients used by k_apply (set-up):
// om = |T| v_k + hr_k G_T, the same expression apply_at_lanes forms per row, and
// oc = |T| alpha_r^S w_k of the row's lower face.
__global__ void __launch_bounds__(256) k_outer_products(OpView o, int N, double *__restrict__ om,
                                                        double *__restrict__ oc, double *__restrict__ ocs)
{
    for (int i = blockIdx.x * 256 + threadIdx.x; i < N; i += gridDim.x * 256) {
        const int T = i / o.n_r, k = i - T * o.n_r;
        om[i] = fma(o.area[T], o.vol[k], o.hr[k] * o.g[T].w);
        oc[i] = o.area_r[T] * o.w[k];
        if (ocs) {
            const dbl4 g = o.g[T];
            ocs[i] = o.hr[k] * g.x;
            ocs[(size_t)N + i] = o.hr[k] * g.y;
            ocs[2 * (size_t)N + i] = o.hr[k] * g.z;
        }
    }
}

// r = f - A u with partial ||r||^2.  With the stored row products (the finest
// level of the factorised operator) the rows are formed as in k_apply; otherwise in
// flux form, where a warp whose stencil reads exact zeros on every lane (A u exactly
// zero) skips its FP64 arithmetic -- the test is on bit patterns, so it costs no FP64
// instruction.  Either way a guess that k_nonzero found to be zero is not read at all.
template <int NT, bool FULL, bool ADV, bool R32>
__device__ __forceinline__ void residual_body(const OpView &o, const FullView &full, const double *__restrict__ f,
                                              const double *__restrict__ u, double *__restrict__ r, int N,
                                              double *__restrict__ partials, const int *__restrict__ nz, int n_nz,
                                              int bid, int nblk, float *__restrict__ r32)
{
    double acc = 0.0;
    const int stride = nblk * NT, n_r = o.n_r;
    // nz: the blocks' flags of k_nonzero over u; with none set u is exactly zero, so
    // r = f, accumulated in the same order as below (bit-identical), without the stencil's loads
    int any = nz ? 0 : 1;
    for (int t = threadIdx.x; t < n_nz; t += NT) any |= nz[t];
    const bool copy = !__syncthreads_or(any);
    if (!FULL && !ADV && o.om) {
        // the stored row products (as k_apply): each warp takes 32 consecutive rows and
        // writes the first 31; the flux through a row's lower face, F_k = oc_k (u_k - u_{k-1}),
        // is formed once and handed to the row below by a shuffle, and
        // r = f - (om u_k - hr_k sum_e g_e u_e + F_k - F_{k+1}): 10 FP64 operations a row
        // with the partial sum of r^2, where the flux form takes 16
        const int lane = threadIdx.x & 31;
        const int wstride = nblk * (NT / 32) * 31;
        const int base0 = (bid * (NT / 32) + (threadIdx.x >> 5)) * 31;
        if (copy) {
            // a zero guess: r = f over the same rows, accumulated in the same order as below,
            // with four rows' loads in flight per thread
            for (int base = base0; base < N; base += 4 * wstride) {
                double v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = base + q * wstride + lane;
                    v[q] = (lane < 31 && i < N) ? f[i] : 0.0;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = base + q * wstride + lane;
                    if (lane < 31 && i < N) {
                        r[i] = v[q];
                        if (R32) r32[i] = (float)v[q];
                        acc = fma(v[q], v[q], acc);
                    }
                }
            }
        }
        for (int base = copy ? N : base0; base < N; base += wstride) {
            const int i = base + lane;
            int T = 0, k = 0;
            double xc = 0.0, F = 0.0;
            if (i < N) {
                T = i / n_r;
                k = i - T * n_r;
                xc = u[i];
                if (k > 0) F = __ldg(&o.oc[i]) * (xc - u[i - 1]);
            }
            const double Fu = __shfl_down_sync(0xffffffffu, F, 1);
            if (lane < 31 && i < N) {
                const double v = f[i] - fma(__ldg(&o.om[i]), xc, outer_horizontal(o, u, T, k, i, N, F - Fu));
                r[i] = v;
                if (R32) r32[i] = (float)v;
                acc = fma(v, v, acc);
            }
        }
        if (partials) {
            acc = block_sum<NT>(acc);
            if (threadIdx.x == 0) partials[bid] = acc;
        }
        return;
    }
    if (copy) {
        for (int i = bid * NT + threadIdx.x; i < N; i += stride) {
            const double v = f[i];
            r[i] = v;
            if (R32) r32[i] = (float)v;
            acc = fma(v, v, acc);
        }
        if (partials) {
            acc = block_sum<NT>(acc);
            if (threadIdx.x == 0) partials[bid] = acc;
        }
        return;
    }
    for (int i0 = bid * NT + threadIdx.x; i0 < N; i0 += 2 * stride) {
        double fv[2], uc[2], um[2], up[2], u0[2], u1[2], u2[2];
        int T[2], k[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = i0 + q * stride;
            fv[q] = uc[q] = um[q] = up[q] = u0[q] = u1[q] = u2[q] = 0.0;
            T[q] = k[q] = 0;
            if (i < N) {
                T[q] = i / n_r;
                k[q] = i - T[q] * n_r;
                const int4 nb = __ldg(&o.nbr[T[q]]);
                fv[q] = f[i];
                uc[q] = u[i];
                if (k[q] > 0) um[q] = u[i - 1];
                if (k[q] < n_r - 1) up[q] = u[i + 1];
                u0[q] = u[nb.x * n_r + k[q]];
                u1[q] = u[nb.y * n_r + k[q]];
                u2[q] = u[nb.z * n_r + k[q]];
            }
        }
        bool zero = true;
#pragma unroll
        for (int q = 0; q < 2; ++q)
            zero = zero && is_zero(uc[q]) && is_zero(um[q]) && is_zero(up[q]) && is_zero(u0[q]) && is_zero(u1[q]) &&
                   is_zero(u2[q]);
        const bool skip = __all_sync(__activemask(), zero);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = i0 + q * stride;
            if (i >= N) continue;
            double v = fv[q];
            if (!skip) v = v - apply_any<NT, FULL, ADV>(o, full, u, T[q], k[q], i);
            r[i] = v;
            if (R32) r32[i] = (float)v;
            acc = fma(v, v, acc);
        }
    }
    if (partials) {
        acc = block_sum<NT>(acc);
        if (threadIdx.x == 0) partials[bid] = acc;
    }
}

// R32: r is also written in FP32 (the mixed V-cycle's copy).  A compile-time choice:
// the double -> float conversion runs on the FP64 pipe, and a kernel that only skips
// its store at run time may still issue it.
// 8 blocks of NT threads per SM (at most 32 registers): the n_part = 8 x SMs blocks of the
// reductions in one wave (40 registers left a second, partial wave: 0.88 against 0.85 ms at
// 41.9 M unknowns)
template <int NT, bool FULL, bool ADV, bool R32>
__global__ void __launch_bounds__(NT, 8) k_residual(OpView o, FullView full, const double *__restrict__ f,
                                                 const double *__restrict__ u, double *__restrict__ r, int N,
                                                 double *__restrict__ partials, const int *__restrict__ nz,
                                                 int n_nz, float *__restrict__ r32)
{
    pdl_wait();
    pdl_trigger();
    residual_body<NT, FULL, ADV, R32>(o, full, f, u, r, N, partials, nz, n_nz, blockIdx.x, gridDim.x, r32);
}

// Per block, whether x has a nonzero element in the block's grid-stride range (a test
// of bit patterns, no FP64 instruction): the probe of k_residual's zero-guess path.
template <int NT>
__device__ __forceinline__ void nonzero_body(const double *__restrict__ x, int N, int *__restrict__ nz, int bid,
                                             int nblk)
{
    int any = 0;
    const int stride = nblk * NT;
    int i = bid * NT + threadIdx.x;
    for (; i + 3 * stride < N; i += 4 * stride) {
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = x[i + q * stride];
#pragma unroll
        for (int q = 0; q < 4; ++q) any |= !is_zero(v[q]);
    }
    for (; i < N; i += stride) any |= !is_zero(x[i]);
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) nz[bid] = any;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_nonzero(const double *__restrict__ x, int N, int *__restrict__ nz)
{
    pdl_wait();
    pdl_trigger();
    nonzero_body<NT>(x, N, nz, blockIdx.x, gridDim.x);
}

// f_c[T][k] = sum_j (f - A u)[4T + j][k]  (Algorithm 1 residual + restriction, Sec. 5)
template <int NT, int CM, bool ADV>
__global__ void __launch_bounds__(NT) k_resid_restrict(OpView o, const double *__restrict__ f,
                                                       const double *__restrict__ u, double *__restrict__ fc, int Nc)
{
    pdl_wait();
    pdl_trigger();
    if (CM != CM_FAC) {
        for (int ic = blockIdx.x * NT + threadIdx.x; ic < Nc; ic += gridDim.x * NT) {
            const int Tc = ic / o.n_r, k = ic - Tc * o.n_r;
            double s = 0.0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int T = 4 * Tc + j, i = T * o.n_r + k;
                s += f[i] - apply_vc<CM, ADV>(o, u, T, k, i);
            }
            fc[ic] = s;
        }
        return;
    }
    // factorised: warps of 32 consecutive coarse rows (31 written), so that lane l + 1 holds
    // the next row of each child column as well (apply_at_lanes)
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * (NT / 32) * 31;
    for (int base = (blockIdx.x * (NT / 32) + (threadIdx.x >> 5)) * 31; base < Nc; base += stride) {
        const int ic = base + lane;
        const bool act = ic < Nc;
        const int Tc = act ? ic / o.n_r : 0, k = act ? ic - Tc * o.n_r : 0;
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int T = 4 * Tc + j, i = T * o.n_r + k;
            double xc = 0.0, d = 0.0;
            if (act) {
                xc = u[i];
                if (k > 0) d = xc - u[i - 1];
            }
            const double du = __shfl_down_sync(0xffffffffu, d, 1);
            if (act && lane < 31) s += f[i] - apply_at_lanes<ADV>(o, u, T, k, xc, d, du);
        }
        if (act && lane < 31) fc[ic] = s;
    }
}

// The same restriction for the factorised operator without advection, from the sums
// over the 4 children instead of each child's residual:
//   f_c = sum_j f_j - vol_k sum_j A_j u_j - (w_k D_k - w_{k+1} D_{k+1})
//         - hr_k (sum_j Gext_j u_j - sum_{outside edges e} g_e u_e),
// with D_k = sum_j Ar_j (u_{j,k} - u_{j,k-1}) the children's lower-face differences
// (taken from the next lane for face k+1), and the horizontal fluxes across the edges
// between the children dropped, as they cancel in the sum (RestrictGeo).  32 FP64
// operations per coarse row where summing 4 child residuals takes 52.
template <int NT>
__global__ void __launch_bounds__(NT) k_restrict_fac(const RestrictGeo *__restrict__ geo, const double *__restrict__ vol,
                                                     const double *__restrict__ w, const double *__restrict__ hr,
                                                     const double *__restrict__ f, const double *__restrict__ u,
                                                     double *__restrict__ fc, int n_r, int Nc)
{
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * (NT / 32) * 31;
    for (int base = (blockIdx.x * (NT / 32) + (threadIdx.x >> 5)) * 31; base < Nc; base += stride) {
        const int ic = base + lane;
        const bool act = ic < Nc;
        const int Tc = act ? ic / n_r : 0, k = act ? ic - Tc * n_r : 0;
        double D = 0.0, F = 0.0, M = 0.0, H = 0.0;
        if (act) {
            const RestrictGeo &G = geo[Tc];
            const int4 x0 = G.x0, x1 = G.x1;
            const dbl4 g0 = G.g0, g1 = G.g1, gx = G.gext, A = G.A, Ar = G.Ar;
            const int i0 = 4 * Tc * n_r + k;
            double uc[4], um[4], fv[4], ue[6];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uc[j] = u[i0 + j * n_r];
                um[j] = k > 0 ? u[i0 + j * n_r - 1] : uc[j];
                fv[j] = f[i0 + j * n_r];
            }
            ue[0] = u[x0.x * n_r + k];
            ue[1] = u[x0.y * n_r + k];
            ue[2] = u[x0.z * n_r + k];
            ue[3] = u[x0.w * n_r + k];
            ue[4] = u[x1.x * n_r + k];
            ue[5] = u[x1.y * n_r + k];
            D = fma(Ar.w, uc[3] - um[3], fma(Ar.z, uc[2] - um[2], fma(Ar.y, uc[1] - um[1], Ar.x * (uc[0] - um[0]))));
            M = fma(A.w, uc[3], fma(A.z, uc[2], fma(A.y, uc[1], A.x * uc[0])));
            const double H1 = fma(gx.w, uc[3], fma(gx.z, uc[2], fma(gx.y, uc[1], gx.x * uc[0])));
            const double H2 = fma(g1.y, ue[5], fma(g1.x, ue[4], fma(g0.w, ue[3], fma(g0.z, ue[2], fma(g0.y, ue[1],
                                                                                                    g0.x * ue[0])))));
            H = H1 - H2;
            F = (fv[0] + fv[1]) + (fv[2] + fv[3]);
        }
        const double Du = __shfl_down_sync(0xffffffffu, D, 1);
        if (act && lane < 31) {
            const double vert = fma(__ldg(&w[k]), D, -__ldg(&w[k + 1]) * Du);
            fc[ic] = F - fma(__ldg(&vol[k]), M, fma(__ldg(&hr[k]), H, vert));
        }
    }
}

// Linear prolongation (Sec. 5): child j of coarse cell T takes
//   u_T + sum_e w_{T,j,e} (u_{nbr e} - u_T)
// per vertical index, the weights those of the least-squares tangent-plane gradient
// (set-up); one thread per fine unknown, coalesced along k.
template <int NT>
__global__ void __launch_bounds__(NT) k_prolong_linear(const int4 *__restrict__ nbr_c, const double *__restrict__ w,
                                                       const double *__restrict__ uc, double *__restrict__ u,
                                                       int n_r, int N)
{
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * NT + threadIdx.x; i < N; i += gridDim.x * NT) {
        const int t = i / n_r, k = i - t * n_r, T = t >> 2, j = t & 3;
        const int4 nb = __ldg(&nbr_c[T]);
        const double *wt = w + (size_t)T * 12 + 3 * j;
        const double v = uc[(size_t)T * n_r + k];
        double s = fma(__ldg(&wt[0]), uc[(size_t)nb.x * n_r + k] - v, v);
        s = fma(__ldg(&wt[1]), uc[(size_t)nb.y * n_r + k] - v, s);
        s = fma(__ldg(&wt[2]), uc[(size_t)nb.z * n_r + k] - v, s);
        u[i] += s;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_prolong_add(const double *__restrict__ uc, double *__restrict__ u, int n_r, int N)
{
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * NT + threadIdx.x; i < N; i += gridDim.x * NT) {
        const int T = i / n_r, k = i - T * n_r;
        u[i] += uc[(T >> 2) * n_r + k];
    }
}

// Twisted Thomas factors of the column blocks A_T (Sec. 4.1; set-up, one
// thread per column of a task).  A_T has couplings c_k = |T| w_k between rows
// k-1 and k and diagonal c_k + c_{k+1} + m_k with excess m_k = |T| v_k +
// hr_k G_T.  Rows 0..j-1 are eliminated from the top and rows n_r-1..j+1 from
// the bottom; each pivot is carried through its excess over the coupling it
// has not yet eliminated:
//   top:    e_0 = m_0,          e_k = m_k + c_k e_{k-1} / p_{k-1},       p_k = e_k + c_{k+1}
//   bottom: e'_{n-1} = m_{n-1}, e'_k = m_k + c_{k+1} e'_{k+1} / q_{k+1}, q_k = e'_k + c_k
//   meeting row: gamma_j = m_j + c_j e_{j-1} / p_{j-1} + c_{j+1} e'_{j+1} / q_{j+1}.
// Only sums of non-negative terms: full relative precision although c_k / m_k
// reaches 1e6-1e9 in a thin shell.  With t_k = d_k / pivot_k the solve is
//   top:    y_k = t_k + (c_k / p_k) y_{k-1},      x_k = y_k + (c_{k+1} / p_k) x_{k+1}
//   bottom: z_k = t_k + (c_{k+1} / q_k) z_{k+1},  x_k = z_k + (c_k / q_k) x_{k-1}
//   x_j = t_j + (c_j / gamma) y_{j-1} + (c_{j+1} / gamma) z_{j+1}.
// Stored: rinv [cell][k] = 1 / pivot of row k (cell-major, read with d);
// fb, fc [task][step][lane] the forward and backward multipliers; fm
// [task][2][16] the two multipliers of the meeting row.
__global__ void k_twisted_factors(int n_tasks, OpView o, const int *__restrict__ cells, int S, int j,
                                  double *__restrict__ rinv, double *__restrict__ fb, double *__restrict__ fc,
                                  double *__restrict__ fm)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n_tasks * kRelaxCols) return;
    const int t = gid / kRelaxCols, col = gid - t * kRelaxCols;
    const int T = cells[gid];
    const int n = o.n_r;
    const size_t base = (size_t)t * S * 32;
    for (int s = 0; s < S; ++s) {
        fb[base + s * 32 + col] = fc[base + s * 32 + col] = 0.0;
        fb[base + s * 32 + col + 16] = fc[base + s * 32 + col + 16] = 0.0;
    }
    double *M = fm + (size_t)t * 2 * kRelaxCols;
    M[col] = M[kRelaxCols + col] = 0.0;
    if (T < 0) return;
    double *ri = rinv + (size_t)T * n;
    const double A = o.area[T], Ar = o.area_r[T], G = o.g[T].w, Ax = o.area_x ? o.area_x[T] : 0.0;
    double e = 0.0, p = 1.0;
    for (int k = 0; k < j; ++k) {
        const double m = col_excess(o, T, k, A, G);
        const double c = col_down(o, T, k, Ar, Ax), cu = col_up(o, T, k, Ar, Ax);
        e = k == 0 ? m : m + c * e / p;
        p = e + cu;
        const double iv = 1.0 / p;
        ri[k] = iv;
        fb[base + k * 32 + col] = c * iv;
        fc[base + k * 32 + col] = cu * iv;
    }
    double eb = 0.0, q = 1.0;
    for (int k = n - 1, s = 0; k > j; --k, ++s) {
        const double m = col_excess(o, T, k, A, G);
        const double cd = col_down(o, T, k, Ar, Ax), cu = col_up(o, T, k, Ar, Ax);
        eb = k == n - 1 ? m : m + cu * eb / q;
        q = eb + cd;
        const double iv = 1.0 / q;
        ri[k] = iv;
        fb[base + s * 32 + col + 16] = cu * iv;
        fc[base + s * 32 + col + 16] = cd * iv;
    }
    const double cj = col_down(o, T, j, Ar, Ax), cj1 = col_up(o, T, j, Ar, Ax);
    double gam = col_excess(o, T, j, A, G);
    if (j > 0) gam += cj * e / p;
    if (j < n - 1) gam += cj1 * eb / q;
    const double ig = 1.0 / gam;
    ri[j] = ig;
    M[col] = cj * ig;
    M[kRelaxCols + col] = cj1 * ig;
}

// Scaled couplings of the twisted relaxation (set-up, after k_twisted_factors): three
// planes of n n_r doubles, cs_e [T][k] = hr_k g_e(T) rinv [T][k] (e = 0, 1, 2).
__global__ void k_scaled_couplings(OpView o, long nn, const double *__restrict__ rinv, double *__restrict__ cs)
{
    const int n_r = o.n_r;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const long T = i / n_r;
        const int k = (int)(i - T * n_r);
        const dbl4 g = o.g[T];
        const double h = o.hr[k], iv = rinv[i];
        cs[i] = (h * g.x) * iv;
        cs[nn + i] = (h * g.y) * iv;
        cs[2 * nn + i] = (h * g.z) * iv;
    }
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

// Twisted Thomas solve of one column pair (one warp of k_relax): lane =
// column + 16 * half.  B, C point at the task's [step][32] multiplier blocks
// (global or shared memory), tc at the column's row of the shared tile, which
// holds t = d / pivot on entry and x on exit.  Each half is a chain of `rows`
// dependent FMAs forward and back; the loads of the next P steps are issued
// while the current P are computed.
template <int P>
__device__ __forceinline__ void twisted_solve(const double *B, const double *C, const double *M, double *tc,
                                              int n_r, int j, int lane)
{
    const int c = lane & (kRelaxCols - 1), half = lane >> 4;
    const int rows = half ? n_r - 1 - j : j;
    auto row_of = [&](int s) { return half ? n_r - 1 - s : s; };
    double y = 0.0;
    {
        double b[P], d[P];
#pragma unroll
        for (int q = 0; q < P; ++q)
            if (q < rows) { b[q] = B[q * 32]; d[q] = tc[row_of(q)]; }
        for (int s0 = 0; s0 < rows; s0 += P) {
            double bn[P], dn[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int s = s0 + P + q;
                if (s < rows) { bn[q] = B[s * 32]; dn[q] = tc[row_of(s)]; }
            }
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int s = s0 + q;
                if (s < rows) {
                    y = fma(b[q], y, d[q]);
                    tc[row_of(s)] = y;
                }
            }
#pragma unroll
            for (int q = 0; q < P; ++q) { b[q] = bn[q]; d[q] = dn[q]; }
        }
    }
    __syncwarp();
    const double other = __shfl_xor_sync(0xffffffffu, y, 16);
    const double ytop = half ? other : y, zbot = half ? y : other;
    const double xj = fma(M[kRelaxCols + c], zbot, fma(M[c], ytop, tc[j]));
    __syncwarp();
    if (half == 0) tc[j] = xj;
    double x = xj;
    {
        double cc[P], yy[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int s = rows - 1 - q;
            if (s >= 0) { cc[q] = C[s * 32]; yy[q] = tc[row_of(s)]; }
        }
        for (int s0 = rows - 1; s0 >= 0; s0 -= P) {
            double cn[P], yn[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int s = s0 - P - q;
                if (s >= 0) { cn[q] = C[s * 32]; yn[q] = tc[row_of(s)]; }
            }
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int s = s0 - q;
                if (s >= 0) {
                    x = fma(cc[q], x, yy[q]);
                    tc[row_of(s)] = x;
                }
            }
#pragma unroll
            for (int q = 0; q < P; ++q) { cc[q] = cn[q]; yy[q] = yn[q]; }
        }
    }
}

// Right-hand-side forms of a twisted relaxation pass (phase A), per row k of a
// column T with the neighbours' iterates u_e and pivot p_k:
//   SK_FAC           t = (f + hr_k sum_e g_e u_e) / p_k    (factorised couplings)
//   SK_FULL          t = (f + sum_e c_e u_e) / p_k         (stencil stored per unknown)
//   SK_SCALED_FIRST  t = f / p_k + sum_e cs_e u_e, also writing f / p_k to ft
//   SK_SCALED        t = ft + sum_e cs_e u_e
// with the scaled couplings cs_e = hr_k g_e / p_k stored per unknown.  The same
// value in exact arithmetic; the scaled forms take 3 FP64 operations a row instead
// of 5 once the colour's ft is written (by its first pass in a visit of the level).
enum RhsForm { SK_FAC = 0, SK_FULL = 1, SK_SCALED_FIRST = 2, SK_SCALED = 3 };

// Phase A for the elements e = tid, tid + NTH, ... of the task's [16][n_r] block:
// t into the shared tile [16][n_r + 1], U elements' loads in flight per thread.
// Padding columns (cell -1) get t = 0.  SK_SCALED reads ft through f.
template <int MODE, int SK, int U, int NTH>
__device__ __forceinline__ void gather_rhs(const OpView &o, const int *s_cell, const int4 *s_nb, const dbl4 *s_g,
                                           const double *__restrict__ rinv, const double *__restrict__ csc,
                                           size_t plane, const double *__restrict__ f, const double *u_in,
                                           double *__restrict__ ft_out, double *tile, int tid)
{
    const int n_r = o.n_r, ld = n_r + 1, ne = kRelaxCols * n_r;
    for (int e0 = tid; e0 < ne; e0 += NTH * U) {
        double fv[U], iv[U], v0[U], v1[U], v2[U];
        dbl4 cs[U];   // SK_FULL: the stored stencil; scaled forms: the scaled couplings in x, y, z
        int col[U], kk[U], gi[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int e = e0 + NTH * q;
            col[q] = -1;
            kk[q] = 0;
            gi[q] = -1;
            fv[q] = iv[q] = v0[q] = v1[q] = v2[q] = 0.0;
            if (SK != SK_FAC) cs[q] = dbl4{0.0, 0.0, 0.0, 0.0};
            if (e < ne) {
                const int c = e / n_r, k = e - c * n_r;
                col[q] = c;
                kk[q] = k;
                const int T = s_cell[c];
                if (T >= 0) {
                    const int i = T * n_r + k;
                    gi[q] = i;
                    fv[q] = f[i];
                    if (SK != SK_SCALED) iv[q] = __ldg(&rinv[i]);
                    if (MODE != PASS_RHS_ONLY) {
                        const int4 nb = s_nb[c];
                        if (MODE == PASS_NORMAL || (nb.w & 1)) v0[q] = u_in[nb.x * n_r + k];
                        if (MODE == PASS_NORMAL || (nb.w & 2)) v1[q] = u_in[nb.y * n_r + k];
                        if (MODE == PASS_NORMAL || (nb.w & 4)) v2[q] = u_in[nb.z * n_r + k];
                        if (SK == SK_FULL) cs[q] = o.c[i];
                        if (SK >= SK_SCALED_FIRST) {
                            cs[q].x = __ldg(&csc[i]);
                            cs[q].y = __ldg(&csc[plane + i]);
                            cs[q].z = __ldg(&csc[2 * plane + i]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (col[q] < 0) continue;
            double d = fv[q];
            if (SK >= SK_SCALED_FIRST) {
                if (SK == SK_SCALED_FIRST) {
                    d = fv[q] * iv[q];
                    if (ft_out && gi[q] >= 0) ft_out[gi[q]] = d;
                }
                if (MODE != PASS_RHS_ONLY) d = fma(cs[q].z, v2[q], fma(cs[q].y, v1[q], fma(cs[q].x, v0[q], d)));
                tile[col[q] * ld + kk[q]] = d;
            } else {
                if (MODE != PASS_RHS_ONLY) {
                    if (SK == SK_FULL) {
                        d = fma(cs[q].z, v2[q], fma(cs[q].y, v1[q], fma(cs[q].x, v0[q], d)));
                    } else {
                        const dbl4 g = s_g[col[q]];
                        d = fma(__ldg(&o.hr[kk[q]]), fma(g.z, v2[q], fma(g.y, v1[q], g.x * v0[q])), d);
                    }
                }
                tile[col[q] * ld + kk[q]] = d * iv[q];
            }
        }
    }
}

// One relaxation pass (eq. BlockJacobi) over whole tasks of 16 columns, one
// task per CTA of NT threads (64, 128 or 256; chosen per level by the autotuner):
//   u_T <- (1 - relax) u_T + relax A_T^{-1} (f_T + hr sum_e g_e u_{T_e}).
// Phase A (all threads, coalesced along k, the loads of several elements in
// flight per thread): t = (f + hr_k sum_e g_e u_{T_e,k}) / pivot_k into a
// [16][n_r+1] shared tile.  STAGE (small levels, where few CTAs cannot hide
// the load latency): the task's multiplier blocks are copied to shared memory
// by cp.async meanwhile, and deeper unrolling keeps more loads in flight;
// otherwise the register budget is kept for 6 resident CTAs per SM.
// Phase B (one warp, rotating with the CTA index so that the serial phases of
// the CTAs resident on an SM spread over its four FP64 units): the twisted
// Thomas solve.  Phase C (all threads): write back, optional relaxation
// weight, optional prolongation into the 4 children (u_fine += P x), loads
// issued before their stores.  In the multicolour passes u_in == u_out: a pass
// reads other colours' columns and its own column before writing it.
// One-directional Thomas factors per unknown (levels relaxed by k_relax_scan):
// the excess-carried recurrence (reading C16) from the bottom row upwards,
//   e_0 = m_0, e_k = m_k + c_k e_{k-1} / p_{k-1}, p_k = e_k + c_{k+1},
// rinv = 1 / p_k, fb = c_k / p_k (0 for k = 0), fc = c_{k+1} / p_k.
__global__ void k_thomas_factors(OpView o, int n_cells, double *__restrict__ rinv, double *__restrict__ fb,
                                 double *__restrict__ fc)
{
    const int T = blockIdx.x * blockDim.x + threadIdx.x;
    if (T >= n_cells) return;
    const int n = o.n_r;
    const size_t row0 = (size_t)T * n;
    const double A = o.area[T], Ar = o.area_r[T], G = o.g[T].w, Ax = o.area_x ? o.area_x[T] : 0.0;
    double e = 0.0, p = 1.0;
    for (int k = 0; k < n; ++k) {
        const double m = col_excess(o, T, k, A, G);
        const double c = k > 0 ? col_down(o, T, k, Ar, Ax) : 0.0, cu = k < n - 1 ? col_up(o, T, k, Ar, Ax) : 0.0;
        e = k == 0 ? m : m + c * e / p;
        p = e + cu;
        const double iv = 1.0 / p;
        rinv[row0 + k] = iv;
        fb[row0 + k] = c * iv;
        fc[row0 + k] = cu * iv;
    }
}

// One relaxation pass (eq. BlockJacobi) in FP64 with one warp per column, for
// levels whose passes are latency-bound (few columns per colour).  Lane l holds the
// R consecutive rows l R .. l R + R - 1 (n_r <= 32 R); each Thomas recurrence,
// y_k = t_k + fb_k y_{k-1} and then x_k = y_k + fc_k x_{k+1}, is the lane's own
// recurrence over its rows, one warp-shuffle scan of the lanes' composite affine
// maps, and a fix-up of each row by its prefix product and the carry from the
// neighbouring lane: 5 + 2 + 10/R FP64 operations a row forward and 2 + 8/R back,
// with a dependent chain of R + 6 steps each way (no shared memory, no barrier).
// The right-hand side is formed exactly as in k_relax (HF: the horizontal
// couplings of the stencil stored per unknown, TPMG^full).
template <int MODE, int R, bool HF>
__global__ void __launch_bounds__(256)
    k_relax_scan(OpView o, const int *__restrict__ cells, const int4 *__restrict__ tnb, const dbl4 *__restrict__ tg,
                 const double *__restrict__ rinv, const double *__restrict__ fb, const double *__restrict__ fcf,
                 int slot0, int n_slots, const double *__restrict__ f, const double *u_in, double *u_out,
                 double *__restrict__ u_fine, double relax)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    // the column's cell, neighbours and couplings are set-up data: read before the wait
    const int T = w < n_slots ? __ldg(&cells[slot0 + w]) : -1;
    const int4 nb = MODE == PASS_RHS_ONLY || T < 0 ? make_int4(0, 0, 0, 0) : __ldg(&tnb[slot0 + w]);
    const dbl4 g = (MODE == PASS_RHS_ONLY || HF || T < 0) ? dbl4{0.0, 0.0, 0.0, 0.0} : tg[slot0 + w];
    pdl_wait();
    pdl_trigger();
    if (T < 0) return;
    const int n_r = o.n_r;
    const bool n0 = MODE == PASS_NORMAL || (nb.w & 1), n1 = MODE == PASS_NORMAL || (nb.w & 2),
               n2 = MODE == PASS_NORMAL || (nb.w & 4);
    const size_t base = (size_t)T * n_r;
    const int k0 = lane * R;   // this lane's rows k0 .. k0 + R - 1
    // forward, y_k = t_k + b_k y_{k-1}: the lane's own recurrence Y_j from y = 0 before its
    // first row, with the prefix products P_j = b_{k0} ... b_{k0+j}; rows past the column
    // are the identity map (b = 1, t = 0)
    // the backward recurrence's coefficients, loaded with the forward ones so that a pass
    // has one round trip to memory on its critical path
    double cf[R];
#pragma unroll
    for (int j = 0; j < R; ++j) cf[j] = k0 + j < n_r ? __ldg(&fcf[base + k0 + j]) : 0.0;
    double y[R], P[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int k = k0 + j;
        double t = 0.0, b = 1.0;
        if (k < n_r) {
            const size_t i = base + k;
            double d = f[i];
            if (MODE != PASS_RHS_ONLY) {
                const double v0 = n0 ? u_in[(size_t)nb.x * n_r + k] : 0.0;
                const double v1 = n1 ? u_in[(size_t)nb.y * n_r + k] : 0.0;
                const double v2 = n2 ? u_in[(size_t)nb.z * n_r + k] : 0.0;
                if (HF) {
                    const dbl4 c = o.c[i];
                    d = fma(c.z, v2, fma(c.y, v1, fma(c.x, v0, d)));
                } else {
                    d = fma(__ldg(&o.hr[k]), fma(g.z, v2, fma(g.y, v1, g.x * v0)), d);
                }
            }
            t = d * __ldg(&rinv[i]);
            b = __ldg(&fb[i]);
        }
        y[j] = j == 0 ? t : fma(b, y[j - 1], t);
        P[j] = j == 0 ? b : P[j - 1] * b;
    }
    {   // inclusive scan of the lanes' maps y -> P y + Y; the carry into lane l is lane l-1's
        double A = P[R - 1], B = y[R - 1];
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const double Ap = __shfl_up_sync(full, A, s), Bp = __shfl_up_sync(full, B, s);
            if (lane >= s) {
                B = fma(A, Bp, B);
                A *= Ap;
            }
        }
        double cin = __shfl_up_sync(full, B, 1);
        if (lane == 0) cin = 0.0;
#pragma unroll
        for (int j = 0; j < R; ++j) y[j] = fma(P[j], cin, y[j]);
    }
    // backward, x_k = y_k + c_k x_{k+1}: the lane's own recurrence X_j from x = 0 after its
    // last row, with the suffix products Q_j = c_{k0+j} ... c_{k0+R-1}; rows past the
    // column take c = 0 (the column's last row has c = 0 anyway)
    double Q[R];
#pragma unroll
    for (int j = R - 1; j >= 0; --j) {
        const int k = k0 + j;
        const double c = cf[j];
        if (k >= n_r) y[j] = 0.0;
        if (j < R - 1) y[j] = fma(c, y[j + 1], y[j]);
        Q[j] = j == R - 1 ? c : c * Q[j + 1];
    }
    {   // inclusive suffix scan of the maps x -> Q x + X; the carry into lane l is lane l+1's
        double A = Q[0], B = y[0];
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const double Ad = __shfl_down_sync(full, A, s), Bd = __shfl_down_sync(full, B, s);
            if (lane + s < 32) {
                B = fma(A, Bd, B);
                A *= Ad;
            }
        }
        double cin = __shfl_down_sync(full, B, 1);
        if (lane == 31) cin = 0.0;
#pragma unroll
        for (int j = 0; j < R; ++j) y[j] = fma(Q[j], cin, y[j]);
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int k = k0 + j;
        if (k >= n_r) continue;
        const size_t i = base + k;
        double v = y[j];
        if (relax != 1.0) {   // from a zero guess (ZERO, RHS_ONLY) the old value is 0
            const double uo = MODE == PASS_NORMAL ? u_in[i] : 0.0;
            v = fma(relax, v - uo, uo);
        }
        u_out[i] = v;
        if (u_fine) {
            const size_t fi = (size_t)4 * T * n_r + k;
#pragma unroll
            for (int h = 0; h < 4; ++h) u_fine[fi + (size_t)h * n_r] += v;
        }
    }
}

template <int MODE, bool STAGE, int NT, int SK>
__global__ void __launch_bounds__(NT, STAGE ? 1 : 6)
    k_relax(OpView o, const int *__restrict__ cells, const int4 *__restrict__ tnb, const dbl4 *__restrict__ tg,
            const double *__restrict__ rinv, const double *__restrict__ fb, const double *__restrict__ fcf,
            const double *__restrict__ fm, int S, int j, int task0, const double *__restrict__ f, const double *u_in,
            double *u_out, double *__restrict__ u_fine, double relax, const double *__restrict__ csc, size_t plane,
            double *__restrict__ ft_out)
{
    extern __shared__ double smem[];
    __shared__ int s_cell[kRelaxCols];
    __shared__ int4 s_nb[kRelaxCols];
    __shared__ dbl4 s_g[kRelaxCols];
    __shared__ double s_m[2 * kRelaxCols];
    const int t = task0 + blockIdx.x;
    const int n_r = o.n_r, ld = n_r + 1, ne = kRelaxCols * n_r;
    double *tile = smem;
    double *sf = smem + ((kRelaxCols * ld + 1) & ~1);   // staged multipliers, 16-byte aligned
    const size_t fbase = (size_t)t * S * 32;
    if (STAGE) {
        const int chunks = S * 16;   // 16-byte chunks per multiplier block
        for (int q = threadIdx.x; q < 2 * chunks; q += NT) {
            const int a = q >= chunks, r = q - a * chunks;
            cp_async16(sf + (size_t)a * S * 32 + 2 * r, (a ? fcf : fb) + fbase + 2 * r);
        }
    }
    if (threadIdx.x < kRelaxCols) {
        const int q = t * kRelaxCols + threadIdx.x;
        s_cell[threadIdx.x] = __ldg(&cells[q]);
        s_nb[threadIdx.x] = __ldg(&tnb[q]);
        s_g[threadIdx.x] = tg[q];
    } else if (threadIdx.x < 3 * kRelaxCols) {
        const int q = threadIdx.x - kRelaxCols;
        s_m[q] = __ldg(&fm[(size_t)t * 2 * kRelaxCols + q]);
    }
    // everything above is set-up data; f and u come from earlier launches
    pdl_wait();
    pdl_trigger();
    __syncthreads();
    // elements per thread with loads in flight (fewer with couplings per unknown,
    // whose rows take registers of their own)
    constexpr int U = SK != SK_FAC ? (STAGE ? 4 : 2) : (STAGE ? 8 : 4);
    gather_rhs<MODE, SK, U, NT>(o, s_cell, s_nb, s_g, rinv, csc, plane, f, u_in, ft_out, tile, threadIdx.x);
    if (STAGE) cp_async_wait_all();
    __syncthreads();
    if ((threadIdx.x >> 5) == (int)(blockIdx.x % (NT / 32))) {
        const int lane = threadIdx.x & 31;
        const double *B = STAGE ? sf + lane : fb + fbase + lane;
        const double *C = STAGE ? sf + (size_t)S * 32 + lane : fcf + fbase + lane;
        twisted_solve<STAGE ? 8 : 4>(B, C, s_m, tile + (lane & (kRelaxCols - 1)) * ld, n_r, j, lane);
    }
    __syncthreads();
    constexpr int W = STAGE ? 4 : 2;
    for (int e0 = threadIdx.x; e0 < ne; e0 += NT * W) {
        double x[W], uo[W], uf[W][4];
        int idx[W], fi[W];
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const int e = e0 + NT * q;
            idx[q] = -1;
            if (e >= ne) continue;
            const int c = e / n_r, k = e - c * n_r;
            const int T = s_cell[c];
            if (T < 0) continue;
            idx[q] = T * n_r + k;
            fi[q] = 4 * T * n_r + k;
            x[q] = tile[c * ld + k];
            uo[q] = (MODE == PASS_NORMAL && relax != 1.0) ? u_in[idx[q]] : 0.0;
            if (u_fine) {
#pragma unroll
                for (int h = 0; h < 4; ++h) uf[q][h] = u_fine[fi[q] + h * n_r];
            }
        }
#pragma unroll
        for (int q = 0; q < W; ++q) {
            if (idx[q] < 0) continue;
            double v = x[q];
            if (relax != 1.0) v = fma(relax, v - uo[q], uo[q]);
            u_out[idx[q]] = v;
            if (u_fine) {
#pragma unroll
                for (int h = 0; h < 4; ++h) u_fine[fi[q] + h * n_r] = uf[q][h] + v;
            }
        }
    }
}

// The same relaxation pass with one warp per task and no block barriers, for
// passes with many tasks: each warp gathers, solves and writes back its own
// 16 columns, so the serial phases of the tasks resident on an SM overlap
// with the gather and write-back phases of others and keep its four FP64
// units busy.  One warp per CTA spreads the tasks evenly over the SMs and
// their sub-partitions.  DEEP: 6 elements per lane in flight in the gather
// instead of 4 -- fewer rounds of load latency, which bound a warp's gather --
// for more registers per warp.
// Registers are capped (without DEEP: 20 resident one-warp CTAs per SM, 5 warps per
// sub-partition, at most 96 registers) so that
// a finest-level pass of up to 3040 tasks fits in one wave: with 102 registers the first sweep's
// ZERO pass held 4 warps per SM sub-partition instead of 5 and ran its last 105 tasks as a
// second wave (73 us against 44 us for a NORMAL pass).
template <int MODE, int SK, bool DEEP>
__global__ void __launch_bounds__(32, DEEP ? 16 : 20)
    k_relax_warp(OpView o, const int *__restrict__ cells, const int4 *__restrict__ tnb, const dbl4 *__restrict__ tg,
                 const double *__restrict__ rinv, const double *__restrict__ fb, const double *__restrict__ fcf,
                 const double *__restrict__ fm, int S, int j, int task0, const double *__restrict__ f,
                 const double *u_in, double *u_out, double *__restrict__ u_fine, double relax,
                 const double *__restrict__ csc, size_t plane, double *__restrict__ ft_out)
{
    extern __shared__ double tile[];
    __shared__ int s_cell[kRelaxCols];
    __shared__ int4 s_nb[kRelaxCols];
    __shared__ dbl4 s_g[kRelaxCols];
    __shared__ double s_m[2 * kRelaxCols];
    const int t = task0 + blockIdx.x, lane = threadIdx.x;
    const int n_r = o.n_r, ld = n_r + 1, ne = kRelaxCols * n_r;
    s_m[lane] = __ldg(&fm[(size_t)t * 2 * kRelaxCols + lane]);
    if (lane < kRelaxCols) {
        const int q = t * kRelaxCols + lane;
        s_cell[lane] = __ldg(&cells[q]);
        s_nb[lane] = __ldg(&tnb[q]);
        s_g[lane] = tg[q];
    }
    pdl_wait();
    pdl_trigger();
    __syncwarp();
    constexpr int U = DEEP ? 6 : 4;
    gather_rhs<MODE, SK, U, 32>(o, s_cell, s_nb, s_g, rinv, csc, plane, f, u_in, ft_out, tile, lane);
    __syncwarp();
    const size_t fbase = (size_t)t * S * 32 + lane;
    twisted_solve<4>(fb + fbase, fcf + fbase, s_m, tile + (lane & (kRelaxCols - 1)) * ld, n_r, j, lane);
    __syncwarp();
    constexpr int W = 2;
    for (int e0 = lane; e0 < ne; e0 += 32 * W) {
        double x[W], uo[W], uf[W][4];
        int idx[W], fi[W];
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const int e = e0 + 32 * q;
            idx[q] = -1;
            if (e >= ne) continue;
            const int c = e / n_r, k = e - c * n_r;
            const int T = s_cell[c];
            if (T < 0) continue;
            idx[q] = T * n_r + k;
            fi[q] = 4 * T * n_r + k;
            x[q] = tile[c * ld + k];
            uo[q] = (MODE == PASS_NORMAL && relax != 1.0) ? u_in[idx[q]] : 0.0;
            if (u_fine) {
#pragma unroll
                for (int h = 0; h < 4; ++h) uf[q][h] = u_fine[fi[q] + h * n_r];
            }
        }
#pragma unroll
        for (int q = 0; q < W; ++q) {
            if (idx[q] < 0) continue;
            double v = x[q];
            if (relax != 1.0) v = fma(relax, v - uo[q], uo[q]);
            u_out[idx[q]] = v;
            if (u_fine) {
#pragma unroll
                for (int h = 0; h < 4; ++h) u_fine[fi[q] + h * n_r] = uf[q][h] + v;
            }
        }
    }
}

// The vector kernels below are HBM-bound: each thread keeps the loads of 4
// grid-stride iterations in flight, and the grid holds 8 blocks per SM.

// partial <a, b>
template <int NT>
__device__ __forceinline__ void dot_body(const double *__restrict__ a, const double *__restrict__ b, int N,
                                         double *__restrict__ partials, int bid, int nblk)
{
    double acc = 0.0;
    const int stride = nblk * NT;
    int i = bid * NT + threadIdx.x;
    for (; i + 3 * stride < N; i += 4 * stride) {
        double x[4], y[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { x[q] = a[i + q * stride]; y[q] = b[i + q * stride]; }
#pragma unroll
        for (int q = 0; q < 4; ++q) acc = fma(x[q], y[q], acc);
    }
    for (; i < N; i += stride) acc = fma(a[i], b[i], acc);
    acc = block_sum<NT>(acc);
    if (threadIdx.x == 0) partials[bid] = acc;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_dot(const double *__restrict__ a, const double *__restrict__ b, int N,
                                            double *__restrict__ partials)
{
    pdl_wait();
    pdl_trigger();
    dot_body<NT>(a, b, N, partials, blockIdx.x, gridDim.x);
}

// u += alpha p; r -= alpha q; partial ||r||^2.  With z_old (flexible CG) also
// the partial <r_new, z_old> of the Polak-Ribiere coefficient, in partials[gridDim.x + block].
template <int NT, bool CROSS, bool R32>
__device__ __forceinline__ void axpy_pair_body(const Scalars *__restrict__ sc, const double *__restrict__ p,
                                               const double *__restrict__ q, double *__restrict__ u,
                                               double *__restrict__ r, int N, double *__restrict__ partials,
                                               const double *__restrict__ z_old, int bid, int nblk,
                                               float *__restrict__ r32)
{
    const double alpha = sc->alpha;
    double acc = 0.0, accz = 0.0;
    const int stride = nblk * NT;
    int i = bid * NT + threadIdx.x;
    for (; i + 3 * stride < N; i += 4 * stride) {
        double pv[4], qv[4], uv[4], rv[4], zv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = i + k * stride;
            pv[k] = p[j]; qv[k] = q[j]; uv[k] = u[j]; rv[k] = r[j];
            if (CROSS) zv[k] = z_old[j];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = i + k * stride;
            u[j] = fma(alpha, pv[k], uv[k]);
            const double x = fma(-alpha, qv[k], rv[k]);
            r[j] = x;
            if (R32) r32[j] = (float)x;
            acc = fma(x, x, acc);
            if (CROSS) accz = fma(x, zv[k], accz);
        }
    }
    for (; i < N; i += stride) {
        u[i] = fma(alpha, p[i], u[i]);
        const double x = fma(-alpha, q[i], r[i]);
        r[i] = x;
        if (R32) r32[i] = (float)x;
        acc = fma(x, x, acc);
        if (CROSS) accz = fma(x, z_old[i], accz);
    }
    acc = block_sum<NT>(acc);
    if (threadIdx.x == 0) partials[bid] = acc;
    if (CROSS) {
        __syncthreads();   // block_sum's shared scratch is reused
        accz = block_sum<NT>(accz);
        if (threadIdx.x == 0) partials[nblk + bid] = accz;
    }
}

template <int NT, bool CROSS, bool R32>
__global__ void __launch_bounds__(NT) k_axpy_pair(const Scalars *__restrict__ sc, const double *__restrict__ p,
                                                  const double *__restrict__ q, double *__restrict__ u,
                                                  double *__restrict__ r, int N, double *__restrict__ partials,
                                                  const double *__restrict__ z_old, float *__restrict__ r32)
{
    pdl_wait();
    pdl_trigger();
    axpy_pair_body<NT, CROSS, R32>(sc, p, q, u, r, N, partials, z_old, blockIdx.x, gridDim.x, r32);
}

// p = z + beta p
template <int NT>
__device__ __forceinline__ void xpby_body(const Scalars *__restrict__ sc, const double *__restrict__ z,
                                          double *__restrict__ p, int N, int bid, int nblk)
{
    const double beta = sc->beta;
    const int stride = nblk * NT;
    int i = bid * NT + threadIdx.x;
    for (; i + 3 * stride < N; i += 4 * stride) {
        double zv[4], pv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) { zv[k] = z[i + k * stride]; pv[k] = p[i + k * stride]; }
#pragma unroll
        for (int k = 0; k < 4; ++k) p[i + k * stride] = fma(beta, pv[k], zv[k]);
    }
    for (; i < N; i += stride) p[i] = fma(beta, p[i], z[i]);
}

template <int NT>
__global__ void __launch_bounds__(NT) k_xpby(const Scalars *__restrict__ sc, const double *__restrict__ z,
                                             double *__restrict__ p, int N)
{
    pdl_wait();
    pdl_trigger();
    xpby_body<NT>(sc, z, p, N, blockIdx.x, gridDim.x);
}

// The decision of a device-side loop: the loop's conditional handle, or, for a member
// of a batched solve (loop.go set), the member's flag, which the batch's loop reads.
__device__ __forceinline__ void set_loop(const LoopCtl &loop, bool go)
{
    if (loop.go)
        *loop.go = go ? 1 : 0;
    else
        cudaGraphSetConditional(loop.cond, go ? 1u : 0u);
}

// Deterministic reduction of the block partials (fixed order) and the PCG scalar step.
__device__ __forceinline__ void finish_body(int what, const double *__restrict__ partials, int n, Scalars *sc,
                                            const LoopCtl &loop)
{
    double v = 0.0, v2 = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) v += partials[i];
    v = block_sum<256>(v);
    if (what == FIN_LOOP_RR0F || what == FIN_RR0F) {   // second set of partials: ||f||^2
        for (int i = threadIdx.x; i < n; i += 256) v2 += partials[n + i];
        __syncthreads();
        v2 = block_sum<256>(v2);
    }
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
    case FIN_RZC:
        sc->rzc = v;
        break;
    case FIN_SUM:
        sc->sum = v;
        break;
    case FIN_BETA_PR:   // flexible CG: beta = (<r, z_new> - <r, z_old>) / <r_old, z_old>
        sc->rz_new = v;
        sc->beta = (v - sc->rzc) / sc->rz;
        sc->rz = v;
        if (!isfinite(v)) sc->flag |= 2;
        break;
    case FIN_LOOP_RR0: {
        sc->rr0 = v;
        sc->rr = v;
        sc->it = 0;
        sc->flag = isfinite(v) ? 0 : 2;
        if (loop.hist) loop.hist[0] = 1.0;
        set_loop(loop, isfinite(v) && v > 0.0 && loop.max_iter > 0);
        break;
    }
    case FIN_RR0F:
    case FIN_LOOP_RR0F: {
        // judge of the initial guess: kept only if its residual is below that of u = 0
        const bool keep = v < v2;
        const double rr = keep ? v : v2;
        sc->ff = v2;
        sc->info = keep ? 1 : 2;
        sc->rr0 = v2;
        sc->rr = rr;
        sc->it = 0;
        sc->flag = isfinite(rr) ? 0 : 2;
        const double rel = v2 > 0.0 ? sqrt(rr / v2) : 0.0;
        if (what == FIN_LOOP_RR0F) {
            if (loop.hist) loop.hist[0] = rel;
            set_loop(loop, isfinite(rr) && rr > 0.0 && !(rel <= loop.rtol) && loop.max_iter > 0);
        }
        break;
    }
    case FIN_LOOP_BETA:
    case FIN_LOOP_BETA_PR:
        sc->rz_new = v;
        sc->beta = sc->it == 0 ? 0.0 : (what == FIN_LOOP_BETA ? v : v - sc->rzc) / sc->rz;
        sc->rz = v;
        if (!isfinite(v)) sc->flag |= 2;
        break;
    case FIN_LOOP_RR: {
        sc->rr = v;
        const int it = ++sc->it;
        if (!isfinite(v)) sc->flag |= 2;
        const double rel = sqrt(v / sc->rr0);
        if (loop.hist) loop.hist[it] = rel;
        const bool go = sc->flag == 0 && !(rel <= loop.rtol) && it < loop.max_iter;
        set_loop(loop, go);
        break;
    }
    default:
        break;
    }
}

__global__ void __launch_bounds__(256) k_finish(int what, const double *__restrict__ partials, int n, Scalars *sc,
                                                LoopCtl loop)
{
    pdl_wait();
    pdl_trigger();
    finish_body(what, partials, n, sc, loop);
}

// ---- batched form: the outer FP64 kernels over the members of a batch -----------
__device__ __forceinline__ OpView batch_view(const BatchMemberDev &m)
{
    return OpView{m.nbr,   m.g,     m.area,  m.area_r, m.vol,   m.w,   m.hr,  m.n_r, nullptr,
                  nullptr, nullptr, nullptr, nullptr,  nullptr, nullptr, m.om, m.oc, m.ocs};
}

// Member m's block b of n_part is virtual block m n_part + b; each CTA runs virtual
// blocks blockIdx.x, blockIdx.x + gridDim.x, ... with the body of the member's own
// kernel, so every member gets the partition (and the partial sums) of its own solve.
template <int NT, int WHAT>
__global__ void __launch_bounds__(NT) k_outer_batch(const BatchMemberDev *__restrict__ mem, int M, int n_part,
                                                    const int *__restrict__ active)
{
    pdl_wait();
    pdl_trigger();
    const int nv = M * n_part;
    for (int vb = blockIdx.x; vb < nv; vb += gridDim.x) {
        const int m = vb / n_part, b = vb - m * n_part;
        if (!active[m]) continue;   // the same for every thread of the block
        const BatchMemberDev &x = mem[m];
        if (WHAT == BATCH_NONZERO) nonzero_body<NT>(x.u, x.N, x.zflags, b, n_part);
        if (WHAT == BATCH_RESIDUAL)
            residual_body<NT, false, false, true>(batch_view(x), FullView{}, x.f, x.u, x.r, x.N, x.partials, x.zflags, n_part,
                                            b, n_part, x.r32);
        if (WHAT == BATCH_DOT_RZ) dot_body<NT>(x.r, x.z, x.N, x.partials, b, n_part);
        if (WHAT == BATCH_XPBY) xpby_body<NT>(x.sc, x.z, x.p, x.N, b, n_part);
        if (WHAT == BATCH_APPLY)
            apply_body<NT, false, false>(batch_view(x), FullView{}, x.p, x.q, x.N, x.partials, b, n_part);
        if (WHAT == BATCH_AXPY)
            axpy_pair_body<NT, true, true>(x.sc, x.p, x.q, x.u, x.r, x.N, x.partials, x.z, b, n_part, x.r32);
        if (WHAT == BATCH_CLEAR_P)
            for (int i = b * NT + threadIdx.x; i < x.N; i += n_part * NT) x.p[i] = 0.0;
        __syncthreads();   // the next virtual block reuses block_sum's shared scratch
    }
}

// The members' finishes, one block each: member m's k_finish with its loop decision
// written to go[m] (active members only).
__global__ void __launch_bounds__(256) k_finish_batch(int what, const BatchMemberDev *__restrict__ mem, int n_part,
                                                      int offset, const int *__restrict__ active, int *go)
{
    pdl_wait();
    pdl_trigger();
    const int m = blockIdx.x;
    if (!active[m]) return;
    const BatchMemberDev &x = mem[m];
    LoopCtl loop{0, x.rtol, x.max_iter, x.hist};
    loop.go = go + m;
    finish_body(what, x.partials + offset, n_part, x.sc, loop);
}

// The end of a batched iteration: the members whose finish decided to go on stay
// active; the batch's loop continues while any member is active.
__global__ void __launch_bounds__(256) k_batch_continue(int M, const int *__restrict__ go, int *active,
                                                        cudaGraphConditionalHandle cond)
{
    pdl_wait();
    pdl_trigger();
    int any = 0;
    for (int m = threadIdx.x; m < M; m += 256) {
        const int g = go[m];
        active[m] = g;
        any |= g;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) cudaGraphSetConditional(cond, any ? 1u : 0u);
}

__global__ void __launch_bounds__(256) k_lincomb(long n, double a, const double *x, double b, const double *y,
                                                 double c, const double *z, double *out)
{
    pdl_wait();
    pdl_trigger();
    for (long i = blockIdx.x * 256L + threadIdx.x; i < n; i += (long)gridDim.x * 256) {
        double v = a * x[i];
        if (y) v = fma(b, y[i], v);
        if (z) v = fma(c, z[i], v);
        out[i] = v;
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

}  // namespace

cudaError_t launch_apply(const Launch &L, const LevelDev &lv, const VertDev &v, const double *x, double *y,
                         double *partials, int n_part)
{
    const int N = lv.n * L.n_r;
    const int grid = partials ? n_part : grid_for(N, kThreads, L.sm_count);
    const FullView fv{lv.cfull, lv.cvr, lv.cvx};
    // ADV: the factorised operator with vertical advection (compiled out without it)
    auto kern = lv.cfull ? k_apply<kThreads, true, false>
                         : (lv.area_x ? k_apply<kThreads, false, true> : k_apply<kThreads, false, false>);
    return launch_k(L, kern, grid, kThreads, 0, make_view(lv, v, L.n_r), fv, x, y, N, partials);
}

cudaError_t launch_nonzero(const Launch &L, long n, const double *x, int *nz, int n_blocks)
{
    return launch_k(L, k_nonzero<kThreads>, n_blocks, kThreads, 0, x, (int)n, nz);
}

cudaError_t launch_residual(const Launch &L, const LevelDev &lv, const VertDev &v, const double *f, const double *u,
                            double *r, double *partials, int n_part, const int *nz, float *r32)
{
    const int N = lv.n * L.n_r;
    const int grid = partials ? n_part : grid_for(N, kThreads, L.sm_count);
    const FullView fv{lv.cfull, lv.cvr, lv.cvx};
    auto kern = r32 ? (lv.cfull ? k_residual<kThreads, true, false, true>
                                : (lv.area_x ? k_residual<kThreads, false, true, true>
                                             : k_residual<kThreads, false, false, true>))
                    : (lv.cfull ? k_residual<kThreads, true, false, false>
                                : (lv.area_x ? k_residual<kThreads, false, true, false>
                                             : k_residual<kThreads, false, false, false>));
    return launch_k(L, kern, grid, kThreads, 0, make_view(lv, v, L.n_r), fv, f, u, r, N, partials, nz,
                    nz ? n_part : 0, r32);
}

cudaError_t launch_resid_restrict(const Launch &L, const LevelDev &fine, const LevelDev &coarse, const VertDev &v,
                                  const double *f, const double *u, double *fc)
{
    const int Nc = coarse.n * L.n_r, grid = grid_for(Nc, kThreads, L.sm_count);
    if (fine.rgeo && stencil_form(fine) == CM_FAC && !fine.area_x)
        return launch_k(L, k_restrict_fac<kThreads>, grid, kThreads, 0, (const RestrictGeo *)fine.rgeo, v.vol, v.w, v.hr,
                        f, u, fc, L.n_r, Nc);    const OpView o = make_view(fine, v, L.n_r);
    void (*kern)(OpView, const double *, const double *, double *, int);
    switch (stencil_form(fine)) {
    case CM_FULL: kern = k_resid_restrict<kThreads, CM_FULL, false>; break;
    case CM_PARTIAL:
        kern = fine.area_x ? k_resid_restrict<kThreads, CM_PARTIAL, true> : k_resid_restrict<kThreads, CM_PARTIAL, false>;
        break;
    default: kern = fine.area_x ? k_resid_restrict<kThreads, CM_FAC, true> : k_resid_restrict<kThreads, CM_FAC, false>;
    }
    return launch_k(L, kern, grid, kThreads, 0, o, f, u, fc, Nc);
}

cudaError_t launch_prolong_add(const Launch &L, const LevelDev &fine, const double *uc, double *u)
{
    const int N = fine.n * L.n_r;
    return launch_k(L, k_prolong_add<kThreads>, grid_for(N, kThreads, L.sm_count), kThreads, 0, uc, u, L.n_r, N);
}

cudaError_t launch_prolong_linear(const Launch &L, const LevelDev &fine, const LevelDev &coarse, const double *uc,
                                  double *u)
{
    const int N = fine.n * L.n_r;
    return launch_k(L, k_prolong_linear<kThreads>, grid_for(N, kThreads, L.sm_count), kThreads, 0, coarse.nbr,
                    coarse.plin, uc, u, L.n_r, N);
}

cudaError_t launch_outer_products(const Launch &L, const LevelDev &lv, const VertDev &v)
{
    const int N = lv.n * L.n_r;
    k_outer_products<<<grid_for(N, 256, L.sm_count), 256, 0, L.s>>>(make_view(lv, v, L.n_r), N, lv.om, lv.oc, lv.ocs);
    return cudaGetLastError();
}

cudaError_t launch_twisted_factors(const Launch &L, const LevelDev &lv, const VertDev &v)
{
    const int n = lv.n_tasks * kRelaxCols;
    k_twisted_factors<<<(n + 127) / 128, 128, 0, L.s>>>(lv.n_tasks, make_view(lv, v, L.n_r), lv.task_cells, lv.steps,
                                                         lv.jmid, lv.rinv, lv.fb, lv.fc, lv.fm);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && lv.cs) e = launch_scaled_couplings(L, lv, v);
    return e;
}

cudaError_t launch_scaled_couplings(const Launch &L, const LevelDev &lv, const VertDev &v)
{
    if (!lv.cs) return cudaSuccess;
    const long nn = (long)lv.n * L.n_r;
    k_scaled_couplings<<<grid_for(nn, 256, L.sm_count), 256, 0, L.s>>>(make_view(lv, v, L.n_r), nn, lv.rinv, lv.cs);
    return cudaGetLastError();
}

template <int MODE, bool STAGE, int NT, int SK>
static cudaError_t relax_launch_t(const Launch &L, const LevelDev &lv, const VertDev &v, int task0, int n_tasks,
                                  double relax, const double *f, const double *u_in, double *u_out, double *u_fine,
                                  size_t smem)
{
    auto kern = k_relax<MODE, STAGE, NT, SK>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_k(L, kern, n_tasks, NT, smem, make_view(lv, v, L.n_r), lv.task_cells, lv.task_nbr, lv.task_g,
                    lv.rinv, lv.fb, lv.fc, lv.fm, lv.steps, lv.jmid, task0, f, u_in, u_out, u_fine, relax,
                    (const double *)lv.cs, (size_t)lv.n * L.n_r, SK == SK_SCALED_FIRST ? lv.ft : (double *)nullptr);
}

// Kernel choice (RELAX_*): the level's autotuned variant, or without one the
// heuristic -- more tasks than one wave of CTAs holds (8 per SM) and a tile of
// at most 32 KB -> one warp per task, otherwise one 128-thread CTA per task.
// CTA variants stage the multipliers in shared memory by cp.async when they
// fit; a column too tall for that runs unstaged with 128 threads.
template <int MODE, int R, bool HF>
static cudaError_t relax_scan_r(const Launch &L, const LevelDev &lv, const VertDev &v, int var, int task0, int n_tasks,
                                double relax, const double *f, const double *u_in, double *u_out, double *u_fine)
{
    const int wpb = 1 << var;   // CTAs of 1, 2, 4 or 8 warps: the autotuner's variants, same arithmetic
    const int n_slots = n_tasks * kRelaxCols;
    return launch_k(L, k_relax_scan<MODE, R, HF>, (n_slots + wpb - 1) / wpb, 32 * wpb, 0, make_view(lv, v, L.n_r),
                    lv.task_cells, lv.task_nbr, lv.task_g, lv.rinv1, lv.fb1, lv.fc1, task0 * kRelaxCols, n_slots, f,
                    u_in, u_out, u_fine, relax);
}

template <int MODE, bool HF>
static cudaError_t relax_scan(const Launch &L, const LevelDev &lv, const VertDev &v, int var, int task0, int n_tasks,
                              double relax, const double *f, const double *u_in, double *u_out, double *u_fine)
{
    const int n = L.n_r;
    if (n <= 32) return relax_scan_r<MODE, 1, HF>(L, lv, v, var, task0, n_tasks, relax, f, u_in, u_out, u_fine);
    if (n <= 64) return relax_scan_r<MODE, 2, HF>(L, lv, v, var, task0, n_tasks, relax, f, u_in, u_out, u_fine);
    if (n <= 128) return relax_scan_r<MODE, 4, HF>(L, lv, v, var, task0, n_tasks, relax, f, u_in, u_out, u_fine);
    if (n <= 256) return relax_scan_r<MODE, 8, HF>(L, lv, v, var, task0, n_tasks, relax, f, u_in, u_out, u_fine);
    if (n <= 512) return relax_scan_r<MODE, 16, HF>(L, lv, v, var, task0, n_tasks, relax, f, u_in, u_out, u_fine);
    return relax_scan_r<MODE, 32, HF>(L, lv, v, var, task0, n_tasks, relax, f, u_in, u_out, u_fine);
}

template <int MODE, int SK>
static cudaError_t relax_launch_sk(const Launch &L0, const LevelDev &lv, const VertDev &v, int task0, int n_tasks,
                                   double relax, const double *f, const double *u_in, double *u_out, double *u_fine)
{
    constexpr bool HF = SK == SK_FULL;
    if (lv.scan) {   // CTAs of 1, 2, 4 or 8 warps (variants 0..3; the deep-pipeline variant 4 is for tasks)
        const int var = (lv.relax_variant < 0 || lv.relax_variant > RELAX_CTA256) ? RELAX_CTA128 : lv.relax_variant;
        return relax_scan<MODE, HF>(L0, lv, v, var, task0, n_tasks, relax, f, u_in, u_out, u_fine);
    }
    // a small colour of a larger level: warp scans in CTAs of 4 warps (the level's tuned
    // variant is a twisted-task kernel's); they form their right-hand side from f
    if (n_tasks <= lv.scan_pass_tasks)
        return relax_scan<MODE, HF>(L0, lv, v, RELAX_CTA128, task0, n_tasks, relax, f, u_in, u_out, u_fine);
    // The twisted-task kernels are launched plainly: measured on GB300, programmatic
    // launch made the FP64 solves that use them 1-2% slower (refinement 6 x 64 and
    // 7 x 128), while it speeds up the scan, transfer and vector kernels.
    Launch L = L0;
    L.pdl = false;
    const double *rhs = SK == SK_SCALED ? lv.ft : f;   // the scaled form reads f / pivot
    const size_t tile = (((size_t)kRelaxCols * (L.n_r + 1) + 1) & ~(size_t)1) * sizeof(double);
    int var = lv.relax_variant;
    if (var < 0) var = (n_tasks >= 8 * L.sm_count && tile <= 32 * 1024) ? RELAX_WARP : RELAX_CTA128;
    if ((var == RELAX_WARP || var == RELAX_WARP_DEEP) && tile <= 32 * 1024) {
        auto kern = var == RELAX_WARP_DEEP ? k_relax_warp<MODE, SK, true> : k_relax_warp<MODE, SK, false>;
        return launch_k(L, kern, n_tasks, 32, tile, make_view(lv, v, L.n_r), lv.task_cells, lv.task_nbr, lv.task_g,
                        lv.rinv, lv.fb, lv.fc, lv.fm, lv.steps, lv.jmid, task0, rhs, u_in, u_out, u_fine, relax,
                        (const double *)lv.cs, (size_t)lv.n * L.n_r,
                        SK == SK_SCALED_FIRST ? lv.ft : (double *)nullptr);
    }
    const size_t staged = tile + (size_t)2 * lv.steps * 32 * sizeof(double);
    if (staged > 160 * 1024)
        return relax_launch_t<MODE, false, 128, SK>(L, lv, v, task0, n_tasks, relax, rhs, u_in, u_out, u_fine, tile);
    if (var == RELAX_CTA64)
        return relax_launch_t<MODE, true, 64, SK>(L, lv, v, task0, n_tasks, relax, rhs, u_in, u_out, u_fine, staged);
    if (var == RELAX_CTA256)
        return relax_launch_t<MODE, true, 256, SK>(L, lv, v, task0, n_tasks, relax, rhs, u_in, u_out, u_fine, staged);
    return relax_launch_t<MODE, true, 128, SK>(L, lv, v, task0, n_tasks, relax, rhs, u_in, u_out, u_fine, staged);
}

// The right-hand-side form of a pass: the stored stencil (TPMG^full) where the level
// has one; otherwise, with the level's scaled couplings, SK_SCALED_FIRST for the first
// pass over a colour in a visit of the level (ft_mode 1) and SK_SCALED after it
// (ft_mode 2); else the factorised couplings.
template <int MODE>
static cudaError_t relax_launch(const Launch &L, const LevelDev &lv, const VertDev &v, int task0, int n_tasks,
                                double relax, const double *f, const double *u_in, double *u_out, double *u_fine,
                                int ft_mode)
{
    if (n_tasks <= 0) return cudaSuccess;
    if (lv.vc) return relax_launch_sk<MODE, SK_FULL>(L, lv, v, task0, n_tasks, relax, f, u_in, u_out, u_fine);
    if (lv.cs && lv.ft && ft_mode == 1)
        return relax_launch_sk<MODE, SK_SCALED_FIRST>(L, lv, v, task0, n_tasks, relax, f, u_in, u_out, u_fine);
    if (lv.cs && lv.ft && ft_mode == 2)
        return relax_launch_sk<MODE, SK_SCALED>(L, lv, v, task0, n_tasks, relax, f, u_in, u_out, u_fine);
    return relax_launch_sk<MODE, SK_FAC>(L, lv, v, task0, n_tasks, relax, f, u_in, u_out, u_fine);
}

cudaError_t launch_thomas_factors(const Launch &L, const LevelDev &lv, const VertDev &v)
{
    k_thomas_factors<<<(lv.n + 127) / 128, 128, 0, L.s>>>(make_view(lv, v, L.n_r), lv.n, lv.rinv1, lv.fb1, lv.fc1);
    return cudaGetLastError();
}

cudaError_t launch_relax(const Launch &L, const LevelDev &lv, const VertDev &v, int mode, int task0, int n_tasks,
                         double relax, const double *f, const double *u_in, double *u_out, double *u_fine,
                         int ft_mode)
{
    switch (mode) {
    case PASS_ZERO: return relax_launch<PASS_ZERO>(L, lv, v, task0, n_tasks, relax, f, u_in, u_out, u_fine, ft_mode);
    case PASS_RHS_ONLY:
        return relax_launch<PASS_RHS_ONLY>(L, lv, v, task0, n_tasks, relax, f, u_in, u_out, u_fine, ft_mode);
    default: return relax_launch<PASS_NORMAL>(L, lv, v, task0, n_tasks, relax, f, u_in, u_out, u_fine, ft_mode);
    }
}

cudaError_t launch_dot(const Launch &L, long n, const double *a, const double *b, double *partials, int n_part)
{
    return launch_k(L, k_dot<kThreads>, n_part, kThreads, 0, a, b, (int)n, partials);
}

cudaError_t launch_finish(const Launch &L, int what, const double *partials, int n_part, Scalars *sc,
                          const LoopCtl *loop)
{
    return launch_k(L, k_finish, 1, 256, 0, what, partials, n_part, sc, loop ? *loop : LoopCtl{0, 0.0, 0, nullptr});
}

cudaError_t launch_axpy_pair(const Launch &L, long n, const Scalars *sc, const double *p, const double *q, double *u,
                             double *r, double *partials, int n_part, const double *z_old, float *r32)
{
    auto kern = r32 ? (z_old ? k_axpy_pair<kThreads, true, true> : k_axpy_pair<kThreads, false, true>)
                    : (z_old ? k_axpy_pair<kThreads, true, false> : k_axpy_pair<kThreads, false, false>);
    return launch_k(L, kern, n_part, kThreads, 0, sc, p,
                    q, u, r, (int)n, partials, z_old, r32);
}

cudaError_t launch_outer_batch(const Launch &L, int what, const BatchMemberDev *mem, int M, int n_part,
                               const int *active)
{
    if (M <= 0) return cudaSuccess;
    const int grid = 2 * 8 * L.sm_count;   // 2 x 8 CTAs per SM, each over M n_part / grid virtual blocks
    switch (what) {
    case BATCH_NONZERO: return launch_k(L, k_outer_batch<kThreads, BATCH_NONZERO>, grid, kThreads, 0, mem, M, n_part, active);
    case BATCH_RESIDUAL: return launch_k(L, k_outer_batch<kThreads, BATCH_RESIDUAL>, grid, kThreads, 0, mem, M, n_part, active);
    case BATCH_DOT_RZ: return launch_k(L, k_outer_batch<kThreads, BATCH_DOT_RZ>, grid, kThreads, 0, mem, M, n_part, active);
    case BATCH_XPBY: return launch_k(L, k_outer_batch<kThreads, BATCH_XPBY>, grid, kThreads, 0, mem, M, n_part, active);
    case BATCH_APPLY: return launch_k(L, k_outer_batch<kThreads, BATCH_APPLY>, grid, kThreads, 0, mem, M, n_part, active);
    case BATCH_AXPY: return launch_k(L, k_outer_batch<kThreads, BATCH_AXPY>, grid, kThreads, 0, mem, M, n_part, active);
    case BATCH_CLEAR_P: return launch_k(L, k_outer_batch<kThreads, BATCH_CLEAR_P>, grid, kThreads, 0, mem, M, n_part, active);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_finish_batch(const Launch &L, int what, const BatchMemberDev *mem, int M, int n_part,
                                const int *active, int *go, int partial_offset)
{
    if (M <= 0) return cudaSuccess;
    return launch_k(L, k_finish_batch, M, 256, 0, what, mem, n_part, partial_offset, active, go);
}

cudaError_t launch_batch_continue(const Launch &L, int M, const int *go, int *active, cudaGraphConditionalHandle cond)
{
    return launch_k(L, k_batch_continue, 1, 256, 0, M, go, active, cond);
}

cudaError_t launch_lincomb(const Launch &L, long n, double a, const double *x, double b, const double *y, double c,
                           const double *z, double *out)
{
    return launch_k(L, k_lincomb, grid_for(n, 256, L.sm_count), 256, 0, n, a, x, b, y, c, z, out);
}

cudaError_t launch_xpby(const Launch &L, long n, const Scalars *sc, const double *z, double *p)
{
    return launch_k(L, k_xpby<kThreads>, grid_for(n, kThreads, L.sm_count), kThreads, 0, sc, z, p, (int)n);
}

}  // namespace tpmg
