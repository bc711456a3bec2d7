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
// blocks' Thomas pivots are computed once per level in FP64 from those
// coefficients (excess-carried pivots) and their reciprocals stored per
// unknown in FP32; the two multipliers of a row are formed in the pass as the
// BF16 couplings times that reciprocal (stored as well only with vertical
// advection, whose couplings differ from alphar_hat).  The outer Krylov
// vectors stay in FP64: the finest level reads the outer residual in FP32 (a
// copy written by the kernel that forms it, or the FP64 vector itself) and
// writes its result as double.
#include <cuda_runtime.h>

#include "tpmg_internal.h"

namespace tpmg {

namespace {

constexpr int kThreads32 = 256;

__device__ __forceinline__ float bf(unsigned short h) { return __uint_as_float((unsigned)h << 16); }

// Thomas factors of the BF16 column blocks (set-up, one thread per column):
// the recurrence of the FP64 path (excess-carried pivots, reading C16)
// evaluated in FP64 on the BF16 coefficients -- diagonal excess
// m_k = beta_hat + sum_e alphaS_hat_e, couplings c_k = alphar_hat of face k
// (c_0 = c_{n} = 0) -- from the bottom row upwards:
//   e_0 = m_0,  e_k = m_k + c_k e_{k-1} / p_{k-1},  p_k = e_k + c_{k+1},
// stored per unknown in FP32: rinv = 1 / p_k, and, where fb / fg are given (vertical
// advection), b = c_k / p_k (b_0 = 0) and g = c_{k+1} / p_k, so that A_T x = d is
//   y_k = d_k rinv_k + b_k y_{k-1},   x_k = y_k + g_k x_{k+1}.
// Without advection the relaxation forms b = c_k rinv_k and g = c_{k+1} rinv_k
// itself from the BF16 couplings (exact in FP32).  With vertical advection (cxv: X
// of face k in BF16, dr the row thickness) row k couples downwards with
// c_k - dr_k X_k and upwards with c_{k+1} + dr_k X_{k+1}, in place of c_k and c_{k+1}.
__global__ void k_thomas_factors32(int n_cells, const bf16x4 *__restrict__ cpack,
                                   const unsigned short *__restrict__ cvert, const unsigned short *__restrict__ cxv,
                                   const double *__restrict__ dr, int n, float *__restrict__ rinv,
                                   float *__restrict__ fb, float *__restrict__ fg)
{
    const int T = blockIdx.x * blockDim.x + threadIdx.x;
    if (T >= n_cells) return;
    const size_t row0 = (size_t)T * n;
    auto m_of = [&](int k) {
        const bf16x4 c = cpack[row0 + k];
        return (double)bf(c.w) + (double)bf(c.x) + (double)bf(c.y) + (double)bf(c.z);
    };
    auto c_of = [&](int k) { return k > 0 && k < n ? (double)bf(cvert[row0 + k]) : 0.0; };
    auto x_of = [&](int k) { return cxv && k > 0 && k < n ? (double)bf(cxv[row0 + k]) : 0.0; };
    double e = 0.0, p = 1.0;
    for (int k = 0; k < n; ++k) {
        const double m = m_of(k);
        double c = c_of(k), cu = c_of(k + 1);
        if (cxv) {
            c -= dr[k] * x_of(k);
            cu += dr[k] * x_of(k + 1);
        }
        e = k == 0 ? m : m + c * e / p;
        p = e + cu;
        rinv[row0 + k] = (float)(1.0 / p);
        if (fb) fb[row0 + k] = (float)(c / p);
        if (fg) fg[row0 + k] = (float)(cu / p);
    }
}

// One relaxation pass (eq. BlockJacobi) in FP32 with one warp per column T:
//   u_T <- (1 - relax) u_T + relax A_T^{-1} (f_T + sum_e alphaS_hat_e u_{T_e}).
// The Thomas algorithm's two first-order recurrences (factors of
// k_thomas_factors32),
//   y_k = t_k + b_k y_{k-1},  t_k = d_k / p_k,     x_k = y_k + g_k x_{k+1},
// are solved with parallel scans of the affine maps y -> b y + t over the
// lanes (Kogge-Stone, 5 shuffle rounds), in one of two row layouts (R =
// ceil(n_r / 32) rows per lane):
// * R == 2 (33 to 64 levels): lane l holds the adjacent rows 2l and 2l + 1.
//   Each recurrence is the lane's own step over its two rows with the prefix
//   (suffix) product of their coefficients, one scan of the lanes' composite
//   maps, and a fix-up of both rows by that product times the carry from the
//   neighbouring lane;
// * otherwise: row k lives on lane k mod 32, so that every load and store of
//   the warp is one coalesced access of 32 consecutive values, and the column
//   is scanned 32 rows at a time, each segment starting from the previous
//   segment's last value.
// Either way there is no shared memory and no block barrier, and the warp
// never waits on a serial chain of n_r steps.  Slots are the relaxation
// tasks' cell lists ([task][16], padding -1), so a colour pass covers slots
// [16 task0, 16 (task0 + n_tasks)).
// The column T (neighbour record nb) of one pass, by one warp (the body of
// k_relax32_scan, shared with the batched form).
template <int MODE, typename TF, int R, bool SF>
__device__ __forceinline__ void relax32_column(const bf16x4 *__restrict__ cpack,
                                               const unsigned short *__restrict__ cvert,
                                               const float *__restrict__ rinv, const float *__restrict__ fb,
                                               const float *__restrict__ fg, int n_r,
                                               const TF *__restrict__ f, const float *u_in, float *u_out,
                                               float *__restrict__ u_fine, double *__restrict__ out64, float relax,
                                               int T, int4 nb, int lane)
{
    const unsigned full = 0xffffffffu;
    const bool n0 = MODE == PASS_NORMAL || (nb.w & 1), n1 = MODE == PASS_NORMAL || (nb.w & 2),
               n2 = MODE == PASS_NORMAL || (nb.w & 4);
    const size_t base = (size_t)T * n_r;
    // CH (two rows per lane, n_r <= 64): lane l holds rows 2l and 2l + 1, each recurrence is
    // the lane's own step, one scan of the lanes' composite affine maps and a fix-up by the
    // prefix products -- a chain of 8 steps each way instead of 12; otherwise row k sits on
    // lane k mod 32 and the 32-row segments are scanned one after another
    constexpr bool CH = R == 2;
    auto row = [&](int r) { return CH ? 2 * lane + r : 32 * r + lane; };
    // the multipliers of row k: c_k rinv_k below and c_{k+1} rinv_k above (SF: the
    // stored ones, with advection).  Face 0 of every column stores the coupling 0 (no
    // flux through the bottom), which is also face n_r of the column before, and one
    // zero element follows the level's last column, so both loads are unconditional.
    auto below = [&](int k, size_t i, float ri) { return SF ? __ldg(&fb[i]) : bf(__ldg(&cvert[i])) * ri; };
    // the coupling above row k (or its stored multiplier): with at most two rows per lane
    // loaded with the forward pass's operands, so that the pass has one round trip to
    // memory on its critical path; with more rows per lane in the backward pass (the
    // registers would cost resident warps on the HBM-bound large levels)
    constexpr bool PF = R <= 2;
    auto above_load = [&](size_t i) { return SF ? __ldg(&fg[i]) : bf(__ldg(&cvert[i + 1])); };
    auto above = [&](float cu, float ri) { return SF ? cu : cu * ri; };
    float cu[R];
    float x[R], ri[R];
    if (CH) {
        float P[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int k = row(j);
            float t = 0.f, b = 1.f;
            ri[j] = cu[j] = 0.f;
            if (k < n_r) {
                const size_t i = base + k;
                float d = (float)f[i];
                if (MODE != PASS_RHS_ONLY) {
                    const bf16x4 cp = cpack[i];
                    const float v0 = n0 ? u_in[(size_t)nb.x * n_r + k] : 0.f;
                    const float v1 = n1 ? u_in[(size_t)nb.y * n_r + k] : 0.f;
                    const float v2 = n2 ? u_in[(size_t)nb.z * n_r + k] : 0.f;
                    d = fmaf(bf(cp.z), v2, fmaf(bf(cp.y), v1, fmaf(bf(cp.x), v0, d)));
                }
                ri[j] = __ldg(&rinv[i]);
                cu[j] = above_load(i);
                t = d * ri[j];
                b = below(k, i, ri[j]);
            }
            x[j] = j == 0 ? t : fmaf(b, x[j - 1], t);
            P[j] = j == 0 ? b : P[j - 1] * b;
        }
        {
            float A = P[R - 1], B = x[R - 1];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float Ap = __shfl_up_sync(full, A, o), Bp = __shfl_up_sync(full, B, o);
                if (lane >= o) {
                    B = fmaf(A, Bp, B);
                    A *= Ap;
                }
            }
            float cin = __shfl_up_sync(full, B, 1);
            if (lane == 0) cin = 0.f;
#pragma unroll
            for (int j = 0; j < R; ++j) x[j] = fmaf(P[j], cin, x[j]);
        }
#pragma unroll
        for (int j = R - 1; j >= 0; --j) {
            const int k = row(j);
            const float c = k < n_r ? above(cu[j], ri[j]) : 0.f;
            if (k >= n_r) x[j] = 0.f;
            if (j < R - 1) x[j] = fmaf(c, x[j + 1], x[j]);
            P[j] = j == R - 1 ? c : c * P[j + 1];
        }
        {
            float A = P[0], B = x[0];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float Ad = __shfl_down_sync(full, A, o), Bd = __shfl_down_sync(full, B, o);
                if (lane + o < 32) {
                    B = fmaf(A, Bd, B);
                    A *= Ad;
                }
            }
            float cin = __shfl_down_sync(full, B, 1);
            if (lane == 31) cin = 0.f;
#pragma unroll
            for (int j = 0; j < R; ++j) x[j] = fmaf(P[j], cin, x[j]);
        }
    } else {
        // forward recurrence, segment by segment
        float carry = 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = 32 * r + lane;
            float A = 0.f, B = 0.f;
            ri[r] = cu[r] = 0.f;
            if (k < n_r) {
                const size_t i = base + k;
                float d = (float)f[i];
                if (MODE != PASS_RHS_ONLY) {
                    const bf16x4 cp = cpack[i];
                    const float v0 = n0 ? u_in[(size_t)nb.x * n_r + k] : 0.f;
                    const float v1 = n1 ? u_in[(size_t)nb.y * n_r + k] : 0.f;
                    const float v2 = n2 ? u_in[(size_t)nb.z * n_r + k] : 0.f;
                    d = fmaf(bf(cp.z), v2, fmaf(bf(cp.y), v1, fmaf(bf(cp.x), v0, d)));
                }
                ri[r] = __ldg(&rinv[i]);
                if (PF) cu[r] = above_load(i);
                B = d * ri[r];
                A = below(k, i, ri[r]);
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float Ap = __shfl_up_sync(full, A, o), Bp = __shfl_up_sync(full, B, o);
                if (lane >= o) {
                    B = fmaf(A, Bp, B);
                    A *= Ap;
                }
            }
            x[r] = fmaf(A, carry, B);
            carry = __shfl_sync(full, x[r], 31);
        }
        // backward recurrence, from the top segment down
        carry = 0.f;
#pragma unroll
        for (int r = R - 1; r >= 0; --r) {
            const int k = 32 * r + lane;
            float A = 0.f, B = 0.f;
            if (k < n_r) {
                A = above(PF ? cu[r] : above_load(base + k), ri[r]);
                B = x[r];
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float Ad = __shfl_down_sync(full, A, o), Bd = __shfl_down_sync(full, B, o);
                if (lane + o < 32) {
                    B = fmaf(A, Bd, B);
                    A *= Ad;
                }
            }
            x[r] = fmaf(A, carry, B);
            carry = __shfl_sync(full, x[r], 0);
        }
    }
    // write-back: relaxation weight, the double copy of the finest level's
    // result, the prolongation into the 4 children (P = R^T)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int k = row(r);
        if (k >= n_r) continue;
        const size_t i = base + k;
        float v = x[r];
        if (relax != 1.f) {   // from a zero guess (ZERO, RHS_ONLY) the old value is 0
            const float uo = MODE == PASS_NORMAL ? u_in[i] : 0.f;
            v = fmaf(relax, v - uo, uo);
        }
        u_out[i] = v;
        if (out64) out64[i] = (double)v;
        if (u_fine) {
            const size_t fi = (size_t)4 * T * n_r + k;
#pragma unroll
            for (int h = 0; h < 4; ++h) u_fine[fi + (size_t)h * n_r] += v;
        }
    }
}

// The same pass for columns of exactly 32 R rows (R = 2: 64, R = 4: 128) without
// vertical advection, in the row-chunk layout (lane l: rows R l .. R l + R - 1) with
// every array moved in pieces of 4 to 32 bytes: f, 1/pivot, u and the neighbours' u
// as one float2 / float4 per lane (f in FP64 as R / 2 double2), the lane's R stencil
// records as R / 2 loads of 16 bytes, its R lower-face couplings as one 4- or 8-byte
// load.  The upper face of row R l + R - 1 is the next lane's first lower face (a
// shuffle; 0 above the top row).  Each recurrence is the lane's own R steps, one scan
// of the lanes' composite maps and a fix-up, with the arithmetic per row of the
// other layouts, so the pass differs from them only in the order of the scan's
// roundings.
__host__ __device__ inline bool relax32_vec_ok(int R, int n_r, bool advection, const void *cpack, const void *cvert,
                                               const void *rinv, const void *f, const void *u_in, const void *u_out,
                                               const void *u_fine, const void *out64)
{
    // every array on a 16-byte boundary (the couplings on 8); null pointers are unused
    const uintptr_t a = (uintptr_t)cpack | (uintptr_t)rinv | (uintptr_t)f | (uintptr_t)u_in | (uintptr_t)u_out |
                        (uintptr_t)u_fine | (uintptr_t)out64;
    return (R == 2 || R == 4) && n_r == 32 * R && !advection && (a & 15) == 0 && ((uintptr_t)cvert & 7) == 0;
}

__device__ __forceinline__ float bf_lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }

// R consecutive floats starting at p (8- or 16-byte aligned) into v[0 .. R-1]
template <int R, bool LDG>
__device__ __forceinline__ void load_rows(const float *p, float *v)
{
    if constexpr (R == 2) {
        const float2 t = LDG ? __ldg(reinterpret_cast<const float2 *>(p)) : *reinterpret_cast<const float2 *>(p);
        v[0] = t.x, v[1] = t.y;
    } else {
        const float4 t = LDG ? __ldg(reinterpret_cast<const float4 *>(p)) : *reinterpret_cast<const float4 *>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    }
}

template <int MODE, typename TF, int R>
__device__ __forceinline__ void relax32_column_vec(const bf16x4 *__restrict__ cpack,
                                                   const unsigned short *__restrict__ cvert,
                                                   const float *__restrict__ rinv, const TF *__restrict__ f,
                                                   const float *u_in, float *u_out, float *__restrict__ u_fine,
                                                   double *__restrict__ out64, float relax, int T, int4 nb, int lane)
{
    static_assert(R == 2 || R == 4, "16-byte layout: 2 or 4 rows per lane");
    constexpr int n_r = 32 * R;
    const unsigned full = 0xffffffffu;
    const bool n0 = MODE == PASS_NORMAL || (nb.w & 1), n1 = MODE == PASS_NORMAL || (nb.w & 2),
               n2 = MODE == PASS_NORMAL || (nb.w & 4);
    const int k0 = R * lane;
    const size_t i0 = (size_t)T * n_r + k0;
    float d[R];
    if constexpr (sizeof(TF) == 4) {
        load_rows<R, true>(reinterpret_cast<const float *>(f) + i0, d);
    } else {
#pragma unroll
        for (int h = 0; h < R / 2; ++h) {
            const double2 t = __ldg(reinterpret_cast<const double2 *>(f + i0) + h);
            d[2 * h] = (float)t.x, d[2 * h + 1] = (float)t.y;
        }
    }
    if (MODE != PASS_RHS_ONLY) {
        // stencil records of rows k0 .. k0 + R - 1: {alphaS_hat 0, 1, 2, beta_hat} in 8 bytes each,
        // as 32-bit words: lo = alphaS_hat 0 | 1, hi = alphaS_hat 2 | beta_hat
        unsigned lo[R], hi[R];
#pragma unroll
        for (int h = 0; h < R / 2; ++h) {
            const uint4 w = __ldg(reinterpret_cast<const uint4 *>(cpack + i0) + h);
            lo[2 * h] = w.x, hi[2 * h] = w.y, lo[2 * h + 1] = w.z, hi[2 * h + 1] = w.w;
        }
        float a0[R], a1[R], a2[R];
#pragma unroll
        for (int j = 0; j < R; ++j) a0[j] = a1[j] = a2[j] = 0.f;
        if (n0) load_rows<R, false>(u_in + (size_t)nb.x * n_r + k0, a0);
        if (n1) load_rows<R, false>(u_in + (size_t)nb.y * n_r + k0, a1);
        if (n2) load_rows<R, false>(u_in + (size_t)nb.z * n_r + k0, a2);
#pragma unroll
        for (int j = 0; j < R; ++j)
            d[j] = fmaf(bf_lo(hi[j]), a2[j], fmaf(bf_hi(lo[j]), a1[j], fmaf(bf_lo(lo[j]), a0[j], d[j])));
    }
    float ri[R];
    load_rows<R, true>(rinv + i0, ri);
    // lower-face couplings c_k of the lane's rows; c_{k+1} above them
    float cb[R];
    if constexpr (R == 2) {
        const unsigned w = __ldg(reinterpret_cast<const unsigned *>(cvert + i0));
        cb[0] = bf_lo(w), cb[1] = bf_hi(w);
    } else {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(cvert + i0));
        cb[0] = bf_lo(w.x), cb[1] = bf_hi(w.x), cb[2] = bf_lo(w.y), cb[3] = bf_hi(w.y);
    }
    float ctop = __shfl_down_sync(full, cb[0], 1);
    if (lane == 31) ctop = 0.f;
    float x[R], P[R];
    // y_k = d_k / p_k + (c_k / p_k) y_{k-1}
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const float t = d[j] * ri[j], b = cb[j] * ri[j];
        x[j] = j == 0 ? t : fmaf(b, x[j - 1], t);
        P[j] = j == 0 ? b : P[j - 1] * b;
    }
    {
        float A = P[R - 1], B = x[R - 1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float Ap = __shfl_up_sync(full, A, o), Bp = __shfl_up_sync(full, B, o);
            if (lane >= o) {
                B = fmaf(A, Bp, B);
                A *= Ap;
            }
        }
        float cin = __shfl_up_sync(full, B, 1);
        if (lane == 0) cin = 0.f;
#pragma unroll
        for (int j = 0; j < R; ++j) x[j] = fmaf(P[j], cin, x[j]);
    }
    // x_k = y_k + (c_{k+1} / p_k) x_{k+1}
#pragma unroll
    for (int j = R - 1; j >= 0; --j) {
        const float c = (j < R - 1 ? cb[j + 1] : ctop) * ri[j];
        if (j < R - 1) x[j] = fmaf(c, x[j + 1], x[j]);
        P[j] = j == R - 1 ? c : c * P[j + 1];
    }
    {
        float A = P[0], B = x[0];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float Ad = __shfl_down_sync(full, A, o), Bd = __shfl_down_sync(full, B, o);
            if (lane + o < 32) {
                B = fmaf(A, Bd, B);
                A *= Ad;
            }
        }
        float cin = __shfl_down_sync(full, B, 1);
        if (lane == 31) cin = 0.f;
#pragma unroll
        for (int j = 0; j < R; ++j) x[j] = fmaf(P[j], cin, x[j]);
    }
    // write-back: relaxation weight, the double copy of the finest level's result, the
    // prolongation into the 4 children (P = R^T)
    if (relax != 1.f) {   // from a zero guess (ZERO, RHS_ONLY) the old value is 0
        float uo[R];
#pragma unroll
        for (int j = 0; j < R; ++j) uo[j] = 0.f;
        if (MODE == PASS_NORMAL) load_rows<R, false>(u_in + i0, uo);
#pragma unroll
        for (int j = 0; j < R; ++j) x[j] = fmaf(relax, x[j] - uo[j], uo[j]);
    }
    auto store_rows = [&](float *p, const float *v) {
        if constexpr (R == 2)
            *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
        else
            *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    };
    store_rows(u_out + i0, x);
    if (out64) {
#pragma unroll
        for (int h = 0; h < R / 2; ++h)
            reinterpret_cast<double2 *>(out64 + i0)[h] = make_double2((double)x[2 * h], (double)x[2 * h + 1]);
    }
    if (u_fine) {
        const size_t fi = (size_t)4 * T * n_r + k0;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float v[R];
            load_rows<R, false>(u_fine + fi + (size_t)h * n_r, v);
#pragma unroll
            for (int j = 0; j < R; ++j) v[j] += x[j];
            store_rows(u_fine + fi + (size_t)h * n_r, v);
        }
    }
}

template <int MODE, typename TF, int R, bool SF, bool VEC = false>
__global__ void __launch_bounds__(256, VEC ? 8 : 1)
    k_relax32_scan(const int *__restrict__ cells, const int4 *__restrict__ tnb, const bf16x4 *__restrict__ cpack,
                   const unsigned short *__restrict__ cvert, const float *__restrict__ rinv,
                   const float *__restrict__ fb, const float *__restrict__ fg, int n_r, int slot0, int n_slots,
                   const TF *__restrict__ f, const float *u_in, float *u_out, float *__restrict__ u_fine,
                   double *__restrict__ out64, float relax)
{
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    // the column's cell and neighbours are set-up data: read before the wait
    const int T = w < n_slots ? __ldg(&cells[slot0 + w]) : -1;
    const int4 nb = MODE == PASS_RHS_ONLY || T < 0 ? make_int4(0, 0, 0, 0) : __ldg(&tnb[slot0 + w]);
    pdl_wait();
    pdl_trigger();
    if (T < 0) return;
    if constexpr (VEC)
        relax32_column_vec<MODE, TF, R>(cpack, cvert, rinv, f, u_in, u_out, u_fine, out64, relax, T, nb, lane);
    else
        relax32_column<MODE, TF, R, SF>(cpack, cvert, rinv, fb, fg, n_r, f, u_in, u_out, u_fine, out64, relax, T, nb,
                                        lane);
}

// Index of the work-list item of a warp-uniform position x: the last item whose first
// position off[it] (ascending, off[0] = 0) is <= x.  A binary search over the launch's
// parameter block: every lane of the warp reads the same entries (broadcast from the
// constant cache), with no global-memory round trip before the column's own loads.
__device__ __forceinline__ int batch_item(const int *off, int n_items, int x)
{
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// One pass of the batched form: the columns of several members' colour passes of one
// mode, right-hand-side type and rows-per-lane class in one launch.  Warp w relaxes
// slot w - woff[it] of item it, with that item's level data and vectors, exactly as
// k_relax32_scan does for the item's own pass; members whose loop has stopped
// (active == 0) are skipped.
template <int MODE, typename TF, int R, int CAP>
__global__ void __launch_bounds__(256) k_relax32_batch(const __grid_constant__ RelaxBatchArgsT<CAP> a,
                                                       const int *__restrict__ active)
{
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int it = batch_item(a.off, a.n_items, w);
    const BatchRelaxItem &I = a.items[it];
    const int ws = w - a.off[it];
    const int T = ws < I.n_slots ? __ldg(&I.cells[I.slot0 + ws]) : -1;
    const int4 nb = MODE == PASS_RHS_ONLY || T < 0 ? make_int4(0, 0, 0, 0) : __ldg(&I.tnb[I.slot0 + ws]);
    pdl_wait();
    pdl_trigger();
    if (T < 0 || !active[I.member]) return;
    // the layout the member's own pass takes (the same rounding as its single solve)
    if constexpr (R == 2 || R == 4) {
        if (relax32_vec_ok(R, I.n_r, false, I.cpack, I.cvert, I.rinv, I.f, I.u_in, I.u_out, I.u_fine, I.out64)) {
            relax32_column_vec<MODE, TF, R>(I.cpack, I.cvert, I.rinv, static_cast<const TF *>(I.f), I.u_in, I.u_out,
                                            I.u_fine, I.out64, I.relax, T, nb, lane);
            return;
        }
    }
    relax32_column<MODE, TF, R, false>(I.cpack, I.cvert, I.rinv, nullptr, nullptr, I.n_r,
                                       static_cast<const TF *>(I.f), I.u_in, I.u_out, I.u_fine, I.out64, I.relax, T,
                                       nb, lane);
}

// f_c[T][k] = sum_j (f - A u)[4T + j][k] in FP32 with the BF16 stencil, the row
// in the flux form of Appendix A (Algorithm 1 residual + restriction).
template <typename TF>
__device__ __forceinline__ void restrict32_row(const int4 *__restrict__ nbr, const bf16x4 *__restrict__ cpack,
                                               const unsigned short *__restrict__ cvert,
                                               const unsigned short *__restrict__ cxv, const float *__restrict__ dr32,
                                               int n_r, const TF *__restrict__ f, const float *__restrict__ u,
                                               float *__restrict__ fc, int ic)
{
    {
        const int Tc = ic / n_r, k = ic - Tc * n_r;
        float s = 0.f;
#pragma unroll
        for (int jc = 0; jc < 4; ++jc) {
            const int T = 4 * Tc + jc, i = T * n_r + k;
            const int4 nb = __ldg(&nbr[T]);
            const bf16x4 cp = cpack[i];
            const float uc = u[i];
            const float um = k > 0 ? u[i - 1] : uc, up = k < n_r - 1 ? u[i + 1] : uc;
            float cl = bf(__ldg(&cvert[i])), cu = k < n_r - 1 ? bf(__ldg(&cvert[i + 1])) : 0.f;
            if (cxv) {   // centred vertical advection (face k's X is zero for k = 0)
                const float d = __ldg(&dr32[k]);
                cl = fmaf(-d, bf(__ldg(&cxv[i])), cl);
                if (k < n_r - 1) cu = fmaf(d, bf(__ldg(&cxv[i + 1])), cu);
            }
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

template <typename TF>
__global__ void __launch_bounds__(kThreads32)
    k_resid_restrict32(const int4 *__restrict__ nbr, const bf16x4 *__restrict__ cpack,
                       const unsigned short *__restrict__ cvert, const unsigned short *__restrict__ cxv,
                       const float *__restrict__ dr32, int n_r, const TF *__restrict__ f,
                       const float *__restrict__ u, float *__restrict__ fc, int Nc)
{
    pdl_wait();
    pdl_trigger();
    for (int ic = blockIdx.x * kThreads32 + threadIdx.x; ic < Nc; ic += gridDim.x * kThreads32)
        restrict32_row<TF>(nbr, cpack, cvert, cxv, dr32, n_r, f, u, fc, ic);
}

// The same residual + restriction for columns of exactly 32 R rows (R = 2: 64, R = 4:
// 128) without vertical advection: one warp per coarse column, lane l forming the
// coarse rows R l .. R l + R - 1, every array moved R rows at a time (f, u, the
// neighbours' u and f_c as one float2 / float4 per lane, f in FP64 as R / 2 double2,
// the stencil as R / 2 loads of 16 bytes, the lower-face couplings as 4 or 8 bytes).
// The rows just below and above a lane's rows, and the coupling above its last row,
// come from the neighbouring lanes by shuffles.  Each row's operations and their
// order are those of restrict32_row, so the results are the same bit for bit.
template <typename TF, int R>
__global__ void __launch_bounds__(kThreads32)
    k_resid_restrict32_vec(const int4 *__restrict__ nbr, const bf16x4 *__restrict__ cpack,
                           const unsigned short *__restrict__ cvert, const TF *__restrict__ f,
                           const float *__restrict__ u, float *__restrict__ fc, int n_coarse)
{
    constexpr int n_r = 32 * R;
    const unsigned full = 0xffffffffu;
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31, k0 = R * lane;
    const int w0 = blockIdx.x * (kThreads32 >> 5) + (threadIdx.x >> 5), nw = gridDim.x * (kThreads32 >> 5);
    for (int Tc = w0; Tc < n_coarse; Tc += nw) {
        float s[R];
#pragma unroll
        for (int j = 0; j < R; ++j) s[j] = 0.f;
#pragma unroll
        for (int jc = 0; jc < 4; ++jc) {
            const int T = 4 * Tc + jc;
            const size_t i0 = (size_t)T * n_r + k0;
            const int4 nb = __ldg(&nbr[T]);
            unsigned lo[R], hi[R];
#pragma unroll
            for (int h = 0; h < R / 2; ++h) {
                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(cpack + i0) + h);
                lo[2 * h] = q.x, hi[2 * h] = q.y, lo[2 * h + 1] = q.z, hi[2 * h + 1] = q.w;
            }
            float uc[R], v0[R], v1[R], v2[R], cl[R], fr[R];
            load_rows<R, true>(u + i0, uc);
            load_rows<R, true>(u + (size_t)nb.x * n_r + k0, v0);
            load_rows<R, true>(u + (size_t)nb.y * n_r + k0, v1);
            load_rows<R, true>(u + (size_t)nb.z * n_r + k0, v2);
            if constexpr (R == 2) {
                const unsigned q = __ldg(reinterpret_cast<const unsigned *>(cvert + i0));
                cl[0] = bf_lo(q), cl[1] = bf_hi(q);
            } else {
                const uint2 q = __ldg(reinterpret_cast<const uint2 *>(cvert + i0));
                cl[0] = bf_lo(q.x), cl[1] = bf_hi(q.x), cl[2] = bf_lo(q.y), cl[3] = bf_hi(q.y);
            }
            if constexpr (sizeof(TF) == 4) {
                load_rows<R, true>(reinterpret_cast<const float *>(f) + i0, fr);
            } else {
#pragma unroll
                for (int h = 0; h < R / 2; ++h) {
                    const double2 t = __ldg(reinterpret_cast<const double2 *>(f + i0) + h);
                    fr[2 * h] = (float)t.x, fr[2 * h + 1] = (float)t.y;
                }
            }
            // the row below the lane's first (u of the column's row 0 itself at k = 0), the row
            // above its last (the top row itself at k = n_r - 1) and the coupling above its last
            // row (0 at the top face)
            float ubelow = __shfl_up_sync(full, uc[R - 1], 1), uabove = __shfl_down_sync(full, uc[0], 1),
                  ctop = __shfl_down_sync(full, cl[0], 1);
            if (lane == 0) ubelow = uc[0];
            if (lane == 31) uabove = uc[R - 1], ctop = 0.f;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const float um = j > 0 ? uc[j - 1] : ubelow, up = j < R - 1 ? uc[j + 1] : uabove;
                const float cu = j < R - 1 ? cl[j + 1] : ctop;
                float a = bf_hi(hi[j]) * uc[j];
                a = fmaf(cl[j], uc[j] - um, a);
                a = fmaf(cu, uc[j] - up, a);
                a = fmaf(bf_lo(lo[j]), uc[j] - v0[j], a);
                a = fmaf(bf_hi(lo[j]), uc[j] - v1[j], a);
                a = fmaf(bf_lo(hi[j]), uc[j] - v2[j], a);
                s[j] += fr[j] - a;
            }
        }
        float *out = fc + (size_t)Tc * n_r + k0;
        if constexpr (R == 2)
            *reinterpret_cast<float2 *>(out) = make_float2(s[0], s[1]);
        else
            *reinterpret_cast<float4 *>(out) = make_float4(s[0], s[1], s[2], s[3]);
    }
}

// Residual + restriction of the batched form: the coarse rows of several members'
// restrictions in one launch.  Each item's rows occupy a range of the launch's
// positions starting at roff[it], a multiple of 32, so that a warp's positions belong
// to one item; position x is coarse row x - roff[it] of that item.
template <typename TF, int CAP>
__global__ void __launch_bounds__(kThreads32) k_restrict32_batch(const __grid_constant__ RestrictBatchArgsT<CAP> a,
                                                                 int total, const int *__restrict__ active)
{
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    for (int x0 = (blockIdx.x * kThreads32 + threadIdx.x) & ~31; x0 < total; x0 += gridDim.x * kThreads32) {
        const int it = batch_item(a.off, a.n_items, x0);
        const BatchRestrictItem &I = a.items[it];
        const int ic = x0 + lane - a.off[it];
        if (ic < I.Nc && active[I.member])
            restrict32_row<TF>(I.nbr, I.cpack, I.cvert, nullptr, nullptr, I.n_r, static_cast<const TF *>(I.f), I.u,
                               I.fc, ic);
    }
}

// Linear prolongation in FP32 (the FP64 kernel's arithmetic on the FP32 weights).
__global__ void __launch_bounds__(kThreads32) k_prolong_linear32(const int4 *__restrict__ nbr_c,
                                                                 const float *__restrict__ w,
                                                                 const float *__restrict__ uc, float *__restrict__ u,
                                                                 int n_r, int N)
{
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * kThreads32 + threadIdx.x; i < N; i += gridDim.x * kThreads32) {
        const int t = i / n_r, k = i - t * n_r, T = t >> 2, j = t & 3;
        const int4 nb = __ldg(&nbr_c[T]);
        const float *wt = w + (size_t)T * 12 + 3 * j;
        const float v = uc[(size_t)T * n_r + k];
        float s = fmaf(__ldg(&wt[0]), uc[(size_t)nb.x * n_r + k] - v, v);
        s = fmaf(__ldg(&wt[1]), uc[(size_t)nb.y * n_r + k] - v, s);
        s = fmaf(__ldg(&wt[2]), uc[(size_t)nb.z * n_r + k] - v, s);
        u[i] += s;
    }
}

__global__ void __launch_bounds__(kThreads32) k_prolong_add32(const float *__restrict__ uc, float *__restrict__ u,
                                                              int n_r, int N)
{
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * kThreads32 + threadIdx.x; i < N; i += gridDim.x * kThreads32) {
        const int T = i / n_r, k = i - T * n_r;
        u[i] += uc[(T >> 2) * n_r + k];
    }
}

__global__ void __launch_bounds__(kThreads32) k_to_f64(const float *__restrict__ x, double *__restrict__ y, int N)
{
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * kThreads32 + threadIdx.x; i < N; i += gridDim.x * kThreads32) y[i] = (double)x[i];
}

inline int grid32(long work, int sm_count)
{
    long b = (work + kThreads32 - 1) / kThreads32;
    const long cap = (long)sm_count * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <int MODE, typename TF, int R>
cudaError_t relax32_r(const Launch &L, const LevelDev &lv, int task0, int n_tasks, float relax, const TF *f,
                      const float *u_in, float *u_out, float *u_fine, double *out64)
{
    // CTA of 1, 2, 4 or 8 warps (the autotuner's variants; same arithmetic)
    const int var = lv.relax_variant < 0 ? RELAX_CTA128 : lv.relax_variant;
    const int wpb = 1 << var;
    const int n_slots = n_tasks * kRelaxCols;
    // the stored multipliers only with vertical advection (their couplings are not alphar_hat)
    auto kern = lv.cxv_on ? k_relax32_scan<MODE, TF, R, true> : k_relax32_scan<MODE, TF, R, false>;
    // columns of exactly 64 or 128 rows: 2 or 4 rows per lane with 8- and 16-byte accesses
    if constexpr (R == 2 || R == 4)
        if (relax32_vec_ok(R, L.n_r, lv.cxv_on, lv.cpack, lv.cvert, lv.rinv32, f, u_in, u_out, u_fine, out64))
            kern = k_relax32_scan<MODE, TF, R, false, true>;
    return launch_k(L, kern, (n_slots + wpb - 1) / wpb, 32 * wpb, 0, lv.task_cells, lv.task_nbr, lv.cpack, lv.cvert,
                    lv.rinv32, lv.fb32, lv.fc32, L.n_r, task0 * kRelaxCols, n_slots, f, u_in, u_out, u_fine, out64,
                    relax);
}

template <int MODE, typename TF>
cudaError_t relax32_t(const Launch &L, const LevelDev &lv, int task0, int n_tasks, float relax, const TF *f,
                      const float *u_in, float *u_out, float *u_fine, double *out64)
{
    const int n = L.n_r;
    if (n <= 32) return relax32_r<MODE, TF, 1>(L, lv, task0, n_tasks, relax, f, u_in, u_out, u_fine, out64);
    if (n <= 64) return relax32_r<MODE, TF, 2>(L, lv, task0, n_tasks, relax, f, u_in, u_out, u_fine, out64);
    if (n <= 128) return relax32_r<MODE, TF, 4>(L, lv, task0, n_tasks, relax, f, u_in, u_out, u_fine, out64);
    if (n <= 256) return relax32_r<MODE, TF, 8>(L, lv, task0, n_tasks, relax, f, u_in, u_out, u_fine, out64);
    if (n <= 512) return relax32_r<MODE, TF, 16>(L, lv, task0, n_tasks, relax, f, u_in, u_out, u_fine, out64);
    return relax32_r<MODE, TF, 32>(L, lv, task0, n_tasks, relax, f, u_in, u_out, u_fine, out64);
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
    // columns of exactly 64 or 128 rows without advection: one warp per coarse column
    // with 8- and 16-byte accesses (the same arithmetic)
    const int grid_w = grid32((long)coarse.n * 32, L.sm_count);
    if (relax32_vec_ok(2, L.n_r, fine.cxv_on, fine.cpack, fine.cvert, nullptr, f, u, fc, nullptr, nullptr))
        return launch_k(L, k_resid_restrict32_vec<TF, 2>, grid_w, kThreads32, 0, fine.nbr, fine.cpack, fine.cvert, f,
                        u, fc, coarse.n);
    if (relax32_vec_ok(4, L.n_r, fine.cxv_on, fine.cpack, fine.cvert, nullptr, f, u, fc, nullptr, nullptr))
        return launch_k(L, k_resid_restrict32_vec<TF, 4>, grid_w, kThreads32, 0, fine.nbr, fine.cpack, fine.cvert, f,
                        u, fc, coarse.n);
    return launch_k(L, k_resid_restrict32<TF>, grid32(Nc, L.sm_count), kThreads32, 0, fine.nbr, fine.cpack, fine.cvert,
                    fine.cxv_on ? fine.cxv : nullptr, L.dr32, L.n_r, f, u, fc, Nc);
}

// The launch's items in a parameter block of capacity CAP (>= the item count).
template <int CAP>
RelaxBatchArgsT<CAP> shrink_relax(const RelaxBatchArgs &a)
{
    RelaxBatchArgsT<CAP> s{};
    s.n_items = a.n_items;
    for (int i = 0; i < a.n_items && i < CAP; ++i) {
        s.off[i] = a.off[i];
        s.items[i] = a.items[i];
    }
    return s;
}
template <int CAP>
RestrictBatchArgsT<CAP> shrink_restrict(const RestrictBatchArgs &a)
{
    RestrictBatchArgsT<CAP> s{};
    s.n_items = a.n_items;
    for (int i = 0; i < a.n_items && i < CAP; ++i) {
        s.off[i] = a.off[i];
        s.items[i] = a.items[i];
    }
    return s;
}

template <int MODE, typename TF, int CAP>
cudaError_t relax32_batch_c(const Launch &L, int n_r_max, const RelaxBatchArgs &big, unsigned grid, int nt,
                            const int *active)
{
    const RelaxBatchArgsT<CAP> a = shrink_relax<CAP>(big);
    // the items of a launch share the rows-per-lane class of their column height
    if (n_r_max <= 32) return launch_k(L, k_relax32_batch<MODE, TF, 1, CAP>, grid, nt, 0, a, active);
    if (n_r_max <= 64) return launch_k(L, k_relax32_batch<MODE, TF, 2, CAP>, grid, nt, 0, a, active);
    if (n_r_max <= 128) return launch_k(L, k_relax32_batch<MODE, TF, 4, CAP>, grid, nt, 0, a, active);
    if (n_r_max <= 256) return launch_k(L, k_relax32_batch<MODE, TF, 8, CAP>, grid, nt, 0, a, active);
    if (n_r_max <= 512) return launch_k(L, k_relax32_batch<MODE, TF, 16, CAP>, grid, nt, 0, a, active);
    return launch_k(L, k_relax32_batch<MODE, TF, 32, CAP>, grid, nt, 0, a, active);
}

template <int MODE, typename TF>
cudaError_t relax32_batch_t(const Launch &L, int n_r_max, const RelaxBatchArgs &a, long total_warps, int wpb,
                            const int *active)
{
    const unsigned grid = (unsigned)((total_warps + wpb - 1) / wpb);
    const int nt = 32 * wpb;
    if (a.n_items <= 2) return relax32_batch_c<MODE, TF, 2>(L, n_r_max, a, grid, nt, active);
    if (a.n_items <= 8) return relax32_batch_c<MODE, TF, 8>(L, n_r_max, a, grid, nt, active);
    return relax32_batch_c<MODE, TF, kBatchItems>(L, n_r_max, a, grid, nt, active);
}

template <typename TF>
cudaError_t launch_relax32_batch(const Launch &L, int mode, int n_r_max, const RelaxBatchArgs &a, long total_warps,
                                 int wpb, const int *active)
{
    if (a.n_items <= 0 || total_warps <= 0) return cudaSuccess;
    if (a.n_items > kBatchItems || (wpb != 1 && wpb != 2 && wpb != 4 && wpb != 8)) return cudaErrorInvalidValue;
    switch (mode) {
    case PASS_ZERO: return relax32_batch_t<PASS_ZERO, TF>(L, n_r_max, a, total_warps, wpb, active);
    case PASS_RHS_ONLY: return relax32_batch_t<PASS_RHS_ONLY, TF>(L, n_r_max, a, total_warps, wpb, active);
    default: return relax32_batch_t<PASS_NORMAL, TF>(L, n_r_max, a, total_warps, wpb, active);
    }
}

template <typename TF>
cudaError_t launch_restrict32_batch(const Launch &L, const RestrictBatchArgs &a, long total, const int *active)
{
    if (a.n_items <= 0 || total <= 0) return cudaSuccess;
    if (a.n_items > kBatchItems) return cudaErrorInvalidValue;
    const int grid = grid32(total, L.sm_count);
    if (a.n_items <= 2)
        return launch_k(L, k_restrict32_batch<TF, 2>, grid, kThreads32, 0, shrink_restrict<2>(a), (int)total, active);
    if (a.n_items <= 8)
        return launch_k(L, k_restrict32_batch<TF, 8>, grid, kThreads32, 0, shrink_restrict<8>(a), (int)total, active);
    return launch_k(L, k_restrict32_batch<TF, kBatchItems>, grid, kThreads32, 0, a, (int)total, active);
}

cudaError_t launch_prolong_add32(const Launch &L, const LevelDev &fine, const float *uc, float *u)
{
    const int N = fine.n * L.n_r;
    return launch_k(L, k_prolong_add32, grid32(N, L.sm_count), kThreads32, 0, uc, u, L.n_r, N);
}

cudaError_t launch_prolong_linear32(const Launch &L, const LevelDev &fine, const LevelDev &coarse, const float *uc,
                                    float *u)
{
    const int N = fine.n * L.n_r;
    return launch_k(L, k_prolong_linear32, grid32(N, L.sm_count), kThreads32, 0, coarse.nbr, coarse.plin32, uc, u,
                    L.n_r, N);
}

cudaError_t launch_thomas_factors32(const Launch &L, const LevelDev &lv)
{
    k_thomas_factors32<<<(lv.n + 127) / 128, 128, 0, L.s>>>(lv.n, lv.cpack, lv.cvert, lv.cxv_on ? lv.cxv : nullptr,
                                                            L.dr, L.n_r, lv.rinv32, lv.cxv_on ? lv.fb32 : nullptr,
                                                            lv.cxv_on ? lv.fc32 : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_to_f64(const Launch &L, long n, const float *x, double *y)
{
    return launch_k(L, k_to_f64, grid32(n, L.sm_count), kThreads32, 0, x, y, (int)n);
}

template cudaError_t launch_relax32<double>(const Launch &, const LevelDev &, int, int, int, float, const double *,
                                            const float *, float *, float *, double *);
template cudaError_t launch_relax32<float>(const Launch &, const LevelDev &, int, int, int, float, const float *,
                                           const float *, float *, float *, double *);
template cudaError_t launch_relax32_batch<double>(const Launch &, int, int, const RelaxBatchArgs &, long, int,
                                                  const int *);
template cudaError_t launch_relax32_batch<float>(const Launch &, int, int, const RelaxBatchArgs &, long, int,
                                                 const int *);
template cudaError_t launch_restrict32_batch<double>(const Launch &, const RestrictBatchArgs &, long, const int *);
template cudaError_t launch_restrict32_batch<float>(const Launch &, const RestrictBatchArgs &, long, const int *);
template cudaError_t launch_resid_restrict32<double>(const Launch &, const LevelDev &, const LevelDev &,
                                                     const double *, const float *, float *);
template cudaError_t launch_resid_restrict32<float>(const Launch &, const LevelDev &, const LevelDev &, const float *,
                                                    const float *, float *);

}  // namespace tpmg
