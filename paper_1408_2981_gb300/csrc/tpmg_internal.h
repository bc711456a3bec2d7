// Internal declarations of the TPMG library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/tpmg.h"

namespace tpmg {

// ---------------------------------------------------------------------------
// Host grid hierarchy (grid.cpp)
// ---------------------------------------------------------------------------
struct HostLevel {
    int ref = 0;                  // refinement level, n = 20 * 4^ref cells
    int n = 0;
    std::vector<double> corner;   // [n][3][3] corner positions, counter-clockwise from outside
    std::vector<int> nbr;         // [n][3] cell across edge e = (corner e, corner e+1)
    std::vector<double> centre;   // [n][3]
    std::vector<double> area;     // [n]
    std::vector<double> g;        // [n][3] |S| n.(c'-c)/|c'-c|^2
    std::vector<int> colour;      // [n]
    int n_colours = 0;
};

struct HostGrid {
    std::vector<HostLevel> lev;   // refinement 0..L
    std::vector<double> zeta;     // [n_r+1] heights r_k - 1
    std::vector<double> r;        // [n_r+1]
    std::vector<double> dr;       // [n_r]
    std::vector<double> vol;      // [n_r] v_k = (r_{k+1}^3 - r_k^3)/3
    std::vector<double> face;     // [n_r+1] sigma_k 2 r_k^2 / (r_{k+1} - r_{k-1})
    double h_min = 0.0;
    double omega2 = 0.0;
};

// Returns false and sets err on failure.
bool build_host_grid(const tpmg_params &p, HostGrid &grid, std::string &err);

// ---------------------------------------------------------------------------
// Device data (api.cu / kernels.cu)
// ---------------------------------------------------------------------------
struct alignas(32) dbl4 {   // four doubles, one 32-byte load
    double x, y, z, w;
};
struct VertDev {            // vertical factors shared by every level (no vertical coarsening)
    const double *vol;      // [n_r]   v_k = (r_{k+1}^3 - r_k^3)/3
    const double *w;        // [n_r+1] omega^2 sigma_k 2 r_k^2 / (r_{k+1} - r_{k-1})
    const double *hr;       // [n_r]   omega^2 (r_{k+1} - r_k)
    const float *vol32, *w32, *hr32;  // FP32 copies for the mixed-precision V-cycle
};

struct LevelDev {
    int n = 0;              // cells
    int ref = 0;
    int n_colours = 0;
    std::vector<int> colour_off;  // [n_colours+1] offsets into cells_by_colour (host copy)
    int4 *nbr = nullptr;          // [n] {nbr0, nbr1, nbr2, lower-colour mask}
    dbl4 *g = nullptr;            // [n] {g0, g1, g2, g0+g1+g2}
    double *area = nullptr;       // [n]
    int *cells_by_colour = nullptr;   // [n] cell ids grouped by colour, ascending within a colour
    // Thomas factors of the column blocks A_T, [n][n_r]
    double *inv = nullptr;        // 1 / pivot_k
    double *ef = nullptr;         // forward multiplier  area*w_k / pivot_k
    double *cpf = nullptr;        // backward multiplier area*w_{k+1} / pivot_k
    // workspaces (coarse levels; the finest level uses caller / PCG buffers)
    double *f = nullptr, *u = nullptr, *u2 = nullptr;
    // mixed precision copies
    float *f32 = nullptr, *u32 = nullptr, *u2_32 = nullptr;
    float *inv32 = nullptr, *ef32 = nullptr, *cpf32 = nullptr;
    float4 *g32 = nullptr;
    float *area32 = nullptr;
};

struct Scalars {            // PCG scalars kept in device memory
    double rz;              // <r, z> of the current iteration
    double pq;              // <p, A p>
    double alpha, beta;
    double rr;              // ||r||^2
    double rr0;             // ||r_0||^2
    double rz_new;
    int flag;               // bit 0: p.Ap <= 0 or non-finite; bit 1: non-finite residual
    int pad;
};

// kernels.cu launchers ------------------------------------------------------
struct Launch {
    cudaStream_t s;
    int n_r;
    int sm_count;
};

enum PassMode { PASS_NORMAL = 0, PASS_ZERO = 1, PASS_PROLONG = 2 };

cudaError_t launch_apply(const Launch &L, const LevelDev &lv, const VertDev &v, const double *x, double *y,
                         double *partials, int n_part);
cudaError_t launch_residual(const Launch &L, const LevelDev &lv, const VertDev &v, const double *f,
                            const double *u, double *r, double *partials, int n_part);
cudaError_t launch_resid_restrict(const Launch &L, const LevelDev &fine, const LevelDev &coarse, const VertDev &v,
                                  const double *f, const double *u, double *fc);
cudaError_t launch_mcsor_pass(const Launch &L, const LevelDev &lv, const VertDev &v, int colour, int mode,
                              double relax, const double *f, double *u, const double *uc);
cudaError_t launch_jacobi(const Launch &L, const LevelDev &lv, const VertDev &v, int mode, double relax,
                          const double *f, const double *u_in, double *u_out, const double *uc);
cudaError_t launch_prolong_add(const Launch &L, const LevelDev &fine, const double *uc, double *u);
cudaError_t launch_thomas_factors(const Launch &L, const LevelDev &lv, const VertDev &v);
cudaError_t launch_dot(const Launch &L, long n, const double *a, const double *b, double *partials, int n_part);
cudaError_t launch_finish(const Launch &L, int what, const double *partials, int n_part, Scalars *sc);
cudaError_t launch_axpy_pair(const Launch &L, long n, const Scalars *sc, const double *p, const double *q, double *u,
                             double *r, double *partials, int n_part);
cudaError_t launch_xpby(const Launch &L, long n, const Scalars *sc, const double *z, double *p);

// noalloc.cu: device address of the fixed scratch array of
// tpmg_vcycle_noalloc on `device`, which must be the current device (looked
// up once per device).
cudaError_t noalloc_scratch(int device, double **ptr);

enum FinishWhat { FIN_RR0 = 0, FIN_ALPHA = 1, FIN_RR = 2, FIN_BETA = 3, FIN_RZ0 = 4 };

}  // namespace tpmg
