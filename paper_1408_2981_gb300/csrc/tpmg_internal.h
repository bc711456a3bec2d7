// Internal declarations of the TPMG library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include <string>
#include <vector>

#include "../../include/tpmg.h"
#include "../../include/tpmg_learned.h"

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
// One coarse cell seen from the residual restriction of the factorised operator
// (k_restrict_fac).  Summed over the cell's 4 children, the horizontal fluxes across
// the 3 edges between children cancel (each edge's weight is stored once for both
// sides), so only the 6 edges from a child to a cell outside the coarse cell remain.
struct alignas(32) RestrictGeo {
    int4 x0, x1;   // the outside cells of those 6 edges (x1.z = x1.w = 0, with weight 0)
    dbl4 g0, g1;   // the edges' weights g_e (times the edge's alpha_S factor)
    dbl4 gext;     // per child j: the sum of the weights of its outside edges
    dbl4 A, Ar;    // per child j: |T_j| beta^S_T, |T_j| alpha_r^S_T
};
struct alignas(8) bf16x4 {   // four bfloat16 values (raw bits), one 8-byte load
    unsigned short x, y, z, w;
};
struct VertDev {            // vertical factors shared by every level (no vertical coarsening)
    const double *vol;      // [n_r]   v_k = (r_{k+1}^3 - r_k^3)/3
    const double *w;        // [n_r+1] omega^2 sigma_k 2 r_k^2 / (r_{k+1} - r_{k-1})
    const double *hr;       // [n_r]   omega^2 (r_{k+1} - r_k)
    const float *ivol32;    // [n_r]   1 / v_k (network features of the learned form)
    // vertical advection (factorised form): X_face = |T| xi^S_T wx_face with
    // wx_face = omega^2 sigma r_face^2 / (r_face+1 - r_face-1) xi^r_face; row k takes
    // xm_k = dr_k wx_k (face k) and xp_k = dr_k wx_{k+1} (face k+1)
    const double *xm;       // [n_r]
    const double *xp;       // [n_r]
    const double *dr;       // [n_r]   r_{k+1} - r_k (rows of a per-face X stored per cell)
    const float *dr32;      // [n_r]
};

// Line relaxation works on tasks of kRelaxCols columns of one colour (the
// cells of a colour in ascending order, padded with -1 to whole tasks).  The
// column blocks A_T are factorised from both ends (twisted factorisation):
// rows 0..jmid-1 from the top, rows n_r-1..jmid+1 from the bottom, meeting in
// row jmid.  Factors are stored per task as [step][lane] with lane = column +
// 16 * half, so that the serial phase reads 32 consecutive doubles per step.
constexpr int kRelaxCols = 16;

// Kernel variants of a relaxation pass (chosen per level by the autotuner).
// FP64: one warp per 16-column task, one CTA of 64 / 128 / 256 threads per task,
// or one warp per task with 6 elements per lane in flight in the gather instead of 4.  FP32: one warp per column
// in CTAs of 1 / 2 / 4 / 8 warps (the first four variants).
enum RelaxVariant { RELAX_WARP = 0, RELAX_CTA64 = 1, RELAX_CTA128 = 2, RELAX_CTA256 = 3, RELAX_WARP_DEEP = 4,
                    RELAX_VARIANTS = 5 };
constexpr int kRelaxVariants32 = 4;

struct LevelDev {
    int n = 0;              // cells
    int ref = 0;
    int n_colours = 0;
    int n_tasks = 0;        // relaxation tasks over all colours
    int steps = 0;          // S = n_r - 1 - jmid: elimination steps of the longer half
    int jmid = 0;           // meeting row (n_r - 1) / 2
    int relax_variant = -1; // RELAX_* chosen by the autotuner, -1 = heuristic
    float relax_us[RELAX_VARIANTS] = {};   // autotuner timings of the level's largest pass
    std::vector<int> colour_task_off;  // [n_colours+1] first task of each colour (host copy)
    std::vector<int> colour_cells;     // [n_colours] cells of each colour (host copy)
    int4 *nbr = nullptr;          // [n] {nbr0, nbr1, nbr2, lower-colour mask}
    dbl4 *g = nullptr;            // [n] {g0, g1, g2, g0+g1+g2}
    double *area = nullptr;       // [n] |T| beta^S_T (factor of the beta term)
    double *area_r = nullptr;     // [n] |T| alpha_r^S_T (factor of the vertical couplings)
    // finest level with general profiles (tpmg_set_outer_profiles): the problem's operator
    // per unknown, cfull [n][n_r] {alphaS_hat e = 0, 1, 2, beta_hat}, cvr [n][n_r+1] alphar_hat
    dbl4 *cfull = nullptr;
    double *cvr = nullptr;
    // the FP64 V-cycle's stencil stored per unknown (coeff_storage FULL: vc and vcr;
    // PARTIAL: vcr only), the same layout as cfull / cvr
    dbl4 *vc = nullptr;
    double *vcr = nullptr;
    // vertical advection: area_x [n] |T| xi^S_T (factorised form), or null; vcx
    // [n][n_r+1] X per face stored per column (FULL storage), used while vcx_on;
    // cvx [n][n_r+1] X of the outer operator's general profiles (finest level), or null
    double *area_x = nullptr;
    double *vcx = nullptr;
    bool vcx_on = false;
    double *cvx = nullptr;
    // mixed precision: X of face k in BF16 per unknown [n][n_r], used while cxv_on
    unsigned short *cxv = nullptr;
    bool cxv_on = false;
    // linear prolongation to the next finer level (coarse levels only): [n][4][3] the
    // weight of child j on (u_{nbr e} - u_T), in FP64 and FP32
    double *plin = nullptr;
    float *plin32 = nullptr;
    float *iarea32 = nullptr;     // [n] 1 / |T| (network features of the learned form)
    float4 *wnb32 = nullptr;      // [n] {g0, g1, g2} / (g0 + g1 + g2), 0
    int *task_cells = nullptr;    // [n_tasks][16] cell ids, -1 = padding
    int4 *task_nbr = nullptr;     // [n_tasks][16] nbr of the task's cells (zero for padding)
    dbl4 *task_g = nullptr;       // [n_tasks][16] g of the task's cells (zero for padding)
    // twisted Thomas factors of the column blocks A_T:
    // rinv [n][n_r] (cell-major) 1 / pivot of row k (p_k above jmid, gamma at jmid, q_k below);
    // fb, fc [n_tasks][steps][32] forward / backward multipliers,
    //   top lane (row k = s):          fb = c_k/p_k,     fc = c_{k+1}/p_k
    //   bottom lane (row k = n_r-1-s): fb = c_{k+1}/q_k, fc = c_k/q_k
    // fm [n_tasks][2][16] meeting row: c_j/gamma, c_{j+1}/gamma
    double *rinv = nullptr, *fb = nullptr, *fc = nullptr, *fm = nullptr;
    // FP64 levels with at most params.scan_max_cells cells: relaxed one warp per column
    // (k_relax_scan) with one-directional factors per unknown [n][n_r]:
    // rinv1 = 1 / p_k, fb1 = c_k / p_k, fc1 = c_{k+1} / p_k.  On larger levels a colour
    // pass of at most scan_pass_tasks tasks (a small colour of the colouring) is relaxed
    // the same way, with the factors held for the whole level; -1: none
    bool scan = false;
    int scan_pass_tasks = -1;
    // finest level, factorised operator without advection: per-row products of its
    // coefficients [n][n_r], om = |T| v_k + hr_k G_T (the row's excess) and
    // oc = |T| alpha_r^S w_k (the coupling through the row's lower face), so that the
    // outer operator costs 8 FP64 operations a row instead of 11; null if they did not fit
    double *om = nullptr, *oc = nullptr;
    // with them where they fit, the horizontal couplings per unknown, three planes [3][n][n_r]
    // ocs_e = hr_k g_e, so that the outer operator's horizontal part costs 3 FMAs a row
    double *ocs = nullptr;
    // FP64 levels with a coarser level below them: the restriction's view of each
    // coarse cell [n / 4], or null (then the kernel forms every child's residual)
    RestrictGeo *rgeo = nullptr;
    double *rinv1 = nullptr, *fb1 = nullptr, *fc1 = nullptr;
    // FP64 levels relaxed by twisted tasks, factorised stencil (params.scaled_rhs, where
    // they fit): the horizontal couplings scaled by the pivots, three planes [3][n][n_r]
    // cs_e = hr_k g_e rinv, and the work vector ft [n][n_r] = f rinv, written by the
    // first pass over each colour in a visit of the level and read by the later ones
    double *cs = nullptr, *ft = nullptr;
    // workspaces (coarse levels; the finest level uses caller / PCG buffers)
    double *f = nullptr, *u = nullptr, *u2 = nullptr;
    // mixed-precision form: the stencil stored per unknown in BF16 (full
    // storage, Sec. 4.2) and FP32 work vectors on every level
    bf16x4 *cpack = nullptr;        // [n][n_r] {alphaS_hat e = 0, 1, 2, beta_hat}
    unsigned short *cvert = nullptr;   // [n][n_r] alphar_hat of face k (coupling to level k-1; 0 for k = 0),
                                       // followed by one 0 (face n_r of the last column)
    // Thomas factors of the BF16 column blocks in FP32, per unknown [n][n_r] (bottom-up
    // elimination): rinv32 = 1 / p_k; with vertical advection also the multipliers
    // fb32 = c_k / p_k, fc32 = c_{k+1} / p_k (allocated with the advection; without it
    // the relaxation forms them from cvert and rinv32)
    float *rinv32 = nullptr, *fb32 = nullptr, *fc32 = nullptr;
    float *f32 = nullptr, *u32 = nullptr, *u2_32 = nullptr;
};

struct Scalars {            // PCG scalars kept in device memory
    double rz;              // <r, z> of the current iteration
    double pq;              // <p, A p>
    double alpha, beta;
    double rr;              // ||r||^2
    double rr0;             // ||r_0||^2
    double rz_new;
    double rzc;             // <r_{k+1}, z_k> (flexible CG)
    int flag;               // bit 0: p.Ap <= 0 or non-finite; bit 1: non-finite residual
    int it;                 // iterations done by the device-side loop
    double ff;              // ||f||^2 (learned solve: the stop test is relative to ||f||)
    double sum;             // FIN_SUM: a reduced dot product for the host-driven outer loops
    int info;               // learned solve: bit 0 initial guess kept, bit 1 rejected (u_0 = 0)
};

// Control of a PCG loop that runs on the device (a CUDA graph with a
// conditional WHILE node): the finish kernels record the residual history,
// count the iterations and set the loop condition.
struct LoopCtl {
    cudaGraphConditionalHandle cond;   // 0: host-driven loop
    double rtol;                       // stop when sqrt(||r||^2 / ||r_0||^2) <= rtol (as the host loop)
    int max_iter;
    double *hist;                      // [max_iter + 1] ||r_k|| / ||r_0|| (device), or NULL
    int *go = nullptr;                 // member of a batched solve: the decision goes here, not to cond
};

// ---------------------------------------------------------------------------
// Batched form (tpmg_batch with the work-list schedule): one launch per step of the
// V-cycle covers that step's passes of every member, each pass an item of the
// launch's work list; the outer Krylov kernels loop over the members' virtual blocks.
// ---------------------------------------------------------------------------
constexpr int kBatchItems = 64;   // items per launch (two ballots of the lanes' entries)

struct BatchRelaxItem {     // one member's colour pass (or Jacobi sweep) of the FP32 V-cycle
    const int *cells;       // the level's task cell lists; the pass covers slots [slot0, slot0 + n_slots)
    const int4 *tnb;
    const bf16x4 *cpack;
    const unsigned short *cvert;
    const float *rinv;
    const void *f;          // double (the member's finest level) or float
    const float *u_in;
    float *u_out, *u_fine;  // u_fine: the next finer level's iterate (fused prolongation), or null
    double *out64;          // the member's z on its finest level's last pass, or null
    int n_r, slot0, n_slots, member;
    float relax;
};

struct BatchRestrictItem {  // one member's FP32 residual + restriction
    const int4 *nbr;
    const bf16x4 *cpack;
    const unsigned short *cvert;
    const void *f;          // double (finest level) or float
    const float *u;
    float *fc;
    int n_r, Nc, member;
};

// The work list of one launch, passed by value as the kernel's parameter (read through
// the constant cache): items [n_items] with their first warps / positions.  CAP is the
// capacity of the launch's parameter block: the smallest of 2, 8 and kBatchItems that
// holds its items, since a launch's cost grows with the size of its parameters.
template <int CAP>
struct RelaxBatchArgsT {
    int n_items;
    int off[CAP];           // first warp of each item (ascending, off[0] = 0)
    BatchRelaxItem items[CAP];
};
template <int CAP>
struct RestrictBatchArgsT {
    int n_items;
    int off[CAP];           // first position of each item (multiples of 32, ascending, off[0] = 0)
    BatchRestrictItem items[CAP];
};
using RelaxBatchArgs = RelaxBatchArgsT<kBatchItems>;
using RestrictBatchArgs = RestrictBatchArgsT<kBatchItems>;

struct BatchMemberDev {     // one member's outer FP64 iteration (finest level, factorised operator)
    const int4 *nbr;
    const dbl4 *g;
    const double *area, *area_r, *om, *oc, *ocs;
    const double *vol, *w, *hr;
    int n_r, N;
    const double *f;
    double *u, *r, *z, *p, *q;
    float *r32;             // r in FP32: the right-hand side of the finest level's V-cycle passes
    double *partials;       // [2 n_part]
    int *zflags;            // [n_part]
    Scalars *sc;
    double *hist;           // [kHistCap]
    double rtol;
    int max_iter;
};

// kernels.cu launchers ------------------------------------------------------
struct Launch {
    cudaStream_t s;
    int n_r;
    int sm_count;
    const double *dr = nullptr;    // [n_r] r_{k+1} - r_k (mixed precision: advection rows)
    const float *dr32 = nullptr;
    bool pdl = false;              // launch with programmatic stream serialisation (launch_k)
};

#ifdef __CUDACC__
// Programmatic dependent launch.  A kernel launched by launch_k with L.pdl set
// may be scheduled while its predecessor in the stream is still running, so
// that its launch and its reads of set-up data overlap the predecessor's tail.
// Every such kernel calls pdl_wait() before it touches memory that an earlier
// launch writes or reads; the wait returns once the predecessor has completed
// and its writes are visible (at once for a kernel launched without the
// attribute).  Since every kernel of the chain waits, the memory effects keep
// the order of plain launches and the results are bit-identical.
// pdl_trigger() lets the successor be scheduled; each kernel issues it right
// after its wait, so at most one launch runs ahead.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_k(const Launch &L, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, Args... args)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = L.s;
    cfg.attrs = at;
    cfg.numAttrs = L.pdl ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    const cudaError_t last = cudaGetLastError();
    return e != cudaSuccess ? e : last;
}
#endif

// Right-hand side of a relaxation pass: NORMAL f + sum of all neighbours;
// ZERO (first forward sweep from a zero guess) only neighbours of a smaller
// colour (mask bits); RHS_ONLY f alone (colour 0 of a ZERO sweep, Jacobi ZERO).
enum PassMode { PASS_NORMAL = 0, PASS_ZERO = 1, PASS_RHS_ONLY = 2 };

cudaError_t launch_apply(const Launch &L, const LevelDev &lv, const VertDev &v, const double *x, double *y,
                         double *partials, int n_part);
// nz (optional): per-block flags of launch_nonzero over u, n_part of them
// r32 (optional): r also in FP32 (the mixed V-cycle's copy of the outer residual)
cudaError_t launch_residual(const Launch &L, const LevelDev &lv, const VertDev &v, const double *f,
                            const double *u, double *r, double *partials, int n_part, const int *nz = nullptr,
                            float *r32 = nullptr);
cudaError_t launch_nonzero(const Launch &L, long n, const double *x, int *nz, int n_blocks);
cudaError_t launch_resid_restrict(const Launch &L, const LevelDev &fine, const LevelDev &coarse, const VertDev &v,
                                  const double *f, const double *u, double *fc);
// One relaxation pass over tasks [task0, task0 + n_tasks) of level lv:
// u_out_T = (1 - relax) u_in_T + relax A_T^{-1} (f_T + sum_T' alphaS_hat u_in_T').
// If u_fine is not NULL the new values are also added to the 4 children of
// each cell in u_fine (prolongation P = R^T of Algorithm 1, fused into the
// last pass that writes a colour).
// ft_mode (levels with scaled couplings): 1 the pass is the first over its columns in
// this visit of the level and writes their f / pivot into lv.ft; 2 it reads lv.ft;
// 0 the factorised form.  Colours relaxed by the warp scans always read f.
cudaError_t launch_relax(const Launch &L, const LevelDev &lv, const VertDev &v, int mode, int task0, int n_tasks,
                         double relax, const double *f, const double *u_in, double *u_out, double *u_fine,
                         int ft_mode = 0);
// cs of a level from its pivots (rinv): after launch_twisted_factors, which also calls it
cudaError_t launch_scaled_couplings(const Launch &L, const LevelDev &lv, const VertDev &v);
cudaError_t launch_prolong_add(const Launch &L, const LevelDev &fine, const double *uc, double *u);
cudaError_t launch_prolong_linear(const Launch &L, const LevelDev &fine, const LevelDev &coarse, const double *uc,
                                  double *u);
cudaError_t launch_twisted_factors(const Launch &L, const LevelDev &lv, const VertDev &v);
cudaError_t launch_outer_products(const Launch &L, const LevelDev &lv, const VertDev &v);
cudaError_t launch_thomas_factors(const Launch &L, const LevelDev &lv, const VertDev &v);
// Mixed-precision V-cycle (FP32 arithmetic, BF16 stencil).  TF is the type of
// the right-hand side (double on the finest level, float below).
template <typename TF>
cudaError_t launch_relax32(const Launch &L, const LevelDev &lv, int mode, int task0, int n_tasks, float relax,
                           const TF *f, const float *u_in, float *u_out, float *u_fine, double *out64);
template <typename TF>
cudaError_t launch_resid_restrict32(const Launch &L, const LevelDev &fine, const LevelDev &coarse, const TF *f,
                                    const float *u, float *fc);
cudaError_t launch_prolong_add32(const Launch &L, const LevelDev &fine, const float *uc, float *u);
cudaError_t launch_prolong_linear32(const Launch &L, const LevelDev &fine, const LevelDev &coarse, const float *uc,
                                    float *u);
cudaError_t launch_to_f64(const Launch &L, long n, const float *x, double *y);
cudaError_t launch_thomas_factors32(const Launch &L, const LevelDev &lv);
cudaError_t launch_dot(const Launch &L, long n, const double *a, const double *b, double *partials, int n_part);
cudaError_t launch_finish(const Launch &L, int what, const double *partials, int n_part, Scalars *sc,
                          const LoopCtl *loop = nullptr);
// z_old != NULL (flexible CG): also partials of <r_new, z_old> in partials[n_part..2 n_part)
cudaError_t launch_axpy_pair(const Launch &L, long n, const Scalars *sc, const double *p, const double *q, double *u,
                             double *r, double *partials, int n_part, const double *z_old, float *r32 = nullptr);
cudaError_t launch_xpby(const Launch &L, long n, const Scalars *sc, const double *z, double *p);
// out = a x + b y + c z (y, z nullable: terms dropped); out may alias x, y or z elementwise
cudaError_t launch_lincomb(const Launch &L, long n, double a, const double *x, double b, const double *y, double c,
                           const double *z, double *out);

// Batched form.  Relaxation: one launch per (mode, right-hand-side type, rows per lane)
// over args.n_items <= kBatchItems items, total_warps the sum of their slots, wpb warps
// per CTA.  Restriction: total the end of the last item's range of positions.
template <typename TF>
cudaError_t launch_relax32_batch(const Launch &L, int mode, int n_r_max, const RelaxBatchArgs &args, long total_warps,
                                 int wpb, const int *active);
template <typename TF>
cudaError_t launch_restrict32_batch(const Launch &L, const RestrictBatchArgs &args, long total, const int *active);
// The outer kernels over the M members (each member's n_part virtual blocks, skipped
// where active[m] == 0).  what: BATCH_* below; finish: FIN_* with the members' loop
// decisions written to go[m].
enum BatchOuter { BATCH_NONZERO = 0, BATCH_RESIDUAL = 1, BATCH_DOT_RZ = 2, BATCH_XPBY = 3, BATCH_APPLY = 4,
                  BATCH_AXPY = 5, BATCH_CLEAR_P = 6 };
cudaError_t launch_outer_batch(const Launch &L, int what, const BatchMemberDev *mem, int M, int n_part,
                               const int *active);
cudaError_t launch_finish_batch(const Launch &L, int what, const BatchMemberDev *mem, int M, int n_part,
                                const int *active, int *go, int partial_offset);
// active[m] = go[m] for every member, and the batch loop's condition = any member active
cudaError_t launch_batch_continue(const Launch &L, int M, const int *go, int *active, cudaGraphConditionalHandle cond);

// noalloc.cu: device address of the fixed scratch array of
// tpmg_vcycle_noalloc on `device`, which must be the current device (looked
// up once per device).
cudaError_t noalloc_scratch(int device, double **ptr);

enum FinishWhat { FIN_RR0 = 0, FIN_ALPHA = 1, FIN_RR = 2, FIN_BETA = 3, FIN_RZ0 = 4, FIN_RZC = 5, FIN_BETA_PR = 6,
                  // device-side loop: RR0 and RR also drive the loop condition; BETA and
                  // BETA_PR give beta = 0 on the first pass (p is cleared before the loop)
                  FIN_LOOP_RR0 = 7, FIN_LOOP_RR = 8, FIN_LOOP_BETA = 9, FIN_LOOP_BETA_PR = 10,
                  // learned solve: partials [0, n) of ||r_0||^2 and [n, 2n) of ||f||^2; the
                  // initial guess is rejected unless ||r_0|| < ||f||; rr0 = ||f||^2
                  FIN_LOOP_RR0F = 11,
                  // the same for the host-driven loop (no loop condition)
                  FIN_RR0F = 12,
                  // Richardson / BiCGStab: the reduced dot product into sum
                  FIN_SUM = 13 };

// learned.cu: the network of the learned form (tpmg_learned.h) -----------------
struct NetView {            // device pointers of a network's weights
    int sizes[5];           // 2 n_r, h, h, h, n_r
    const uint16_t *w[4];   // bfloat16 W_l [sizes[l+1]][sizes[l]]
    const float *b[4];      // FP32 b_l
};
NetView net_view(const tpmg_net *net);
// y [rows][sizes[l+1]] = act(x W_l^T + b_l), ReLU for l < 3
cudaError_t launch_net_layer(cudaStream_t s, const NetView &v, int l, const float *x, long rows, float *y);
// the whole network in one tensor-core kernel (hidden width 64, n_r % 8 == 0):
// out [rows][n_r] = s * network(X), activations rounded to bfloat16 between layers
bool net_fused_ok(const NetView &v);
// the same network on tcgen05 (tiles of 128 columns, FP32 accumulators in tensor memory;
// n_r a multiple of 16, at most 128), from the inputs of launch_net_features_tiled
// (bfloat16 in the kernel's tile layout, net_tc_input_elems of them); *err set if a
// CTA gave up waiting (its outputs NaN)
bool net_tc_ok(const NetView &v);
size_t net_tc_input_elems(long rows, int n_r);
cudaError_t launch_net_features_tiled(const Launch &L, const LevelDev &lv, const float *p, long rows,
                                      const double *s, uint16_t *Xt);
template <typename TO>
cudaError_t launch_net_tc(const Launch &L, const NetView &v, const uint16_t *Xt, long rows, const double *s, TO *out,
                          int *err);
template <typename TO>
cudaError_t launch_net_fused(const Launch &L, const NetView &v, const float *X, long rows, const double *s, TO *out);
// p = f / (|T| v_k) in FP32 (level size) and partials [n_part] of sum p^2; the finish writes s.
// f32 (optional): f in FP32 as well (the conversion the kernel makes anyway)
template <typename TF>
cudaError_t launch_net_prepare(const Launch &L, const LevelDev &lv, const VertDev &vert, const TF *f, float *p,
                               double *partials, int n_part, float *f32 = nullptr);
cudaError_t launch_net_scale_finish(const Launch &L, const LevelDev &lv, const double *partials, int n_part, double *s);
// X [rows][2 n_r] network inputs from the point values p of the level (cells NULL: rows 0..rows-1)
cudaError_t launch_net_features(const Launch &L, const LevelDev &lv, const float *p, const int *cells, long rows,
                                const double *s, float *X);
cudaError_t launch_net_targets(const Launch &L, const double *u, const int *cells, long rows, const double *s, float *t);
template <typename TO>
cudaError_t launch_net_output(const Launch &L, const float *y, long n, const double *s, TO *u);
cudaError_t launch_judge_reset(const Launch &L, const Scalars *sc, long n, const double *f, double *u, double *r,
                               float *r32 = nullptr);
cudaError_t launch_to_f32(const Launch &L, long n, const double *x, float *y);

}  // namespace tpmg
