/*
 * tpmg.h -- C ABI of the GB300 tensor-product multigrid (TPMG) library.
 *
 * Solves the pressure-correction equation of Dedner, Mueller & Scheichl,
 * "Efficient multigrid preconditioners for atmospheric flow simulations at
 * high aspect ratio" (arXiv:1408.2981), Sec. 2 eq. HelmholtzVector with
 * constant profiles (alpha_r = alpha_S = beta = 1, xi_r = 0):
 *
 *     -omega^2 div grad u + u = f      in  S^2 x [1, 1+H],
 *     du/dr = 0 at r = 1 and r = 1 + H,
 *
 * discretised by the cell-centred finite volumes of Appendix A on an
 * icosahedral grid (Sec. 4.1-4.2) times a graded vertical column, with
 * preconditioned conjugate gradients whose preconditioner is one TPMG V-cycle
 * (Algorithm 1): vertical line (column tridiagonal) relaxation, eq. BlockJacobi,
 * and horizontal-only coarsening.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Field vectors are double arrays of length n_cells * n_r in the library's
 * cell order (cell T of refinement level L, children of a coarse cell T are
 * 4T..4T+3) with the vertical index k fastest: element (T, k) at T*n_r + k.
 * A right-hand side holds cell integrals (Sec. 5), i.e. the finite-volume
 * discretisation of the source times the cell volume |T| v_k.
 *
 * Pointers named d_* are DEVICE pointers on the current CUDA device (for
 * example the data pointer of a float64 torch tensor); h_* are HOST pointers.
 * The caller owns every buffer it passes and keeps it alive until the work
 * on the context's stream that uses it has completed; the library never
 * frees caller memory.  The library owns every internal workspace: all of it
 * is allocated by tpmg_setup and released by tpmg_destroy.
 *
 * All device work is ordered on the stream given to tpmg_setup.
 * tpmg_apply_operator and tpmg_vcycle are asynchronous; tpmg_solve,
 * tpmg_solve_host and tpmg_solve_host_many return after their solves have
 * finished.
 *
 * Errors are returned as tpmg_status values; no C++ exception crosses this
 * interface.  A context is not thread-safe: one thread at a time per context.
 * tpmg_last_error gives a human-readable message for the last failed call.
 */
#ifndef TPMG_H
#define TPMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tpmg_ctx tpmg_ctx;

typedef enum {
    TPMG_OK = 0,
    TPMG_ERR_INVALID_ARG = 1,   /* a parameter or pointer was rejected; nothing was launched */
    TPMG_ERR_CUDA = 2,          /* a CUDA runtime call failed; see tpmg_last_error */
    TPMG_ERR_OOM = 3,           /* device memory allocation failed in tpmg_setup */
    TPMG_ERR_NOT_CONVERGED = 4, /* tpmg_solve used max_iter iterations without reaching rtol */
    TPMG_ERR_BREAKDOWN = 5      /* p.Ap <= 0 or a non-finite residual (not SPD, or NaN/Inf input) */
} tpmg_status;

/* Block relaxation of eq. BlockJacobi: u_T <- u_T + relax A_T^{-1} (f - A u)_T. */
enum { TPMG_SMOOTH_MCSOR = 0,   /* multicolour block-SOR: forward colours before, reverse after the correction */
       TPMG_SMOOTH_JACOBI = 1 }; /* weighted block-Jacobi */

/* Storage of the V-cycle's stencil (Sec. 4.2):
 *   FACTORISED: recomputed on the fly from O(n_r + n_cells) factorised FP64 data
 *     (TPMG^otimes, TPMG^fac);
 *   FULL: stored per unknown (TPMG^full) -- in FP64 for the FP64 V-cycle (40 bytes
 *     per unknown and level), in BF16 for the mixed-precision V-cycle;
 *   PARTIAL (FP64 only): alpha_r stored per face and column, beta and alpha_S
 *     factorised (the partial factorisation TPMG^partial of Sec. 5.3; 8 bytes per
 *     unknown and level).
 * Until tpmg_set_outer_profiles gives general profiles, FULL and PARTIAL store the
 * factorised profiles' coefficients, so all three are the same preconditioner up to
 * rounding.  The outer operator of tpmg_solve and tpmg_apply_operator is the exact
 * factorised FP64 one, or the general one of tpmg_set_outer_profiles. */
enum { TPMG_COEFF_FACTORISED = 0, TPMG_COEFF_FULL = 1, TPMG_COEFF_PARTIAL = 2 };

/* Outer iteration of tpmg_solve (Sec. 5 uses Richardson and BiCGStab; with constant
 * profiles the operator and the V-cycle are symmetric positive definite, so CG applies). */
enum { TPMG_OUTER_CG = 0,          /* preconditioned CG (flexible CG in the mixed-precision form) */
       TPMG_OUTER_RICHARDSON = 1,  /* u <- u + B (f - A u) */
       TPMG_OUTER_BICGSTAB = 2 };  /* BiCGStab, preconditioned from the right (2 V-cycles per iteration) */

/* Prolongation of the V-cycle (Algorithm 1's correction u_h += P u_2h).  The restriction
 * is always the sum over the 4 children (Sec. 5).
 *   CONSTANT: each child takes its parent's value, P = R^T, which keeps B symmetric for CG;
 *   LINEAR:   linear interpolation, the paper's own choice (Sec. 5): the coarse field is
 *             linear in the plane tangent to the sphere at the parent's centre, with the
 *             least-squares gradient of the differences to its 3 neighbours, and each child
 *             takes its value at the child's centre.  B is then not symmetric: tpmg_solve
 *             needs params.outer Richardson or BiCGStab. */
enum { TPMG_PROLONG_CONSTANT = 0, TPMG_PROLONG_LINEAR = 1 };

/* Cell centre used by the two-point flux of Appendix A. */
enum { TPMG_CENTRE_CIRCUM = 0,      /* spherical circumcentre (centre chord normal to the edge) */
       TPMG_CENTRE_VERTEX_MEAN = 1 };

/* Arithmetic of the V-cycle.  FP64: everything in double (any TPMG_COEFF_*).
 * MIXED (requires TPMG_COEFF_FULL): the V-cycle
 * (operator, line smoother, transfers) in FP32 on the BF16 stencil, with the
 * column factors precomputed per level in FP32; the outer Krylov vectors,
 * residual, dot products and updates in FP64.  Because the FP32 V-cycle is not
 * exactly symmetric, tpmg_solve then runs flexible CG (Polak-Ribiere
 * coefficient), which reaches the FP64 solution to the requested tolerance. */
enum { TPMG_PREC_FP64 = 0, TPMG_PREC_MIXED = 1 };

typedef struct {
    int    refinement;   /* fine icosahedral level L >= 0: n_cells = 20 * 4^L (L <= 9) */
    int    n_levels;     /* multigrid levels, 1 .. L+1 (level 0 coarsest = refinement L-n_levels+1) */
    int    n_r;          /* vertical cells, 1 .. 1024 */
    double H;            /* shell depth over the sphere radius, e.g. 10/6371 (> 0) */
    double grading;      /* geometric ratio dr_{k+1}/dr_k, finest at k = 0; 1.0 = uniform (> 0) */
    double omega2;       /* omega^2 in unit-sphere units; if <= 0, omega^2 = courant_c * h_min^2,
                            h_min = smallest distance between neighbouring fine-level centres */
    double courant_c;    /* Courant-type ratio omega^2 / h_min^2 used when omega2 <= 0 */
    int    nu_pre;       /* pre-smoothing sweeps on levels > 0 (>= 0) */
    int    nu_post;      /* post-smoothing sweeps on levels > 0 (>= 0; = nu_pre for a symmetric B) */
    int    nu_coarse;    /* symmetric sweeps on the coarsest level (>= 0) */
    int    smoother;     /* TPMG_SMOOTH_* */
    double relax;        /* relaxation factor rho_relax (0 < relax < 2) */
    int    coeff_storage;/* TPMG_COEFF_* */
    int    centre;       /* TPMG_CENTRE_* */
    int    precision;    /* TPMG_PREC_* */
    int    graphs;       /* 1: tpmg_solve runs as one CUDA graph launch with its loop on the device
                            (captured at the first solve with given vectors); 0: kernel by kernel
                            from a host loop.  The results are identical. */
    int    autotune;     /* 1: tpmg_setup times the relaxation kernel variants on every level and
                            keeps the fastest (see tpmg_query_tuning); 0: a fixed heuristic.  The
                            results are identical. */
    int    scan_max_cells; /* FP64 V-cycle: levels with at most this many cells relax one warp per
                            column with the Thomas recurrences as warp scans (short latency, more
                            FP64 work); larger levels use the 16-column twisted-factorisation tasks,
                            except for their colours of at most scan_max_cells / 2 cells, which
                            are relaxed by the warp scans too.  A fixed rule, so the results do
                            not depend on timings (>= 0). */
    int    outer;        /* TPMG_OUTER_*: the outer iteration of tpmg_solve.  Richardson and
                            BiCGStab run their loop from the host (one read-back per dot product)
                            and are not available in a batch. */
    int    prolongation; /* TPMG_PROLONG_*: the V-cycle's coarse-to-fine transfer */
    int    pdl;          /* 1: the kernels of the V-cycle and of the outer loop are launched with
                            programmatic dependent launch, so each one is scheduled, and reads its
                            set-up data, while its predecessor in the stream finishes; every kernel
                            still waits for its predecessor's results.  The FP64 relaxation of
                            levels above scan_max_cells (16-column twisted tasks) is launched
                            plainly, where programmatic launch measured slower.  0: plain
                            launches.  The results are identical. */
    int    relax_variant;/* -1: the autotuner's (or the heuristic's) relaxation kernel per level;
                            0..4 (mixed precision 0..3): that variant of tpmg_query_tuning on every
                            level (variant 4 on a warp-scan level: its default CTA shape).  The
                            results are identical. */
    int    scaled_rhs;   /* FP64 V-cycle, factorised stencil: 1 (default) the levels relaxed by
                            twisted tasks keep their horizontal couplings divided by the pivots,
                            hr_k g_e / p_k, per unknown (24 bytes), and the relaxation writes
                            f / p_k once per colour and visit of a level, so that a pass forms its
                            right-hand side in 3 FP64 operations a row instead of 5 (allocated
                            only where they fit; otherwise the factorised form).  0: the
                            factorised form.  Equal in exact arithmetic; the rounding differs by
                            a few ulp of the right-hand side. */
    int    net_tcgen05;  /* learned form (tpmg_learned.h), hidden width 64 and n_r a multiple of 16
                            up to 128: 1 (default) the network runs as one tcgen05 kernel (MMAs
                            from shared memory into tensor memory), 0 as one mma.sync kernel.
                            Both round inputs and activations to bfloat16 and accumulate in FP32;
                            the accumulation order differs. */
} tpmg_params;

/* Fills *p with the defaults: refinement 3, n_levels 4, n_r 16, H = 10/6371,
 * grading 1, omega2 0 with courant_c 8, nu 2/2/1, block-SOR with relax 1,
 * factorised storage, circumcentres, FP64, graphs and autotuning on,
 * scan_max_cells 5120, outer CG, constant prolongation, programmatic launch, relax_variant -1,
 * scaled_rhs 1, net_tcgen05 1.
 * Returns TPMG_ERR_INVALID_ARG if p is NULL. */
tpmg_status tpmg_default_params(tpmg_params *p);

/* Factorised profiles (Sec. 2, eq. profiles): alpha_r(r, x) = alpha_r^r(r) alpha_r^S(x),
 * alpha_S(r, x) = alpha_S^r(r) alpha_S^S(x), beta(r, x) = beta^r(r) beta^S(x), the form
 * the tensor-product V-cycle handles exactly.  Host arrays, positive and finite; a
 * NULL array is the constant 1.
 *   beta_r, alphaS_r  [n_r]      vertical factors at the cell centres (level k)
 *   alphar_r          [n_r + 1]  vertical factor at the faces (face k between levels k-1, k)
 *   beta_s, alphar_s, alphaS_s   [20 * 4^refinement] horizontal factors on the cells of
 *                                the finest level, in the library's cell order
 * Coarse multigrid levels use the area-weighted mean of each cell's 4 children; an
 * edge uses the mean of its two cells' alphaS_s, so the operator stays symmetric.
 *   xi_r [n_r + 1], xi_s [20 * 4^refinement]  vertical advection xi_r(r, x) = xi_r^r(r)
 *                                xi_r^S(x) at the faces (finite, any sign); both NULL =
 *                                no advection, one NULL = that factor 1.
 * Vertical advection (the -omega^2 xi_r d_r u term of eq. HelmholtzVector, centred as in
 * Appendix A) makes the operator non-symmetric: row k of a column couples to the row
 * below with down_k = alphar_hat_k - dr_k X_k and to the row above with up_k =
 * alphar_hat_{k+1} + dr_k X_{k+1}, X_face = omega^2 |T| r_face^2 / (r_{face+1} -
 * r_{face-1}) xi_face.  tpmg_setup rejects profiles for which a coupling of a V-cycle
 * level is negative (the column blocks must stay M-matrices for the line smoother's
 * elimination), and tpmg_solve then needs params.outer Richardson or BiCGStab. */
typedef struct {
    const double *beta_r;
    const double *alphaS_r;
    const double *alphar_r;
    const double *beta_s;
    const double *alphar_s;
    const double *alphaS_s;
    const double *xi_r;
    const double *xi_s;
} tpmg_profiles;

/* Builds the grid hierarchy, geometry, colouring and coefficients on the host
 * (Sec. 4.1-4.2, Appendix A), uploads them, and allocates all workspaces on the
 * current device.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).  On success *out owns everything and must be released with
 * tpmg_destroy.  Errors: INVALID_ARG (bad parameter, *out untouched),
 * OOM, CUDA. */
tpmg_status tpmg_setup(const tpmg_params *p, void *cuda_stream, tpmg_ctx **out);

/* tpmg_setup with factorised profiles (prof NULL: constant profiles, as tpmg_setup).
 * The arrays are copied.  Errors as tpmg_setup; INVALID_ARG also for a profile value
 * that is not positive and finite. */
tpmg_status tpmg_setup_profiles(const tpmg_params *p, const tpmg_profiles *prof, void *cuda_stream, tpmg_ctx **out);

/* The problem's operator with general (non-factorising) profiles on the finest level
 * (Sec. 2, eq. profiles; the TPMG^full storage of Sec. 4.2 for the operator only):
 * h_beta, h_alphaS [n_cells * n_r] at the cell centres and h_alphar [n_cells * (n_r + 1)]
 * at the faces (cell-major), host arrays, positive and finite; h_xi [n_cells * (n_r + 1)]
 * the vertical advection at the faces (finite), or NULL for none; three NULLs restore the
 * factorised operator (h_xi is then ignored).  From then on the outer iteration -- tpmg_solve, tpmg_apply_operator,
 * the learned and batched solves -- applies this operator with per-unknown FP64
 * coefficients (edges: the mean of the two cells' alpha_S).  The V-cycle follows its
 * coefficient storage (Sec. 3.2.2, Sec. 5, Sec. 5.3):
 *   FACTORISED keeps the factorised profiles given to tpmg_setup_profiles (TPMG^fac
 *     preconditioning the full operator);
 *   FULL (FP64 or mixed precision) adopts all three general profiles (TPMG^full);
 *   PARTIAL adopts alpha_r and keeps the factorised beta and alpha_S (TPMG^partial).
 * Each coarse level takes the area-weighted mean of a general profile over the 4
 * children per vertical index.  Synchronous.  Errors: INVALID_ARG, OOM, CUDA. */
tpmg_status tpmg_set_outer_profiles(tpmg_ctx *ctx, const double *h_beta, const double *h_alphar,
                                    const double *h_alphaS, const double *h_xi);

/* y = A x on the finest level (eq. ColumnEquation: matrix-free finite-volume
 * operator).  d_x, d_y: device, n_cells*n_r doubles, must not overlap.
 * Asynchronous on the context stream.  Errors: INVALID_ARG (NULL pointer), CUDA. */
tpmg_status tpmg_apply_operator(tpmg_ctx *ctx, const double *d_x, double *d_y);

/* z = B r: one V-cycle (Algorithm 1) on the finest level from a zero initial
 * guess; B is the preconditioner used inside tpmg_solve.  d_r, d_z: device,
 * n_cells*n_r doubles, must not overlap; d_r is not modified.  Asynchronous.
 * Errors: INVALID_ARG, CUDA. */
tpmg_status tpmg_vcycle(tpmg_ctx *ctx, const double *d_r, double *d_z);

/* Capacity, in doubles, of the fixed scratch array of tpmg_vcycle_noalloc
 * (2^21 doubles = 16 MiB). */
#define TPMG_VCYCLE_NOALLOC_MAX_DOUBLES (1u << 21)

/* z = B r exactly as tpmg_vcycle computes it, for callers that must not let
 * the library allocate device memory on their behalf: a host model that owns
 * the device memory through its own pool and forbids other allocations once
 * its time loop runs, or code for which the device synchronisation that
 * cudaMalloc / cudaFree can cause is not acceptable.  This call allocates
 * nothing: the work vectors of the coarse levels (the second buffer of the
 * block-Jacobi smoother, and the f / pivot vectors of levels relaxed with
 * scaled couplings, params.scaled_rhs) come from one fixed device array built into the
 * library, of TPMG_VCYCLE_NOALLOC_MAX_DOUBLES doubles, which every GPU that
 * loads the library holds until the process exits.  The context itself still
 * comes from tpmg_setup, and this call neither reads nor writes the context's
 * own work vectors.  The paper has no counterpart: this is an interface
 * convenience, not part of the method.
 *
 * d_r, d_z: device, n_cells*n_r doubles, must not overlap; d_r is not modified.
 * FP64 contexts only (TPMG_ERR_INVALID_ARG otherwise).  The context's device must be current.  Scratch needed: 2 * sum over the
 * coarse levels of n_cells_l * n_r doubles for block-SOR, plus sum over all
 * levels of n_cells_l * n_r for block Jacobi, plus n_cells_l * n_r for every
 * level relaxed with scaled couplings (each part rounded up to 32 doubles); a
 * larger problem is rejected with INVALID_ARG before anything is
 * launched.  tpmg_setup looks up the array's device address (with the
 * context's device current), so this call only reads it.  Every call on a device shares the one array and leaves
 * the last call's values in it; no element is read before the call has written
 * it, so nothing needs clearing.  Calls whose work overlaps on the GPU (other
 * streams, other contexts, other threads) race on the array: order them.
 * Asynchronous on the context stream.  Errors: INVALID_ARG, CUDA. */
tpmg_status tpmg_vcycle_noalloc(tpmg_ctx *ctx, const double *d_r, double *d_z);

/* The outer iteration params.outer (preconditioned CG by default) for A u = f
 * with B = one V-cycle.  d_u holds the initial guess on entry and the solution
 * on return.  Stops when ||r_k||_2 <= rtol * ||r_0||_2 (recursively updated
 * residual for CG and BiCGStab, the true residual for Richardson; Sec. 5 uses
 * rtol = 1e-5).  *iters counts outer iterations (BiCGStab: 2 V-cycles each).
 * *iters = number of products q = A p; *rel_resid = ||r_k|| / ||r_0||.
 * resid_hist (host, nullable, max_iter+1 doubles) receives ||r_k|| / ||r_0||
 * for k = 0..*iters.  Synchronises the context stream before returning.
 * Returns OK, NOT_CONVERGED (iters = max_iter), BREAKDOWN (p.Ap <= 0 or a
 * non-finite norm; the solution holds the last finite iterate), INVALID_ARG, CUDA.
 * With vertical advection (xi in the profiles) the operator, and with linear
 * prolongation the V-cycle, is not symmetric, and CG does not apply: INVALID_ARG unless
 * params.outer is Richardson or BiCGStab.
 * With graphs on (and no kernel class being timed) the whole solve is one graph
 * launch with the loop on the device; otherwise the host drives the loop.
 * Both run the same kernels in the same order. */
tpmg_status tpmg_solve(tpmg_ctx *ctx, const double *d_f, double *d_u, double rtol, int max_iter,
                       int *iters, double *rel_resid, double *resid_hist);

/* tpmg_solve with HOST buffers: copies h_f and the initial guess h_u to the
 * device, solves, and copies the solution back into h_u, all inside the call
 * (pinned host memory gives full copy bandwidth; pageable memory works).
 * The solve is tpmg_solve's on the context's own staging vectors, so its
 * device-side loop graph is captured once for them (a tpmg_solve on other
 * vectors in between captures its own, and the next call here captures again).
 * Same arguments and returns as tpmg_solve. */
tpmg_status tpmg_solve_host(tpmg_ctx *ctx, const double *h_f, double *h_u, double rtol, int max_iter,
                            int *iters, double *rel_resid, double *resid_hist);

/* n solves with HOST buffers, one after another, with the copies overlapped
 * (tpmg_solve's PCG of Sec. 5 for each right-hand side in turn; the paper has no
 * host-transfer layer).  System j solves A u_j = f_j: h_f[j] (N doubles, read)
 * and h_u[j] (N doubles, receives the solution; with guess = 1 it also holds the
 * initial guess, with guess = 0 the guess is zero and nothing is copied in for
 * it).  While system j is solved on the device, system j + 1's inputs are copied
 * to the device and system j - 1's solution back to the host, on two copy
 * streams of the context, through two staging slots (2 N doubles of device
 * memory allocated on the first call, kept with the context; one cached solve
 * graph per slot).  Each system's solution, iterations and residual are those
 * of tpmg_solve on the same vectors, bit for bit.  The overlap needs page-locked
 * host memory (cudaHostAlloc, cudaHostRegister); pageable arrays give the same
 * results with the copies serialised by CUDA.  The h_f[j] may repeat; no h_u[j]
 * may overlap another system's h_f or h_u (INVALID_ARG, nothing launched).
 * iters[n], rel_resid[n]: per system, as tpmg_solve; status[n] (or NULL): each
 * system's tpmg_solve status.  Where tpmg_solve runs its loop on the device
 * (CG, graphs on, no kernel class timed, max_iter < 4096), all n solves are
 * enqueued back to back and their results read after the last one; otherwise
 * each returns before the next is enqueued.  A system that ends NOT_CONVERGED
 * or BREAKDOWN does not stop the others; the call returns the first such
 * status, or OK.  A CUDA error stops the call (the outputs of systems not yet
 * reported are unset).  Nothing of the call is in flight when it returns. */
tpmg_status tpmg_solve_host_many(tpmg_ctx *ctx, int n, const double *const *h_f, double *const *h_u, int guess,
                                 double rtol, int max_iter, int *iters, double *rel_resid, int *status);

/* Many independent solves in one graph launch (the batched form, Sec. 5's
 * method applied to many problems at once; the paper has no batching layer).
 * A batch holds one PCG solve (tpmg_solve's algorithm and arithmetic, rtol,
 * max_iter) for each of n (context, right-hand side) pairs -- of any sizes and
 * parameters, on the current device -- with the loop of every solve on the
 * device, in one CUDA graph.  d_f[i], d_u[i]: device vectors of ctxs[i] as in
 * tpmg_solve (d_u[i] = initial guess, overwritten by the solution); the
 * pointers are baked into the batch, which stays valid while the contexts and
 * vectors live.  Every problem's solution, iterations and residuals are those
 * of its own tpmg_solve, bit for bit.  max_iter < 4096.  Two forms (this
 * call builds the work-list form when a context appears more than once, the
 * branch form otherwise; tpmg_batch_create_ex chooses explicitly):
 *   TPMG_BATCH_WORKLIST, possible when every context is a mixed-precision CG
 *   context with constant prolongation, no vertical advection, the factorised
 *   outer operator (no tpmg_set_outer_profiles) and nu_pre, nu_post,
 *   nu_coarse >= 1: the members' V-cycles are merged into one schedule of
 *   steps (aligned at the coarsest level: the same phase, level counted from
 *   the coarsest, and pass of that level), and each step is one launch per
 *   kernel class whose work list holds that step's pass of every member (a
 *   member, its level, colour and column range); the outer FP64 kernels run
 *   every member's blocks in one launch each.  A context may appear several
 *   times (several right-hand sides on one operator): its grid, stencil and
 *   factors are shared and the batch allocates each member's work vectors
 *   (about 48 bytes per unknown).  The relaxation launches' CTA shapes (1, 2,
 *   4 or 8 warps) are timed at creation and the fastest kept (same arithmetic).
 *   TPMG_BATCH_BRANCHES: each problem is an independent branch of the graph
 *   (the contexts' own device-side solves), any context kind; a context may
 *   appear once, and must not run another solve while its batch runs.  On 48
 *   distinct mixed-precision problems it measured faster than the work list
 *   (the problems' graphs overlap freely; the work list's launches carry an
 *   item lookup and a member flag on their critical path).
 * Errors: INVALID_ARG (NULL, a repeated context outside the work-list form,
 * aliased vectors, other device, a context with vertical advection or linear
 * prolongation), OOM, CUDA. */
enum { TPMG_BATCH_AUTO = -1, TPMG_BATCH_BRANCHES = 0, TPMG_BATCH_WORKLIST = 1 };
typedef struct tpmg_batch tpmg_batch;
tpmg_status tpmg_batch_create(tpmg_ctx *const *ctxs, int n, const double *const *d_f, double *const *d_u,
                              double rtol, int max_iter, tpmg_batch **out);

/* tpmg_batch_create with the form chosen by the caller: form TPMG_BATCH_AUTO (the
 * rule of tpmg_batch_create), TPMG_BATCH_BRANCHES, or TPMG_BATCH_WORKLIST
 * (INVALID_ARG if a member does not qualify); groups = the work-list form's number
 * of root branches, each a work-list schedule over a share of the members of about
 * equal size (0: the default; at most n).  Results are those of tpmg_batch_create
 * bit for bit whatever the form and the groups.  Errors as tpmg_batch_create. */
tpmg_status tpmg_batch_create_ex(tpmg_ctx *const *ctxs, int n, const double *const *d_f, double *const *d_u,
                                 double rtol, int max_iter, int form, int groups, tpmg_batch **out);

/* Runs the batch on cuda_stream and waits for it.  iters[i], rel_resid[i]
 * (host, n entries) as tpmg_solve; status (nullable, n entries) per problem;
 * kernel_launches (nullable) = kernels the run executed.  Returns OK when every
 * problem converged, otherwise the first problem's non-OK status. */
tpmg_status tpmg_batch_run(tpmg_batch *b, void *cuda_stream, int *iters, double *rel_resid, int *status,
                           long long *kernel_launches);

/* The form tpmg_batch_create built (TPMG_BATCH_*), or -1 for NULL. */
int tpmg_batch_form(const tpmg_batch *b);

/* Releases the batch (not the contexts).  NULL is ignored. */
void tpmg_batch_destroy(tpmg_batch *b);

/* Sizes of multigrid level `level` (0 = coarsest, n_levels-1 = finest):
 * cells, vertical cells, omega^2 actually used, number of colours.  Any output
 * may be NULL.  Errors: INVALID_ARG. */
tpmg_status tpmg_query(const tpmg_ctx *ctx, int level, int *n_cells, int *n_r, double *omega2, int *n_colours);

/* The autotuner's choice on multigrid level `level`: variant = relaxation kernel
 * (FP64: 0 one warp per 16-column task, 1/2/3 one CTA of 64/128/256 threads per
 * task, 4 one warp per task with 6 elements per lane in flight in the gather
 * instead of 4); mixed precision: one warp per
 * column in CTAs of 1/2/4/8 warps; -1 heuristic: not tuned) and us[5] =
 * measured microseconds of the level's largest colour pass with each variant
 * (us[4] = 0 where only four apply: mixed precision, and FP64 levels relaxed by
 * the warp scans, whose variants 0..3 are CTAs of 1/2/4/8 warps).  Any output
 * may be NULL.
 * Errors: INVALID_ARG. */
tpmg_status tpmg_query_tuning(const tpmg_ctx *ctx, int level, int *variant, float *us);

/* Host copies of the grid of multigrid level `level`: centres [n][3] (unit
 * vectors), areas [n] (spherical), nbrs [n][3] (cell across edge e of the
 * counter-clockwise corners (v_e, v_{e+1})), g [n][3] (two-point flux factor
 * |S| n.(c'-c)/|c'-c|^2), colour [n], r_faces [n_r+1] (1 = r_0 < ... < r_nr = 1+H).
 * Any output may be NULL.  Errors: INVALID_ARG. */
tpmg_status tpmg_export_mesh(const tpmg_ctx *ctx, int level, double *centres, double *areas, int *nbrs,
                             double *g, int *colour, double *r_faces);

/* Tracing: kernel classes of the library, for launch counts and timings. */
enum { TPMG_K_APPLY = 0,      /* y = A x (with the fused dot of CG) */
       TPMG_K_RESIDUAL = 1,   /* r = f - A u (initial residual of CG) */
       TPMG_K_RESTRICT = 2,   /* fused residual + restriction of Algorithm 1 */
       TPMG_K_RELAX = 3,      /* one colour pass / one Jacobi sweep of the line relaxation */
       TPMG_K_PROLONG = 4,    /* u += P u_c when no post-smoothing follows */
       TPMG_K_DOT = 5,        /* <r, z> block partials */
       TPMG_K_AXPY = 6,       /* u += alpha p, r -= alpha q, ||r||^2 partials */
       TPMG_K_XPBY = 7,       /* p = z + beta p */
       TPMG_K_FINISH = 8,     /* deterministic reduction of partials + CG scalar step */
       TPMG_K_COPY = 9,       /* device-to-device copies and clears issued by the library */
       TPMG_K_NET = 10,       /* learned form (tpmg_learned.h): features, network layers, output */
       TPMG_K_COUNT = 11 };

/* Resets the tracing counters of ctx and times (with a CUDA event pair on the
 * context stream around each launch) the kernel classes whose bit is set in
 * class_mask (bit i = class i; 0 = count launches only).  Launch counts and
 * processed unknowns are always accumulated.  Errors: INVALID_ARG, CUDA. */
tpmg_status tpmg_profile(tpmg_ctx *ctx, unsigned class_mask);

/* Reads the counters of one kernel class since the last tpmg_profile call:
 * launches, units = number of (cell, level) unknowns the launches processed
 * (for the algorithmic bytes / flops per launch), and -- if the class is
 * timed -- total_ms, the summed device time of the `timed` launches that carry
 * an event pair.  Launches made one by one are all timed, each with its own
 * pair.  In a captured graph one pair of event-record nodes spans each run of
 * consecutive launches of the class (so that the timing adds few nodes and
 * keeps the kernels of a run back to back); those pairs hold the most recent
 * replay only (timed counts one replay's launches).  The average duration of
 * a launch is total_ms / timed.  Synchronises the context stream.
 * Any output may be NULL.  Errors: INVALID_ARG, CUDA. */
tpmg_status tpmg_profile_read(tpmg_ctx *ctx, int kernel_class, long long *launches, double *total_ms,
                              double *units, long long *timed);

/* Algorithmic work of one kernel class since the last tpmg_profile call, for the
 * roofline of the class: the HBM bytes the method itself must move (each array
 * it needs streamed once, neighbour re-reads cached, per-column metadata
 * amortised; arrays a kernel stores only to save arithmetic -- the Thomas
 * factors, the outer operator's row products -- are not counted) and the flops
 * of its formulas (FMA = 2).  bytes / flops cover every launch counted by
 * tpmg_profile_read; timed_bytes / timed_flops the launches inside the class's
 * event pairs, so that timed_bytes / total_ms is the class's achieved
 * algorithmic rate.  Per unknown of a launch:
 *   line relaxation (eq. BlockJacobi), FP64: 24 B (read f and u, write u), 16 B
 *     from a zero guess; 12 flops (the right-hand side f + sum of the neighbour
 *     couplings and its scaling by the pivot, 3 FMA and 2 multiplies, then one FMA
 *     per recurrence), 5 for the first colour from a zero guess (no neighbour
 *     terms); the prolongation fused into a coarse level's last
 *     pass adds 8 B (2 B per fine unknown) and 4 flops per coarse unknown;
 *   line relaxation, FP32 on the BF16 stencil: f (8 B on the finest level, 4 B
 *     below) + stencil 10 B + u read 4 B (not from a zero guess) + u write 4 B,
 *     +8 B for the finest level's FP64 result, +4 B per coarse unknown of fused
 *     prolongation; flops as in FP64;
 *   residual + restriction (Algorithm 1) per fine unknown: FP64 18 B, 12 flops;
 *     FP32 f + u 4 B + stencil 10 B + 1 B, 20 flops;
 *   operator apply 16 B, 14 flops; initial residual 24 B, 17 flops (+8 B for the
 *   zero-guess probe); axpy 48 B (56 B in flexible CG); dot 16 B; xpby 24 B;
 *   clears 8 B (FP32: 4 B); copies 16 B.
 * Any output may be NULL.  Synchronises the context stream.  Errors: INVALID_ARG, CUDA. */
tpmg_status tpmg_profile_work(tpmg_ctx *ctx, int kernel_class, double *bytes, double *timed_bytes, double *flops,
                              double *timed_flops);

/* Measured FP64 throughput of the current device in TFLOP/s (FMA = 2 flops):
 * kernels of 2, 4 or 8 independent FMA chains per thread on every SM, with 1, 2,
 * 4 or the most resident 256-thread blocks per SM; per configuration one warm-up
 * launch and three launches timed with CUDA events on cuda_stream; the best rate
 * of all.  It is the denominator of the FP64-pipe roofline of the FP64 kernels.
 * The paper has no counterpart: a measurement utility.  Allocates and frees a
 * small device buffer; synchronises the stream; takes about 0.5 s.
 * Errors: INVALID_ARG (tflops NULL), OOM, CUDA. */
tpmg_status tpmg_fp64_peak(void *cuda_stream, double *tflops);

/* Static description of a status value. */
const char *tpmg_status_string(tpmg_status s);

/* Message of the last failed call on ctx ("" if none); valid until the next call. */
const char *tpmg_last_error(const tpmg_ctx *ctx);

/* Releases every device and host resource of ctx (after synchronising its
 * stream).  NULL is ignored. */
void tpmg_destroy(tpmg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* TPMG_H */
