// C ABI of the TPMG library: context set-up, V-cycle orchestration (Algorithm 1
// of Dedner, Mueller & Scheichl, arXiv:1408.2981) and preconditioned CG.
// Every step of the solve runs in the kernels of kernels.cu on the context's
// stream; the host only sequences launches and reads one scalar per iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "tpmg_internal.h"

using namespace tpmg;

// Launch counters (always on) and optional CUDA-event timing per kernel class.
struct Tracer {
    unsigned mask = 0;
    long long launches[TPMG_K_COUNT] = {};
    double units[TPMG_K_COUNT] = {};
    double bytes[TPMG_K_COUNT] = {};   // algorithmic HBM bytes of the launches (alg_* below)
    double flops[TPMG_K_COUNT] = {};   // algorithmic flops of the launches (FMA = 2)
    std::vector<cudaEvent_t> ev;   // pairs: ev[2i] before the first, ev[2i+1] after the last launch of bracket i
    std::vector<int> cls;          // class of bracket i
    std::vector<int> nl;           // launches in bracket i
    std::vector<double> nb;        // algorithmic bytes of the launches in bracket i
    std::vector<double> nf;        // algorithmic flops of the launches in bracket i
    size_t used = 0;
    int open = -1;                 // class of the bracket being captured, -1 if none
    cudaStream_t open_s = nullptr; // its stream
};

// Launches and processed unknowns per kernel class of a captured solve: its initial
// part and one iteration of its device-side loop.
struct ClassCounts {
    long long init[TPMG_K_COUNT] = {}, iter[TPMG_K_COUNT] = {};
    double uinit[TPMG_K_COUNT] = {}, uiter[TPMG_K_COUNT] = {};
    double binit[TPMG_K_COUNT] = {}, biter[TPMG_K_COUNT] = {};
    double finit[TPMG_K_COUNT] = {}, fiter[TPMG_K_COUNT] = {};
};

// The V-cycle of tpmg_solve (r -> z on the context's own vectors) replayed
// from a captured CUDA graph, with the launch counts of one replay.
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    long long launches[TPMG_K_COUNT] = {};
    double units[TPMG_K_COUNT] = {};
    double bytes[TPMG_K_COUNT] = {};
    double flops[TPMG_K_COUNT] = {};
};

struct tpmg_ctx {
    tpmg_params p{};
    Tracer tr;
    cudaStream_t stream = nullptr;
    cudaStream_t issue = nullptr;       // stream the next launches go to (stream, or cap_stream while capturing)
    cudaStream_t cap_stream = nullptr;  // private stream on which graphs are captured
    bool capturing = false;
    GraphCache vc;
    // whole solve as one graph (device-side loop), cached for the two argument sets used
    // last (two, so that the pipelined host solves alternate between their staging slots)
    struct SolveGraph {
        cudaGraphExec_t exec = nullptr;
        const double *f = nullptr;
        double *u = nullptr;
        double rtol = 0.0;
        int max_iter = -1;
        long long init = 0, iter = 0;   // launches of the initial part and of one iteration
        ClassCounts cls;                // the same per kernel class, with the unknowns processed
        unsigned long long used = 0;    // last use, for replacing the older entry
    } sg[2];
    unsigned long long sg_clock = 0;
    long long last_launches = 0;          // kernels executed by the last solve
    // learned form (tpmg_learned.h): attached networks (COARSE, WARM), their
    // inference workspaces, scales, the learned solve's graph and the
    // coarsest-level recording
    tpmg_net *net[2] = {nullptr, nullptr};
    struct NetWs {
        float *p = nullptr, *x = nullptr, *h0 = nullptr, *h1 = nullptr, *y = nullptr;
        uint16_t *xt = nullptr;   // the tcgen05 kernel's inputs, bfloat16 in its tile layout
        long rows = 0;
    } nws[2];
    float *net_p = nullptr;       // point values of tpmg_net_features / tpmg_net_targets
    long net_p_cap = 0;
    double *d_net_s = nullptr;    // [2] feature scales s (COARSE, WARM)
    int *d_net_err = nullptr;     // set by the tcgen05 network kernel if a CTA gave up waiting
    bool net_coarse_on = false;   // the V-cycle being issued uses the COARSE network
    struct {
        cudaGraphExec_t exec = nullptr;
        const double *f = nullptr;
        double *u = nullptr;
        double rtol = 0.0;
        int max_iter = -1;
        const tpmg_net *nets[2] = {nullptr, nullptr};
        long long init = 0, iter = 0;
        ClassCounts cls;
    } lg;
    double *bv = nullptr, *bs = nullptr, *bz = nullptr, *bh = nullptr;   // BiCGStab's v, s, z, r^ (on first use)
    // factorised profiles (tpmg_setup_profiles): vertical factors and the horizontal
    // factors of every refinement level; empty = the constant 1
    std::vector<double> pr_beta, pr_aS, pr_ar;
    std::vector<std::vector<double>> ps_beta, ps_ar, ps_aS;
    // factorised vertical advection: xi_fac set when given; empty factor = 1
    bool xi_fac = false;
    std::vector<double> pr_xi;
    std::vector<std::vector<double>> ps_xi;
    dbl4 *cfull_store = nullptr;   // the finest level's general-profile coefficients (on first use)
    double *cvx_store = nullptr;   // the finest level's general advection X (on first use)
    double *rec = nullptr;        // coarsest-level right-hand sides being recorded
    int rec_cap = 0, rec_n = 0;
    double *d_hist = nullptr;     // [kHistCap] residual history of the device-side loop
    int device = 0;
    int sm_count = 0;
    double *noalloc_base = nullptr;   // device address of tpmg_vcycle_noalloc's fixed array (set-up)
    HostGrid host;
    std::vector<LevelDev> lv;     // multigrid levels, 0 = coarsest
    VertDev vert{};
    double *d_vert = nullptr;     // backing store of vert (vol | w | hr)
    long N = 0;                   // fine-level unknowns
    // PCG vectors (fine level)
    double *r = nullptr, *z = nullptr, *pv = nullptr, *q = nullptr;
    // mixed precision: r in FP32, written by every kernel that writes r (initial residual,
    // axpy, the learned solve's judge), read by the finest level of the V-cycle of r
    float *r32 = nullptr;
    double *hf = nullptr, *hu = nullptr;   // device staging for tpmg_solve_host
    // tpmg_solve_host_many (on first use): its second staging slot, the streams of its
    // copies in and out, and its events (per slot: inputs copied, solved, solution copied out)
    double *hf2 = nullptr, *hu2 = nullptr;
    cudaStream_t xin = nullptr, xout = nullptr;
    cudaEvent_t xev_in[2] = {}, xev_solved[2] = {}, xev_out[2] = {};
    Scalars *h_many = nullptr;   // pinned: each system's scalars, read after the last solve
    int h_many_cap = 0;
    double *partials = nullptr;
    int n_part = 0;
    int *zflags = nullptr;        // [n_part] per-block flags of the initial guess's zero probe
    Scalars *sc = nullptr;        // device
    Scalars *h_sc = nullptr;      // pinned host mirror
    std::vector<void *> allocs;   // every device allocation, freed by tpmg_destroy
    std::string err;
};

// One launch of the work-list form's schedule: a kernel class and its items.
struct BatchLaunch {
    int kind = 0;            // 0 relaxation, 1 residual + restriction
    int mode = 0;            // PASS_* (relaxation)
    bool f64 = false;        // right-hand side in FP64 (a member's finest level)
    int n_r_max = 0;         // rows-per-lane class of the items' columns
    int args = 0;            // index of the launch's work list (tpmg_batch::rargs or cargs)
    int count = 0;           // its items
    long total = 0;          // warps (relaxation) or positions (restriction) of the launch
    int wpb = 4;             // warps per CTA of a relaxation launch (tuned)
    float us[4] = {};        // tuner timings for 1 / 2 / 4 / 8 warps per CTA
};

struct tpmg_batch {
    std::vector<tpmg_ctx *> ctx;
    std::vector<long long> init_launches, iter_launches;   // per problem
    double rtol = 0.0;
    int max_iter = 0;
    cudaGraphExec_t exec = nullptr;
    // work-list form (TPMG_BATCH_WORKLIST): one graph whose launches each cover one step
    // of every member's V-cycle or outer iteration; members may share a context
    int form = TPMG_BATCH_BRANCHES;
    int n_part = 0;
    Scalars *h_sc = nullptr;                // [M] pinned host mirror of the members' scalars
    std::vector<Scalars *> d_sc;            // [M] device
    // The members are split into groups of about equal work; each group is one work-list
    // schedule with its own loop, a root branch of the graph, so that the groups drift
    // apart and one group's FP64-bound outer operator overlaps another's HBM-bound V-cycle.
    struct Group {
        std::vector<int> members;           // batch members, in the group's order
        BatchMemberDev *d_mem = nullptr;    // [members]
        int *d_active = nullptr, *d_go = nullptr;
        std::vector<BatchLaunch> launches;  // the group's V-cycle launches in order
        std::vector<RelaxBatchArgs> rargs;  // their work lists (kernel parameters)
        std::vector<RestrictBatchArgs> cargs;
        long long init = 0, iter = 0;       // launches of the initial part and of one iteration
    };
    std::vector<Group> groups;
    std::vector<void *> allocs;             // device allocations of the work-list form
};

namespace {

const char *kStatus[] = {"TPMG_OK", "TPMG_ERR_INVALID_ARG", "TPMG_ERR_CUDA", "TPMG_ERR_OOM",
                         "TPMG_ERR_NOT_CONVERGED", "TPMG_ERR_BREAKDOWN"};

tpmg_status fail(tpmg_ctx *c, tpmg_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

#define CU(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? TPMG_ERR_OOM : TPMG_ERR_CUDA,      \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

template <typename T>
cudaError_t dalloc(tpmg_ctx *ctx, T **ptr, size_t count)
{
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    ctx->allocs.push_back(p);
    *ptr = static_cast<T *>(p);
    return cudaMemsetAsync(p, 0, std::max<size_t>(count, 1) * sizeof(T), ctx->stream);
}

bool validate(const tpmg_params *p, std::string &msg)
{
    if (!p) { msg = "params is NULL"; return false; }
    if (p->refinement < 0 || p->refinement > 9) { msg = "refinement must be in 0..9"; return false; }
    if (p->n_levels < 1 || p->n_levels > p->refinement + 1) { msg = "n_levels must be in 1..refinement+1"; return false; }
    if (p->n_r < 1 || p->n_r > 1024) { msg = "n_r must be in 1..1024"; return false; }
    const double N = 20.0 * std::pow(4.0, p->refinement) * p->n_r;
    if (N > 2147483647.0) { msg = "n_cells * n_r must fit in a 32-bit index"; return false; }
    if (!(p->H > 0.0) || !std::isfinite(p->H)) { msg = "H must be positive"; return false; }
    if (!(p->grading > 0.0) || !std::isfinite(p->grading)) { msg = "grading must be positive"; return false; }
    if (!(p->omega2 > 0.0) && !(p->courant_c > 0.0)) { msg = "omega2 or courant_c must be positive"; return false; }
    if (p->nu_pre < 0 || p->nu_post < 0 || p->nu_coarse < 0 || p->nu_pre > 64 || p->nu_post > 64 || p->nu_coarse > 64) {
        msg = "smoothing counts must be in 0..64"; return false;
    }
    if (p->smoother != TPMG_SMOOTH_MCSOR && p->smoother != TPMG_SMOOTH_JACOBI) { msg = "unknown smoother"; return false; }
    if (!(p->relax > 0.0 && p->relax < 2.0)) { msg = "relax must be in (0, 2)"; return false; }
    if (p->coeff_storage != TPMG_COEFF_FACTORISED && p->coeff_storage != TPMG_COEFF_FULL &&
        p->coeff_storage != TPMG_COEFF_PARTIAL) {
        msg = "unknown coefficient storage"; return false;
    }
    if (p->centre != TPMG_CENTRE_CIRCUM && p->centre != TPMG_CENTRE_VERTEX_MEAN) { msg = "unknown centre kind"; return false; }
    if (p->precision != TPMG_PREC_FP64 && p->precision != TPMG_PREC_MIXED) { msg = "unknown precision"; return false; }
    if (p->precision == TPMG_PREC_MIXED && p->coeff_storage != TPMG_COEFF_FULL) {
        msg = "the mixed-precision V-cycle stores its stencil per unknown in BF16 (TPMG_COEFF_FULL)";
        return false;
    }
    if (p->graphs != 0 && p->graphs != 1) { msg = "graphs must be 0 or 1"; return false; }
    if (p->autotune != 0 && p->autotune != 1) { msg = "autotune must be 0 or 1"; return false; }
    if (p->scan_max_cells < 0) { msg = "scan_max_cells must be >= 0"; return false; }
    if (p->outer < TPMG_OUTER_CG || p->outer > TPMG_OUTER_BICGSTAB) { msg = "unknown outer iteration"; return false; }
    if (p->prolongation != TPMG_PROLONG_CONSTANT && p->prolongation != TPMG_PROLONG_LINEAR) {
        msg = "unknown prolongation"; return false;
    }
    if (p->pdl != 0 && p->pdl != 1) { msg = "pdl must be 0 or 1"; return false; }
    if (p->relax_variant < -1 ||
        p->relax_variant >= (p->precision == TPMG_PREC_MIXED ? kRelaxVariants32 : (int)RELAX_VARIANTS)) {
        msg = "relax_variant must be -1 or a relaxation kernel variant";
        return false;
    }
    if (p->scaled_rhs != 0 && p->scaled_rhs != 1) { msg = "scaled_rhs must be 0 or 1"; return false; }
    if (p->net_tcgen05 != 0 && p->net_tcgen05 != 1) { msg = "net_tcgen05 must be 0 or 1"; return false; }
    return true;
}

Launch launch_of(const tpmg_ctx *ctx)
{
    return Launch{ctx->issue, ctx->p.n_r, ctx->sm_count, ctx->vert.dr, ctx->vert.dr32, ctx->p.pdl == 1};
}

double vfac(const std::vector<double> &v, int k) { return v.empty() ? 1.0 : v[k]; }
double hfac(const std::vector<std::vector<double>> &h, int ref, int T) { return h.empty() ? 1.0 : h[ref][T]; }

// horizontal profile factors on every refinement level: the finest as given, each
// coarser cell the area-weighted mean of its 4 children
bool level_means(const HostGrid &G, int L, const double *fine, std::vector<std::vector<double>> &out,
                 bool any_sign = false)
{
    out.clear();
    if (!fine) return true;
    out.assign(L + 1, std::vector<double>());
    out[L].assign(fine, fine + G.lev[L].n);
    for (double v : out[L])
        if (!std::isfinite(v) || (!any_sign && !(v > 0.0))) return false;
    for (int l = L - 1; l >= 0; --l) {
        out[l].resize(G.lev[l].n);
        for (int T = 0; T < G.lev[l].n; ++T) {
            double sum = 0.0, a = 0.0;
            for (int j = 0; j < 4; ++j) {
                const double aj = G.lev[l + 1].area[4 * T + j];
                sum += aj * out[l + 1][4 * T + j];
                a += aj;
            }
            out[l][T] = sum / a;
        }
    }
    return true;
}

bool copy_vertical(const double *v, int n, std::vector<double> &out, bool any_sign = false)
{
    out.clear();
    if (!v) return true;
    out.assign(v, v + n);
    for (double x : out)
        if (!std::isfinite(x) || (!any_sign && !(x > 0.0))) return false;
    return true;
}

// The solver may run CG only with a symmetric operator and V-cycle: vertical advection
// (factorised, or in the outer operator's general profiles) makes the operator
// non-symmetric, linear prolongation the V-cycle.
bool has_advection(const tpmg_ctx *ctx) { return ctx->xi_fac || (!ctx->lv.empty() && ctx->lv.back().cvx); }
bool nonsymmetric(const tpmg_ctx *ctx) { return has_advection(ctx) || ctx->p.prolongation == TPMG_PROLONG_LINEAR; }

cudaError_t grow_events(Tracer &t, size_t pairs)
{
    while (t.ev.size() < 2 * pairs) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        t.ev.push_back(e);
    }
    if (t.cls.size() < pairs) t.cls.resize(pairs);
    if (t.nl.size() < pairs) t.nl.resize(pairs);
    if (t.nb.size() < pairs) t.nb.resize(pairs);
    if (t.nf.size() < pairs) t.nf.resize(pairs);
    return cudaSuccess;
}

// Records the end of the open bracket, if any.
cudaError_t close_bracket(tpmg_ctx *ctx)
{
    Tracer &t = ctx->tr;
    if (t.open < 0) return cudaSuccess;
    const cudaError_t e =
        cudaEventRecordWithFlags(t.ev[2 * t.used + 1], t.open_s, ctx->capturing ? cudaEventRecordExternal : 0);
    t.cls[t.used] = t.open;
    ++t.used;
    t.open = -1;
    return e;
}

// Every device operation of the library goes through run(): it counts the
// launch and the unknowns it processes, and brackets it with an event pair on
// the issuing stream when its class is being timed.  While a graph is being
// captured the pair becomes two event-record nodes of the graph, re-recorded
// by every replay, and one pair spans each run of consecutive launches of the
// timed class (for example all post-smoothing passes of a V-cycle): an event
// node between two kernels costs microseconds of its own and would cut the
// programmatic overlap of the kernels around it.  The capture closes the last
// bracket before it ends (end_capture).
// Algorithmic HBM bytes per unit of the kernel classes whose launches do not state
// their own: each array the method needs streamed once (neighbour re-reads cached,
// per-column metadata amortised), FP64 vectors of the outer iteration.  The line
// relaxation, the restriction, the prolongation, the copies and the initial residual
// state their bytes at the launch (alg_* below).
double class_bytes_per_unit(int kclass)
{
    switch (kclass) {
    case TPMG_K_APPLY: return 16.0;    // read x, write y
    case TPMG_K_RESIDUAL: return 24.0; // read f, u, write r
    case TPMG_K_RESTRICT: return 18.0; // read f, u, write f_c (a quarter of the fine size)
    case TPMG_K_PROLONG: return 18.0;  // read u_c (a quarter), read and write u
    case TPMG_K_DOT: return 16.0;
    case TPMG_K_AXPY: return 48.0;     // read p, q, u, r, write u, r (+8 with z_old: alg_axpy)
    case TPMG_K_XPBY: return 24.0;
    case TPMG_K_COPY: return 8.0;      // a clear (a copy states 16)
    default: return 0.0;               // finish (scalars), network (not part of the roofline)
    }
}

// Algorithmic FP64 flops per unit (FMA = 2) of the same classes: the arithmetic of the
// method's formulas as the kernels evaluate them.  The apply's row (8 operations from
// its stored products) and its fused dot; the residual's flux-form row; the
// restriction's row per fine unknown; the axpy pair with ||r||^2; dot, xpby one FMA.
double class_flops_per_unit(int kclass)
{
    switch (kclass) {
    case TPMG_K_APPLY: return 14.0;
    case TPMG_K_RESIDUAL: return 17.0;
    case TPMG_K_RESTRICT: return 12.0;
    case TPMG_K_PROLONG: return 1.0;
    case TPMG_K_DOT: return 2.0;
    case TPMG_K_AXPY: return 6.0;
    case TPMG_K_XPBY: return 2.0;
    default: return 0.0;
    }
}

struct Alg {         // algorithmic work of one launch
    double bytes, flops;
};

template <class F>
cudaError_t run_w(tpmg_ctx *ctx, int kclass, double units, Alg w, F &&launch)
{
    Tracer &t = ctx->tr;
    t.launches[kclass] += 1;
    t.units[kclass] += units;
    t.bytes[kclass] += w.bytes;
    t.flops[kclass] += w.flops;
    const bool timed = (t.mask >> kclass) & 1u;
    cudaError_t e = cudaSuccess;
    if (t.open >= 0 && (t.open != kclass || t.open_s != ctx->issue)) e = close_bracket(ctx);
    if (e != cudaSuccess) return e;
    if (timed && t.open < 0) {
        if (2 * t.used + 2 > t.ev.size()) {
            e = grow_events(t, t.used + 1024);
            if (e != cudaSuccess) return e;
        }
        e = cudaEventRecordWithFlags(t.ev[2 * t.used], ctx->issue, ctx->capturing ? cudaEventRecordExternal : 0);
        if (e != cudaSuccess) return e;
        t.open = kclass;
        t.open_s = ctx->issue;
        t.nl[t.used] = 0;
        t.nb[t.used] = 0.0;
        t.nf[t.used] = 0.0;
    }
    e = launch();
    if (timed) {
        if (e == cudaSuccess) {
            t.nl[t.used] += 1;
            t.nb[t.used] += w.bytes;
            t.nf[t.used] += w.flops;
        }
        if (!ctx->capturing) {
            const cudaError_t ec = close_bracket(ctx);
            if (e == cudaSuccess) e = ec;
        }
    }
    return e;
}

// a launch whose flops follow from its class (class_flops_per_unit) and whose bytes are given
template <class F>
cudaError_t run_b(tpmg_ctx *ctx, int kclass, double units, double bytes, F &&launch)
{
    return run_w(ctx, kclass, units, Alg{bytes, units * class_flops_per_unit(kclass)}, std::forward<F>(launch));
}

template <class F>
cudaError_t run(tpmg_ctx *ctx, int kclass, double units, F &&launch)
{
    return run_b(ctx, kclass, units, units * class_bytes_per_unit(kclass), std::forward<F>(launch));
}

// Algorithmic bytes of one line-relaxation pass over `units` unknowns (the survey of
// the method's traffic: the arrays the method needs, each streamed once).  FP64: read
// f, the neighbours' u (one read of u over a sweep) and write u, 24 B per unknown;
// a pass from a zero guess reads no u, 16 B; the prolongation fused into a coarse
// level's last pass adds the read of the coarse value, 2 B per fine unknown = 8 B per
// coarse unknown.  The stored twisted factors are this design's extra traffic, not
// the method's.
// Flops per unknown: the right-hand side f + hr_k sum_e g_e u_e (3 FMA + 1 multiply)
// scaled by the pivot (1), the forward and backward recurrences (1 FMA each): 12; from
// a zero guess the first colour has no neighbour terms, 5; the fused prolongation adds
// 4 per coarse unknown.  (The kernels evaluate the neighbour terms of the other colours
// of a first sweep with zeros for the not yet relaxed ones, as counted here.)
Alg alg_relax64(double units, int mode, bool fused)
{
    return Alg{units * ((mode == PASS_NORMAL ? 24.0 : 16.0) + (fused ? 8.0 : 0.0)),
               units * ((mode == PASS_RHS_ONLY ? 5.0 : 12.0) + (fused ? 4.0 : 0.0))};
}
// The FP32 V-cycle on the BF16 stencil: f (8 B in FP64 on the finest level, 4 B
// below), the stencil of the column (alphaS_hat x 3 and beta_hat: 8 B; alphar_hat of
// the lower face: 2 B), u read (4 B, not from a zero guess), u written (4 B), the
// finest level's result also written in FP64 (8 B), the fused prolongation 1 B per
// fine unknown (4 B per coarse unknown).  The stored FP32 Thomas factors (12 B) are
// this design's extra traffic.
// Flops (FP32) per unknown as in FP64: 12, 5 for the first colour from a zero guess,
// +4 per coarse unknown for the fused prolongation.
Alg alg_relax32(double units, int mode, bool f64, bool out64, bool fused)
{
    return Alg{units * ((f64 ? 8.0 : 4.0) + 10.0 + (mode == PASS_NORMAL ? 4.0 : 0.0) + 4.0 + (out64 ? 8.0 : 0.0) +
                        (fused ? 4.0 : 0.0)),
               units * ((mode == PASS_RHS_ONLY ? 5.0 : 12.0) + (fused ? 4.0 : 0.0))};
}
// Residual + restriction in FP32 per fine unknown: f (8 or 4 B), u (4 B), the stencil
// (10 B), f_c written (4 B over 4 children).
// Flops per fine unknown: the flux-form row (6 FMA, 1 multiply, 6 differences) and the sum.
Alg alg_restrict32(double units, bool f64) { return Alg{units * ((f64 ? 8.0 : 4.0) + 4.0 + 10.0 + 1.0), units * 20.0}; }

#define LCHK(call)                                                                                \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(ctx, TPMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// r = f - A u on the finest level with the partials of ||r||^2: a probe of u first (its own
// launch), so that where the guess is exactly zero -- how a solve normally starts -- the
// residual kernel copies f instead of loading the stencil; the result is the same either way.
cudaError_t residual_probed(tpmg_ctx *ctx, const Launch &L, const double *f, const double *u, double *r)
{
    const LevelDev &fl = ctx->lv.back();
    const long N = ctx->N;
    float *const r32 = r == ctx->r ? ctx->r32 : nullptr;   // the context's r keeps its FP32 copy in step
    cudaError_t e = run_w(ctx, TPMG_K_RESIDUAL, (double)N, Alg{8.0 * N, 0.0},   // the probe reads u
                          [&] { return launch_nonzero(L, N, u, ctx->zflags, ctx->n_part); });
    if (e != cudaSuccess) return e;
    return run_b(ctx, TPMG_K_RESIDUAL, (double)N, (r32 ? 28.0 : 24.0) * N, [&] {
        return launch_residual(L, fl, ctx->vert, f, u, r, ctx->partials, ctx->n_part, ctx->zflags, r32);
    });
}

// Algorithm 1 on multigrid level l: u = V-cycle(f) from a zero initial guess.
// `scratch` is a second vector of the level size (block-Jacobi ping-pong).
// Below the finest level the result is a coarse-grid correction: it is added
// to the 4 children of every cell in u_fine (prolongation P = R^T) by the pass
// that writes that column's final value, so no separate prolongation pass and
// no re-read of the correction is needed.
tpmg_status vcycle_level(tpmg_ctx *ctx, int l, const double *f, double *u, double *scratch, double *u_fine)
{
    const Launch L = launch_of(ctx);
    const tpmg_params &p = ctx->p;
    const LevelDev &lv = ctx->lv[l];
    const int C = lv.n_colours;
    const bool jac = p.smoother == TPMG_SMOOTH_JACOBI;
    const double nunits = (double)lv.n * p.n_r;
    const size_t nbytes = sizeof(double) * lv.n * p.n_r;
    double *cur = u, *oth = scratch;   // Jacobi: current iterate / other buffer
    // a coarse level adds its result into the 4 children of u_fine: fused into the pass
    // that writes each column's final value (P = R^T), or after the level's last pass
    // (linear prolongation, which reads the 3 neighbours' final values too)
    const bool lin = u_fine && p.prolongation == TPMG_PROLONG_LINEAR;
    double *const fuse = lin ? nullptr : u_fine;
    auto prolong_linear = [&]() -> tpmg_status {
        const LevelDev &fl = ctx->lv[l + 1];
        const double *cc = cur;
        LCHK(run(ctx, TPMG_K_PROLONG, (double)fl.n * p.n_r,
                 [&] { return launch_prolong_linear(L, fl, lv, cc, u_fine); }));
        return TPMG_OK;
    };
    // scaled couplings: the first pass over a colour in this visit of the level writes
    // its columns' f / pivot into lv.ft, the later passes read it (bit c: colour c;
    // bit 63: the whole level, block Jacobi)
    unsigned long long ft_seen = 0;
    auto ft_mode = [&](int c) {
        if (!lv.cs || !lv.ft) return 0;
        const unsigned long long bit = 1ull << c;
        const int m = (ft_seen & bit) ? 2 : 1;
        ft_seen |= bit;
        return m;
    };
    // one multicolour block-SOR pass over colour c, in place in u
    auto pass = [&](int c, int mode, double *fine) -> cudaError_t {
        const int t0 = lv.colour_task_off[c], nt = lv.colour_task_off[c + 1] - t0;
        const int m = (mode == PASS_ZERO && c == 0) ? PASS_RHS_ONLY : mode;
        const double units = (double)lv.colour_cells[c] * p.n_r;
        const int ftm = ft_mode(c);
        return run_w(ctx, TPMG_K_RELAX, units, alg_relax64(units, m, fine != nullptr), [&] {
            return launch_relax(L, lv, ctx->vert, m, t0, nt, p.relax, f, u, u, fine, ftm);
        });
    };
    // one block-Jacobi sweep from cur into oth
    auto jacobi = [&](int mode, double *fine) -> cudaError_t {
        const int m = mode == PASS_ZERO ? PASS_RHS_ONLY : mode;
        const int ftm = ft_mode(63);
        cudaError_t e = run_w(ctx, TPMG_K_RELAX, nunits, alg_relax64(nunits, m, fine != nullptr), [&] {
            return launch_relax(L, lv, ctx->vert, m, 0, lv.n_tasks, p.relax, f, cur, oth, fine, ftm);
        });
        std::swap(cur, oth);
        return e;
    };
    auto clear = [&](double *x) -> cudaError_t {
        return run(ctx, TPMG_K_COPY, nunits, [&] { return cudaMemsetAsync(x, 0, nbytes, ctx->issue); });
    };
    if (l == 0) {
        // coarsest level: nu_coarse symmetric sweeps (a zero correction prolongates to nothing)
        if (p.nu_coarse == 0) LCHK(clear(u));
        for (int s = 0; s < p.nu_coarse; ++s) {
            const bool last = s == p.nu_coarse - 1;
            if (jac) {
                LCHK(jacobi(s == 0 ? PASS_ZERO : PASS_NORMAL, last ? fuse : nullptr));
                continue;
            }
            for (int c = 0; c < C; ++c)
                LCHK(pass(c, s == 0 ? PASS_ZERO : PASS_NORMAL, last && c == C - 1 ? fuse : nullptr));
            for (int c = C - 2; c >= 0; --c) LCHK(pass(c, PASS_NORMAL, last ? fuse : nullptr));
        }
        if (lin) {
            const tpmg_status st = prolong_linear();
            if (st != TPMG_OK) return st;
        }
    } else {
        // pre-smoothing (forward colour order)
        if (p.nu_pre == 0) LCHK(clear(cur));
        for (int s = 0; s < p.nu_pre; ++s) {
            if (jac) {
                LCHK(jacobi(s == 0 ? PASS_ZERO : PASS_NORMAL, nullptr));
                continue;
            }
            for (int c = 0; c < C; ++c) LCHK(pass(c, s == 0 ? PASS_ZERO : PASS_NORMAL, nullptr));
        }
        // residual + restriction, then the coarse V-cycle adds its correction into cur
        LevelDev &co = ctx->lv[l - 1];
        const double *uc = cur;
        LCHK(run(ctx, TPMG_K_RESTRICT, nunits,
                 [&] { return launch_resid_restrict(L, lv, co, ctx->vert, f, uc, co.f); }));
        tpmg_status st = vcycle_level(ctx, l - 1, co.f, co.u, co.u2, cur);
        if (st != TPMG_OK) return st;
        // post-smoothing (reverse colour order, the adjoint of the pre-smoothing)
        for (int s = 0; s < p.nu_post; ++s) {
            const bool last = s == p.nu_post - 1;
            if (jac) {
                LCHK(jacobi(PASS_NORMAL, last ? fuse : nullptr));
                continue;
            }
            for (int c = C - 1; c >= 0; --c) LCHK(pass(c, PASS_NORMAL, last ? fuse : nullptr));
        }
        if (lin) {
            const tpmg_status st = prolong_linear();
            if (st != TPMG_OK) return st;
        } else if (p.nu_post == 0 && u_fine) {
            const LevelDev &fl = ctx->lv[l + 1];
            const double *cc = cur;
            LCHK(run(ctx, TPMG_K_PROLONG, (double)fl.n * p.n_r,
                     [&] { return launch_prolong_add(L, fl, cc, u_fine); }));
        }
    }
    // the finest level returns its result in u (coarse levels have handed theirs on already)
    if (!u_fine && cur != u) {
        const double *cc = cur;
        LCHK(run_b(ctx, TPMG_K_COPY, nunits, 16.0 * nunits,
                   [&] { return cudaMemcpyAsync(u, cc, nbytes, cudaMemcpyDeviceToDevice, ctx->issue); }));
    }
    return TPMG_OK;
}

// The bfloat16 bits of the value nearest to x (8 significant bits, ties to the
// even significand), for finite x in the binary32 range: the 45 low
// significand bits of the double are rounded away in integer arithmetic, and
// the result, exact in binary32, gives its upper 16 bits.
unsigned short bf16_bits(double x)
{
    uint64_t b;
    std::memcpy(&b, &x, sizeof b);
    const uint64_t lsb = (b >> 45) & 1u;
    b += (((uint64_t)1 << 44) - 1) + lsb;
    b &= ~(((uint64_t)1 << 45) - 1);
    double r;
    std::memcpy(&r, &b, sizeof r);
    const float f = (float)r;
    uint32_t fb;
    std::memcpy(&fb, &f, sizeof fb);
    return (unsigned short)(fb >> 16);
}

// The network attached in `role` on level lv: u_out = s network(features(f))
// for every column of the level (scale, features, four layers, output).
template <typename TF, typename TO>
tpmg_status net_infer(tpmg_ctx *ctx, int role, const LevelDev &lv, const TF *f, TO *u_out, float *f32 = nullptr)
{
    const Launch L = launch_of(ctx);
    const NetView v = net_view(ctx->net[role]);
    const auto &w = ctx->nws[role];
    double *s = ctx->d_net_s + role;
    const long rows = lv.n;
    const double nunits = (double)lv.n * ctx->p.n_r;
    LCHK(run(ctx, TPMG_K_NET, nunits, [&] {
        return launch_net_prepare<TF>(L, lv, ctx->vert, f, w.p, ctx->partials, ctx->n_part, f32);
    }));
    LCHK(run(ctx, TPMG_K_NET, 1.0, [&] { return launch_net_scale_finish(L, lv, ctx->partials, ctx->n_part, s); }));
    if (ctx->p.net_tcgen05 && net_tc_ok(v) && w.xt) {   // the whole network on tcgen05
        LCHK(run(ctx, TPMG_K_NET, nunits, [&] { return launch_net_features_tiled(L, lv, w.p, rows, s, w.xt); }));
        LCHK(run(ctx, TPMG_K_NET, nunits,
                 [&] { return launch_net_tc<TO>(L, v, w.xt, rows, s, u_out, ctx->d_net_err); }));
        return TPMG_OK;
    }
    LCHK(run(ctx, TPMG_K_NET, nunits, [&] { return launch_net_features(L, lv, w.p, nullptr, rows, s, w.x); }));
    if (net_fused_ok(v)) {   // one tensor-core kernel for the whole network (mma.sync)
        LCHK(run(ctx, TPMG_K_NET, nunits, [&] { return launch_net_fused<TO>(L, v, w.x, rows, s, u_out); }));
        return TPMG_OK;
    }
    const float *in = w.x;
    float *bufs[2] = {w.h0, w.h1};
    for (int l = 0; l < 4; ++l) {
        float *out = l == 3 ? w.y : bufs[l & 1];
        LCHK(run(ctx, TPMG_K_NET, nunits, [&] { return launch_net_layer(ctx->issue, v, l, in, rows, out); }));
        in = out;
    }
    LCHK(run(ctx, TPMG_K_NET, nunits, [&] { return launch_net_output<TO>(L, w.y, rows * ctx->p.n_r, s, u_out); }));
    return TPMG_OK;
}

// The learned solve's initial guess: the WARM network's prediction, then one block-Jacobi
// line relaxation (eq. BlockJacobi, the V-cycle's smoother in FP32) from it on the finest
// level, which removes the vertically oscillating part of the network's error; written to
// u in FP64.  The network's first kernel converts f to FP32 anyway, and stores it in the
// FP32 copy of r (free until the initial residual is formed), so that the relaxation reads
// f in FP32 instead of converting every double again on the FP64 pipe.
tpmg_status warm_start(tpmg_ctx *ctx, const Launch &L, const double *f, double *u)
{
    LevelDev &fl = ctx->lv[ctx->p.n_levels - 1];
    const long N = ctx->N;
    float *const f32 = ctx->r32;
    const tpmg_status s1 = net_infer<double, float>(ctx, TPMG_NET_WARM, fl, f, fl.u32, f32);
    if (s1 != TPMG_OK) return s1;
    LCHK(run_w(ctx, TPMG_K_RELAX, (double)N, alg_relax32((double)N, PASS_NORMAL, !f32, true, false), [&] {
        return f32 ? launch_relax32<float>(L, fl, PASS_NORMAL, 0, fl.n_tasks, (float)ctx->p.relax, f32, fl.u32,
                                           fl.u2_32, nullptr, u)
                   : launch_relax32<double>(L, fl, PASS_NORMAL, 0, fl.n_tasks, (float)ctx->p.relax, f, fl.u32,
                                            fl.u2_32, nullptr, u);
    }));
    return TPMG_OK;
}

// Algorithm 1 in the mixed-precision form on level l: u = V-cycle(f), FP32
// arithmetic on the BF16 stencil.  TF is double on the finest level (the
// FP64 residual of the outer Krylov loop is read directly) and float below.
// As in vcycle_level, a coarse level adds its result into the 4 children in
// u_fine in the pass that writes each column's final value; the finest level
// writes its final values also as double into z64.
template <typename TF>
tpmg_status vcycle_mixed(tpmg_ctx *ctx, int l, const TF *f, float *u, float *scratch, float *u_fine, double *z64)
{
    const Launch L = launch_of(ctx);
    const tpmg_params &p = ctx->p;
    const LevelDev &lv = ctx->lv[l];
    const int C = lv.n_colours;
    const bool jac = p.smoother == TPMG_SMOOTH_JACOBI;
    const float relax = (float)p.relax;
    const double nunits = (double)lv.n * p.n_r;
    const size_t nbytes = sizeof(float) * lv.n * p.n_r;
    constexpr bool kF64 = std::is_same<TF, double>::value;   // the finest level's FP64 right-hand side
    float *cur = u, *oth = scratch;
    // the coarse-to-fine transfer as in vcycle_level: fused into the final pass, or the
    // linear prolongation after the level's last pass
    const bool lin = u_fine && p.prolongation == TPMG_PROLONG_LINEAR;
    float *const fuse = lin ? nullptr : u_fine;
    auto prolong_linear = [&](const float *cc) -> tpmg_status {
        const LevelDev &fl = ctx->lv[l + 1];
        LCHK(run_b(ctx, TPMG_K_PROLONG, (double)fl.n * p.n_r, 9.0 * fl.n * p.n_r,
                   [&] { return launch_prolong_linear32(L, fl, lv, cc, u_fine); }));
        return TPMG_OK;
    };
    auto pass = [&](int c, int mode, float *fine, double *out) -> cudaError_t {
        const int t0 = lv.colour_task_off[c], nt = lv.colour_task_off[c + 1] - t0;
        const int m = (mode == PASS_ZERO && c == 0) ? PASS_RHS_ONLY : mode;
        const double units = (double)lv.colour_cells[c] * p.n_r;
        return run_w(ctx, TPMG_K_RELAX, units, alg_relax32(units, m, kF64, out != nullptr, fine != nullptr),
                     [&] { return launch_relax32<TF>(L, lv, m, t0, nt, relax, f, u, u, fine, out); });
    };
    auto jacobi = [&](int mode, float *fine, double *out) -> cudaError_t {
        const int m = mode == PASS_ZERO ? PASS_RHS_ONLY : mode;
        cudaError_t e = run_w(ctx, TPMG_K_RELAX, nunits, alg_relax32(nunits, m, kF64, out != nullptr, fine != nullptr),
                              [&] { return launch_relax32<TF>(L, lv, m, 0, lv.n_tasks, relax, f, cur, oth, fine, out); });
        std::swap(cur, oth);
        return e;
    };
    auto clear = [&](float *x) -> cudaError_t {
        return run_b(ctx, TPMG_K_COPY, nunits, 4.0 * nunits, [&] { return cudaMemsetAsync(x, 0, nbytes, ctx->issue); });
    };
    if (l == 0) {
        if constexpr (std::is_same<TF, float>::value) {
            // recording of the coarsest-level right-hand sides (training data of the learned form)
            if (ctx->rec && !ctx->capturing && ctx->rec_n < ctx->rec_cap && ctx->p.n_levels > 1) {
                double *dst = ctx->rec + (size_t)ctx->rec_n * lv.n * p.n_r;
                LCHK(run_b(ctx, TPMG_K_COPY, nunits, 12.0 * nunits,
                           [&] { return launch_to_f64(L, (long)lv.n * p.n_r, f, dst); }));
                ++ctx->rec_n;
            }
            // learned form: the network's prediction and one block-Jacobi line
            // relaxation from it replace the coarsest-level solve; the relaxation
            // pass adds the result into u_fine (prolongation)
            if (ctx->net_coarse_on && ctx->p.n_levels > 1) {
                tpmg_status st = net_infer<float, float>(ctx, TPMG_NET_COARSE, lv, f, scratch);
                if (st != TPMG_OK) return st;
                LCHK(run_w(ctx, TPMG_K_RELAX, nunits, alg_relax32(nunits, PASS_NORMAL, false, false, fuse != nullptr), [&] {
                    return launch_relax32<float>(L, lv, PASS_NORMAL, 0, lv.n_tasks, relax, f, scratch, u, fuse, nullptr);
                }));
                return lin ? prolong_linear(u) : TPMG_OK;
            }
        }
        if (p.nu_coarse == 0) {
            LCHK(clear(u));
            if (z64)
                LCHK(run_b(ctx, TPMG_K_COPY, nunits, 12.0 * nunits,
                           [&] { return launch_to_f64(L, (long)lv.n * p.n_r, u, z64); }));
        }
        for (int s = 0; s < p.nu_coarse; ++s) {
            const bool last = s == p.nu_coarse - 1;
            if (jac) {
                LCHK(jacobi(s == 0 ? PASS_ZERO : PASS_NORMAL, last ? fuse : nullptr, last ? z64 : nullptr));
                continue;
            }
            for (int c = 0; c < C; ++c) {
                const bool fin = last && c == C - 1;
                LCHK(pass(c, s == 0 ? PASS_ZERO : PASS_NORMAL, fin ? fuse : nullptr, fin ? z64 : nullptr));
            }
            for (int c = C - 2; c >= 0; --c)
                LCHK(pass(c, PASS_NORMAL, last ? fuse : nullptr, last ? z64 : nullptr));
        }
        return lin ? prolong_linear(cur) : TPMG_OK;
    }
    if (p.nu_pre == 0) LCHK(clear(cur));
    for (int s = 0; s < p.nu_pre; ++s) {
        if (jac) {
            LCHK(jacobi(s == 0 ? PASS_ZERO : PASS_NORMAL, nullptr, nullptr));
            continue;
        }
        for (int c = 0; c < C; ++c) LCHK(pass(c, s == 0 ? PASS_ZERO : PASS_NORMAL, nullptr, nullptr));
    }
    LevelDev &co = ctx->lv[l - 1];
    const float *uc = cur;
    LCHK(run_w(ctx, TPMG_K_RESTRICT, nunits, alg_restrict32(nunits, kF64),
               [&] { return launch_resid_restrict32<TF>(L, lv, co, f, uc, co.f32); }));
    tpmg_status st = vcycle_mixed<float>(ctx, l - 1, co.f32, co.u32, co.u2_32, cur, nullptr);
    if (st != TPMG_OK) return st;
    for (int s = 0; s < p.nu_post; ++s) {
        const bool last = s == p.nu_post - 1;
        if (jac) {
            LCHK(jacobi(PASS_NORMAL, last ? fuse : nullptr, last ? z64 : nullptr));
            continue;
        }
        for (int c = C - 1; c >= 0; --c) LCHK(pass(c, PASS_NORMAL, last ? fuse : nullptr, last ? z64 : nullptr));
    }
    if (lin) {
        const tpmg_status st2 = prolong_linear(cur);
        if (st2 != TPMG_OK) return st2;
    }
    if (p.nu_post == 0) {
        const float *cc = cur;
        if (fuse) {
            const LevelDev &fl = ctx->lv[l + 1];
            LCHK(run_b(ctx, TPMG_K_PROLONG, (double)fl.n * p.n_r, 9.0 * fl.n * p.n_r,
                       [&] { return launch_prolong_add32(L, fl, cc, u_fine); }));
        }
        if (z64)
            LCHK(run_b(ctx, TPMG_K_COPY, nunits, 12.0 * nunits,
                       [&] { return launch_to_f64(L, (long)lv.n * p.n_r, cc, z64); }));
    }
    return TPMG_OK;
}

tpmg_status vcycle_fine(tpmg_ctx *ctx, const double *r, double *z)
{
    const int l = ctx->p.n_levels - 1;
    LevelDev &fl = ctx->lv[l];
    if (ctx->p.precision == TPMG_PREC_MIXED) {
        // the V-cycle of the context's own residual reads its FP32 copy: the same values
        // the passes would round r to, in half the bytes
        if (r == ctx->r && ctx->r32) return vcycle_mixed<float>(ctx, l, ctx->r32, fl.u32, fl.u2_32, nullptr, z);
        return vcycle_mixed<double>(ctx, l, r, fl.u32, fl.u2_32, nullptr, z);
    }
    return vcycle_level(ctx, l, r, z, fl.u2, nullptr);
}

void drop_graph(tpmg_ctx *ctx)
{
    if (ctx->vc.exec) cudaGraphExecDestroy(ctx->vc.exec);
    ctx->vc = GraphCache{};
    for (auto &e : ctx->sg) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        e = tpmg_ctx::SolveGraph{};
    }
    if (ctx->lg.exec) cudaGraphExecDestroy(ctx->lg.exec);
    ctx->lg.exec = nullptr;
    ctx->lg.max_iter = -1;
}

// z = B r on the PCG vectors of the context.  With graphs enabled the V-cycle
// (about 90 launches for 6 levels) is captured once on the private stream and
// then replayed on the context stream as one graph launch.
tpmg_status vcycle_pcg(tpmg_ctx *ctx)
{
    if (!ctx->p.graphs) return vcycle_fine(ctx, ctx->r, ctx->z);
    Tracer &t = ctx->tr;
    if (!ctx->vc.exec) {
        long long l0[TPMG_K_COUNT];
        double u0[TPMG_K_COUNT], b0[TPMG_K_COUNT], f0[TPMG_K_COUNT];
        std::copy(t.launches, t.launches + TPMG_K_COUNT, l0);
        std::copy(t.units, t.units + TPMG_K_COUNT, u0);
        std::copy(t.bytes, t.bytes + TPMG_K_COUNT, b0);
        std::copy(t.flops, t.flops + TPMG_K_COUNT, f0);
        CU(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        ctx->capturing = true;
        ctx->issue = ctx->cap_stream;
        tpmg_status st = vcycle_fine(ctx, ctx->r, ctx->z);
        if (close_bracket(ctx) != cudaSuccess && st == TPMG_OK) st = fail(ctx, TPMG_ERR_CUDA, "event record");
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
        ctx->capturing = false;
        ctx->issue = ctx->stream;
        cudaGraphExec_t exec = nullptr;
        cudaError_t ei = cudaErrorUnknown;
        if (st == TPMG_OK && e == cudaSuccess && g) ei = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        for (int c = 0; c < TPMG_K_COUNT; ++c) {   // the captured launches belong to every replay
            ctx->vc.launches[c] = t.launches[c] - l0[c];
            ctx->vc.units[c] = t.units[c] - u0[c];
            ctx->vc.bytes[c] = t.bytes[c] - b0[c];
            ctx->vc.flops[c] = t.flops[c] - f0[c];
            t.launches[c] = l0[c];
            t.units[c] = u0[c];
            t.bytes[c] = b0[c];
            t.flops[c] = f0[c];
        }
        if (st != TPMG_OK) return st;
        if (e != cudaSuccess) return fail(ctx, TPMG_ERR_CUDA, std::string("V-cycle capture: ") + cudaGetErrorString(e));
        if (ei != cudaSuccess) return fail(ctx, TPMG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
        ctx->vc.exec = exec;
    }
    CU(cudaGraphLaunch(ctx->vc.exec, ctx->stream));
    for (int c = 0; c < TPMG_K_COUNT; ++c) {
        t.launches[c] += ctx->vc.launches[c];
        t.units[c] += ctx->vc.units[c];
        t.bytes[c] += ctx->vc.bytes[c];
        t.flops[c] += ctx->vc.flops[c];
    }
    return TPMG_OK;
}

tpmg_status read_scalars(tpmg_ctx *ctx)
{
    CU(cudaMemcpyAsync(ctx->h_sc, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return TPMG_OK;
}

constexpr int kHistCap = 4096;   // longest residual history of the device-side loop

// Stream capture into an existing graph (after `deps`), launches issued on the
// private stream; *leaves receives the capture's final nodes.
template <class F>
tpmg_status capture_into(tpmg_ctx *ctx, cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps,
                         std::vector<cudaGraphNode_t> *leaves, F &&body)
{
    CU(cudaStreamBeginCaptureToGraph(ctx->cap_stream, g, deps, nullptr, ndeps, cudaStreamCaptureModeThreadLocal));
    ctx->issue = ctx->cap_stream;
    ctx->capturing = true;
    tpmg_status st = body();
    if (close_bracket(ctx) != cudaSuccess && st == TPMG_OK) st = fail(ctx, TPMG_ERR_CUDA, "event record");
    const cudaGraphNode_t *out = nullptr;
    size_t nout = 0;
    cudaStreamCaptureStatus cs;
    const cudaError_t ei = cudaStreamGetCaptureInfo(ctx->cap_stream, &cs, nullptr, nullptr, &out, nullptr, &nout);
    if (leaves && ei == cudaSuccess) leaves->assign(out, out + nout);
    cudaGraph_t gout = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &gout);
    ctx->capturing = false;
    ctx->issue = ctx->stream;
    if (st != TPMG_OK) return st;
    if (ei != cudaSuccess || ee != cudaSuccess)
        return fail(ctx, TPMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ei != cudaSuccess ? ei : ee));
    return TPMG_OK;
}

// Appends one whole PCG solve of ctx to graph g (no dependencies: a root
// branch): the initial residual, then a conditional WHILE node whose body is
// one iteration, in the order
//   z = B r;  beta (0 on the first pass, p cleared before the loop);  p = z + beta p;
//   q = A p, alpha;  u += alpha p, r -= alpha q;  stop test,
// which performs the arithmetic of the host-driven loop of pcg() step for step.
// The finish kernels record the history in ctx->d_hist, count the iterations
// in the device scalars and set the loop condition.  The launch counters of
// the captured kernels are restored (a graph's launches are counted per run).
// learned = true (tpmg_solve_learned): the initial guess is the WARM network's
// prediction if one is attached, the stop test is relative to ||f||, and the
// judge replaces a guess whose residual is not below ||f|| by zero.
tpmg_status append_solve(tpmg_ctx *ctx, cudaGraph_t g, const double *f, double *u, double rtol, int max_iter,
                         long long *init_launches = nullptr, long long *iter_launches = nullptr, bool learned = false,
                         ClassCounts *cls = nullptr)
{
    Tracer &t = ctx->tr;
    long long l0[TPMG_K_COUNT];
    double u0[TPMG_K_COUNT], b0[TPMG_K_COUNT], f0[TPMG_K_COUNT];
    std::copy(t.launches, t.launches + TPMG_K_COUNT, l0);
    std::copy(t.units, t.units + TPMG_K_COUNT, u0);
    std::copy(t.bytes, t.bytes + TPMG_K_COUNT, b0);
    std::copy(t.flops, t.flops + TPMG_K_COUNT, f0);
    cudaGraphConditionalHandle h;
    CU(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    const LoopCtl loop{h, rtol, max_iter, ctx->d_hist};
    LevelDev &fl = ctx->lv[ctx->p.n_levels - 1];
    const long N = ctx->N;
    const int np = ctx->n_part;
    const bool flexible = ctx->p.precision == TPMG_PREC_MIXED || learned;
    std::vector<cudaGraphNode_t> leaves;
    tpmg_status st = capture_into(ctx, g, nullptr, 0, &leaves, [&]() -> tpmg_status {
        const Launch L = launch_of(ctx);
        if (learned && ctx->net[TPMG_NET_WARM]) {   // the network's guess and one relaxation
            const tpmg_status s1 = warm_start(ctx, L, f, u);
            if (s1 != TPMG_OK) return s1;
        }
        LCHK(residual_probed(ctx, L, f, u, ctx->r));
        if (learned) {
            LCHK(run(ctx, TPMG_K_DOT, (double)N, [&] { return launch_dot(L, N, f, f, ctx->partials + np, np); }));
            LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_LOOP_RR0F, ctx->partials, np, ctx->sc, &loop); }));
            LCHK(run(ctx, TPMG_K_COPY, (double)N, [&] { return launch_judge_reset(L, ctx->sc, N, f, u, ctx->r, ctx->r32); }));
        } else {
            LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_LOOP_RR0, ctx->partials, np, ctx->sc, &loop); }));
        }
        LCHK(run(ctx, TPMG_K_COPY, (double)N, [&] { return cudaMemsetAsync(ctx->pv, 0, sizeof(double) * N, ctx->issue); }));
        return TPMG_OK;
    });
    if (st != TPMG_OK) return st;
    long long after_init = 0;
    long long l1[TPMG_K_COUNT];
    double u1[TPMG_K_COUNT], b1[TPMG_K_COUNT], f1[TPMG_K_COUNT];
    for (int c = 0; c < TPMG_K_COUNT; ++c) {
        after_init += t.launches[c] - l0[c];
        l1[c] = t.launches[c];
        u1[c] = t.units[c];
        b1[c] = t.bytes[c];
        f1[c] = t.flops[c];
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CU(cudaGraphAddNode(&node, g, leaves.data(), nullptr, leaves.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    st = capture_into(ctx, body, nullptr, 0, nullptr, [&]() -> tpmg_status {
        const Launch L = launch_of(ctx);
        ctx->net_coarse_on = learned && ctx->net[TPMG_NET_COARSE];
        tpmg_status s2 = vcycle_fine(ctx, ctx->r, ctx->z);
        ctx->net_coarse_on = false;
        if (s2 != TPMG_OK) return s2;
        LCHK(run(ctx, TPMG_K_DOT, (double)N, [&] { return launch_dot(L, N, ctx->r, ctx->z, ctx->partials, np); }));
        LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] {
            return launch_finish(L, flexible ? FIN_LOOP_BETA_PR : FIN_LOOP_BETA, ctx->partials, np, ctx->sc, &loop);
        }));
        LCHK(run(ctx, TPMG_K_XPBY, (double)N, [&] { return launch_xpby(L, N, ctx->sc, ctx->z, ctx->pv); }));
        LCHK(run(ctx, TPMG_K_APPLY, (double)N, [&] { return launch_apply(L, fl, ctx->vert, ctx->pv, ctx->q, ctx->partials, np); }));
        LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_ALPHA, ctx->partials, np, ctx->sc); }));
        const double *z_old = flexible ? ctx->z : nullptr;
        LCHK(run_w(ctx, TPMG_K_AXPY, (double)N,
                   Alg{((z_old ? 56.0 : 48.0) + (ctx->r32 ? 4.0 : 0.0)) * N, (z_old ? 8.0 : 6.0) * N}, [&] {
                       return launch_axpy_pair(L, N, ctx->sc, ctx->pv, ctx->q, u, ctx->r, ctx->partials, np, z_old,
                                               ctx->r32);
                   }));
        LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_LOOP_RR, ctx->partials, np, ctx->sc, &loop); }));
        if (flexible)
            LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_RZC, ctx->partials + np, np, ctx->sc); }));
        return TPMG_OK;
    });
    long long total = 0;
    for (int c = 0; c < TPMG_K_COUNT; ++c) total += t.launches[c] - l0[c];
    if (init_launches) *init_launches = after_init;
    if (iter_launches) *iter_launches = total - after_init;
    if (cls)
        for (int c = 0; c < TPMG_K_COUNT; ++c) {
            cls->init[c] = l1[c] - l0[c];
            cls->iter[c] = t.launches[c] - l1[c];
            cls->uinit[c] = u1[c] - u0[c];
            cls->uiter[c] = t.units[c] - u1[c];
            cls->binit[c] = b1[c] - b0[c];
            cls->biter[c] = t.bytes[c] - b1[c];
            cls->finit[c] = f1[c] - f0[c];
            cls->fiter[c] = t.flops[c] - f1[c];
        }
    std::copy(l0, l0 + TPMG_K_COUNT, t.launches);
    std::copy(u0, u0 + TPMG_K_COUNT, t.units);
    std::copy(b0, b0 + TPMG_K_COUNT, t.bytes);
    std::copy(f0, f0 + TPMG_K_COUNT, t.flops);
    return st;
}

// Result of a device-side solve from the scalars (and history) read back.
tpmg_status loop_result(tpmg_ctx *ctx, const Scalars &s, double rtol, int max_iter, int *iters, double *rel)
{
    *iters = s.it;
    if (s.flag & 2) return fail(ctx, TPMG_ERR_BREAKDOWN, "non-finite residual");
    if (s.flag & 1) return fail(ctx, TPMG_ERR_BREAKDOWN, "p.Ap <= 0: operator or preconditioner not SPD");
    if (s.rr0 == 0.0) {
        *rel = 0.0;
        return TPMG_OK;
    }
    *rel = std::sqrt(s.rr / s.rr0);
    if (*rel <= rtol && s.it <= max_iter) return TPMG_OK;
    return fail(ctx, TPMG_ERR_NOT_CONVERGED, "max_iter reached before rtol");
}

// tpmg_solve with the loop on the device: one graph launch per solve (the
// graph is captured once per argument set), one read-back at the end.  In two
// parts, so that several solves can be enqueued before their results are read:
// pcg_graph_launch enqueues the solve and the copy of its scalars into *h_out;
// pcg_graph_result turns those scalars, once the stream has reached them, into
// the solve's results (and counts its launches).
tpmg_status pcg_graph_launch(tpmg_ctx *ctx, const double *f, double *u, double rtol, int max_iter, Scalars *h_out,
                             const tpmg_ctx::SolveGraph **used)
{
    auto hit = [&](const tpmg_ctx::SolveGraph &e) {
        return e.exec && e.f == f && e.u == u && e.rtol == rtol && e.max_iter == max_iter;
    };
    tpmg_ctx::SolveGraph *slot = hit(ctx->sg[0]) ? &ctx->sg[0] : hit(ctx->sg[1]) ? &ctx->sg[1] : nullptr;
    if (!slot) {
        slot = ctx->sg[0].used <= ctx->sg[1].used ? &ctx->sg[0] : &ctx->sg[1];
        auto &sg = *slot;
        if (sg.exec) cudaGraphExecDestroy(sg.exec);
        sg = tpmg_ctx::SolveGraph{};
        cudaGraph_t g;
        CU(cudaGraphCreate(&g, 0));
        tpmg_status st = append_solve(ctx, g, f, u, rtol, max_iter, &sg.init, &sg.iter, false, &sg.cls);
        cudaError_t e = st == TPMG_OK ? cudaGraphInstantiate(&sg.exec, g, 0) : cudaSuccess;
        cudaGraphDestroy(g);
        if (st != TPMG_OK) return st;
        if (e != cudaSuccess) {
            sg.exec = nullptr;
            return fail(ctx, TPMG_ERR_CUDA, std::string("solve graph: ") + cudaGetErrorString(e));
        }
        sg.f = f;
        sg.u = u;
        sg.rtol = rtol;
        sg.max_iter = max_iter;
    }
    slot->used = ++ctx->sg_clock;
    CU(cudaGraphLaunch(slot->exec, ctx->stream));
    CU(cudaMemcpyAsync(h_out, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
    *used = slot;
    return TPMG_OK;
}

tpmg_status pcg_graph_result(tpmg_ctx *ctx, const Scalars &s, const tpmg_ctx::SolveGraph &sg, double rtol,
                             int max_iter, int *iters, double *rel)
{
    ctx->last_launches = sg.init + (long long)s.it * sg.iter;
    // the replay's launches count like launches made one by one (tpmg_profile_read)
    if (s.it >= 0)
        for (int c = 0; c < TPMG_K_COUNT; ++c) {
            ctx->tr.launches[c] += sg.cls.init[c] + (long long)s.it * sg.cls.iter[c];
            ctx->tr.units[c] += sg.cls.uinit[c] + s.it * sg.cls.uiter[c];
            ctx->tr.bytes[c] += sg.cls.binit[c] + s.it * sg.cls.biter[c];
            ctx->tr.flops[c] += sg.cls.finit[c] + s.it * sg.cls.fiter[c];
        }
    return loop_result(ctx, s, rtol, max_iter, iters, rel);
}

tpmg_status pcg_graph(tpmg_ctx *ctx, const double *f, double *u, double rtol, int max_iter, int *iters, double *rel,
                      double *hist)
{
    const tpmg_ctx::SolveGraph *sg = nullptr;
    const tpmg_status st = pcg_graph_launch(ctx, f, u, rtol, max_iter, ctx->h_sc, &sg);
    if (st != TPMG_OK) return st;
    CU(cudaStreamSynchronize(ctx->stream));
    const Scalars s = *ctx->h_sc;
    if (hist && s.it >= 0) CU(cudaMemcpy(hist, ctx->d_hist, sizeof(double) * (s.it + 1), cudaMemcpyDeviceToHost));
    return pcg_graph_result(ctx, s, *sg, rtol, max_iter, iters, rel);
}

// The sum of a dot product on the host (block partials, fixed-order finish, one read-back).
tpmg_status dot_host(tpmg_ctx *ctx, const double *a, const double *b, double *out)
{
    const Launch L = launch_of(ctx);
    const long N = ctx->N;
    const int np = ctx->n_part;
    LCHK(run(ctx, TPMG_K_DOT, (double)N, [&] { return launch_dot(L, N, a, b, ctx->partials, np); }));
    LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_SUM, ctx->partials, np, ctx->sc); }));
    tpmg_status st = read_scalars(ctx);
    if (st == TPMG_OK) *out = ctx->h_sc->sum;
    return st;
}

// Preconditioned Richardson iteration (Sec. 5): r = f - A u (the true residual,
// with ||r||^2), z = B r, u <- u + z, until ||r|| <= rtol ||r_0||.
tpmg_status richardson(tpmg_ctx *ctx, const double *f, double *u, double rtol, int max_iter, int *iters, double *rel,
                       double *hist)
{
    const Launch L = launch_of(ctx);
    LevelDev &fl = ctx->lv[ctx->p.n_levels - 1];
    const long N = ctx->N;
    const int np = ctx->n_part;
    *iters = 0;
    *rel = 1.0;
    double rr0 = 0.0;
    for (int it = 0;; ++it) {
        LCHK(residual_probed(ctx, L, f, u, ctx->r));
        LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_SUM, ctx->partials, np, ctx->sc); }));
        tpmg_status st = read_scalars(ctx);
        if (st != TPMG_OK) return st;
        const double rr = ctx->h_sc->sum;
        if (!std::isfinite(rr)) return fail(ctx, TPMG_ERR_BREAKDOWN, "non-finite residual");
        if (it == 0) {
            rr0 = rr;
            if (hist) hist[0] = 1.0;
            if (rr0 == 0.0) { *rel = 0.0; return TPMG_OK; }
        } else {
            *iters = it;
            *rel = std::sqrt(rr / rr0);
            if (hist) hist[it] = *rel;
            if (*rel <= rtol) return TPMG_OK;
        }
        if (it == max_iter) break;
        if ((st = vcycle_fine(ctx, ctx->r, ctx->z)) != TPMG_OK) return st;
        LCHK(run(ctx, TPMG_K_AXPY, (double)N, [&] { return launch_lincomb(L, N, 1.0, u, 1.0, ctx->z, 0.0, nullptr, u); }));
    }
    return fail(ctx, TPMG_ERR_NOT_CONVERGED, "max_iter reached before rtol");
}

// BiCGStab (van der Vorst 1992) preconditioned from the right by one V-cycle per
// application, the oracle's steps in the same order: with r^ = r_0,
//   rho = <r^, r>, beta = (rho / rho_prev)(alpha / omega), p = r + beta (p - omega v),
//   y = B p, v = A y, alpha = rho / <r^, v>, s = r - alpha v,
//   z = B s, t = A z, omega = <t, s> / <t, t>, u += alpha y + omega z, r = s - omega t.
tpmg_status bicgstab(tpmg_ctx *ctx, const double *f, double *u, double rtol, int max_iter, int *iters, double *rel,
                     double *hist)
{
    const Launch L = launch_of(ctx);
    LevelDev &fl = ctx->lv[ctx->p.n_levels - 1];
    const long N = ctx->N;
    const int np = ctx->n_part;
    if (!ctx->bv) {
        CU(dalloc(ctx, &ctx->bv, (size_t)N));
        CU(dalloc(ctx, &ctx->bs, (size_t)N));
        CU(dalloc(ctx, &ctx->bz, (size_t)N));
        CU(dalloc(ctx, &ctx->bh, (size_t)N));
    }
    double *r = ctx->r, *rh = ctx->bh, *p = ctx->pv, *v = ctx->bv, *y = ctx->z, *sv = ctx->bs, *z = ctx->bz, *t = ctx->q;
    *iters = 0;
    *rel = 1.0;
    LCHK(residual_probed(ctx, L, f, u, r));
    LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_SUM, ctx->partials, np, ctx->sc); }));
    tpmg_status st = read_scalars(ctx);
    if (st != TPMG_OK) return st;
    const double rr0 = ctx->h_sc->sum;
    if (hist) hist[0] = 1.0;
    if (!std::isfinite(rr0)) return fail(ctx, TPMG_ERR_BREAKDOWN, "initial residual is not finite");
    if (rr0 == 0.0) { *rel = 0.0; return TPMG_OK; }
    LCHK(run(ctx, TPMG_K_COPY, (double)N, [&] { return cudaMemcpyAsync(rh, r, sizeof(double) * N, cudaMemcpyDeviceToDevice, ctx->issue); }));
    LCHK(run(ctx, TPMG_K_COPY, (double)N, [&] { return cudaMemsetAsync(p, 0, sizeof(double) * N, ctx->issue); }));
    LCHK(run(ctx, TPMG_K_COPY, (double)N, [&] { return cudaMemsetAsync(v, 0, sizeof(double) * N, ctx->issue); }));
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    for (int it = 0; it < max_iter; ++it) {
        double rho, rv, ts, tt, rr;
        if ((st = dot_host(ctx, rh, r, &rho)) != TPMG_OK) return st;
        if (!(rho != 0.0) || !std::isfinite(rho)) return fail(ctx, TPMG_ERR_BREAKDOWN, "BiCGStab: <r^, r> = 0");
        const double beta = (rho / rho_prev) * (alpha / omega);
        // p = r + beta (p - omega v)
        LCHK(run(ctx, TPMG_K_XPBY, (double)N, [&] { return launch_lincomb(L, N, 1.0, r, beta, p, -beta * omega, v, p); }));
        if ((st = vcycle_fine(ctx, p, y)) != TPMG_OK) return st;
        LCHK(run(ctx, TPMG_K_APPLY, (double)N, [&] { return launch_apply(L, fl, ctx->vert, y, v, ctx->partials, np); }));
        if ((st = dot_host(ctx, rh, v, &rv)) != TPMG_OK) return st;
        if (!(rv != 0.0) || !std::isfinite(rv)) return fail(ctx, TPMG_ERR_BREAKDOWN, "BiCGStab: <r^, v> = 0");
        alpha = rho / rv;
        LCHK(run(ctx, TPMG_K_AXPY, (double)N, [&] { return launch_lincomb(L, N, 1.0, r, -alpha, v, 0.0, nullptr, sv); }));
        if ((st = vcycle_fine(ctx, sv, z)) != TPMG_OK) return st;
        LCHK(run(ctx, TPMG_K_APPLY, (double)N, [&] { return launch_apply(L, fl, ctx->vert, z, t, ctx->partials, np); }));
        if ((st = dot_host(ctx, t, t, &tt)) != TPMG_OK) return st;
        if (!(tt > 0.0) || !std::isfinite(tt)) return fail(ctx, TPMG_ERR_BREAKDOWN, "BiCGStab: <t, t> = 0");
        if ((st = dot_host(ctx, t, sv, &ts)) != TPMG_OK) return st;
        omega = ts / tt;
        LCHK(run(ctx, TPMG_K_AXPY, (double)N, [&] { return launch_lincomb(L, N, 1.0, u, alpha, y, omega, z, u); }));
        LCHK(run(ctx, TPMG_K_AXPY, (double)N, [&] { return launch_lincomb(L, N, 1.0, sv, -omega, t, 0.0, nullptr, r); }));
        rho_prev = rho;
        if ((st = dot_host(ctx, r, r, &rr)) != TPMG_OK) return st;
        *iters = it + 1;
        *rel = std::sqrt(rr / rr0);
        if (hist) hist[it + 1] = *rel;
        if (!std::isfinite(*rel)) return fail(ctx, TPMG_ERR_BREAKDOWN, "non-finite residual");
        if (*rel <= rtol) return TPMG_OK;
    }
    return fail(ctx, TPMG_ERR_NOT_CONVERGED, "max_iter reached before rtol");
}

// learned = true: the host-driven form of tpmg_solve_learned's loop (same
// kernels, same order as append_solve with learned set).
tpmg_status pcg(tpmg_ctx *ctx, const double *f, double *u, double rtol, int max_iter, int *iters, double *rel,
                double *hist, bool learned = false)
{
    const Launch L = launch_of(ctx);
    LevelDev &fl = ctx->lv[ctx->p.n_levels - 1];
    const long N = ctx->N;
    const int np = ctx->n_part;
    // the FP32 V-cycle is not exactly symmetric: Polak-Ribiere coefficient (flexible CG)
    const bool flexible = ctx->p.precision == TPMG_PREC_MIXED || learned;
    *iters = 0;
    *rel = 1.0;
    if (learned && ctx->net[TPMG_NET_WARM]) {   // the network's guess and one relaxation
        const tpmg_status s1 = warm_start(ctx, L, f, u);
        if (s1 != TPMG_OK) return s1;
    }
    LCHK(residual_probed(ctx, L, f, u, ctx->r));
    if (learned) {
        LCHK(run(ctx, TPMG_K_DOT, (double)N, [&] { return launch_dot(L, N, f, f, ctx->partials + np, np); }));
        LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_RR0F, ctx->partials, np, ctx->sc); }));
        LCHK(run(ctx, TPMG_K_COPY, (double)N, [&] { return launch_judge_reset(L, ctx->sc, N, f, u, ctx->r, ctx->r32); }));
    } else {
        LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_RR0, ctx->partials, np, ctx->sc); }));
    }
    tpmg_status st = read_scalars(ctx);
    if (st != TPMG_OK) return st;
    const double rr0 = ctx->h_sc->rr0;
    const double rel0 = learned && rr0 > 0.0 ? std::sqrt(ctx->h_sc->rr / rr0) : 1.0;
    if (hist) hist[0] = rel0;
    if (!std::isfinite(rr0) || !std::isfinite(rel0)) return fail(ctx, TPMG_ERR_BREAKDOWN, "initial residual is not finite");
    if (rr0 == 0.0) { *rel = 0.0; return TPMG_OK; }
    *rel = rel0;
    if (learned && (rel0 <= rtol || max_iter == 0)) return rel0 <= rtol ? TPMG_OK : fail(ctx, TPMG_ERR_NOT_CONVERGED, "max_iter reached before rtol");
    // z = B r: the learned form's V-cycle runs kernel by kernel with the COARSE network
    auto precondition = [&]() -> tpmg_status {
        if (!learned) return vcycle_pcg(ctx);
        ctx->net_coarse_on = ctx->net[TPMG_NET_COARSE] != nullptr;
        const tpmg_status s2 = vcycle_fine(ctx, ctx->r, ctx->z);
        ctx->net_coarse_on = false;
        return s2;
    };
    if ((st = precondition()) != TPMG_OK) return st;
    LCHK(run(ctx, TPMG_K_DOT, (double)N, [&] { return launch_dot(L, N, ctx->r, ctx->z, ctx->partials, np); }));
    LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_RZ0, ctx->partials, np, ctx->sc); }));
    LCHK(run(ctx, TPMG_K_COPY, (double)N, [&] { return cudaMemcpyAsync(ctx->pv, ctx->z, sizeof(double) * N, cudaMemcpyDeviceToDevice, ctx->stream); }));
    for (int it = 0; it < max_iter; ++it) {
        LCHK(run(ctx, TPMG_K_APPLY, (double)N, [&] { return launch_apply(L, fl, ctx->vert, ctx->pv, ctx->q, ctx->partials, np); }));
        LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_ALPHA, ctx->partials, np, ctx->sc); }));
        // flexible CG (mixed precision): the axpy also forms <r_new, z_old>
        const double *z_old = flexible ? ctx->z : nullptr;
        LCHK(run_w(ctx, TPMG_K_AXPY, (double)N,
                   Alg{((z_old ? 56.0 : 48.0) + (ctx->r32 ? 4.0 : 0.0)) * N, (z_old ? 8.0 : 6.0) * N}, [&] {
                       return launch_axpy_pair(L, N, ctx->sc, ctx->pv, ctx->q, u, ctx->r, ctx->partials, np, z_old,
                                               ctx->r32);
                   }));
        LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_RR, ctx->partials, np, ctx->sc); }));
        if (flexible) LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, FIN_RZC, ctx->partials + np, np, ctx->sc); }));
        if ((st = read_scalars(ctx)) != TPMG_OK) return st;
        const Scalars &s = *ctx->h_sc;
        if (s.flag & 1) return fail(ctx, TPMG_ERR_BREAKDOWN, "p.Ap <= 0: operator or preconditioner not SPD");
        if (s.flag & 2) return fail(ctx, TPMG_ERR_BREAKDOWN, "non-finite residual");
        *iters = it + 1;
        *rel = std::sqrt(s.rr / rr0);
        if (hist) hist[it + 1] = *rel;
        if (*rel <= rtol) return TPMG_OK;
        if (it + 1 == max_iter) break;
        if ((st = precondition()) != TPMG_OK) return st;
        LCHK(run(ctx, TPMG_K_DOT, (double)N, [&] { return launch_dot(L, N, ctx->r, ctx->z, ctx->partials, np); }));
        LCHK(run(ctx, TPMG_K_FINISH, 1.0, [&] { return launch_finish(L, flexible ? FIN_BETA_PR : FIN_BETA, ctx->partials, np, ctx->sc); }));
        LCHK(run(ctx, TPMG_K_XPBY, (double)N, [&] { return launch_xpby(L, N, ctx->sc, ctx->z, ctx->pv); }));
    }
    return fail(ctx, TPMG_ERR_NOT_CONVERGED, "max_iter reached before rtol");
}

// The host-driven outer iteration of params.outer.
tpmg_status outer_host(tpmg_ctx *ctx, const double *f, double *u, double rtol, int max_iter, int *iters, double *rel,
                       double *hist)
{
    if (ctx->p.outer == TPMG_OUTER_RICHARDSON) return richardson(ctx, f, u, rtol, max_iter, iters, rel, hist);
    if (ctx->p.outer == TPMG_OUTER_BICGSTAB) return bicgstab(ctx, f, u, rtol, max_iter, iters, rel, hist);
    return pcg(ctx, f, u, rtol, max_iter, iters, rel, hist);
}

// The BF16 stencil of one multigrid level (refinement of H), full storage (Sec. 4.2):
// with pb == NULL from the factorised profiles; otherwise from general profiles of
// this level, pb, ps [n][n_r] (beta, alpha_S at the cells) and pr [n][n_r+1] (alpha_r
// at the faces), an edge taking the mean of its two cells' alpha_S.
void bf16_stencil(const tpmg_ctx *ctx, const HostLevel &H, const double *pb, const double *pr, const double *ps,
                  std::vector<bf16x4> &cp, std::vector<unsigned short> &cv)
{
    const HostGrid &G = ctx->host;
    const int n_r = ctx->p.n_r;
    cp.resize((size_t)H.n * n_r);
    cv.resize((size_t)H.n * n_r);
    for (int T = 0; T < H.n; ++T) {
        double ge[3], aB = 0.0, aR = 0.0;
        if (!pb) {
            for (int e = 0; e < 3; ++e)
                ge[e] = H.g[3 * T + e] * (ctx->ps_aS.empty() ? 1.0
                                          : 0.5 * (ctx->ps_aS[H.ref][T] + ctx->ps_aS[H.ref][H.nbr[3 * T + e]]));
            aB = H.area[T] * hfac(ctx->ps_beta, H.ref, T);
            aR = H.area[T] * hfac(ctx->ps_ar, H.ref, T);
        }
        for (int k = 0; k < n_r; ++k) {
            const size_t i = (size_t)T * n_r + k;
            if (!pb) {
                const double hr = G.omega2 * G.dr[k] * vfac(ctx->pr_aS, k);
                cp[i] = bf16x4{bf16_bits(hr * ge[0]), bf16_bits(hr * ge[1]), bf16_bits(hr * ge[2]),
                               bf16_bits(aB * (G.vol[k] * vfac(ctx->pr_beta, k)))};
                cv[i] = bf16_bits(aR * (G.omega2 * G.face[k] * vfac(ctx->pr_ar, k)));
            } else {
                unsigned short a[3];
                for (int e = 0; e < 3; ++e) {
                    const double edge = 0.5 * (ps[i] + ps[(size_t)H.nbr[3 * T + e] * n_r + k]);
                    a[e] = bf16_bits(G.omega2 * G.dr[k] * H.g[3 * T + e] * edge);
                }
                cp[i] = bf16x4{a[0], a[1], a[2], bf16_bits(H.area[T] * G.vol[k] * pb[i])};
                cv[i] = bf16_bits(G.omega2 * H.area[T] * G.face[k] * pr[(size_t)T * (n_r + 1) + k]);
            }
        }
    }
}

// The FP64 stencil of one multigrid level stored per unknown (Sec. 4.2; Appendix A,
// eq. hatFunctionsNonFac), horizontal part: c [n][n_r] {alphaS_hat e = 0, 1, 2, beta_hat}.
// With pb == NULL from the factorised profiles (the products the factorised kernels
// form); otherwise from general profiles of this level, pb, ps [n][n_r] (beta, alpha_S
// at the cells), an edge taking the mean of its two cells' alpha_S.
void fp64_horizontal(const tpmg_ctx *ctx, const HostLevel &H, const double *pb, const double *ps, std::vector<dbl4> &c)
{
    const HostGrid &G = ctx->host;
    const int n_r = ctx->p.n_r;
    c.resize((size_t)H.n * n_r);
    for (int T = 0; T < H.n; ++T) {
        double ge[3];
        for (int e = 0; e < 3; ++e)
            ge[e] = H.g[3 * T + e] * (ctx->ps_aS.empty() ? 1.0
                                      : 0.5 * (ctx->ps_aS[H.ref][T] + ctx->ps_aS[H.ref][H.nbr[3 * T + e]]));
        const double aB = H.area[T] * hfac(ctx->ps_beta, H.ref, T);
        for (int k = 0; k < n_r; ++k) {
            const size_t i = (size_t)T * n_r + k;
            if (!pb) {
                const double hr = G.omega2 * G.dr[k] * vfac(ctx->pr_aS, k);
                c[i] = dbl4{hr * ge[0], hr * ge[1], hr * ge[2], aB * (G.vol[k] * vfac(ctx->pr_beta, k))};
            } else {
                const double hr = G.omega2 * G.dr[k];
                double a[3];
                for (int e = 0; e < 3; ++e)
                    a[e] = hr * H.g[3 * T + e] * (0.5 * (ps[i] + ps[(size_t)H.nbr[3 * T + e] * n_r + k]));
                c[i] = dbl4{a[0], a[1], a[2], H.area[T] * G.vol[k] * pb[i]};
            }
        }
    }
}

// Vertical part: cr [n][n_r + 1] alphar_hat of face k, zero on the two boundary faces
// (no flux through the bottom and the top).  With pr == NULL from the factorised
// profiles, otherwise from a general alpha_r of this level [n][n_r + 1].
void fp64_vertical(const tpmg_ctx *ctx, const HostLevel &H, const double *pr, std::vector<double> &cr)
{
    const HostGrid &G = ctx->host;
    const int n_r = ctx->p.n_r;
    cr.resize((size_t)H.n * (n_r + 1));
    for (int T = 0; T < H.n; ++T) {
        const double aR = H.area[T] * hfac(ctx->ps_ar, H.ref, T);
        for (int k = 0; k <= n_r; ++k) {
            const size_t fi = (size_t)T * (n_r + 1) + k;
            if (k == 0 || k == n_r)
                cr[fi] = 0.0;
            else if (!pr)
                cr[fi] = aR * (G.omega2 * G.face[k] * vfac(ctx->pr_ar, k));
            else
                cr[fi] = G.omega2 * H.area[T] * G.face[k] * pr[fi];
        }
    }
}

// Vertical advection of one level per face (Appendix A, centred): x [n][n_r + 1]
// X_{T,face} = omega^2 sigma_face |T| r_face^2 / (r_{face+1} - r_{face-1}) xi_{T,face}
// (half the face factor of alphar_hat), from the factorised xi with pxi == NULL,
// otherwise from a general xi of this level [n][n_r + 1]; zero on the boundary faces.
void fp64_advection(const tpmg_ctx *ctx, const HostLevel &H, const double *pxi, std::vector<double> &x)
{
    const HostGrid &G = ctx->host;
    const int n_r = ctx->p.n_r;
    x.assign((size_t)H.n * (n_r + 1), 0.0);
    for (int T = 0; T < H.n; ++T) {
        const double aX = H.area[T] * hfac(ctx->ps_xi, H.ref, T);
        for (int k = 1; k < n_r; ++k) {
            const size_t fi = (size_t)T * (n_r + 1) + k;
            if (!pxi)
                x[fi] = aX * (0.5 * G.omega2 * G.face[k] * vfac(ctx->pr_xi, k));
            else
                x[fi] = G.omega2 * H.area[T] * (0.5 * G.face[k]) * pxi[fi];
        }
    }
}

// Every row of every column must couple to its neighbours with non-negative weights
// (down_k = cr_k - dr_k X_k, up_k = cr_{k+1} + dr_k X_{k+1}) for the excess-carried
// elimination of the line smoother: an M-matrix column block.
bool couplings_ok(const tpmg_ctx *ctx, int n_cells, const std::vector<double> &cr, const std::vector<double> &x)
{
    const int n_r = ctx->p.n_r;
    for (int T = 0; T < n_cells; ++T)
        for (int k = 0; k < n_r; ++k) {
            const size_t f = (size_t)T * (n_r + 1) + k;
            const double dr = ctx->host.dr[k];
            if (k > 0 && !(cr[f] - dr * x[f] >= 0.0)) return false;
            if (k < n_r - 1 && !(cr[f + 1] + dr * x[f + 1] >= 0.0)) return false;
        }
    return true;
}

// The vertical advection a level's V-cycle uses: its stored X (FULL: vcx; mixed: cxv in
// BF16) or its factor |T| xi^S (area_x), from the factorised xi (pxi == NULL) or a
// general one of this level; none when neither is given.  Checks the column blocks.
tpmg_status upload_advection(tpmg_ctx *ctx, const HostLevel &H, LevelDev &D, const double *pxi, const double *pr)
{
    const tpmg_params &p = ctx->p;
    const bool mixed = p.precision == TPMG_PREC_MIXED, stored = p.coeff_storage == TPMG_COEFF_FULL;
    const bool on = pxi ? true : (stored && pr ? false : ctx->xi_fac);   // FULL with general profiles: their xi only
    const size_t nn = (size_t)H.n * p.n_r;
    D.vcx_on = D.cxv_on = false;
    if (!on) return TPMG_OK;
    std::vector<double> x, cr;
    fp64_advection(ctx, H, pxi, x);
    fp64_vertical(ctx, H, pr, cr);
    if (!couplings_ok(ctx, H.n, cr, x))
        return fail(ctx, TPMG_ERR_INVALID_ARG, "vertical advection too strong: a column block is no M-matrix "
                                               "(dr |xi| > 2 alpha_r on some face)");
    if (mixed) {
        std::vector<unsigned short> xb(nn);
        for (int T = 0; T < H.n; ++T)
            for (int k = 0; k < p.n_r; ++k) xb[(size_t)T * p.n_r + k] = bf16_bits(x[(size_t)T * (p.n_r + 1) + k]);
        if (!D.cxv) CU(dalloc(ctx, &D.cxv, nn));
        if (!D.fb32) CU(dalloc(ctx, &D.fb32, nn));   // the column blocks' multipliers, stored with advection
        if (!D.fc32) CU(dalloc(ctx, &D.fc32, nn));
        CU(cudaMemcpyAsync(D.cxv, xb.data(), nn * sizeof(unsigned short), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        D.cxv_on = true;
    } else if (stored) {
        if (!D.vcx) CU(dalloc(ctx, &D.vcx, x.size()));
        CU(cudaMemcpyAsync(D.vcx, x.data(), x.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        D.vcx_on = true;
    } else if (!D.area_x) {   // factorised or partial: xi stays factorised
        std::vector<double> ax(H.n);
        for (int T = 0; T < H.n; ++T) ax[T] = H.area[T] * hfac(ctx->ps_xi, H.ref, T);
        CU(dalloc(ctx, &D.area_x, ax.size()));
        CU(cudaMemcpyAsync(D.area_x, ax.data(), ax.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    return TPMG_OK;
}

// Weights of the linear prolongation from coarse level H to its children on level
// Hf (Sec. 5; see TPMG_PROLONG_LINEAR): for coarse cell T with centre c and unit
// normal n, an orthonormal basis (a, b) of the tangent plane is built from the
// coordinate axis least aligned with n; the 3 neighbours' offsets c_e - c give rows
// x_e = ((c_e - c).a, (c_e - c).b), the children's offsets y_j likewise, and child j's
// weight on u_e - u_T is y_j^T (X^T X)^{-1} x_e (the least-squares gradient).
void prolong_weights(const HostLevel &H, const HostLevel &Hf, std::vector<double> &w)
{
    w.assign((size_t)H.n * 12, 0.0);
    auto cen = [](const HostLevel &L, int T) { return &L.centre[3 * (size_t)T]; };
    for (int T = 0; T < H.n; ++T) {
        const double *c = cen(H, T);
        const double len = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        const double n[3] = {c[0] / len, c[1] / len, c[2] / len};
        int ax = 0;
        for (int d = 1; d < 3; ++d)
            if (std::fabs(n[d]) < std::fabs(n[ax])) ax = d;
        double a[3] = {0.0, 0.0, 0.0};
        a[ax] = 1.0;
        const double an = a[ax] * n[ax];
        for (int d = 0; d < 3; ++d) a[d] -= an * n[d];
        const double al = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        for (int d = 0; d < 3; ++d) a[d] /= al;
        const double b[3] = {n[1] * a[2] - n[2] * a[1], n[2] * a[0] - n[0] * a[2], n[0] * a[1] - n[1] * a[0]};
        auto coords = [&](const double *p, double &x, double &y) {
            const double d0 = p[0] - c[0], d1 = p[1] - c[1], d2 = p[2] - c[2];
            x = d0 * a[0] + d1 * a[1] + d2 * a[2];
            y = d0 * b[0] + d1 * b[1] + d2 * b[2];
        };
        double ex[3], ey[3], sxx = 0.0, sxy = 0.0, syy = 0.0;
        for (int e = 0; e < 3; ++e) {
            coords(cen(H, H.nbr[3 * T + e]), ex[e], ey[e]);
            sxx += ex[e] * ex[e];
            sxy += ex[e] * ey[e];
            syy += ey[e] * ey[e];
        }
        const double det = sxx * syy - sxy * sxy;
        for (int j = 0; j < 4; ++j) {
            double yx, yy;
            coords(cen(Hf, 4 * T + j), yx, yy);
            const double gx = (syy * yx - sxy * yy) / det, gy = (sxx * yy - sxy * yx) / det;
            for (int e = 0; e < 3; ++e) w[(size_t)T * 12 + 3 * j + e] = gx * ex[e] + gy * ey[e];
        }
    }
}

// General per-unknown profiles of one level from the next finer (m values per cell):
// each coarse (cell, j) the area-weighted mean over the 4 children's (cell, j).
std::vector<double> average_children(const HostLevel &fine, const std::vector<double> &pf, int m)
{
    const int nc = fine.n / 4;
    std::vector<double> pc((size_t)nc * m);
    for (int T = 0; T < nc; ++T)
        for (int j = 0; j < m; ++j) {
            double s = 0.0, a = 0.0;
            for (int c = 0; c < 4; ++c) {
                const double ac = fine.area[4 * T + c];
                s += ac * pf[(size_t)(4 * T + c) * m + j];
                a += ac;
            }
            pc[(size_t)T * m + j] = s / a;
        }
    return pc;
}

tpmg_status upload_level(tpmg_ctx *ctx, int l)
{
    const tpmg_params &p = ctx->p;
    const HostLevel &H = ctx->host.lev[p.refinement - (p.n_levels - 1 - l)];
    LevelDev &D = ctx->lv[l];
    D.n = H.n;
    D.ref = H.ref;
    D.n_colours = H.n_colours;
    std::vector<int4> nb(H.n);
    std::vector<dbl4> g(H.n);
    std::vector<double> areaB(H.n), areaR(H.n);
    // an edge's alpha_S^S: the mean of its two cells' factors (symmetric operator)
    auto edge = [&](int T, int e) {
        return ctx->ps_aS.empty() ? 1.0 : 0.5 * (ctx->ps_aS[H.ref][T] + ctx->ps_aS[H.ref][H.nbr[3 * T + e]]);
    };
    for (int T = 0; T < H.n; ++T) {
        int mask = 0;
        for (int e = 0; e < 3; ++e)
            if (H.colour[H.nbr[3 * T + e]] < H.colour[T]) mask |= 1 << e;
        nb[T] = make_int4(H.nbr[3 * T], H.nbr[3 * T + 1], H.nbr[3 * T + 2], mask);
        const double g0 = H.g[3 * T] * edge(T, 0), g1 = H.g[3 * T + 1] * edge(T, 1), g2 = H.g[3 * T + 2] * edge(T, 2);
        g[T] = dbl4{g0, g1, g2, (g0 + g1) + g2};
        areaB[T] = H.area[T] * hfac(ctx->ps_beta, H.ref, T);
        areaR[T] = H.area[T] * hfac(ctx->ps_ar, H.ref, T);
    }
    // relaxation tasks: the cells of each colour in ascending order, padded to whole tasks
    std::vector<int> tasks;
    D.colour_task_off.assign(H.n_colours + 1, 0);
    D.colour_cells.assign(H.n_colours, 0);
    for (int c = 0; c < H.n_colours; ++c) {
        D.colour_task_off[c] = (int)(tasks.size() / kRelaxCols);
        for (int T = 0; T < H.n; ++T)
            if (H.colour[T] == c) {
                tasks.push_back(T);
                ++D.colour_cells[c];
            }
        while (tasks.size() % kRelaxCols) tasks.push_back(-1);
    }
    D.n_tasks = (int)(tasks.size() / kRelaxCols);
    D.colour_task_off[H.n_colours] = D.n_tasks;
    D.jmid = (p.n_r - 1) / 2;
    D.steps = p.n_r - 1 - D.jmid;
    const size_t n = H.n, nn = (size_t)H.n * p.n_r;
    const size_t nf = (size_t)D.n_tasks * std::max(D.steps, 1) * 32;
    CU(dalloc(ctx, &D.nbr, n));
    CU(dalloc(ctx, &D.g, n));
    CU(dalloc(ctx, &D.area, n));
    CU(dalloc(ctx, &D.area_r, n));
    CU(dalloc(ctx, &D.task_cells, tasks.size()));
    CU(dalloc(ctx, &D.task_nbr, tasks.size()));
    CU(dalloc(ctx, &D.task_g, tasks.size()));
    const bool mixed = p.precision == TPMG_PREC_MIXED;
    std::vector<dbl4> hc;     // FP64 stencil per unknown (FULL, PARTIAL), alive until the final synchronise
    std::vector<double> hcr;
    if (!mixed && p.coeff_storage != TPMG_COEFF_FACTORISED) {
        fp64_vertical(ctx, H, nullptr, hcr);
        CU(dalloc(ctx, &D.vcr, hcr.size()));
        CU(cudaMemcpyAsync(D.vcr, hcr.data(), hcr.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        if (p.coeff_storage == TPMG_COEFF_FULL) {
            fp64_horizontal(ctx, H, nullptr, nullptr, hc);
            CU(dalloc(ctx, &D.vc, nn));
            CU(cudaMemcpyAsync(D.vc, hc.data(), nn * sizeof(dbl4), cudaMemcpyHostToDevice, ctx->stream));
        }
    }
    if (!mixed) {
        D.scan = H.n <= p.scan_max_cells;
        // on a larger level, colours of at most scan_max_cells / 2 cells are relaxed by the
        // warp scans too: such a pass is latency-bound, and a twisted-task pass takes the
        // time of one task's serial column solve however few tasks it has
        D.scan_pass_tasks = -1;
        if (!D.scan)
            for (int c = 0; c < H.n_colours; ++c)
                if (D.colour_cells[c] <= p.scan_max_cells / 2)
                    D.scan_pass_tasks = std::max(D.scan_pass_tasks, D.colour_task_off[c + 1] - D.colour_task_off[c]);
        if (D.scan || D.scan_pass_tasks >= 0) {
            CU(dalloc(ctx, &D.rinv1, nn));
            CU(dalloc(ctx, &D.fb1, nn));
            CU(dalloc(ctx, &D.fc1, nn));
        }
        CU(dalloc(ctx, &D.rinv, nn));
        CU(dalloc(ctx, &D.fb, nf));
        CU(dalloc(ctx, &D.fc, nf));
        CU(dalloc(ctx, &D.fm, (size_t)D.n_tasks * 2 * kRelaxCols));
        CU(dalloc(ctx, &D.u2, nn));
        if (l < p.n_levels - 1) {
            CU(dalloc(ctx, &D.f, nn));
            CU(dalloc(ctx, &D.u, nn));
        }
    } else {
        // BF16 stencil, full storage: per (T, k) alphaS_hat of the 3 edges and beta_hat,
        // and alphar_hat of face k (Appendix A, eq. hatFunctionsNonFac)
        std::vector<bf16x4> cp;
        std::vector<unsigned short> cv;
        bf16_stencil(ctx, H, nullptr, nullptr, nullptr, cp, cv);
        CU(dalloc(ctx, &D.cpack, nn));
        CU(dalloc(ctx, &D.cvert, nn + 1));   // + a zero coupling after the last column (face n_r)
        CU(cudaMemsetAsync(D.cvert + nn, 0, sizeof(unsigned short), ctx->stream));
        CU(dalloc(ctx, &D.rinv32, nn));
        CU(dalloc(ctx, &D.u32, nn));
        CU(dalloc(ctx, &D.u2_32, nn));
        if (l < p.n_levels - 1) CU(dalloc(ctx, &D.f32, nn));
        CU(cudaMemcpyAsync(D.cpack, cp.data(), nn * sizeof(bf16x4), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemcpyAsync(D.cvert, cv.data(), nn * sizeof(unsigned short), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));   // cp, cv are local
    }
    CU(cudaMemcpyAsync(D.nbr, nb.data(), n * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(D.g, g.data(), n * sizeof(dbl4), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(D.area, areaB.data(), n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(D.area_r, areaR.data(), n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    // learned-form features: geometric cell areas and flux weights
    std::vector<float> ia(H.n);
    std::vector<float4> wn(H.n);
    for (int T = 0; T < H.n; ++T) {
        ia[T] = (float)(1.0 / H.area[T]);
        const double g0 = H.g[3 * T], g1 = H.g[3 * T + 1], g2 = H.g[3 * T + 2], sg = (g0 + g1) + g2;
        wn[T] = make_float4((float)(g0 / sg), (float)(g1 / sg), (float)(g2 / sg), 0.f);
    }
    CU(dalloc(ctx, &D.iarea32, n));
    CU(dalloc(ctx, &D.wnb32, n));
    CU(cudaMemcpyAsync(D.iarea32, ia.data(), n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(D.wnb32, wn.data(), n * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(D.task_cells, tasks.data(), tasks.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    std::vector<int4> tnb(tasks.size(), make_int4(0, 0, 0, 0));
    std::vector<dbl4> tg(tasks.size(), dbl4{0.0, 0.0, 0.0, 0.0});
    for (size_t q = 0; q < tasks.size(); ++q)
        if (tasks[q] >= 0) { tnb[q] = nb[tasks[q]]; tg[q] = g[tasks[q]]; }
    CU(cudaMemcpyAsync(D.task_nbr, tnb.data(), tnb.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(D.task_g, tg.data(), tg.size() * sizeof(dbl4), cudaMemcpyHostToDevice, ctx->stream));
    // the restriction's view of the coarse cells (FP64 levels with a coarser one): each
    // coarse cell's edges to outside cells, which must be 6 (3 of the 12 child-edge
    // sides pair up inside), else the level keeps the child-by-child kernel
    std::vector<RestrictGeo> rg;   // alive until the final synchronise
    if (!mixed && l > 0) {
        const int nc = H.n / 4;
        rg.resize(nc);
        bool ok = true;
        for (int Tc = 0; Tc < nc && ok; ++Tc) {
            int xe[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            double ge[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, gx[4], A[4], Ar[4];
            int m = 0;
            for (int j = 0; j < 4; ++j) {
                const int T = 4 * Tc + j;
                const int nbT[3] = {nb[T].x, nb[T].y, nb[T].z};
                const double gT[3] = {g[T].x, g[T].y, g[T].z};
                gx[j] = 0.0;
                for (int e = 0; e < 3; ++e) {
                    if (nbT[e] / 4 == Tc) continue;
                    if (m == 6) { ok = false; break; }
                    xe[m] = nbT[e];
                    ge[m++] = gT[e];
                    gx[j] += gT[e];
                }
                A[j] = areaB[T];
                Ar[j] = areaR[T];
            }
            ok = ok && m == 6;
            rg[Tc] = RestrictGeo{make_int4(xe[0], xe[1], xe[2], xe[3]), make_int4(xe[4], xe[5], 0, 0),
                                 dbl4{ge[0], ge[1], ge[2], ge[3]}, dbl4{ge[4], ge[5], 0.0, 0.0},
                                 dbl4{gx[0], gx[1], gx[2], gx[3]}, dbl4{A[0], A[1], A[2], A[3]},
                                 dbl4{Ar[0], Ar[1], Ar[2], Ar[3]}};
        }
        if (ok) {
            CU(dalloc(ctx, &D.rgeo, (size_t)nc));
            CU(cudaMemcpyAsync(D.rgeo, rg.data(), rg.size() * sizeof(RestrictGeo), cudaMemcpyHostToDevice, ctx->stream));
        }
    }
    {
        const tpmg_status st = upload_advection(ctx, H, D, nullptr, nullptr);
        if (st != TPMG_OK) return st;
    }
    std::vector<double> pw;   // linear prolongation weights, alive until the final synchronise
    std::vector<float> pw32;
    if (p.prolongation == TPMG_PROLONG_LINEAR && l < p.n_levels - 1) {
        prolong_weights(H, ctx->host.lev[H.ref + 1], pw);
        if (mixed) {
            pw32.assign(pw.begin(), pw.end());
            CU(dalloc(ctx, &D.plin32, pw32.size()));
            CU(cudaMemcpyAsync(D.plin32, pw32.data(), pw32.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
        } else {
            CU(dalloc(ctx, &D.plin, pw.size()));
            CU(cudaMemcpyAsync(D.plin, pw.data(), pw.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        }
    }
    if (!mixed) {
        CU(launch_twisted_factors(launch_of(ctx), D, ctx->vert));
        if (D.rinv1) CU(launch_thomas_factors(launch_of(ctx), D, ctx->vert));
    } else {
        CU(launch_thomas_factors32(launch_of(ctx), D));
    }
    // the host vectors above must outlive the asynchronous copies
    CU(cudaStreamSynchronize(ctx->stream));
    return TPMG_OK;
}

// Autotuner: on every level each relaxation kernel variant (one warp per task,
// or one CTA of 64 / 128 / 256 threads per task) is timed on the level's
// largest colour pass -- NORMAL mode, on the level's zeroed work vectors, one
// warm-up and three timed launches -- and the fastest is kept.  All variants
// perform the same arithmetic in the same order, so the choice changes no
// result, only the time.
tpmg_status autotune(tpmg_ctx *ctx)
{
    const Launch L = launch_of(ctx);
    const bool mixed = ctx->p.precision == TPMG_PREC_MIXED;
    cudaEvent_t a, b;
    CU(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return fail(ctx, TPMG_ERR_CUDA, "autotune: cudaEventCreate");
    }
    tpmg_status st = TPMG_OK;
    for (LevelDev &D : ctx->lv) {
        int c = 0;
        for (int k = 1; k < D.n_colours; ++k)
            if (D.colour_cells[k] > D.colour_cells[c]) c = k;
        const int t0 = D.colour_task_off[c], nt = D.colour_task_off[c + 1] - t0;
        auto pass = [&]() {
            return mixed ? launch_relax32<float>(L, D, PASS_NORMAL, t0, nt, 1.f, D.u2_32, D.u32, D.u32, nullptr, nullptr)
                         : launch_relax(L, D, ctx->vert, PASS_NORMAL, t0, nt, 1.0, D.u2, D.u2, D.u2, nullptr, 2);
        };
        float best = 0.f;
        int best_var = RELAX_CTA128;
        // the warp-scan levels (FP32, and FP64 levels of at most scan_max_cells) have four CTA shapes
        const int n_var = (mixed || D.scan) ? kRelaxVariants32 : (int)RELAX_VARIANTS;
        for (int var = 0; var < n_var && st == TPMG_OK; ++var) {
            D.relax_variant = var;
            cudaError_t e = pass();
            if (e == cudaSuccess) e = cudaEventRecord(a, ctx->stream);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = pass();
            if (e == cudaSuccess) e = cudaEventRecord(b, ctx->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (e != cudaSuccess) st = fail(ctx, TPMG_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
            D.relax_us[var] = 1e3f * ms / 3.f;
            if (var == 0 || D.relax_us[var] < best) {
                best = D.relax_us[var];
                best_var = var;
            }
        }
        D.relax_variant = best_var;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

// ---- the work-list form of the batch ------------------------------------------

// One step of a member's mixed-precision V-cycle, generated in the order vcycle_mixed
// issues it.  Buffers of a level: 0 = u32, 1 = u2_32 (block Jacobi's second buffer).
struct VOp {
    int kind = 0;            // 0 relaxation pass, 1 residual + restriction (lvl -> lvl - 1)
    int phase = 0;           // 0 pre-smoothing (and restriction), 1 coarsest level, 2 post-smoothing
    int lvl = 0;             // multigrid level, 0 = coarsest
    int idx = 0;             // position among the same (phase, lvl, kind)
    int mode = PASS_NORMAL, task0 = 0, n_tasks = 0;
    int uin = 0, uout = 0;   // relaxation: buffers read and written; restriction: uin = the iterate
    int fine_buf = -1;       // fused prolongation into this buffer of level lvl + 1, or none
    bool out64 = false;      // writes the member's FP64 result z
};

// The member's V-cycle (Algorithm 1, mixed precision, P = R^T fused), as vcycle_mixed.
void member_ops(const tpmg_ctx *ctx, int l, bool finest, int fine_cur, std::vector<VOp> &ops)
{
    const tpmg_params &p = ctx->p;
    const LevelDev &lv = ctx->lv[l];
    const int C = lv.n_colours;
    const bool jac = p.smoother == TPMG_SMOOTH_JACOBI;
    const int fuse = finest ? -1 : fine_cur;
    int cur = 0, oth = 1;
    int counter[3] = {0, 0, 0};
    auto relax = [&](int phase, int mode, int c, int in, int out, int fine, bool o64) {
        VOp o;
        o.kind = 0;
        o.phase = phase;
        o.lvl = l;
        o.idx = counter[phase]++;
        o.mode = mode;
        if (c < 0) {
            o.task0 = 0;
            o.n_tasks = lv.n_tasks;
        } else {
            o.task0 = lv.colour_task_off[c];
            o.n_tasks = lv.colour_task_off[c + 1] - o.task0;
        }
        o.uin = in;
        o.uout = out;
        o.fine_buf = fine;
        o.out64 = o64;
        if (o.n_tasks > 0) ops.push_back(o);
    };
    auto colour_mode = [](int sweep, int c) { return sweep == 0 ? (c == 0 ? PASS_RHS_ONLY : PASS_ZERO) : PASS_NORMAL; };
    if (l == 0) {
        for (int s = 0; s < p.nu_coarse; ++s) {
            const bool last = s == p.nu_coarse - 1;
            if (jac) {
                relax(1, s == 0 ? PASS_RHS_ONLY : PASS_NORMAL, -1, cur, oth, last ? fuse : -1, last && finest);
                std::swap(cur, oth);
                continue;
            }
            for (int c = 0; c < C; ++c) {
                const bool fin = last && c == C - 1;
                relax(1, colour_mode(s, c), c, 0, 0, fin ? fuse : -1, fin && finest);
            }
            for (int c = C - 2; c >= 0; --c) relax(1, PASS_NORMAL, c, 0, 0, last ? fuse : -1, last && finest);
        }
        return;
    }
    for (int s = 0; s < p.nu_pre; ++s) {
        if (jac) {
            relax(0, s == 0 ? PASS_RHS_ONLY : PASS_NORMAL, -1, cur, oth, -1, false);
            std::swap(cur, oth);
            continue;
        }
        for (int c = 0; c < C; ++c) relax(0, colour_mode(s, c), c, 0, 0, -1, false);
    }
    VOp r;
    r.kind = 1;
    r.phase = 0;
    r.lvl = l;
    r.uin = cur;
    ops.push_back(r);
    member_ops(ctx, l - 1, false, cur, ops);
    for (int s = 0; s < p.nu_post; ++s) {
        const bool last = s == p.nu_post - 1;
        if (jac) {
            relax(2, PASS_NORMAL, -1, cur, oth, last ? fuse : -1, last && finest);
            std::swap(cur, oth);
            continue;
        }
        for (int c = C - 1; c >= 0; --c) relax(2, PASS_NORMAL, c, 0, 0, last ? fuse : -1, last && finest);
    }
}

// Position of an op in the merged schedule: pre-smoothing and restriction from the
// finest level down, the coarsest level, post-smoothing from the coarsest level up;
// levels are counted from the coarsest, so that the members' small coarse passes
// fall into the same steps.  Every member's own order is kept.
std::array<int, 4> op_key(const VOp &o)
{
    if (o.phase == 0) return {0, -o.lvl, o.kind, o.idx};
    if (o.phase == 1) return {1, 0, 0, o.idx};
    return {2, o.lvl, 0, o.idx};
}

int rows_class(int n_r)
{
    int c = 32;
    while (c < n_r && c < 1024) c *= 2;
    return c;
}

bool worklist_member_ok(const tpmg_ctx *c)
{
    const tpmg_params &p = c->p;
    return p.precision == TPMG_PREC_MIXED && p.outer == TPMG_OUTER_CG && p.prolongation == TPMG_PROLONG_CONSTANT &&
           !has_advection(c) && !c->lv.back().cfull && p.nu_pre >= 1 && p.nu_post >= 1 && p.nu_coarse >= 1;
}

template <typename T>
cudaError_t balloc(tpmg_batch *b, T **ptr, size_t count)
{
    void *q = nullptr;
    const cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    b->allocs.push_back(q);
    *ptr = static_cast<T *>(q);
    return cudaSuccess;
}

// A group's V-cycle for every active member: the schedule's launches in order.
cudaError_t batch_vcycle(const tpmg_batch::Group &G, const Launch &L)
{
    for (const BatchLaunch &bl : G.launches) {
        cudaError_t e;
        if (bl.kind == 0) {
            const RelaxBatchArgs &a = G.rargs[bl.args];
            e = bl.f64 ? launch_relax32_batch<double>(L, bl.mode, bl.n_r_max, a, bl.total, bl.wpb, G.d_active)
                       : launch_relax32_batch<float>(L, bl.mode, bl.n_r_max, a, bl.total, bl.wpb, G.d_active);
        } else {
            const RestrictBatchArgs &a = G.cargs[bl.args];
            e = bl.f64 ? launch_restrict32_batch<double>(L, a, bl.total, G.d_active)
                       : launch_restrict32_batch<float>(L, a, bl.total, G.d_active);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

constexpr int kBatchGroups = 4;   // root branches of a work-list batch (fewer for small batches)

// Builds the work-list form of a batch whose members all pass worklist_member_ok.
tpmg_status build_worklist(tpmg_batch *b, tpmg_ctx *const *ctxs, int M, const double *const *d_f, double *const *d_u,
                           cudaStream_t s, int groups)
{
    const int n_part = ctxs[0]->n_part;
    for (int m = 0; m < M; ++m)
        if (ctxs[m]->n_part != n_part) return TPMG_ERR_INVALID_ARG;
    b->form = TPMG_BATCH_WORKLIST;
    b->n_part = n_part;
    // the members' work vectors: outer FP64 r, z, p, q (r also in FP32) and every level's
    // FP32 iterate (and block Jacobi's second buffer), the coarse levels' FP32 right-hand sides
    std::vector<BatchMemberDev> mem(M);
    std::vector<std::vector<float *>> u32(M), u2(M), f32(M);
    b->d_sc.assign(M, nullptr);
    for (int m = 0; m < M; ++m) {
        const tpmg_ctx *c = ctxs[m];
        const LevelDev &fl = c->lv.back();
        const long N = c->N;
        const int n_r = c->p.n_r, L = c->p.n_levels;
        BatchMemberDev &x = mem[m];
        x = BatchMemberDev{fl.nbr, fl.g, fl.area, fl.area_r, fl.om, fl.oc, fl.ocs, c->vert.vol, c->vert.w, c->vert.hr, n_r,
                           (int)N, d_f[m], d_u[m]};
        if (balloc(b, &x.r, N) != cudaSuccess || balloc(b, &x.r32, N) != cudaSuccess || balloc(b, &x.z, N) != cudaSuccess ||
            balloc(b, &x.p, N) != cudaSuccess ||
            balloc(b, &x.q, N) != cudaSuccess || balloc(b, &x.partials, 2 * (size_t)n_part) != cudaSuccess ||
            balloc(b, &x.zflags, (size_t)n_part) != cudaSuccess || balloc(b, &b->d_sc[m], 1) != cudaSuccess ||
            balloc(b, &x.hist, kHistCap) != cudaSuccess)
            return TPMG_ERR_OOM;
        x.sc = b->d_sc[m];
        x.rtol = b->rtol;
        x.max_iter = b->max_iter;
        const bool jac = c->p.smoother == TPMG_SMOOTH_JACOBI;
        u32[m].assign(L, nullptr);
        u2[m].assign(L, nullptr);
        f32[m].assign(L, nullptr);
        for (int l = 0; l < L; ++l) {
            const size_t n = (size_t)c->lv[l].n * n_r;
            if (balloc(b, &u32[m][l], n) != cudaSuccess || (jac && balloc(b, &u2[m][l], n) != cudaSuccess) ||
                (l < L - 1 && balloc(b, &f32[m][l], n) != cudaSuccess))
                return TPMG_ERR_OOM;
        }
    }
    auto clear_work = [&]() -> bool {   // every work vector zero (at creation, and after the tuner)
        for (int m = 0; m < M; ++m) {
            const long N = ctxs[m]->N;
            if (cudaMemsetAsync(mem[m].r, 0, N * sizeof(double), s) != cudaSuccess ||
                cudaMemsetAsync(mem[m].r32, 0, N * sizeof(float), s) != cudaSuccess ||
                cudaMemsetAsync(mem[m].z, 0, N * sizeof(double), s) != cudaSuccess)
                return false;
            for (size_t l = 0; l < u32[m].size(); ++l) {
                const size_t n = (size_t)ctxs[m]->lv[l].n * ctxs[m]->p.n_r;
                if (cudaMemsetAsync(u32[m][l], 0, n * sizeof(float), s) != cudaSuccess ||
                    (u2[m][l] && cudaMemsetAsync(u2[m][l], 0, n * sizeof(float), s) != cudaSuccess) ||
                    (f32[m][l] && cudaMemsetAsync(f32[m][l], 0, n * sizeof(float), s) != cudaSuccess))
                    return false;
            }
        }
        return cudaStreamSynchronize(s) == cudaSuccess;
    };
    if (!clear_work()) return TPMG_ERR_CUDA;
    // groups of about equal work: members by decreasing size, each to the lightest group
    const int G = groups > 0 ? std::min(groups, M) : std::max(1, std::min(M / 2, kBatchGroups));
    b->groups.assign(G, tpmg_batch::Group{});
    {
        std::vector<int> order(M);
        for (int m = 0; m < M; ++m) order[m] = m;
        std::stable_sort(order.begin(), order.end(), [&](int a, int c2) { return ctxs[a]->N > ctxs[c2]->N; });
        std::vector<double> load(G, 0.0);
        for (int m : order) {
            const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            b->groups[g].members.push_back(m);
            load[g] += (double)ctxs[m]->N;
        }
        for (auto &grp : b->groups) std::sort(grp.members.begin(), grp.members.end());   // the caller's order
    }
    // each group's merged schedule: its members' ops under their keys, steps in key order,
    // each step split into launches by kernel class; item member = index within the group
    struct Tagged {
        std::array<int, 4> key;
        int member;   // within the group
        VOp op;
    };
    for (tpmg_batch::Group &grp : b->groups) {
        const int Mg = (int)grp.members.size();
        std::vector<Tagged> all;
        for (int j = 0; j < Mg; ++j) {
            std::vector<VOp> ops;
            const tpmg_ctx *c = ctxs[grp.members[j]];
            member_ops(c, c->p.n_levels - 1, true, -1, ops);
            for (const VOp &o : ops) all.push_back(Tagged{op_key(o), j, o});
        }
        std::stable_sort(all.begin(), all.end(), [](const Tagged &a, const Tagged &b2) { return a.key < b2.key; });
        for (size_t i0 = 0; i0 < all.size();) {
            size_t i1 = i0;
            while (i1 < all.size() && all[i1].key == all[i0].key) ++i1;
            // launch classes of the step: (kind, mode, rows class); every member's finest level
            // reads its FP32 copy of r, so all right-hand sides are FP32
            auto class_of = [&](const Tagged &t) {
                const tpmg_ctx *c = ctxs[grp.members[t.member]];
                return std::array<int, 3>{t.op.kind, t.op.kind == 0 ? t.op.mode : 0,
                                          t.op.kind == 0 ? rows_class(c->p.n_r) : 0};
            };
            std::vector<std::array<int, 3>> classes;
            for (size_t i = i0; i < i1; ++i) {
                const auto cl = class_of(all[i]);
                if (std::find(classes.begin(), classes.end(), cl) == classes.end()) classes.push_back(cl);
            }
            for (const auto &cl : classes) {
                BatchLaunch bl;
                bl.kind = cl[0];
                bl.mode = cl[1];
                bl.f64 = false;
                bl.n_r_max = cl[2];
                auto open = [&]() {   // a new work list for the launch
                    bl.count = 0;
                    bl.total = 0;
                    if (bl.kind == 0) {
                        bl.args = (int)grp.rargs.size();
                        grp.rargs.emplace_back();
                        std::memset(&grp.rargs.back(), 0, sizeof(RelaxBatchArgs));
                    } else {
                        bl.args = (int)grp.cargs.size();
                        grp.cargs.emplace_back();
                        std::memset(&grp.cargs.back(), 0, sizeof(RestrictBatchArgs));
                    }
                };
                open();
                for (size_t i = i0; i < i1; ++i) {
                    const Tagged &t = all[i];
                    if (class_of(t) != cl) continue;
                    if (bl.count == kBatchItems) {
                        grp.launches.push_back(bl);
                        open();
                    }
                    const int m = grp.members[t.member], l = t.op.lvl;
                    const tpmg_ctx *c = ctxs[m];
                    const int n_r = c->p.n_r;
                    const LevelDev &lv = c->lv[l];
                    auto buf = [&](int lvl, int id) { return id == 0 ? u32[m][lvl] : u2[m][lvl]; };
                    const bool finest = l == c->p.n_levels - 1;
                    const void *f = finest ? (const void *)mem[m].r32 : (const void *)f32[m][l];
                    if (bl.kind == 0) {
                        BatchRelaxItem it{lv.task_cells, lv.task_nbr, lv.cpack, lv.cvert, lv.rinv32, f,
                                          buf(l, t.op.uin), buf(l, t.op.uout),
                                          t.op.fine_buf >= 0 ? buf(l + 1, t.op.fine_buf) : nullptr,
                                          t.op.out64 ? mem[m].z : nullptr, n_r, t.op.task0 * kRelaxCols,
                                          t.op.n_tasks * kRelaxCols, t.member, (float)c->p.relax};
                        RelaxBatchArgs &a = grp.rargs[bl.args];
                        a.off[bl.count] = (int)bl.total;
                        a.items[bl.count] = it;
                        a.n_items = bl.count + 1;
                        bl.total += it.n_slots;
                    } else {
                        const int Nc = c->lv[l - 1].n * n_r;
                        BatchRestrictItem it{lv.nbr, lv.cpack, lv.cvert, f, buf(l, t.op.uin), f32[m][l - 1], n_r, Nc,
                                             t.member};
                        RestrictBatchArgs &a = grp.cargs[bl.args];
                        a.off[bl.count] = (int)bl.total;
                        a.items[bl.count] = it;
                        a.n_items = bl.count + 1;
                        bl.total += (Nc + 31) & ~31;
                    }
                    ++bl.count;
                }
                if (bl.count > 0) grp.launches.push_back(bl);   // (an empty last list stays unused)
            }
            i0 = i1;
        }
        for (const BatchLaunch &bl : grp.launches)
            if (bl.total > INT32_MAX / 2) return TPMG_ERR_INVALID_ARG;   // positions are 32-bit in the kernels
        std::vector<BatchMemberDev> gm(Mg);
        for (int j = 0; j < Mg; ++j) gm[j] = mem[grp.members[j]];
        if (balloc(b, &grp.d_mem, Mg) != cudaSuccess || balloc(b, &grp.d_active, Mg) != cudaSuccess ||
            balloc(b, &grp.d_go, Mg) != cudaSuccess)
            return TPMG_ERR_OOM;
        if (cudaMemcpyAsync(grp.d_mem, gm.data(), sizeof(BatchMemberDev) * Mg, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemsetAsync(grp.d_active, 1, sizeof(int) * Mg, s) != cudaSuccess ||
            cudaMemsetAsync(grp.d_go, 0, sizeof(int) * Mg, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            return TPMG_ERR_CUDA;
    }
    if (cudaMallocHost(&b->h_sc, sizeof(Scalars) * M) != cudaSuccess) return TPMG_ERR_OOM;
    // tuner: CTAs of 1, 2, 4 or 8 warps for each relaxation launch of more than two waves
    // of warps, timed on the batch's zeroed work vectors (every variant is the same arithmetic)
    const int sm = ctxs[0]->sm_count;
    const Launch L0{s, 0, sm, nullptr, nullptr, false};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TPMG_ERR_CUDA;
    tpmg_status st = TPMG_OK;
    for (tpmg_batch::Group &grp : b->groups)
        for (BatchLaunch &bl : grp.launches) {
            if (bl.kind != 0 || bl.total < 2L * 32 * sm) continue;
            float best = 0.f;
            for (int v = 0; v < 4 && st == TPMG_OK; ++v) {
                BatchLaunch t = bl;
                t.wpb = 1 << v;
                auto go = [&]() {
                    return launch_relax32_batch<float>(L0, t.mode, t.n_r_max, grp.rargs[t.args], t.total, t.wpb,
                                                       grp.d_active);
                };
                float ms = 0.f;
                if (go() != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess) st = TPMG_ERR_CUDA;
                for (int k = 0; k < 3 && st == TPMG_OK; ++k)
                    if (go() != cudaSuccess) st = TPMG_ERR_CUDA;
                if (st == TPMG_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    st = TPMG_ERR_CUDA;
                bl.us[v] = 1e3f * ms / 3.f;
                if (st == TPMG_OK && (best == 0.f || bl.us[v] < best)) {
                    best = bl.us[v];
                    bl.wpb = t.wpb;
                }
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != TPMG_OK) return st;
    if (!clear_work()) return TPMG_ERR_CUDA;   // the tuner wrote into them
    // the graph: per group a root branch -- its members' initial residuals and first
    // decisions, then a conditional WHILE node whose body is one iteration of every
    // active member of the group
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return TPMG_ERR_CUDA;
    const Launch L{cs, 0, sm, nullptr, nullptr, ctxs[0]->p.pdl != 0};
    cudaGraph_t g = nullptr;
    auto capture = [&](cudaGraph_t into, std::vector<cudaGraphNode_t> *leaves, auto &&body) -> tpmg_status {
        if (cudaStreamBeginCaptureToGraph(cs, into, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
            cudaSuccess)
            return TPMG_ERR_CUDA;
        const cudaError_t eb = body();
        const cudaGraphNode_t *out = nullptr;
        size_t nout = 0;
        cudaStreamCaptureStatus csx;
        const cudaError_t ei = cudaStreamGetCaptureInfo(cs, &csx, nullptr, nullptr, &out, nullptr, &nout);
        if (leaves && ei == cudaSuccess) leaves->assign(out, out + nout);
        cudaGraph_t gout = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(cs, &gout);
        return (eb == cudaSuccess && ei == cudaSuccess && ee == cudaSuccess) ? TPMG_OK : TPMG_ERR_CUDA;
    };
    auto counted = [](long long &n, cudaError_t e) {
        ++n;
        return e;
    };
    if (cudaGraphCreate(&g, 0) != cudaSuccess) st = TPMG_ERR_CUDA;
    for (tpmg_batch::Group &grp : b->groups) {
        if (st != TPMG_OK) break;
        const int Mg = (int)grp.members.size();
        BatchMemberDev *dm = grp.d_mem;
        int *act = grp.d_active, *go = grp.d_go;
        cudaGraphConditionalHandle h = 0;
        if (cudaGraphConditionalHandleCreate(&h, g, 0, 0) != cudaSuccess) {
            st = TPMG_ERR_CUDA;
            break;
        }
        std::vector<cudaGraphNode_t> leaves;
        long long &n_init = grp.init, &n_iter = grp.iter;
        st = capture(g, &leaves, [&]() -> cudaError_t {
            cudaError_t e = cudaMemsetAsync(act, 1, sizeof(int) * Mg, cs);
            if (e == cudaSuccess) e = counted(n_init, launch_outer_batch(L, BATCH_NONZERO, dm, Mg, n_part, act));
            if (e == cudaSuccess) e = counted(n_init, launch_outer_batch(L, BATCH_RESIDUAL, dm, Mg, n_part, act));
            if (e == cudaSuccess) e = counted(n_init, launch_finish_batch(L, FIN_LOOP_RR0, dm, Mg, n_part, act, go, 0));
            if (e == cudaSuccess) e = counted(n_init, launch_outer_batch(L, BATCH_CLEAR_P, dm, Mg, n_part, act));
            if (e == cudaSuccess) e = counted(n_init, launch_batch_continue(L, Mg, go, act, h));
            return e;
        });
        if (st != TPMG_OK) break;
        cudaGraphNode_t node = nullptr;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if (cudaGraphAddNode(&node, g, leaves.data(), nullptr, leaves.size(), &cp) != cudaSuccess) {
            st = TPMG_ERR_CUDA;
            break;
        }
        st = capture(cp.conditional.phGraph_out[0], nullptr, [&]() -> cudaError_t {
            cudaError_t e = batch_vcycle(grp, L);
            n_iter += (long long)grp.launches.size();
            if (e == cudaSuccess) e = counted(n_iter, launch_outer_batch(L, BATCH_DOT_RZ, dm, Mg, n_part, act));
            if (e == cudaSuccess)
                e = counted(n_iter, launch_finish_batch(L, FIN_LOOP_BETA_PR, dm, Mg, n_part, act, go, 0));
            if (e == cudaSuccess) e = counted(n_iter, launch_outer_batch(L, BATCH_XPBY, dm, Mg, n_part, act));
            if (e == cudaSuccess) e = counted(n_iter, launch_outer_batch(L, BATCH_APPLY, dm, Mg, n_part, act));
            if (e == cudaSuccess) e = counted(n_iter, launch_finish_batch(L, FIN_ALPHA, dm, Mg, n_part, act, go, 0));
            if (e == cudaSuccess) e = counted(n_iter, launch_outer_batch(L, BATCH_AXPY, dm, Mg, n_part, act));
            if (e == cudaSuccess) e = counted(n_iter, launch_finish_batch(L, FIN_LOOP_RR, dm, Mg, n_part, act, go, 0));
            if (e == cudaSuccess)
                e = counted(n_iter, launch_finish_batch(L, FIN_RZC, dm, Mg, n_part, act, go, n_part));
            if (e == cudaSuccess) e = counted(n_iter, launch_batch_continue(L, Mg, go, act, h));
            return e;
        });
    }
    if (st == TPMG_OK && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) st = TPMG_ERR_CUDA;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return st;
}

}  // namespace

extern "C" {

tpmg_status tpmg_default_params(tpmg_params *p)
{
    if (!p) return TPMG_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof(*p));
    p->refinement = 3;
    p->n_levels = 4;
    p->n_r = 16;
    p->H = 10.0 / 6371.0;
    p->grading = 1.0;
    p->omega2 = 0.0;
    p->courant_c = 8.0;
    p->nu_pre = 2;
    p->nu_post = 2;
    p->nu_coarse = 1;
    p->smoother = TPMG_SMOOTH_MCSOR;
    p->relax = 1.0;
    p->coeff_storage = TPMG_COEFF_FACTORISED;
    p->centre = TPMG_CENTRE_CIRCUM;
    p->precision = TPMG_PREC_FP64;
    p->graphs = 1;
    p->autotune = 1;
    p->scan_max_cells = 5120;
    p->outer = TPMG_OUTER_CG;
    p->prolongation = TPMG_PROLONG_CONSTANT;
    p->pdl = 1;
    p->relax_variant = -1;
    p->scaled_rhs = 1;
    p->net_tcgen05 = 1;
    return TPMG_OK;
}

tpmg_status tpmg_setup(const tpmg_params *params, void *cuda_stream, tpmg_ctx **out)
{
    return tpmg_setup_profiles(params, nullptr, cuda_stream, out);
}

tpmg_status tpmg_setup_profiles(const tpmg_params *params, const tpmg_profiles *prof, void *cuda_stream,
                                tpmg_ctx **out)
{
    std::string msg;
    if (!out) return TPMG_ERR_INVALID_ARG;
    if (!validate(params, msg)) return TPMG_ERR_INVALID_ARG;
    if (prof) {   // every profile value positive and finite (checked before any CUDA call)
        const long n_fine = 20L << (2 * params->refinement);
        auto ok = [](const double *v, long n) {
            for (long i = 0; v && i < n; ++i)
                if (!(v[i] > 0.0) || !std::isfinite(v[i])) return false;
            return true;
        };
        auto finite = [](const double *v, long n) {
            for (long i = 0; v && i < n; ++i)
                if (!std::isfinite(v[i])) return false;
            return true;
        };
        if (!ok(prof->beta_r, params->n_r) || !ok(prof->alphaS_r, params->n_r) || !ok(prof->alphar_r, params->n_r + 1) ||
            !ok(prof->beta_s, n_fine) || !ok(prof->alphar_s, n_fine) || !ok(prof->alphaS_s, n_fine) ||
            !finite(prof->xi_r, params->n_r + 1) || !finite(prof->xi_s, n_fine))
            return TPMG_ERR_INVALID_ARG;
    }
    tpmg_ctx *ctx = new (std::nothrow) tpmg_ctx();
    if (!ctx) return TPMG_ERR_OOM;
    auto bail = [&](tpmg_status s) {
        tpmg_destroy(ctx);
        return s;
    };
    ctx->p = *params;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    ctx->issue = ctx->stream;
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(TPMG_ERR_CUDA);
    if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(TPMG_ERR_CUDA);
    if (cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess)
        return bail(TPMG_ERR_CUDA);
    // the fixed array of tpmg_vcycle_noalloc: its address is looked up here, with the
    // context's device current, so that the entry point itself only reads it
    if (noalloc_scratch(ctx->device, &ctx->noalloc_base) != cudaSuccess) return bail(TPMG_ERR_CUDA);
    if (!build_host_grid(ctx->p, ctx->host, msg)) return bail(TPMG_ERR_INVALID_ARG);
    const int n_r = ctx->p.n_r;
    if (prof) {
        const int L = ctx->p.refinement;
        if (!copy_vertical(prof->beta_r, n_r, ctx->pr_beta) || !copy_vertical(prof->alphaS_r, n_r, ctx->pr_aS) ||
            !copy_vertical(prof->alphar_r, n_r + 1, ctx->pr_ar) ||
            !level_means(ctx->host, L, prof->beta_s, ctx->ps_beta) ||
            !level_means(ctx->host, L, prof->alphar_s, ctx->ps_ar) ||
            !level_means(ctx->host, L, prof->alphaS_s, ctx->ps_aS) ||
            !copy_vertical(prof->xi_r, n_r + 1, ctx->pr_xi, true) ||
            !level_means(ctx->host, L, prof->xi_s, ctx->ps_xi, true))
            return bail(TPMG_ERR_INVALID_ARG);
        ctx->xi_fac = prof->xi_r || prof->xi_s;
    }
    // vertical factors: vol | w | hr
    {
        const HostGrid &G = ctx->host;
        std::vector<double> hv(6 * n_r + 1);
        double *vol = hv.data(), *w = vol + n_r, *hr = w + n_r + 1, *xm = hr + n_r, *xp = xm + n_r, *drv = xp + n_r;
        for (int k = 0; k <= n_r; ++k) w[k] = G.omega2 * G.face[k] * vfac(ctx->pr_ar, k);
        // the factorised advection's vertical factor of face k (zero on the boundary faces)
        auto wx = [&](int k) { return (k == 0 || k == n_r) ? 0.0 : 0.5 * G.omega2 * G.face[k] * vfac(ctx->pr_xi, k); };
        for (int k = 0; k < n_r; ++k) {
            vol[k] = G.vol[k] * vfac(ctx->pr_beta, k);
            hr[k] = G.omega2 * G.dr[k] * vfac(ctx->pr_aS, k);
            xm[k] = G.dr[k] * wx(k);
            xp[k] = G.dr[k] * wx(k + 1);
            drv[k] = G.dr[k];
        }
        tpmg_status st = TPMG_OK;
        if (dalloc(ctx, &ctx->d_vert, hv.size()) != cudaSuccess) return bail(TPMG_ERR_OOM);
        if (cudaMemcpyAsync(ctx->d_vert, hv.data(), hv.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            st = TPMG_ERR_CUDA;
        if (st != TPMG_OK) return bail(st);
        ctx->vert.vol = ctx->d_vert;
        ctx->vert.w = ctx->d_vert + n_r;
        ctx->vert.hr = ctx->d_vert + 2 * n_r + 1;
        ctx->vert.xm = ctx->d_vert + 3 * n_r + 1;
        ctx->vert.xp = ctx->d_vert + 4 * n_r + 1;
        ctx->vert.dr = ctx->d_vert + 5 * n_r + 1;
        std::vector<float> iv(2 * n_r);
        for (int k = 0; k < n_r; ++k) {
            iv[k] = (float)(1.0 / G.vol[k]);
            iv[n_r + k] = (float)G.dr[k];
        }
        float *d_iv = nullptr;
        if (dalloc(ctx, &d_iv, 2 * n_r) != cudaSuccess) return bail(TPMG_ERR_OOM);
        if (cudaMemcpyAsync(d_iv, iv.data(), 2 * n_r * sizeof(float), cudaMemcpyHostToDevice, ctx->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            return bail(TPMG_ERR_CUDA);
        ctx->vert.ivol32 = d_iv;
        ctx->vert.dr32 = d_iv + n_r;
    }
    ctx->lv.assign(ctx->p.n_levels, LevelDev());
    for (int l = 0; l < ctx->p.n_levels; ++l) {
        tpmg_status st = upload_level(ctx, l);
        if (st != TPMG_OK) return bail(st);
    }
    ctx->N = (long)ctx->lv.back().n * n_r;
    ctx->n_part = 8 * ctx->sm_count;   // blocks of the reducing kernels, one partial each
    if (dalloc(ctx, &ctx->r, ctx->N) != cudaSuccess || dalloc(ctx, &ctx->z, ctx->N) != cudaSuccess ||
        dalloc(ctx, &ctx->pv, ctx->N) != cudaSuccess || dalloc(ctx, &ctx->q, ctx->N) != cudaSuccess ||
        dalloc(ctx, &ctx->hf, ctx->N) != cudaSuccess || dalloc(ctx, &ctx->hu, ctx->N) != cudaSuccess ||
        dalloc(ctx, &ctx->partials, 2 * (size_t)ctx->n_part) != cudaSuccess ||
        dalloc(ctx, &ctx->zflags, (size_t)ctx->n_part) != cudaSuccess ||
        dalloc(ctx, &ctx->d_hist, kHistCap) != cudaSuccess || dalloc(ctx, &ctx->sc, 1) != cudaSuccess ||
        dalloc(ctx, &ctx->d_net_s, 3) != cudaSuccess || dalloc(ctx, &ctx->d_net_err, 1) != cudaSuccess ||
        (ctx->p.precision == TPMG_PREC_MIXED && dalloc(ctx, &ctx->r32, ctx->N) != cudaSuccess))
        return bail(TPMG_ERR_OOM);
    if (cudaMallocHost(&ctx->h_sc, sizeof(Scalars)) != cudaSuccess) return bail(TPMG_ERR_OOM);
    {
        // finest level: per-row products of the outer operator's coefficients (16 bytes per
        // unknown), allocated after everything the solver needs and only where they fit;
        // without them the operator stays matrix-free
        LevelDev &D = ctx->lv.back();
        if (dalloc(ctx, &D.om, (size_t)ctx->N) != cudaSuccess || dalloc(ctx, &D.oc, (size_t)ctx->N) != cudaSuccess) {
            (void)cudaGetLastError();   // a failed allocation leaves no sticky error
            D.om = D.oc = nullptr;
        } else {
            if (dalloc(ctx, &D.ocs, 3 * (size_t)ctx->N) != cudaSuccess) {   // 24 more bytes per unknown
                (void)cudaGetLastError();
                D.ocs = nullptr;
            }
            if (launch_outer_products(launch_of(ctx), D, ctx->vert) != cudaSuccess) return bail(TPMG_ERR_CUDA);
        }
    }
    // levels relaxed by twisted tasks (FP64, factorised stencil): the scaled couplings
    // (24 bytes per unknown) and the work vector of f / pivot, where they fit
    for (LevelDev &D : ctx->lv) {
        if (ctx->p.precision != TPMG_PREC_FP64 || !ctx->p.scaled_rhs) break;
        if (D.scan || D.vc || D.n_colours > 63) continue;
        const size_t nn = (size_t)D.n * n_r;
        if (dalloc(ctx, &D.cs, 3 * nn) != cudaSuccess || dalloc(ctx, &D.ft, nn) != cudaSuccess) {
            (void)cudaGetLastError();
            D.cs = D.ft = nullptr;
            continue;
        }
        if (launch_scaled_couplings(launch_of(ctx), D, ctx->vert) != cudaSuccess) return bail(TPMG_ERR_CUDA);
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return bail(TPMG_ERR_CUDA);
    if (ctx->p.relax_variant >= 0) {
        for (LevelDev &D : ctx->lv) D.relax_variant = ctx->p.relax_variant;
    } else if (ctx->p.autotune) {
        tpmg_status st = autotune(ctx);
        if (st != TPMG_OK) return bail(st);
    }
    *out = ctx;
    return TPMG_OK;
}

tpmg_status tpmg_apply_operator(tpmg_ctx *ctx, const double *d_x, double *d_y)
{
    if (!ctx || !d_x || !d_y) return fail(ctx, TPMG_ERR_INVALID_ARG, "NULL argument");
    if (d_x == d_y) return fail(ctx, TPMG_ERR_INVALID_ARG, "x and y must not overlap");
    LCHK(run(ctx, TPMG_K_APPLY, (double)ctx->N,
             [&] { return launch_apply(launch_of(ctx), ctx->lv.back(), ctx->vert, d_x, d_y, nullptr, 0); }));
    return TPMG_OK;
}

tpmg_status tpmg_set_outer_profiles(tpmg_ctx *ctx, const double *h_beta, const double *h_alphar,
                                    const double *h_alphaS, const double *h_xi)
{
    if (!ctx) return TPMG_ERR_INVALID_ARG;
    LevelDev &D = ctx->lv.back();
    const HostLevel &H = ctx->host.lev[ctx->p.refinement];
    const int n_r = ctx->p.n_r, n = H.n;
    const size_t nn = (size_t)n * n_r, nf = (size_t)n * (n_r + 1);
    const bool clear = !h_beta && !h_alphar && !h_alphaS;
    if (!clear) {
        if (!h_beta || !h_alphar || !h_alphaS) return fail(ctx, TPMG_ERR_INVALID_ARG, "give all three profiles or none");
        auto ok = [](const double *v, size_t m, bool any_sign) {
            for (size_t i = 0; i < m; ++i)
                if (!std::isfinite(v[i]) || (!any_sign && !(v[i] > 0.0))) return false;
            return true;
        };
        if (!ok(h_beta, nn, false) || !ok(h_alphaS, nn, false) || !ok(h_alphar, nf, false))
            return fail(ctx, TPMG_ERR_INVALID_ARG, "profiles must be positive and finite");
        if (h_xi && !ok(h_xi, nf, true)) return fail(ctx, TPMG_ERR_INVALID_ARG, "xi must be finite");
    }
    const double *px = clear ? nullptr : h_xi;
    // A V-cycle that stores its stencil per unknown adopts the general profiles too
    // (FULL: all of them, advection included, TPMG^full; PARTIAL: alpha_r, with beta,
    // alpha_S and xi factorised, TPMG^partial; coarse levels average them over the
    // children), or goes back to the factorised ones; then its column factors are formed
    // again.  The first pass only checks that every level's column blocks stay M-matrices,
    // so that a rejected call changes nothing.
    const bool stored = ctx->p.coeff_storage == TPMG_COEFF_FULL;
    const bool mixed = ctx->p.precision == TPMG_PREC_MIXED;
    for (int pass = 0; pass < 2 && ctx->p.coeff_storage != TPMG_COEFF_FACTORISED; ++pass) {
        std::vector<double> b, r, a, x;
        if (!clear) {
            b.assign(h_beta, h_beta + nn);
            r.assign(h_alphar, h_alphar + nf);
            a.assign(h_alphaS, h_alphaS + nn);
            if (px) x.assign(px, px + nf);
        }
        if (pass == 1) {
            CU(cudaStreamSynchronize(ctx->stream));
            drop_graph(ctx);   // captured solves hold the V-cycle's kernels
        }
        for (int l = ctx->p.n_levels - 1; l >= 0; --l) {
            const HostLevel &Hl = ctx->host.lev[ctx->p.refinement - (ctx->p.n_levels - 1 - l)];
            if (!clear && l < ctx->p.n_levels - 1) {
                const HostLevel &Hf = ctx->host.lev[Hl.ref + 1];
                b = average_children(Hf, b, n_r);
                r = average_children(Hf, r, n_r + 1);
                a = average_children(Hf, a, n_r);
                if (px) x = average_children(Hf, x, n_r + 1);
            }
            const double *lb = clear ? nullptr : b.data(), *lr = clear ? nullptr : r.data();
            const double *la = clear ? nullptr : a.data(), *lx = (stored && px) ? x.data() : nullptr;
            LevelDev &Dl = ctx->lv[l];
            if (pass == 0) {
                const bool on = lx ? true : (stored && !clear ? false : ctx->xi_fac);
                if (on) {
                    std::vector<double> xv, crv;
                    fp64_advection(ctx, Hl, lx, xv);
                    fp64_vertical(ctx, Hl, lr, crv);
                    if (!couplings_ok(ctx, Hl.n, crv, xv))
                        return fail(ctx, TPMG_ERR_INVALID_ARG, "vertical advection too strong: a column block is no "
                                                               "M-matrix (dr |xi| > 2 alpha_r on some face)");
                }
                continue;
            }
            if (mixed) {
                std::vector<bf16x4> cp;
                std::vector<unsigned short> cv;
                bf16_stencil(ctx, Hl, lb, lr, la, cp, cv);
                CU(cudaMemcpyAsync(Dl.cpack, cp.data(), cp.size() * sizeof(bf16x4), cudaMemcpyHostToDevice, ctx->stream));
                CU(cudaMemcpyAsync(Dl.cvert, cv.data(), cv.size() * sizeof(unsigned short), cudaMemcpyHostToDevice,
                                   ctx->stream));
                CU(cudaStreamSynchronize(ctx->stream));   // cp, cv are local
                const tpmg_status st = upload_advection(ctx, Hl, Dl, lx, lr);
                if (st != TPMG_OK) return st;
                CU(launch_thomas_factors32(launch_of(ctx), Dl));
                CU(cudaStreamSynchronize(ctx->stream));
                continue;
            }
            std::vector<dbl4> c;
            std::vector<double> cr;
            fp64_vertical(ctx, Hl, lr, cr);
            CU(cudaMemcpyAsync(Dl.vcr, cr.data(), cr.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
            if (stored) {
                fp64_horizontal(ctx, Hl, lb, la, c);
                CU(cudaMemcpyAsync(Dl.vc, c.data(), c.size() * sizeof(dbl4), cudaMemcpyHostToDevice, ctx->stream));
            }
            CU(cudaStreamSynchronize(ctx->stream));   // c, cr are local
            const tpmg_status st = upload_advection(ctx, Hl, Dl, lx, lr);
            if (st != TPMG_OK) return st;
            CU(launch_twisted_factors(launch_of(ctx), Dl, ctx->vert));
            if (Dl.rinv1) CU(launch_thomas_factors(launch_of(ctx), Dl, ctx->vert));
            CU(cudaStreamSynchronize(ctx->stream));
        }
    }
    CU(cudaStreamSynchronize(ctx->stream));
    drop_graph(ctx);   // captured solves hold the operator's kernels
    if (clear) {
        D.cfull = nullptr;   // the arrays stay allocated for a later call (freed by tpmg_destroy)
        D.cvx = nullptr;
        return TPMG_OK;
    }
    // the problem's operator per unknown in FP64 (finest level)
    std::vector<dbl4> c;
    std::vector<double> cr;
    fp64_horizontal(ctx, H, h_beta, h_alphaS, c);
    fp64_vertical(ctx, H, h_alphar, cr);
    if (!D.cvr) {
        dbl4 *cf = nullptr;
        CU(dalloc(ctx, &cf, nn));
        CU(dalloc(ctx, &D.cvr, nf));
        ctx->cfull_store = cf;
    }
    CU(cudaMemcpyAsync(ctx->cfull_store, c.data(), nn * sizeof(dbl4), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(D.cvr, cr.data(), nf * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    std::vector<double> xo;
    if (h_xi) {
        fp64_advection(ctx, H, h_xi, xo);
        if (!ctx->cvx_store) CU(dalloc(ctx, &ctx->cvx_store, nf));
        CU(cudaMemcpyAsync(ctx->cvx_store, xo.data(), nf * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    D.cfull = ctx->cfull_store;
    D.cvx = h_xi ? ctx->cvx_store : nullptr;
    return TPMG_OK;
}

tpmg_status tpmg_vcycle(tpmg_ctx *ctx, const double *d_r, double *d_z)
{
    if (!ctx || !d_r || !d_z) return fail(ctx, TPMG_ERR_INVALID_ARG, "NULL argument");
    if (d_r == d_z) return fail(ctx, TPMG_ERR_INVALID_ARG, "r and z must not overlap");
    return vcycle_fine(ctx, d_r, d_z);
}

// The V-cycle of tpmg_vcycle with the level work vectors taken from the fixed
// array of noalloc.cu.  The context's own work-vector pointers are pointed
// into that array for the duration of the call (the launches capture the
// pointer values when they are enqueued) and then restored, so the sequence
// of kernels is exactly the one tpmg_vcycle runs.
tpmg_status tpmg_vcycle_noalloc(tpmg_ctx *ctx, const double *d_r, double *d_z)
{
    if (!ctx || !d_r || !d_z) return fail(ctx, TPMG_ERR_INVALID_ARG, "NULL argument");
    if (d_r == d_z) return fail(ctx, TPMG_ERR_INVALID_ARG, "r and z must not overlap");
    if (ctx->p.precision != TPMG_PREC_FP64)
        return fail(ctx, TPMG_ERR_INVALID_ARG, "the fixed-scratch V-cycle is built for FP64 precision only");
    const int L = ctx->p.n_levels;
    const bool jac = ctx->p.smoother == TPMG_SMOOTH_JACOBI;
    auto padded = [&](int l) { return ((size_t)ctx->lv[l].n * ctx->p.n_r + 31) & ~(size_t)31; };
    size_t need = 0;
    // f, u of the coarse levels; block Jacobi's second buffer; f / pivot where the level
    // relaxes with scaled couplings
    for (int l = 0; l < L; ++l)
        need += (l < L - 1 ? 2 : 0) * padded(l) + (jac ? padded(l) : 0) + (ctx->lv[l].ft ? padded(l) : 0);
    if (need > (size_t)TPMG_VCYCLE_NOALLOC_MAX_DOUBLES) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "problem needs %zu doubles of scratch; the fixed array holds %u", need,
                      (unsigned)TPMG_VCYCLE_NOALLOC_MAX_DOUBLES);
        return fail(ctx, TPMG_ERR_INVALID_ARG, msg);
    }
    int dev = -1;
    CU(cudaGetDevice(&dev));
    if (dev != ctx->device) return fail(ctx, TPMG_ERR_INVALID_ARG, "the context's device must be current");
    double *const base = ctx->noalloc_base;   // looked up by tpmg_setup
    struct Saved { double *f, *u, *u2, *ft; } saved[16];   // n_levels <= 10
    size_t off = 0;
    for (int l = 0; l < L; ++l) {
        LevelDev &D = ctx->lv[l];
        saved[l] = Saved{D.f, D.u, D.u2, D.ft};
        if (l < L - 1) {
            D.f = base + off; off += padded(l);
            D.u = base + off; off += padded(l);
        }
        if (jac) { D.u2 = base + off; off += padded(l); }
        if (D.ft) { D.ft = base + off; off += padded(l); }
    }
    const tpmg_status st = vcycle_fine(ctx, d_r, d_z);
    for (int l = 0; l < L; ++l) {
        ctx->lv[l].f = saved[l].f;
        ctx->lv[l].u = saved[l].u;
        ctx->lv[l].u2 = saved[l].u2;
        ctx->lv[l].ft = saved[l].ft;
    }
    return st;
}

tpmg_status tpmg_solve(tpmg_ctx *ctx, const double *d_f, double *d_u, double rtol, int max_iter, int *iters,
                       double *rel_resid, double *resid_hist)
{
    if (!ctx || !d_f || !d_u || !iters || !rel_resid) return fail(ctx, TPMG_ERR_INVALID_ARG, "NULL argument");
    if (!(rtol >= 0.0) || max_iter < 0) return fail(ctx, TPMG_ERR_INVALID_ARG, "rtol must be >= 0, max_iter >= 0");
    if (d_f == d_u) return fail(ctx, TPMG_ERR_INVALID_ARG, "f and u must not overlap");
    if (nonsymmetric(ctx) && ctx->p.outer == TPMG_OUTER_CG)
        return fail(ctx, TPMG_ERR_INVALID_ARG, "vertical advection or linear prolongation: the operator or the V-cycle is not symmetric, so CG does not apply (use Richardson or BiCGStab)");
    // the device-side loop cannot carry the event pairs of a timed kernel class
    if (ctx->p.outer == TPMG_OUTER_CG && ctx->p.graphs && ctx->tr.mask == 0 && max_iter < kHistCap)
        return pcg_graph(ctx, d_f, d_u, rtol, max_iter, iters, rel_resid, resid_hist);
    long long before = 0, after = 0;
    for (int c = 0; c < TPMG_K_COUNT; ++c) before += ctx->tr.launches[c];
    const tpmg_status st = outer_host(ctx, d_f, d_u, rtol, max_iter, iters, rel_resid, resid_hist);
    for (int c = 0; c < TPMG_K_COUNT; ++c) after += ctx->tr.launches[c];
    ctx->last_launches = after - before;
    return st;
}

tpmg_status tpmg_batch_create(tpmg_ctx *const *ctxs, int n, const double *const *d_f, double *const *d_u, double rtol,
                              int max_iter, tpmg_batch **out)
{
    return tpmg_batch_create_ex(ctxs, n, d_f, d_u, rtol, max_iter, TPMG_BATCH_AUTO, 0, out);
}

tpmg_status tpmg_batch_create_ex(tpmg_ctx *const *ctxs, int n, const double *const *d_f, double *const *d_u,
                                 double rtol, int max_iter, int form, int groups, tpmg_batch **out)
{
    if (!out || !ctxs || !d_f || !d_u || n < 1) return TPMG_ERR_INVALID_ARG;
    if (form != TPMG_BATCH_AUTO && form != TPMG_BATCH_BRANCHES && form != TPMG_BATCH_WORKLIST) return TPMG_ERR_INVALID_ARG;
    if (groups < 0 || groups > n) return TPMG_ERR_INVALID_ARG;
    if (!(rtol >= 0.0) || max_iter < 0 || max_iter >= kHistCap) return TPMG_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return TPMG_ERR_CUDA;
    bool worklist = true, repeated = false;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !d_f[i] || !d_u[i] || d_f[i] == d_u[i] || ctxs[i]->device != dev) return TPMG_ERR_INVALID_ARG;
        if (ctxs[i]->p.outer != TPMG_OUTER_CG) return TPMG_ERR_INVALID_ARG;   // batches hold device-side CG loops
        if (nonsymmetric(ctxs[i])) return TPMG_ERR_INVALID_ARG;              // which need a symmetric A and B
        worklist = worklist && worklist_member_ok(ctxs[i]);
        for (int k = 0; k < i; ++k) {
            if (ctxs[k] == ctxs[i]) repeated = true;
            if (d_u[k] == d_u[i] || d_u[k] == d_f[i] || d_f[k] == d_u[i]) return TPMG_ERR_INVALID_ARG;   // aliased
        }
    }
    if (form == TPMG_BATCH_WORKLIST && !worklist) return TPMG_ERR_INVALID_ARG;   // a member does not qualify
    if (form == TPMG_BATCH_BRANCHES) worklist = false;
    // automatic: branches where every problem has its own context (measured faster on the
    // 48-problem workload: the problems' graphs overlap freely), the work list where a
    // context carries several right-hand sides (a branch holds its context's own solve)
    if (form == TPMG_BATCH_AUTO && !repeated) worklist = false;
    if (repeated && !worklist) return TPMG_ERR_INVALID_ARG;
    tpmg_batch *b = new (std::nothrow) tpmg_batch();
    if (!b) return TPMG_ERR_OOM;
    b->ctx.assign(ctxs, ctxs + n);
    b->init_launches.assign(n, 0);
    b->iter_launches.assign(n, 0);
    b->rtol = rtol;
    b->max_iter = max_iter;
    if (worklist) {
        const tpmg_status st = build_worklist(b, ctxs, n, d_f, d_u, ctxs[0]->stream, groups);
        if (st != TPMG_OK) {
            (void)cudaGetLastError();
            tpmg_batch_destroy(b);
            return st;
        }
        *out = b;
        return TPMG_OK;
    }
    cudaGraph_t g;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) {
        delete b;
        return TPMG_ERR_CUDA;
    }
    tpmg_status st = TPMG_OK;
    for (int i = 0; i < n && st == TPMG_OK; ++i)
        st = append_solve(ctxs[i], g, d_f[i], d_u[i], rtol, max_iter, &b->init_launches[i], &b->iter_launches[i]);
    if (st == TPMG_OK && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) st = TPMG_ERR_CUDA;
    cudaGraphDestroy(g);
    if (st != TPMG_OK) {
        tpmg_batch_destroy(b);
        return st;
    }
    *out = b;
    return TPMG_OK;
}

tpmg_status tpmg_batch_run(tpmg_batch *b, void *cuda_stream, int *iters, double *rel_resid, int *status,
                           long long *kernel_launches)
{
    if (!b || !iters || !rel_resid) return TPMG_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return TPMG_ERR_CUDA;
    if (b->form == TPMG_BATCH_WORKLIST) {
        const int M = (int)b->ctx.size();
        for (int m = 0; m < M; ++m)
            if (cudaMemcpyAsync(b->h_sc + m, b->d_sc[m], sizeof(Scalars), cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return TPMG_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return TPMG_ERR_CUDA;
        tpmg_status first = TPMG_OK;
        for (int m = 0; m < M; ++m) {
            const tpmg_status st = loop_result(b->ctx[m], b->h_sc[m], b->rtol, b->max_iter, &iters[m], &rel_resid[m]);
            if (status) status[m] = st;
            if (st != TPMG_OK && first == TPMG_OK) first = st;
        }
        // each group's loop runs as long as its longest member
        long long launches = 0;
        for (const tpmg_batch::Group &grp : b->groups) {
            int it_max = 0;
            for (int m : grp.members) it_max = std::max(it_max, iters[m]);
            launches += grp.init + (long long)it_max * grp.iter;
        }
        if (kernel_launches) *kernel_launches = launches;
        return first;
    }
    for (tpmg_ctx *c : b->ctx)
        if (cudaMemcpyAsync(c->h_sc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return TPMG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TPMG_ERR_CUDA;
    tpmg_status first = TPMG_OK;
    long long launches = 0;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        const tpmg_status st = loop_result(b->ctx[i], *b->ctx[i]->h_sc, b->rtol, b->max_iter, &iters[i], &rel_resid[i]);
        if (status) status[i] = st;
        if (st != TPMG_OK && first == TPMG_OK) first = st;
        launches += b->init_launches[i] + (long long)iters[i] * b->iter_launches[i];
    }
    if (kernel_launches) *kernel_launches = launches;
    return first;
}

int tpmg_batch_form(const tpmg_batch *b) { return b ? b->form : -1; }

void tpmg_batch_destroy(tpmg_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (!b->allocs.empty() || b->h_sc) cudaDeviceSynchronize();   // no member's kernel still reads them
    for (void *q : b->allocs) cudaFree(q);
    if (b->h_sc) cudaFreeHost(b->h_sc);
    delete b;
}

tpmg_status tpmg_solve_host(tpmg_ctx *ctx, const double *h_f, double *h_u, double rtol, int max_iter, int *iters,
                            double *rel_resid, double *resid_hist)
{
    if (!ctx || !h_f || !h_u || !iters || !rel_resid) return fail(ctx, TPMG_ERR_INVALID_ARG, "NULL argument");
    if (!(rtol >= 0.0) || max_iter < 0) return fail(ctx, TPMG_ERR_INVALID_ARG, "rtol must be >= 0, max_iter >= 0");
    if (nonsymmetric(ctx) && ctx->p.outer == TPMG_OUTER_CG)
        return fail(ctx, TPMG_ERR_INVALID_ARG, "vertical advection or linear prolongation: the operator or the V-cycle is not symmetric, so CG does not apply (use Richardson or BiCGStab)");
    const size_t bytes = sizeof(double) * ctx->N;
    CU(cudaMemcpyAsync(ctx->hf, h_f, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->hu, h_u, bytes, cudaMemcpyHostToDevice, ctx->stream));
    // the solve of tpmg_solve on the staging vectors (the device-side loop where it applies)
    tpmg_status st = tpmg_solve(ctx, ctx->hf, ctx->hu, rtol, max_iter, iters, rel_resid, resid_hist);
    CU(cudaMemcpyAsync(h_u, ctx->hu, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return st;
}

// tpmg_solve_host for a sequence of right-hand sides, with the copies of one system
// overlapping the solves of its neighbours.  Two staging slots alternate: system j is
// solved in slot j % 2 while the copy-in stream fills the other slot with system j + 1's
// inputs and the copy-out stream drains system j - 1's solution from it.  Every solve is
// tpmg_solve's on one slot's vectors (one cached graph per slot), and the events order
// each slot's uses: inputs copied -> solved -> solution copied out -> next inputs.
tpmg_status tpmg_solve_host_many(tpmg_ctx *ctx, int n, const double *const *h_f, double *const *h_u, int guess,
                                 double rtol, int max_iter, int *iters, double *rel_resid, int *status)
{
    if (!ctx) return TPMG_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!h_f || !h_u || !iters || !rel_resid)))
        return fail(ctx, TPMG_ERR_INVALID_ARG, "n < 0 or NULL array");
    if (guess != 0 && guess != 1) return fail(ctx, TPMG_ERR_INVALID_ARG, "guess must be 0 or 1");
    if (!(rtol >= 0.0) || max_iter < 0) return fail(ctx, TPMG_ERR_INVALID_ARG, "rtol must be >= 0, max_iter >= 0");
    if (nonsymmetric(ctx) && ctx->p.outer == TPMG_OUTER_CG)
        return fail(ctx, TPMG_ERR_INVALID_ARG, "vertical advection or linear prolongation: the operator or the V-cycle is not symmetric, so CG does not apply (use Richardson or BiCGStab)");
    // a solution is copied out while later systems' inputs are copied in, so no solution
    // array may overlap another system's arrays
    auto overlap = [&](const double *a, const double *b) { return a < b + ctx->N && b < a + ctx->N; };
    for (int j = 0; j < n; ++j) {
        if (!h_f[j] || !h_u[j]) return fail(ctx, TPMG_ERR_INVALID_ARG, "NULL right-hand side or solution");
        for (int k = 0; k < n; ++k)
            if (k != j && (overlap(h_u[k], h_u[j]) || overlap(h_u[k], h_f[j])))
                return fail(ctx, TPMG_ERR_INVALID_ARG, "a solution array overlaps another system's arrays");
    }
    if (n == 0) return TPMG_OK;
    if (!ctx->hu2) {   // hu2 is set last: a failed first attempt is retried whole
        if (!ctx->hf2 && dalloc(ctx, &ctx->hf2, ctx->N) != cudaSuccess)
            return fail(ctx, TPMG_ERR_OOM, "second staging slot");
        if (dalloc(ctx, &ctx->hu2, ctx->N) != cudaSuccess) return fail(ctx, TPMG_ERR_OOM, "second staging slot");
    }
    if (!ctx->xout) {   // the streams and events, kept only once all of them exist
        cudaStream_t in = nullptr, out = nullptr;
        cudaEvent_t ev[6] = {};
        cudaError_t e = cudaStreamCreateWithFlags(&in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&out, cudaStreamNonBlocking);
        for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (cudaEvent_t x : ev)
                if (x) cudaEventDestroy(x);
            if (in) cudaStreamDestroy(in);
            if (out) cudaStreamDestroy(out);
            return fail(ctx, TPMG_ERR_CUDA, std::string("host solves: ") + cudaGetErrorString(e));
        }
        ctx->xin = in;
        ctx->xout = out;
        for (int i = 0; i < 2; ++i) {
            ctx->xev_in[i] = ev[i];
            ctx->xev_solved[i] = ev[2 + i];
            ctx->xev_out[i] = ev[4 + i];
        }
    }
    double *F[2] = {ctx->hf, ctx->hf2}, *U[2] = {ctx->hu, ctx->hu2};
    const size_t bytes = sizeof(double) * ctx->N;
    // the streams start behind all work already on the context's stream; a slot's events
    // are recorded afresh on every use, so no wait below sees an earlier call's record
    CU(cudaEventRecord(ctx->xev_solved[0], ctx->stream));
    CU(cudaEventRecord(ctx->xev_solved[1], ctx->stream));
    CU(cudaEventRecord(ctx->xev_out[0], ctx->stream));
    CU(cudaEventRecord(ctx->xev_out[1], ctx->stream));
    // system j's inputs into slot j % 2, once the slot's previous system is solved and
    // its solution copied out
    auto copy_in = [&](int j) -> cudaError_t {
        const int sl = j & 1;
        cudaError_t e = cudaStreamWaitEvent(ctx->xin, ctx->xev_solved[sl], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->xin, ctx->xev_out[sl], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(F[sl], h_f[j], bytes, cudaMemcpyHostToDevice, ctx->xin);
        if (e == cudaSuccess && guess) e = cudaMemcpyAsync(U[sl], h_u[j], bytes, cudaMemcpyHostToDevice, ctx->xin);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->xev_in[sl], ctx->xin);
        return e;
    };
    // with the loop on the device every solve is enqueued at once and its scalars read
    // after the last one, so the solves follow each other on the GPU without waiting for
    // the host; otherwise each tpmg_solve returns before the next system is enqueued
    const bool device_loop =
        ctx->p.outer == TPMG_OUTER_CG && ctx->p.graphs && ctx->tr.mask == 0 && max_iter < kHistCap;
    if (device_loop && ctx->h_many_cap < n) {
        if (ctx->h_many) CU(cudaFreeHost(ctx->h_many));
        ctx->h_many = nullptr;
        ctx->h_many_cap = 0;
        CU(cudaMallocHost(&ctx->h_many, sizeof(Scalars) * (size_t)n));
        ctx->h_many_cap = n;
    }
    std::vector<const tpmg_ctx::SolveGraph *> graph(device_loop ? n : 0, nullptr);
    auto body = [&]() -> tpmg_status {
        tpmg_status first = TPMG_OK;
        CU(copy_in(0));
        for (int j = 0; j < n; ++j) {
            const int sl = j & 1;
            if (j + 1 < n) CU(copy_in(j + 1));
            CU(cudaStreamWaitEvent(ctx->stream, ctx->xev_in[sl], 0));
            if (!guess) {
                CU(cudaStreamWaitEvent(ctx->stream, ctx->xev_out[sl], 0));
                CU(cudaMemsetAsync(U[sl], 0, bytes, ctx->stream));
            }
            if (device_loop) {
                const tpmg_status st = pcg_graph_launch(ctx, F[sl], U[sl], rtol, max_iter, ctx->h_many + j, &graph[j]);
                if (st != TPMG_OK) return st;
            } else {
                const tpmg_status st = tpmg_solve(ctx, F[sl], U[sl], rtol, max_iter, &iters[j], &rel_resid[j], nullptr);
                if (status) status[j] = st;
                if (st != TPMG_OK && st != TPMG_ERR_NOT_CONVERGED && st != TPMG_ERR_BREAKDOWN) return st;
                if (st != TPMG_OK && first == TPMG_OK) first = st;
            }
            CU(cudaEventRecord(ctx->xev_solved[sl], ctx->stream));
            CU(cudaStreamWaitEvent(ctx->xout, ctx->xev_solved[sl], 0));
            CU(cudaMemcpyAsync(h_u[j], U[sl], bytes, cudaMemcpyDeviceToHost, ctx->xout));
            CU(cudaEventRecord(ctx->xev_out[sl], ctx->xout));
        }
        if (device_loop) {
            CU(cudaStreamSynchronize(ctx->stream));
            for (int j = 0; j < n; ++j) {
                const tpmg_status st =
                    pcg_graph_result(ctx, ctx->h_many[j], *graph[j], rtol, max_iter, &iters[j], &rel_resid[j]);
                if (status) status[j] = st;
                if (st != TPMG_OK && first == TPMG_OK) first = st;
            }
        }
        return first;
    };
    tpmg_status st = body();
    // nothing of the call is in flight when it returns, whatever failed
    const cudaError_t e1 = cudaStreamSynchronize(ctx->xin), e2 = cudaStreamSynchronize(ctx->xout),
                      e3 = cudaStreamSynchronize(ctx->stream);
    if (st == TPMG_OK || st == TPMG_ERR_NOT_CONVERGED || st == TPMG_ERR_BREAKDOWN) {
        const cudaError_t e = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3;
        if (e != cudaSuccess) return fail(ctx, TPMG_ERR_CUDA, std::string("host solves: ") + cudaGetErrorString(e));
    }
    return st;
}

tpmg_status tpmg_query(const tpmg_ctx *ctx, int level, int *n_cells, int *n_r, double *omega2, int *n_colours)
{
    if (!ctx || level < 0 || level >= ctx->p.n_levels) return TPMG_ERR_INVALID_ARG;
    if (n_cells) *n_cells = ctx->lv[level].n;
    if (n_r) *n_r = ctx->p.n_r;
    if (omega2) *omega2 = ctx->host.omega2;
    if (n_colours) *n_colours = ctx->lv[level].n_colours;
    return TPMG_OK;
}

tpmg_status tpmg_query_tuning(const tpmg_ctx *ctx, int level, int *variant, float *us)
{
    if (!ctx || level < 0 || level >= ctx->p.n_levels) return TPMG_ERR_INVALID_ARG;
    const LevelDev &D = ctx->lv[level];
    if (variant) *variant = D.relax_variant;
    if (us) std::copy(D.relax_us, D.relax_us + RELAX_VARIANTS, us);
    return TPMG_OK;
}

tpmg_status tpmg_export_mesh(const tpmg_ctx *ctx, int level, double *centres, double *areas, int *nbrs, double *g,
                             int *colour, double *r_faces)
{
    if (!ctx || level < 0 || level >= ctx->p.n_levels) return TPMG_ERR_INVALID_ARG;
    const HostLevel &H = ctx->host.lev[ctx->p.refinement - (ctx->p.n_levels - 1 - level)];
    if (centres) std::memcpy(centres, H.centre.data(), H.centre.size() * sizeof(double));
    if (areas) std::memcpy(areas, H.area.data(), H.area.size() * sizeof(double));
    if (nbrs) std::memcpy(nbrs, H.nbr.data(), H.nbr.size() * sizeof(int));
    if (g) std::memcpy(g, H.g.data(), H.g.size() * sizeof(double));
    if (colour) std::memcpy(colour, H.colour.data(), H.colour.size() * sizeof(int));
    if (r_faces) std::memcpy(r_faces, ctx->host.r.data(), ctx->host.r.size() * sizeof(double));
    return TPMG_OK;
}

tpmg_status tpmg_profile(tpmg_ctx *ctx, unsigned class_mask)
{
    if (!ctx) return TPMG_ERR_INVALID_ARG;
    if (class_mask >> TPMG_K_COUNT) return fail(ctx, TPMG_ERR_INVALID_ARG, "unknown kernel class in mask");
    CU(cudaStreamSynchronize(ctx->stream));
    drop_graph(ctx);   // its captured event nodes would alias the reset event pool
    Tracer &t = ctx->tr;
    t.mask = class_mask;
    std::fill(t.launches, t.launches + TPMG_K_COUNT, 0LL);
    std::fill(t.units, t.units + TPMG_K_COUNT, 0.0);
    std::fill(t.bytes, t.bytes + TPMG_K_COUNT, 0.0);
    std::fill(t.flops, t.flops + TPMG_K_COUNT, 0.0);
    t.used = 0;
    t.open = -1;
    if (class_mask) CU(grow_events(t, 8192));   // created here, outside any timed region
    return TPMG_OK;
}

tpmg_status tpmg_profile_read(tpmg_ctx *ctx, int kernel_class, long long *launches, double *total_ms, double *units,
                              long long *timed)
{
    if (!ctx || kernel_class < 0 || kernel_class >= TPMG_K_COUNT) return fail(ctx, TPMG_ERR_INVALID_ARG, "bad class");
    CU(cudaStreamSynchronize(ctx->stream));
    const Tracer &t = ctx->tr;
    double ms = 0.0;
    long long n = 0;
    for (size_t i = 0; i < t.used; ++i) {
        if (t.cls[i] != kernel_class) continue;
        float m = 0.f;
        CU(cudaEventElapsedTime(&m, t.ev[2 * i], t.ev[2 * i + 1]));
        ms += m;
        n += t.nl[i];
    }
    if (launches) *launches = t.launches[kernel_class];
    if (total_ms) *total_ms = ms;
    if (units) *units = t.units[kernel_class];
    if (timed) *timed = n;
    return TPMG_OK;
}

tpmg_status tpmg_profile_work(tpmg_ctx *ctx, int kernel_class, double *bytes, double *timed_bytes, double *flops,
                              double *timed_flops)
{
    if (!ctx || kernel_class < 0 || kernel_class >= TPMG_K_COUNT) return fail(ctx, TPMG_ERR_INVALID_ARG, "bad class");
    CU(cudaStreamSynchronize(ctx->stream));
    const Tracer &t = ctx->tr;
    double b = 0.0, fl = 0.0;
    for (size_t i = 0; i < t.used; ++i)
        if (t.cls[i] == kernel_class) {
            b += t.nb[i];
            fl += t.nf[i];
        }
    if (bytes) *bytes = t.bytes[kernel_class];
    if (timed_bytes) *timed_bytes = b;
    if (flops) *flops = t.flops[kernel_class];
    if (timed_flops) *timed_flops = fl;
    return TPMG_OK;
}

const char *tpmg_status_string(tpmg_status s)
{
    const int i = (int)s;
    return (i >= 0 && i < (int)(sizeof(kStatus) / sizeof(kStatus[0]))) ? kStatus[i] : "TPMG_UNKNOWN_STATUS";
}

const char *tpmg_last_error(const tpmg_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

// ---- learned form (tpmg_learned.h) ------------------------------------------

namespace {

tpmg_status level_arg(tpmg_ctx *ctx, int level, const void *a, const void *b, long rows, const int *cells)
{
    if (!ctx) return TPMG_ERR_INVALID_ARG;
    if (level < 0 || level >= ctx->p.n_levels) return fail(ctx, TPMG_ERR_INVALID_ARG, "level out of range");
    if (!a || !b) return fail(ctx, TPMG_ERR_INVALID_ARG, "NULL argument");
    if (rows < 1 || (!cells && rows > ctx->lv[level].n) || rows > 64L * 65535L ||
        (double)rows * ctx->p.n_r > 2147483647.0)
        return fail(ctx, TPMG_ERR_INVALID_ARG, "rows out of range (rows * n_r must fit in a 32-bit index)");
    return TPMG_OK;
}

// point values of the field f on level into ctx->net_p and its scale s into d_net_s[2]
tpmg_status level_scale(tpmg_ctx *ctx, int level, const double *f)
{
    const Launch L = launch_of(ctx);
    const LevelDev &lv = ctx->lv[level];
    double *s = ctx->d_net_s + 2;
    const long n = (long)lv.n * ctx->p.n_r;
    if (n > ctx->net_p_cap) {   // grows to the finest level at most; freed by tpmg_destroy
        CU(dalloc(ctx, &ctx->net_p, (size_t)n));
        ctx->net_p_cap = n;
    }
    LCHK(run(ctx, TPMG_K_NET, (double)n, [&] {
        return launch_net_prepare<double>(L, lv, ctx->vert, f, ctx->net_p, ctx->partials, ctx->n_part);
    }));
    LCHK(run(ctx, TPMG_K_NET, 1.0, [&] { return launch_net_scale_finish(L, lv, ctx->partials, ctx->n_part, s); }));
    return TPMG_OK;
}

}  // namespace

tpmg_status tpmg_net_features(tpmg_ctx *ctx, int level, const double *d_f, const int *d_cells, long rows, float *d_x,
                              double *h_scale)
{
    tpmg_status st = level_arg(ctx, level, d_f, d_x, rows, d_cells);
    if (st != TPMG_OK || (st = level_scale(ctx, level, d_f)) != TPMG_OK) return st;
    const Launch L = launch_of(ctx);
    const double *s = ctx->d_net_s + 2;
    LCHK(run(ctx, TPMG_K_NET, (double)rows * ctx->p.n_r, [&] {
        return launch_net_features(L, ctx->lv[level], ctx->net_p, d_cells, rows, s, d_x);
    }));
    if (h_scale) {
        CU(cudaMemcpyAsync(&ctx->h_sc->ff, s, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        *h_scale = ctx->h_sc->ff;
    }
    return TPMG_OK;
}

tpmg_status tpmg_net_targets(tpmg_ctx *ctx, int level, const double *d_f, const double *d_u, const int *d_cells,
                             long rows, float *d_t)
{
    tpmg_status st = level_arg(ctx, level, d_f, d_t, rows, d_cells);
    if (st == TPMG_OK && !d_u) st = fail(ctx, TPMG_ERR_INVALID_ARG, "NULL argument");
    if (st != TPMG_OK || (st = level_scale(ctx, level, d_f)) != TPMG_OK) return st;
    const Launch L = launch_of(ctx);
    const double *s = ctx->d_net_s + 2;
    LCHK(run(ctx, TPMG_K_NET, (double)rows * ctx->p.n_r, [&] { return launch_net_targets(L, d_u, d_cells, rows, s, d_t); }));
    return TPMG_OK;
}

tpmg_status tpmg_record_coarse(tpmg_ctx *ctx, double *d_buf, int capacity)
{
    if (!ctx) return TPMG_ERR_INVALID_ARG;
    if (d_buf) {
        if (ctx->p.precision != TPMG_PREC_MIXED || ctx->p.n_levels < 2 || ctx->p.graphs != 0)
            return fail(ctx, TPMG_ERR_INVALID_ARG, "recording needs the mixed-precision form, n_levels >= 2, graphs 0");
        if (capacity < 1) return fail(ctx, TPMG_ERR_INVALID_ARG, "capacity must be >= 1");
    }
    ctx->rec = d_buf;
    ctx->rec_cap = d_buf ? capacity : 0;
    ctx->rec_n = 0;
    return TPMG_OK;
}

tpmg_status tpmg_record_count(const tpmg_ctx *ctx, int *count)
{
    if (!ctx || !count) return TPMG_ERR_INVALID_ARG;
    *count = ctx->rec_n;
    return TPMG_OK;
}

tpmg_status tpmg_coarse_solve(tpmg_ctx *ctx, const double *d_f0, double *d_u0, int sweeps)
{
    if (!ctx || !d_f0 || !d_u0) return fail(ctx, TPMG_ERR_INVALID_ARG, "NULL argument");
    if (ctx->p.precision != TPMG_PREC_MIXED || ctx->p.n_levels < 2)
        return fail(ctx, TPMG_ERR_INVALID_ARG, "the coarse solve needs the mixed-precision form and n_levels >= 2");
    if (sweeps < 1 || sweeps > 64) return fail(ctx, TPMG_ERR_INVALID_ARG, "sweeps must be in 1..64");
    LevelDev &c = ctx->lv[0];
    const long n = (long)c.n * ctx->p.n_r;
    const Launch L = launch_of(ctx);
    LCHK(run(ctx, TPMG_K_COPY, (double)n, [&] { return launch_to_f32(L, n, d_f0, c.f32); }));
    // Algorithm 1's coarsest-level solve with nu_coarse = sweeps, without the
    // network or the recording
    const int nu = ctx->p.nu_coarse;
    double *rec = ctx->rec;
    ctx->p.nu_coarse = sweeps;
    ctx->rec = nullptr;
    ctx->net_coarse_on = false;
    const tpmg_status st = vcycle_mixed<float>(ctx, 0, c.f32, c.u32, c.u2_32, nullptr, nullptr);
    ctx->p.nu_coarse = nu;
    ctx->rec = rec;
    if (st != TPMG_OK) return st;
    LCHK(run(ctx, TPMG_K_COPY, (double)n, [&] { return launch_to_f64(L, n, c.u32, d_u0); }));
    return TPMG_OK;
}

tpmg_status tpmg_net_fault(tpmg_ctx *ctx, int *flag)
{
    if (!ctx || !flag) return fail(ctx, TPMG_ERR_INVALID_ARG, "NULL argument");
    int h = 0;
    CU(cudaMemcpyAsync(&h, ctx->d_net_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *flag = h != 0;
    return TPMG_OK;
}

tpmg_status tpmg_net_predict(tpmg_ctx *ctx, int role, const double *d_f, double *d_u)
{
    if (!ctx || !d_f || !d_u) return fail(ctx, TPMG_ERR_INVALID_ARG, "NULL argument");
    if (role != TPMG_NET_COARSE && role != TPMG_NET_WARM) return fail(ctx, TPMG_ERR_INVALID_ARG, "unknown role");
    if (!ctx->net[role]) return fail(ctx, TPMG_ERR_INVALID_ARG, "no network attached in this role");
    const LevelDev &lv = role == TPMG_NET_COARSE ? ctx->lv[0] : ctx->lv.back();
    return net_infer<double, double>(ctx, role, lv, d_f, d_u);
}

tpmg_status tpmg_vcycle_learned(tpmg_ctx *ctx, const double *d_r, double *d_z)
{
    if (!ctx || !d_r || !d_z) return fail(ctx, TPMG_ERR_INVALID_ARG, "NULL argument");
    if (d_r == d_z) return fail(ctx, TPMG_ERR_INVALID_ARG, "r and z must not overlap");
    if (!ctx->net[TPMG_NET_COARSE]) return fail(ctx, TPMG_ERR_INVALID_ARG, "no COARSE network attached");
    ctx->net_coarse_on = true;
    const tpmg_status st = vcycle_fine(ctx, d_r, d_z);
    ctx->net_coarse_on = false;
    return st;
}

tpmg_status tpmg_attach_net(tpmg_ctx *ctx, int role, tpmg_net *net)
{
    if (!ctx) return TPMG_ERR_INVALID_ARG;
    if (role != TPMG_NET_COARSE && role != TPMG_NET_WARM) return fail(ctx, TPMG_ERR_INVALID_ARG, "unknown role");
    if (net) {
        const NetView v = net_view(net);
        if (v.sizes[0] != 2 * ctx->p.n_r || v.sizes[4] != ctx->p.n_r)
            return fail(ctx, TPMG_ERR_INVALID_ARG, "the network's columns do not have the context's n_r");
        if (role == TPMG_NET_COARSE && (ctx->p.precision != TPMG_PREC_MIXED || ctx->p.n_levels < 2))
            return fail(ctx, TPMG_ERR_INVALID_ARG, "a coarse network needs the mixed-precision form and n_levels >= 2");
        auto &w = ctx->nws[role];
        const long rows = role == TPMG_NET_COARSE ? ctx->lv[0].n : ctx->lv.back().n;
        const long h = v.sizes[1];
        if (w.rows != rows * h) {   // (re)allocate for this hidden width; old blocks are freed at destroy
            const size_t nr = (size_t)ctx->p.n_r;
            CU(dalloc(ctx, &w.p, (size_t)rows * nr));
            CU(dalloc(ctx, &w.x, (size_t)rows * 2 * nr));
            CU(dalloc(ctx, &w.xt, net_tc_input_elems(rows, ctx->p.n_r)));
            CU(dalloc(ctx, &w.h0, (size_t)rows * h));
            CU(dalloc(ctx, &w.h1, (size_t)rows * h));
            CU(dalloc(ctx, &w.y, (size_t)rows * nr));
            w.rows = rows * h;
        }
    }
    ctx->net[role] = net;
    if (ctx->lg.exec) cudaGraphExecDestroy(ctx->lg.exec);
    ctx->lg.exec = nullptr;
    ctx->lg.max_iter = -1;
    return TPMG_OK;
}

tpmg_status tpmg_solve_learned(tpmg_ctx *ctx, const double *d_f, double *d_u, double rtol, int max_iter, int *iters,
                               double *rel_resid, int *info, int *fallback_iters, long long *kernel_launches)
{
    if (!ctx || !d_f || !d_u || !iters || !rel_resid) return fail(ctx, TPMG_ERR_INVALID_ARG, "NULL argument");
    if (ctx->p.precision != TPMG_PREC_MIXED)
        return fail(ctx, TPMG_ERR_INVALID_ARG, "the learned solve needs the mixed-precision form");
    if (nonsymmetric(ctx))
        return fail(ctx, TPMG_ERR_INVALID_ARG, "the learned solve runs flexible CG, which needs a symmetric operator "
                                               "and V-cycle");
    if (!(rtol >= 0.0) || max_iter < 1 || max_iter >= kHistCap)
        return fail(ctx, TPMG_ERR_INVALID_ARG, "rtol must be >= 0, max_iter in 1..4095");
    if (d_f == d_u) return fail(ctx, TPMG_ERR_INVALID_ARG, "f and u must not overlap");
    auto &lg = ctx->lg;
    Scalars s{};
    long long launches = 0;
    int it_learned = 0;
    if (!ctx->p.graphs || ctx->tr.mask != 0) {
        // host-driven loop (graphs off, or a kernel class being timed): same kernels, same order
        long long before = 0, after = 0;
        for (int c = 0; c < TPMG_K_COUNT; ++c) before += ctx->tr.launches[c];
        double rel_h = 1.0;
        const tpmg_status sh = pcg(ctx, d_f, d_u, rtol, max_iter, &it_learned, &rel_h, nullptr, true);
        for (int c = 0; c < TPMG_K_COUNT; ++c) after += ctx->tr.launches[c];
        launches = after - before;
        if (sh != TPMG_OK && sh != TPMG_ERR_NOT_CONVERGED && sh != TPMG_ERR_BREAKDOWN) return sh;
        s = *ctx->h_sc;
        if (sh == TPMG_ERR_BREAKDOWN && s.flag == 0) s.flag = 2;
    } else {
    if (!lg.exec || lg.f != d_f || lg.u != d_u || lg.rtol != rtol || lg.max_iter != max_iter ||
        lg.nets[0] != ctx->net[0] || lg.nets[1] != ctx->net[1]) {
        if (lg.exec) cudaGraphExecDestroy(lg.exec);
        lg.exec = nullptr;
        cudaGraph_t g;
        CU(cudaGraphCreate(&g, 0));
        // event pairs of timed classes cannot live inside the loop body: not timed here
        const unsigned mask = ctx->tr.mask;
        ctx->tr.mask = 0;
        tpmg_status st = append_solve(ctx, g, d_f, d_u, rtol, max_iter, &lg.init, &lg.iter, true, &lg.cls);
        ctx->tr.mask = mask;
        cudaError_t e = st == TPMG_OK ? cudaGraphInstantiate(&lg.exec, g, 0) : cudaSuccess;
        cudaGraphDestroy(g);
        if (st != TPMG_OK) return st;
        if (e != cudaSuccess) return fail(ctx, TPMG_ERR_CUDA, std::string("learned solve graph: ") + cudaGetErrorString(e));
        lg.f = d_f;
        lg.u = d_u;
        lg.rtol = rtol;
        lg.max_iter = max_iter;
        lg.nets[0] = ctx->net[0];
        lg.nets[1] = ctx->net[1];
    }
    CU(cudaGraphLaunch(lg.exec, ctx->stream));
    CU(cudaMemcpyAsync(ctx->h_sc, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    s = *ctx->h_sc;
    launches = lg.init + (long long)s.it * lg.iter;
    if (s.it >= 0)
        for (int c = 0; c < TPMG_K_COUNT; ++c) {
            ctx->tr.launches[c] += lg.cls.init[c] + (long long)s.it * lg.cls.iter[c];
            ctx->tr.units[c] += lg.cls.uinit[c] + s.it * lg.cls.uiter[c];
            ctx->tr.bytes[c] += lg.cls.binit[c] + s.it * lg.cls.biter[c];
            ctx->tr.flops[c] += lg.cls.finit[c] + s.it * lg.cls.fiter[c];
        }
    it_learned = s.it;
    }
    int bits = s.info & 3;
    if (!ctx->net[TPMG_NET_WARM]) bits = 0;   // the guess judged was the caller's, not a network's
    *iters = it_learned;
    double rel = s.ff > 0.0 ? std::sqrt(s.rr / s.ff) : 0.0;
    int it_fb = 0;
    tpmg_status st = TPMG_OK;
    if (s.flag != 0 || !(rel <= rtol)) {
        // fallback: plain TPMG-PCG to the same ||f||-relative tolerance
        bits |= TPMG_LEARNED_FALLBACK;
        double rtol_fb = rtol;
        if (s.flag != 0) CU(cudaMemsetAsync(d_u, 0, sizeof(double) * ctx->N, ctx->stream));
        else rtol_fb = rtol * std::sqrt(s.ff / s.rr);
        double rel_fb = 1.0;
        st = tpmg_solve(ctx, d_f, d_u, rtol_fb, max_iter, &it_fb, &rel_fb, nullptr);
        launches += ctx->last_launches;
        const double rr0_fb = ctx->h_sc->rr0;
        rel = s.ff > 0.0 ? rel_fb * std::sqrt(rr0_fb / s.ff) : 0.0;
        *iters += it_fb;
    }
    *rel_resid = rel;
    if (info) *info = bits;
    if (fallback_iters) *fallback_iters = it_fb;
    if (kernel_launches) *kernel_launches = launches;
    ctx->last_launches = launches;
    return st;
}

void tpmg_destroy(tpmg_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    drop_graph(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (cudaStream_t x : {ctx->xin, ctx->xout})
        if (x) {
            cudaStreamSynchronize(x);
            cudaStreamDestroy(x);
        }
    for (int i = 0; i < 2; ++i)
        for (cudaEvent_t e : {ctx->xev_in[i], ctx->xev_solved[i], ctx->xev_out[i]})
            if (e) cudaEventDestroy(e);
    for (void *p : ctx->allocs) cudaFree(p);
    if (ctx->h_sc) cudaFreeHost(ctx->h_sc);
    if (ctx->h_many) cudaFreeHost(ctx->h_many);
    for (cudaEvent_t e : ctx->tr.ev) cudaEventDestroy(e);
    delete ctx;
}

}  // extern "C"
