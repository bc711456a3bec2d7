/*
 * tpmg_oracle.c -- TEST INFRASTRUCTURE ONLY (not part of the product path).
 *
 * A plain, slow, single-threaded FP64 CPU statement of what the tensor-product
 * multigrid (TPMG) preconditioned conjugate-gradient path computes, written from
 * Dedner, Mueller & Scheichl, "Efficient multigrid preconditioners for
 * atmospheric flow simulations at high aspect ratio" (arXiv:1408.2981).
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load this file.  It shares no code, header, table or helper with the CUDA
 * library and includes nothing from it.
 *
 * Problem (Sec. 2, eq. HelmholtzVector with constant profiles
 * alpha_r = alpha_S = beta = 1, xi_r = 0):
 *     -omega^2 div grad u + u = f   in the shell  S^2 x [1, 1+H],
 * homogeneous Neumann conditions at r = 1 and r = 1+H (Appendix A).
 *
 * Everything is plain loops in the order the paper states the method:
 *   grid (Sec. 4.1, Sec. 4.2) -> finite-volume hat coefficients (Appendix A,
 *   eq. hatFunctionsNonFac) -> column equation (eq. ColumnEquation,
 *   TridiagonalSystem) -> Thomas algorithm -> block relaxation (eq. BlockJacobi)
 *   -> V-cycle (Algorithm 1) -> preconditioned CG.
 *
 * Readings taken where the paper is silent, ambiguous or garbled are marked
 * "Reading Cn" and listed in the design notes of the repository.
 *
 * Build: plain C99, compiled with -O2 -ffp-contract=off so that every
 * operation is one IEEE-754 double rounding on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* 3-vectors                                                                  */
/* ------------------------------------------------------------------------- */
typedef struct { double x, y, z; } vec3;

static vec3 v_make(double x, double y, double z) { vec3 v = {x, y, z}; return v; }
static vec3 v_add(vec3 a, vec3 b) { return v_make(a.x + b.x, a.y + b.y, a.z + b.z); }
static vec3 v_sub(vec3 a, vec3 b) { return v_make(a.x - b.x, a.y - b.y, a.z - b.z); }
static vec3 v_scale(vec3 a, double s) { return v_make(a.x * s, a.y * s, a.z * s); }
static double v_dot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static vec3 v_cross(vec3 a, vec3 b)
{
    return v_make(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double v_norm(vec3 a) { return sqrt(v_dot(a, a)); }
static vec3 v_unit(vec3 a) { return v_scale(a, 1.0 / v_norm(a)); }

/* ------------------------------------------------------------------------- */
/* Horizontal grid: icosahedron refined by edge bisection, vertices projected */
/* onto the unit sphere (Sec. 4.1: each coarse triangle holds four fine ones; */
/* Sec. 4.2: icosahedral grid with points projected onto the sphere).         */
/* ------------------------------------------------------------------------- */
typedef struct {
    int ref;            /* refinement level: 20 * 4^ref cells               */
    int n_cells, n_verts, n_edges;
    vec3 *vert;         /* [n_verts] vertex positions on the unit sphere    */
    int *cv;            /* [n_cells][3] vertex ids, counter-clockwise seen from outside */
    int *nbr;           /* [n_cells][3] cell across edge e = (v_e, v_{(e+1)%3}) */
    int *edge;          /* [n_cells][3] id of the unique edge in slot e     */
    vec3 *centre;       /* [n_cells] cell centre r_T                        */
    double *area;       /* [n_cells] |T|                                    */
    double *g;          /* [n_cells][3] |S_TT'| n.(r_T'-r_T)/|r_T'-r_T|^2  */
    int *colour;        /* [n_cells] DSATUR colour of the neighbour graph   */
    int n_colours;
} ogrid;

static void grid_free(ogrid *G)
{
    free(G->vert); free(G->cv); free(G->nbr); free(G->edge);
    free(G->centre); free(G->area); free(G->g); free(G->colour);
    memset(G, 0, sizeof(*G));
}

static int grid_alloc(ogrid *G, int ref, int n_cells, int n_verts)
{
    G->ref = ref;
    G->n_cells = n_cells;
    G->n_verts = n_verts;
    G->vert = (vec3 *)calloc((size_t)n_verts, sizeof(vec3));
    G->cv = (int *)calloc((size_t)n_cells * 3, sizeof(int));
    G->nbr = (int *)calloc((size_t)n_cells * 3, sizeof(int));
    G->edge = (int *)calloc((size_t)n_cells * 3, sizeof(int));
    G->centre = (vec3 *)calloc((size_t)n_cells, sizeof(vec3));
    G->area = (double *)calloc((size_t)n_cells, sizeof(double));
    G->g = (double *)calloc((size_t)n_cells * 3, sizeof(double));
    G->colour = (int *)calloc((size_t)n_cells, sizeof(int));
    if (!G->vert || !G->cv || !G->nbr || !G->edge || !G->centre || !G->area || !G->g || !G->colour)
        return -1;
    return 0;
}

/* Level 0.  Vertices: the 12 cyclic permutations of (0, +-1, +-phi), taken in
 * the order  index = 4*p + 2*[s1 > 0] + [s2 > 0]  for the cyclic shift p of
 * (0, s1, s2*phi), then normalised.  Faces: every triple of pairwise adjacent
 * vertices, listed as (i, j, k) with i the smallest id and (i, j, k)
 * counter-clockwise seen from outside; faces sorted lexicographically. */
static int build_icosahedron(ogrid *G)
{
    const double phi = 0.5 * (1.0 + sqrt(5.0));
    vec3 raw[12];
    int p, s1, s2, i, j, k, nf = 0;
    if (grid_alloc(G, 0, 20, 12)) return -1;
    for (p = 0; p < 3; ++p)
        for (s1 = 0; s1 < 2; ++s1)
            for (s2 = 0; s2 < 2; ++s2) {
                double a = 0.0, b = s1 ? 1.0 : -1.0, c = s2 ? phi : -phi;
                vec3 v;
                if (p == 0) v = v_make(a, b, c);
                else if (p == 1) v = v_make(c, a, b);
                else v = v_make(b, c, a);
                raw[4 * p + 2 * s1 + s2] = v;
            }
    for (i = 0; i < 12; ++i) G->vert[i] = v_unit(raw[i]);
    /* adjacent vertices of the unnormalised icosahedron are at distance 2 */
    for (i = 0; i < 12; ++i)
        for (j = i + 1; j < 12; ++j)
            for (k = j + 1; k < 12; ++k) {
                vec3 dij = v_sub(raw[i], raw[j]), djk = v_sub(raw[j], raw[k]), dki = v_sub(raw[k], raw[i]);
                if (fabs(v_dot(dij, dij) - 4.0) > 1e-9 || fabs(v_dot(djk, djk) - 4.0) > 1e-9 ||
                    fabs(v_dot(dki, dki) - 4.0) > 1e-9)
                    continue;
                {
                    vec3 nrm = v_cross(v_sub(raw[j], raw[i]), v_sub(raw[k], raw[i]));
                    vec3 mid = v_add(v_add(raw[i], raw[j]), raw[k]);
                    if (nf >= 20) return -1;
                    G->cv[3 * nf + 0] = i;
                    if (v_dot(nrm, mid) > 0.0) { G->cv[3 * nf + 1] = j; G->cv[3 * nf + 2] = k; }
                    else { G->cv[3 * nf + 1] = k; G->cv[3 * nf + 2] = j; }
                    ++nf;
                }
            }
    if (nf != 20) return -1;
    /* lexicographic sort of the (i, j, k) rows (insertion sort, 20 rows) */
    for (i = 1; i < 20; ++i) {
        int row[3] = {G->cv[3 * i], G->cv[3 * i + 1], G->cv[3 * i + 2]};
        j = i - 1;
        while (j >= 0 && (G->cv[3 * j] > row[0] ||
                          (G->cv[3 * j] == row[0] && (G->cv[3 * j + 1] > row[1] ||
                                                      (G->cv[3 * j + 1] == row[1] && G->cv[3 * j + 2] > row[2]))))) {
            memcpy(&G->cv[3 * (j + 1)], &G->cv[3 * j], 3 * sizeof(int));
            --j;
        }
        memcpy(&G->cv[3 * (j + 1)], row, 3 * sizeof(int));
    }
    return 0;
}

/* Neighbours: every edge of the closed surface is shared by exactly two cells.
 * Sort all (cell, slot) half-edges by their unordered vertex pair and pair them. */
typedef struct { int lo, hi, cell, slot; } half_edge;

static int cmp_half_edge(const void *pa, const void *pb)
{
    const half_edge *a = (const half_edge *)pa, *b = (const half_edge *)pb;
    if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
    if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
    if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
    return a->slot - b->slot;
}

static int match_edges(ogrid *G)
{
    int n = 3 * G->n_cells, i;
    half_edge *h = (half_edge *)malloc((size_t)n * sizeof(half_edge));
    if (!h) return -1;
    for (i = 0; i < n; ++i) {
        int T = i / 3, e = i % 3;
        int a = G->cv[3 * T + e], b = G->cv[3 * T + (e + 1) % 3];
        h[i].lo = a < b ? a : b;
        h[i].hi = a < b ? b : a;
        h[i].cell = T;
        h[i].slot = e;
    }
    qsort(h, (size_t)n, sizeof(half_edge), cmp_half_edge);
    if (n % 2) { free(h); return -1; }
    for (i = 0; i < n; i += 2) {
        const half_edge *a = &h[i], *b = &h[i + 1];
        if (a->lo != b->lo || a->hi != b->hi || a->cell == b->cell ||
            (i + 2 < n && h[i + 2].lo == a->lo && h[i + 2].hi == a->hi)) {
            free(h);
            return -1; /* not a closed two-manifold */
        }
        G->nbr[3 * a->cell + a->slot] = b->cell;
        G->nbr[3 * b->cell + b->slot] = a->cell;
        G->edge[3 * a->cell + a->slot] = i / 2;
        G->edge[3 * b->cell + b->slot] = i / 2;
    }
    G->n_edges = n / 2;
    free(h);
    return 0;
}

/* One bisection step.  With m_ab = normalize(v_a + v_b), child j of parent
 * (v0, v1, v2) is cell 4*parent + j:
 *   j = 0: (m01, m12, m20)   j = 1: (v0, m01, m20)
 *   j = 2: (m01, v1, m12)    j = 3: (m20, m12, v2) */
static int refine(const ogrid *P, ogrid *C)
{
    int T, i;
    if (grid_alloc(C, P->ref + 1, 4 * P->n_cells, P->n_verts + P->n_edges)) return -1;
    for (i = 0; i < P->n_verts; ++i) C->vert[i] = P->vert[i];
    for (T = 0; T < P->n_cells; ++T) {
        int v0 = P->cv[3 * T], v1 = P->cv[3 * T + 1], v2 = P->cv[3 * T + 2];
        int m01 = P->n_verts + P->edge[3 * T + 0];
        int m12 = P->n_verts + P->edge[3 * T + 1];
        int m20 = P->n_verts + P->edge[3 * T + 2];
        int *c = &C->cv[12 * T];
        C->vert[m01] = v_unit(v_add(P->vert[v0], P->vert[v1]));
        C->vert[m12] = v_unit(v_add(P->vert[v1], P->vert[v2]));
        C->vert[m20] = v_unit(v_add(P->vert[v2], P->vert[v0]));
        c[0] = m01; c[1] = m12; c[2] = m20;
        c[3] = v0;  c[4] = m01; c[5] = m20;
        c[6] = m01; c[7] = v1;  c[8] = m12;
        c[9] = m20; c[10] = m12; c[11] = v2;
    }
    return 0;
}

/* Geometry (Appendix A).  Reading C3: |T| is the spherical area and |S| the
 * great-circle arc length.  The cell centre r_T is the spherical circumcentre
 * (centre_kind 0): then r_T' - r_T is orthogonal to the shared edge, the
 * condition under which the two-point flux of Appendix A is consistent.  The
 * normalised vertex mean (centre_kind 1) is kept as an option. */
static void compute_geometry(ogrid *G, int centre_kind)
{
    int T, e;
    for (T = 0; T < G->n_cells; ++T) {
        vec3 a = G->vert[G->cv[3 * T]], b = G->vert[G->cv[3 * T + 1]], c = G->vert[G->cv[3 * T + 2]];
        /* spherical excess, Van Oosterom & Strackee: tan(E/2) = |a.(b x c)| / (1 + a.b + b.c + c.a);
         * a.(b x c) is evaluated as a.((b - a) x (c - a)), equal in exact arithmetic,
         * which keeps full relative precision for small cells. */
        double num = fabs(v_dot(a, v_cross(v_sub(b, a), v_sub(c, a))));
        double den = 1.0 + v_dot(a, b) + v_dot(b, c) + v_dot(c, a);
        G->area[T] = 2.0 * atan2(num, den);
        if (centre_kind == 0)
            G->centre[T] = v_unit(v_cross(v_sub(b, a), v_sub(c, a)));  /* equidistant from a, b, c */
        else
            G->centre[T] = v_unit(v_add(v_add(a, b), c));
    }
    /* two-point flux factor g_TT' = |S_TT'| n_TT'.(r_T' - r_T) / |r_T' - r_T|^2,
     * evaluated once per edge (from the cell with the smaller id) so that
     * g_TT' == g_T'T exactly. */
    for (T = 0; T < G->n_cells; ++T)
        for (e = 0; e < 3; ++e) {
            int Tp = G->nbr[3 * T + e], ep;
            vec3 p, q, m, n, d;
            double len, gval;
            if (Tp < T) continue;
            p = G->vert[G->cv[3 * T + e]];
            q = G->vert[G->cv[3 * T + (e + 1) % 3]];
            len = atan2(v_norm(v_cross(p, v_sub(q, p))), v_dot(p, q));   /* |p x q| = |p x (q - p)| */
            m = v_unit(v_add(p, q));                 /* edge midpoint */
            n = v_unit(v_cross(v_sub(q, p), m));     /* tangent to the sphere, normal to the edge */
            d = v_sub(G->centre[Tp], G->centre[T]);
            if (v_dot(n, d) < 0.0) n = v_scale(n, -1.0);
            gval = len * v_dot(n, d) / v_dot(d, d);
            G->g[3 * T + e] = gval;
            for (ep = 0; ep < 3; ++ep)
                if (G->nbr[3 * Tp + ep] == T) G->g[3 * Tp + ep] = gval;
        }
}

/* Colouring by saturation degree (Brelaz's DSATUR; Reading C4: multicolour
 * block-SOR, as few colours -- sequential passes -- as possible): repeatedly
 * take, among the uncoloured cells, one whose coloured neighbours show the
 * most distinct colours, the one with the smallest index among those, and
 * give it the smallest colour none of its neighbours has.  Every cell has 3
 * neighbours, so at most 4 colours are used; on the refined icosahedra 3
 * suffice.  Candidates wait in one binary min-heap of cell indices per
 * saturation value; a popped entry is skipped if its cell has been coloured or
 * has reached a higher saturation since it was pushed. */
typedef struct { int *a; int n; } iheap;

static void iheap_push(iheap *h, int v)
{
    int i = h->n++;
    h->a[i] = v;
    while (i > 0 && h->a[(i - 1) / 2] > h->a[i]) {
        int t = h->a[i]; h->a[i] = h->a[(i - 1) / 2]; h->a[(i - 1) / 2] = t;
        i = (i - 1) / 2;
    }
}

static int iheap_pop(iheap *h)
{
    int top = h->a[0], i = 0;
    h->a[0] = h->a[--h->n];
    for (;;) {
        int l = 2 * i + 1, r = l + 1, m = i, t;
        if (l < h->n && h->a[l] < h->a[m]) m = l;
        if (r < h->n && h->a[r] < h->a[m]) m = r;
        if (m == i) break;
        t = h->a[i]; h->a[i] = h->a[m]; h->a[m] = t;
        i = m;
    }
    return top;
}

static int saturation(const ogrid *G, int T)
{
    int seen[4] = {0, 0, 0, 0}, e, s = 0;
    for (e = 0; e < 3; ++e) {
        int c = G->colour[G->nbr[3 * T + e]];
        if (c >= 0 && !seen[c]) { seen[c] = 1; ++s; }
    }
    return s;
}

static int dsatur_colour(ogrid *G)
{
    int n = G->n_cells, T, e, c, s, step;
    int *sat = (int *)calloc((size_t)n, sizeof(int));
    iheap h[4];
    int ok = sat != NULL;
    for (s = 0; s < 4; ++s) {
        h[s].a = (int *)malloc((size_t)n * sizeof(int));
        h[s].n = 0;
        ok = ok && h[s].a != NULL;
    }
    if (!ok) {
        free(sat);
        for (s = 0; s < 4; ++s) free(h[s].a);
        return -1;
    }
    for (T = 0; T < n; ++T) { G->colour[T] = -1; iheap_push(&h[0], T); }
    G->n_colours = 0;
    for (step = 0; step < n; ++step) {
        int used[4] = {0, 0, 0, 0};
        T = -1;
        for (s = 3; s >= 0 && T < 0; --s)
            while (h[s].n > 0) {
                int cand = iheap_pop(&h[s]);
                if (G->colour[cand] < 0 && sat[cand] == s) { T = cand; break; }
            }
        for (e = 0; e < 3; ++e) {
            c = G->colour[G->nbr[3 * T + e]];
            if (c >= 0) used[c] = 1;
        }
        for (c = 0; c < 4 && used[c]; ++c) {}
        G->colour[T] = c;
        if (c + 1 > G->n_colours) G->n_colours = c + 1;
        for (e = 0; e < 3; ++e) {
            int U = G->nbr[3 * T + e], su;
            if (G->colour[U] >= 0) continue;
            su = saturation(G, U);
            if (su > sat[U]) { sat[U] = su; iheap_push(&h[su], U); }
        }
    }
    free(sat);
    for (s = 0; s < 4; ++s) free(h[s].a);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Oracle context                                                              */
/* ------------------------------------------------------------------------- */
/* Coarsest-level guess supplied by the caller (the learned form's network):
 * u [n_cells * n_r] = guess(f [n_cells * n_r]); the V-cycle follows it with one
 * block-Jacobi line relaxation (eq. BlockJacobi) on the coarsest level. */
typedef void (*coarse_solve_fn)(int n_cells, int n_r, const double *f, double *u);

typedef struct {
    int L, n_levels, n_r;
    double H, grading, omega2, h_min;
    coarse_solve_fn coarse_cb;   /* NULL: Algorithm 1's nu_coarse sweeps */
    int nu_pre, nu_post, nu_coarse, smoother; /* smoother: 0 multicolour block-SOR, 1 block-Jacobi */
    int centre_kind;                          /* 0 circumcentre, 1 normalised vertex mean */
    int vc_bf16;          /* V-cycle of the mixed-precision form: BF16-rounded coefficients */
    int bf16_now;         /* set while such a V-cycle runs                         */
    double relax;
    ogrid *grid;          /* [L+1] refinement levels 0..L                     */
    /* vertical grid (Appendix A), faces k = 0..n_r                           */
    double *zeta;         /* [n_r+1] height r_k - 1                           */
    double *r;            /* [n_r+1] r_k                                      */
    double *dr;           /* [n_r]   r_{k+1} - r_k                            */
    double *vol;          /* [n_r]   v_k = (r_{k+1}^3 - r_k^3)/3              */
    double *arv;          /* [n_r+1] sigma_k 2 r_k^2 / (r_{k+1} - r_{k-1})    */
    /* profiles (Sec. 2, eq. profiles) in factorised form, alpha(r, x) = alpha^r(r) alpha^S(x):
     * vertical factors of beta and alpha_S at the cell centres [n_r] and of alpha_r at the
     * faces [n_r+1]; horizontal factors per refinement level [n_cells] (the finest given,
     * coarser levels the area-weighted mean over the 4 children); NULL = 1 */
    double *pr_beta, *pr_aS, *pr_ar;
    double **ps_beta, **ps_ar, **ps_aS;
    /* vertical advection xi_r (Sec. 2, eq. HelmholtzVector; Appendix A) in factorised
     * form: vertical factor at the faces [n_r+1], horizontal per refinement level; both
     * NULL = no advection (a NULL factor next to a given one counts as 1) */
    double *pr_xi;
    double **ps_xi;
    /* general (non-factorising) profiles of the problem's operator on the finest level:
     * beta, alpha_S per unknown [n_cells][n_r], alpha_r per face [n_cells][n_r + 1];
     * NULL = the V-cycle's operator.  The outer iterations apply this operator; the
     * V-cycle keeps its (factorised) profiles: TPMG preconditioning the full operator. */
    double *pf_beta, *pf_ar, *pf_aS;
    double *pf_xi;        /* general xi_r per face [n_cells][n_r + 1], or NULL (none)   */
    /* the same general profiles on every refinement level (coarse: area-weighted means
     * over the 4 children, per vertical index) and the switch vc_full that makes the
     * V-cycle's operators use them: 0 none (TPMG^fac, the factorised profiles), 1 all
     * three (TPMG^full), 2 alpha_r only, beta and alpha_S factorised (TPMG^partial, Sec. 5.3) */
    double **pl_beta, **pl_ar, **pl_aS, **pl_xi;
    int vc_full;
    int prolong_linear;   /* 0: P = R^T, each child takes its parent's value (Reading C5);
                             1: linear interpolation with a tangent-plane gradient (Reading C25) */
    /* multigrid work arrays per multigrid level (0 = coarsest)               */
    double **mg_f, **mg_u, **mg_r;
    /* column work arrays of the line relaxation, 5 n_r doubles per thread: compiled with
     * OpenMP, the columns of one colour (and the rows of the operator and the transfers)
     * are shared out over threads; each column's arithmetic is unchanged, so the results
     * are the same bits as with one thread (the dot products stay sequential). */
    double *col_ws;
    int ws_threads;
} octx;

static int thread_id(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

static int max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* work arrays for every thread a parallel region may use (called outside any region) */
static int ensure_ws(octx *o)
{
    const int nt = max_threads();
    if (nt <= o->ws_threads) return 0;
    free(o->col_ws);
    o->col_ws = (double *)calloc((size_t)nt * 5 * o->n_r, sizeof(double));
    o->ws_threads = o->col_ws ? nt : 0;
    return o->col_ws ? 0 : -2;
}

static const ogrid *mg_grid(const octx *o, int l) { return &o->grid[o->L - (o->n_levels - 1 - l)]; }

/* Hat coefficients for unit profiles (eq. hatFunctionsNonFac).
 * beta_hat_{T,k}        = |T| v_k
 * alphaS_hat_{TT',k}    = omega^2 (r_{k+1} - r_k) g_TT'
 * alphar_hat_{T,k}      = omega^2 sigma_k |T| 2 r_k^2 / (r_{k+1} - r_{k-1})   (face k)
 * Reading C2: a single factor omega^2 in the horizontal term. */
/* x rounded to the nearest bfloat16 value (8 significant bits, the exponent
 * range of binary32), ties to the even significand.  x = m 2^e with
 * m in [0.5, 1): m 2^8 is rounded to an integer by rint (round-half-even in
 * the default rounding mode) and scaled back.  For finite normal-range x. */
double oracle_bf16(double x)
{
    int e;
    double m;
    if (x == 0.0 || !isfinite(x)) return x;
    m = frexp(x, &e);
    return ldexp(rint(ldexp(m, 8)), e - 8);
}

static double coeff(const octx *o, double v) { return o->bf16_now ? oracle_bf16(v) : v; }

/* factor of profile p: vertical array v at index k times horizontal array of the
 * refinement level of G at cell T (1 where absent) */
static double vfac(const double *v, int k) { return v ? v[k] : 1.0; }
static double hfac(const octx *o, double *const *h, const ogrid *G, int T)
{
    return h ? h[G - o->grid][T] : 1.0;
}

/* With profiles: beta_hat x beta^r_k beta^S_T, alphar_hat x alpha_r^r(face) alpha_r^S_T,
 * alphaS_hat x alpha_S^r_k (alpha_S^S_T + alpha_S^S_T') / 2 (the edge value is the mean
 * of its two cells', so the operator stays symmetric). */
static int full_now(const octx *o) { return o->vc_full == 1 && o->pl_beta; }
static int general_ar_now(const octx *o) { return o->vc_full >= 1 && o->pl_ar; }
static double beta_hat(const octx *o, const ogrid *G, int T, int k)
{
    if (full_now(o)) return coeff(o, G->area[T] * o->vol[k] * o->pl_beta[G - o->grid][(size_t)T * o->n_r + k]);
    return coeff(o, G->area[T] * o->vol[k] * vfac(o->pr_beta, k) * hfac(o, o->ps_beta, G, T));
}
static double alphaS_hat(const octx *o, const ogrid *G, int T, int e, int k)
{
    double edge = 1.0;
    if (full_now(o)) {
        const double *a = o->pl_aS[G - o->grid];
        edge = 0.5 * (a[(size_t)T * o->n_r + k] + a[(size_t)G->nbr[3 * T + e] * o->n_r + k]);
        return coeff(o, o->omega2 * o->dr[k] * G->g[3 * T + e] * edge);
    }
    if (o->ps_aS) edge = 0.5 * (hfac(o, o->ps_aS, G, T) + hfac(o, o->ps_aS, G, G->nbr[3 * T + e]));
    return coeff(o, o->omega2 * o->dr[k] * G->g[3 * T + e] * vfac(o->pr_aS, k) * edge);
}
static double alphar_hat(const octx *o, const ogrid *G, int T, int face)
{
    if (general_ar_now(o))
        return coeff(o, o->omega2 * G->area[T] * o->arv[face] * o->pl_ar[G - o->grid][(size_t)T * (o->n_r + 1) + face]);
    return coeff(o, o->omega2 * G->area[T] * o->arv[face] * vfac(o->pr_ar, face) * hfac(o, o->ps_ar, G, T));
}

/* Vertical advection of face `face` (Appendix A, the cell integral of xi_r d_r u):
 * X_{T,face} = omega^2 sigma_face |T| r_face^2 / (r_{face+1} - r_{face-1}) xi_{T,face},
 * half the alphar_hat factor; row k takes it times its own thickness r_{k+1} - r_k
 * (Reading C24).  Zero without advection. */
static int has_xi(const octx *o) { return full_now(o) ? o->pl_xi != NULL : (o->pr_xi || o->ps_xi); }
static double xi_hat(const octx *o, const ogrid *G, int T, int face)
{
    if (full_now(o)) {
        if (!o->pl_xi) return 0.0;
        return coeff(o, o->omega2 * G->area[T] * (0.5 * o->arv[face]) * o->pl_xi[G - o->grid][(size_t)T * (o->n_r + 1) + face]);
    }
    if (!o->pr_xi && !o->ps_xi) return 0.0;
    return coeff(o, o->omega2 * G->area[T] * (0.5 * o->arv[face]) * vfac(o->pr_xi, face) * hfac(o, o->ps_xi, G, T));
}

/* The vertical couplings of row (T, k): diffusion through face k (resp. k+1) minus
 * (plus) the centred advection across it,
 *   down_k = alphar_hat_{T,k} - dr_k X_{T,k},   up_k = alphar_hat_{T,k+1} + dr_k X_{T,k+1},
 * so that the row's vertical part is down_k (u_k - u_{k-1}) + up_k (u_k - u_{k+1})
 * (eq. TridiagonalNonFactorising: b = -alphar_hat - xi_hat, c = -alphar_hat + xi_hat).
 * Without advection both are the symmetric alphar_hat of the face. */
static double vert_down(const octx *o, const ogrid *G, int T, int k)
{
    const double a = alphar_hat(o, G, T, k);
    return has_xi(o) ? a - o->dr[k] * xi_hat(o, G, T, k) : a;
}
static double vert_up(const octx *o, const ogrid *G, int T, int k)
{
    const double a = alphar_hat(o, G, T, k + 1);
    return has_xi(o) ? a + o->dr[k] * xi_hat(o, G, T, k + 1) : a;
}

/* Column T of the operator as a tridiagonal matrix (eq. ColumnEquation,
 * TridiagonalSystem; Reading C2): off-diagonals -alphar_hat_{T,k} (face k couples
 * levels k-1 and k), d_{TT',k} = -alphaS_hat_{TT',k}, and diagonal a_{T,k} =
 * beta_hat_{T,k} minus the sum of all off-diagonals of the row.  Exported for
 * the tests; the solver itself works with the flux form below. */
static void column_matrix(const octx *o, const ogrid *G, int T, double *sub, double *diag, double *sup)
{
    int k, e, n = o->n_r;
    for (k = 0; k < n; ++k) {
        double lo = vert_down(o, G, T, k), up = vert_up(o, G, T, k), hs = 0.0;
        for (e = 0; e < 3; ++e) hs += alphaS_hat(o, G, T, e, k);
        sub[k] = -lo;
        sup[k] = -up;
        diag[k] = beta_hat(o, G, T, k) + lo + up + hs;
    }
}

/* (A u)_{T,k} in the flux form in which Appendix A derives it: the mass term
 * plus the vertical fluxes through faces k and k+1 (eq. VerticalDiffusion) and
 * the horizontal two-point fluxes through the edges of T, each a coupling times
 * a difference of neighbouring values:
 *   beta_hat u_{T,k} + alphar_hat_{T,k} (u_{T,k} - u_{T,k-1})
 *     + alphar_hat_{T,k+1} (u_{T,k} - u_{T,k+1}) + sum_T' alphaS_hat_{TT',k} (u_{T,k} - u_{T',k}).
 * Reading C2 fixes the signs (a conservative flux difference).  Summing the
 * tridiagonal entries first would round the large diagonal and perturb the
 * nearly singular vertically constant mode of the column by eps * cond. */
static double apply_row(const octx *o, const ogrid *G, const double *u, int T, int k)
{
    int n = o->n_r, e;
    size_t i = (size_t)T * n + k;
    double s = beta_hat(o, G, T, k) * u[i];
    if (k > 0) s += vert_down(o, G, T, k) * (u[i] - u[i - 1]);
    if (k < n - 1) s += vert_up(o, G, T, k) * (u[i] - u[i + 1]);
    for (e = 0; e < 3; ++e) s += alphaS_hat(o, G, T, e, k) * (u[i] - u[(size_t)G->nbr[3 * T + e] * n + k]);
    return s;
}

static void apply_level(octx *o, int l, const double *u, double *y)
{
    const ogrid *G = mg_grid(o, l);
    int n = o->n_r, T, k;
#pragma omp parallel for private(k) schedule(static)
    for (T = 0; T < G->n_cells; ++T)
        for (k = 0; k < n; ++k) y[(size_t)T * n + k] = apply_row(o, G, u, T, k);
}

/* Row (T, k) of the problem's operator with the general profiles: the flux form of
 * apply_row with beta_hat = |T| v_k beta_{T,k}, alphar_hat = omega^2 |T| (face
 * factor) alpha_r at the face, alphaS_hat = omega^2 dr_k g_TT' (alpha_S_{T,k} +
 * alpha_S_{T',k}) / 2. */
static double apply_row_full(const octx *o, const ogrid *G, const double *u, int T, int k)
{
    int n = o->n_r, e;
    size_t i = (size_t)T * n + k, fa = (size_t)T * (n + 1) + k;
    double s = G->area[T] * o->vol[k] * o->pf_beta[i] * u[i];
    double down = o->omega2 * G->area[T] * o->arv[k] * o->pf_ar[fa];
    double up = o->omega2 * G->area[T] * o->arv[k + 1] * o->pf_ar[fa + 1];
    if (o->pf_xi) {   /* centred vertical advection, as in vert_down / vert_up */
        down -= o->dr[k] * (o->omega2 * G->area[T] * (0.5 * o->arv[k]) * o->pf_xi[fa]);
        up += o->dr[k] * (o->omega2 * G->area[T] * (0.5 * o->arv[k + 1]) * o->pf_xi[fa + 1]);
    }
    if (k > 0) s += down * (u[i] - u[i - 1]);
    if (k < n - 1) s += up * (u[i] - u[i + 1]);
    for (e = 0; e < 3; ++e) {
        const int Tn = G->nbr[3 * T + e];
        const double edge = 0.5 * (o->pf_aS[i] + o->pf_aS[(size_t)Tn * n + k]);
        s += o->omega2 * o->dr[k] * G->g[3 * T + e] * edge * (u[i] - u[(size_t)Tn * n + k]);
    }
    return s;
}

/* y = A u with the problem's operator (the general profiles where set) on the finest level */
static void apply_outer(octx *o, const double *u, double *y)
{
    const int lf = o->n_levels - 1;
    const ogrid *G = mg_grid(o, lf);
    int n = o->n_r, T, k;
    if (!o->pf_beta) {
        apply_level(o, lf, u, y);
        return;
    }
#pragma omp parallel for private(k) schedule(static)
    for (T = 0; T < G->n_cells; ++T)
        for (k = 0; k < n; ++k) y[(size_t)T * n + k] = apply_row_full(o, G, u, T, k);
}

/* Textbook Thomas algorithm for a general tridiag(a, b, c) x = d, no pivoting:
 * forward elimination then back substitution.  a[0] and c[n-1] are not used.
 * (Exported for the tests; the smoother uses oracle_column_solve.) */
int oracle_thomas(int n, const double *a, const double *b, const double *c, const double *d, double *x)
{
    double *cp, *dp;
    int i;
    if (n < 1) return -1;
    cp = (double *)malloc((size_t)n * sizeof(double));
    dp = (double *)malloc((size_t)n * sizeof(double));
    if (!cp || !dp) { free(cp); free(dp); return -2; }
    cp[0] = (n > 1) ? c[0] / b[0] : 0.0;
    dp[0] = d[0] / b[0];
    for (i = 1; i < n; ++i) {
        double den = b[i] - a[i] * cp[i - 1];
        cp[i] = (i < n - 1) ? c[i] / den : 0.0;
        dp[i] = (d[i] - a[i] * dp[i - 1]) / den;
    }
    x[n - 1] = dp[n - 1];
    for (i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
    free(cp);
    free(dp);
    return 0;
}

/* Thomas algorithm for the column block A_T, given -- as it arises in the flux
 * form -- by its vertical couplings c_k >= 0 between levels k-1 and k
 * (k = 1..n-1; A_T has -c_k off the diagonal) and the excess m_k > 0 of each
 * diagonal entry over the couplings of its row (diagonal = m_k + c_k + c_{k+1},
 * here m_k = beta_hat + sum_T' alphaS_hat).  Forward elimination and back
 * substitution as in the textbook algorithm; the pivots are carried through
 * their excess e_k = pivot_k - c_{k+1}, which obeys
 *     e_0 = m_0,   e_k = m_k + c_k e_{k-1} / pivot_{k-1},
 * a sum of non-negative terms.  (Eliminating row k-1 from row k subtracts
 * c_k^2 / pivot_{k-1} = c_k - c_k e_{k-1} / pivot_{k-1} from the diagonal.)
 * The textbook pivot b_k - c_k^2 / pivot_{k-1} cancels catastrophically when the
 * couplings dwarf the mass term, as they do in a thin shell. */
int oracle_column_solve2(int n, const double *cd, const double *cu, const double *m, const double *d, double *x);

int oracle_column_solve(int n, const double *c, const double *m, const double *d, double *x)
{
    double *cu;
    int k, st;
    if (n < 1) return -1;
    cu = (double *)malloc((size_t)n * sizeof(double));
    if (!cu) return -2;
    for (k = 0; k < n; ++k) cu[k] = k < n - 1 ? c[k + 1] : 0.0;
    st = oracle_column_solve2(n, c, cu, m, d, x);
    free(cu);
    return st;
}

/* The same elimination for a column block with separate couplings of each row to the
 * row below, cd_k >= 0 (k = 1..n-1), and to the row above, cu_k >= 0 (k = 0..n-2):
 * A_T = tridiag(-cd, m + cd + cu, -cu), the non-symmetric block of vertical advection.
 * Eliminating row k-1 from row k subtracts cd_k cu_{k-1} / pivot_{k-1} =
 * cd_k - cd_k e_{k-1} / pivot_{k-1} from the diagonal, so
 *     e_0 = m_0,   e_k = m_k + cd_k e_{k-1} / pivot_{k-1},   pivot_k = e_k + cu_k. */
int oracle_column_solve2(int n, const double *cd, const double *cu, const double *m, const double *d, double *x)
{
    double *piv, *y;
    int k;
    if (n < 1) return -1;
    piv = (double *)malloc((size_t)n * sizeof(double));
    y = (double *)malloc((size_t)n * sizeof(double));
    if (!piv || !y) { free(piv); free(y); return -2; }
    {
        double e = m[0];
        piv[0] = e + (n > 1 ? cu[0] : 0.0);
        y[0] = d[0] / piv[0];
        for (k = 1; k < n; ++k) {
            e = m[k] + cd[k] * e / piv[k - 1];
            piv[k] = e + (k < n - 1 ? cu[k] : 0.0);
            y[k] = (d[k] + cd[k] * y[k - 1]) / piv[k];
        }
    }
    x[n - 1] = y[n - 1];
    for (k = n - 2; k >= 0; --k) x[k] = y[k] + cu[k] / piv[k] * x[k + 1];
    free(piv);
    free(y);
    return 0;
}

/* Block relaxation of column T (eq. BlockJacobi):
 *   u_T <- u_T + rho * A_T^{-1} (f_T - (A u)_T),
 * A_T the tridiagonal diagonal block of the column. */
static void relax_column(octx *o, int l, int T, const double *f, const double *u_in, double *u_out)
{
    const ogrid *G = mg_grid(o, l);
    int n = o->n_r, k, e;
    double *a = o->col_ws + (size_t)thread_id() * 5 * n, *c = a + n, *b = c + n, *d = b + n, *x = d + n;
    for (k = 0; k < n; ++k) {
        double hs = 0.0;
        for (e = 0; e < 3; ++e) hs += alphaS_hat(o, G, T, e, k);
        a[k] = vert_down(o, G, T, k);            /* coupling to level k-1 */
        c[k] = vert_up(o, G, T, k);              /* coupling to level k+1 */
        b[k] = beta_hat(o, G, T, k) + hs;        /* excess of the diagonal */
        d[k] = f[(size_t)T * n + k] - apply_row(o, G, u_in, T, k);
    }
    oracle_column_solve2(n, a, c, b, d, x);
    for (k = 0; k < n; ++k) u_out[(size_t)T * n + k] = u_in[(size_t)T * n + k] + o->relax * x[k];
}

/* Multicolour block-SOR: columns of one colour do not touch each other, so a
 * sequential in-place sweep over the cells of colour c (index order) is the
 * colour pass.  Reading C4: colour order 0..C-1 (forward) or C-1..0. */
static void colour_pass(octx *o, int l, int c, const double *f, double *u)
{
    const ogrid *G = mg_grid(o, l);
    int T;
    if (ensure_ws(o)) return;
#pragma omp parallel for schedule(static)
    for (T = 0; T < G->n_cells; ++T)
        if (G->colour[T] == c) relax_column(o, l, T, f, u, u);
}

static void jacobi_sweep(octx *o, int l, const double *f, double *u)
{
    const ogrid *G = mg_grid(o, l);
    size_t N = (size_t)G->n_cells * o->n_r;
    double *old = (double *)malloc(N * sizeof(double));
    int T;
    memcpy(old, u, N * sizeof(double));
    if (ensure_ws(o)) { free(old); return; }
#pragma omp parallel for schedule(static)
    for (T = 0; T < G->n_cells; ++T) relax_column(o, l, T, f, old, u);
    free(old);
}

/* dir = +1 forward colours, -1 reverse colours, 0 symmetric (forward then the
 * reverse order without repeating the last colour). */
static void smooth(octx *o, int l, const double *f, double *u, int sweeps, int dir)
{
    const ogrid *G = mg_grid(o, l);
    int s, c;
    for (s = 0; s < sweeps; ++s) {
        if (o->smoother == 1) { jacobi_sweep(o, l, f, u); continue; }
        if (dir >= 0)
            for (c = 0; c < G->n_colours; ++c) colour_pass(o, l, c, f, u);
        if (dir < 0)
            for (c = G->n_colours - 1; c >= 0; --c) colour_pass(o, l, c, f, u);
        if (dir == 0)
            for (c = G->n_colours - 2; c >= 0; --c) colour_pass(o, l, c, f, u);
    }
}

/* Restriction (Sec. 5: sum of the four fine cells of a coarse cell) and the
 * prolongation P = R^T (Reading C5: piecewise-constant injection). */
static void restrict_sum(const octx *o, int l_fine, const double *rf, double *fc)
{
    const ogrid *Gc = mg_grid(o, l_fine - 1);
    int n = o->n_r, T, j, k;
#pragma omp parallel for private(j, k) schedule(static)
    for (T = 0; T < Gc->n_cells; ++T)
        for (k = 0; k < n; ++k) {
            double s = 0.0;
            for (j = 0; j < 4; ++j) s += rf[(size_t)(4 * T + j) * n + k];
            fc[(size_t)T * n + k] = s;
        }
}

/* Linear interpolation from the coarse cell T to its children (Sec. 5 prolongates
 * "by linear interpolation"; Reading C25): the coarse field is taken as linear in the
 * plane tangent to the sphere at the centre c_T, with the gradient g that fits the
 * differences to the 3 coarse neighbours in least squares,
 *     min_g sum_e (u_e - u_T - g . d_e)^2,   d_e = (c_e - c_T) projected onto the plane,
 * and child t takes u_T + g . d_t, d_t = (c_t - c_T) projected.  In a basis (t1, t2) of
 * the plane, with the rows x_e = (d_e . t1, d_e . t2), the normal equations are
 * (sum_e x_e x_e^T) g = sum_e x_e (u_e - u_T); child t's weight on u_e - u_T is therefore
 * w_te = x_t^T (sum x x^T)^{-1} x_e. */
static void linear_weights(const octx *o, int l_fine, int T, double w[4][3])
{
    const ogrid *Gf = mg_grid(o, l_fine), *Gc = mg_grid(o, l_fine - 1);
    const vec3 c = Gc->centre[T], nrm = v_unit(c);
    double x[3][2], m00 = 0.0, m01 = 0.0, m11 = 0.0, det;
    vec3 d[3], t1, t2;
    int e, j;
    for (e = 0; e < 3; ++e) {
        vec3 v = v_sub(Gc->centre[Gc->nbr[3 * T + e]], c);
        d[e] = v_sub(v, v_scale(nrm, v_dot(v, nrm)));
    }
    t1 = v_unit(d[0]);
    t2 = v_cross(nrm, t1);
    for (e = 0; e < 3; ++e) {
        x[e][0] = v_dot(d[e], t1);
        x[e][1] = v_dot(d[e], t2);
        m00 += x[e][0] * x[e][0];
        m01 += x[e][0] * x[e][1];
        m11 += x[e][1] * x[e][1];
    }
    det = m00 * m11 - m01 * m01;
    for (j = 0; j < 4; ++j) {
        vec3 v = v_sub(Gf->centre[4 * T + j], c);
        const vec3 dt = v_sub(v, v_scale(nrm, v_dot(v, nrm)));
        const double px = v_dot(dt, t1), py = v_dot(dt, t2);
        /* (px, py) M^{-1}, M^{-1} = [[m11, -m01], [-m01, m00]] / det */
        const double qx = (px * m11 - py * m01) / det, qy = (py * m00 - px * m01) / det;
        for (e = 0; e < 3; ++e) w[j][e] = qx * x[e][0] + qy * x[e][1];
    }
}

static void prolong_add(const octx *o, int l_fine, const double *uc, double *uf)
{
    const ogrid *Gc = mg_grid(o, l_fine - 1);
    int n = o->n_r, T, j, k, e;
#pragma omp parallel for private(j, k, e) schedule(static)
    for (T = 0; T < Gc->n_cells; ++T) {
        double w[4][3];
        if (o->prolong_linear) linear_weights(o, l_fine, T, w);
        for (j = 0; j < 4; ++j)
            for (k = 0; k < n; ++k) {
                const double uT = uc[(size_t)T * n + k];
                double s = uT;
                if (o->prolong_linear)
                    for (e = 0; e < 3; ++e) s += w[j][e] * (uc[(size_t)Gc->nbr[3 * T + e] * n + k] - uT);
                uf[(size_t)(4 * T + j) * n + k] += s;
            }
    }
}

/* Threads of the parallel loops (the build with OpenMP; 1 otherwise): sets n when
 * n > 0, returns the number in use. */
int oracle_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
    return max_threads();
}

/* on != 0: linear prolongation (Reading C25); 0: P = R^T (Reading C5) */
void oracle_set_prolongation(void *h, int linear) { ((octx *)h)->prolong_linear = linear != 0; }

/* Algorithm 1 on multigrid level l with RHS f and initial guess u (in/out).
 * Coarsest level: nu_coarse smoother sweeps (symmetric for block-SOR). */
static void vcycle_level(octx *o, int l, const double *f, double *u)
{
    const ogrid *G = mg_grid(o, l);
    size_t N = (size_t)G->n_cells * o->n_r, i;
    if (l == 0) {
        if (o->coarse_cb) {
            o->coarse_cb(G->n_cells, o->n_r, f, u);
            jacobi_sweep(o, l, f, u);
        } else {
            smooth(o, l, f, u, o->nu_coarse, 0);
        }
        return;
    }
    smooth(o, l, f, u, o->nu_pre, +1);                       /* pre-smoothing    */
    apply_level(o, l, u, o->mg_r[l]);                        /* residual         */
#pragma omp parallel for schedule(static)
    for (i = 0; i < N; ++i) o->mg_r[l][i] = f[i] - o->mg_r[l][i];
    restrict_sum(o, l, o->mg_r[l], o->mg_f[l - 1]);          /* f_{l-1} = R r_l  */
    memset(o->mg_u[l - 1], 0, (size_t)mg_grid(o, l - 1)->n_cells * o->n_r * sizeof(double));
    vcycle_level(o, l - 1, o->mg_f[l - 1], o->mg_u[l - 1]);  /* recursion        */
    prolong_add(o, l, o->mg_u[l - 1], u);                    /* correction       */
    smooth(o, l, f, u, o->nu_post, -1);                      /* post-smoothing   */
}

/* ------------------------------------------------------------------------- */
/* Exported API (ctypes)                                                       */
/* ------------------------------------------------------------------------- */
static void free_level_profile(const octx *o, double **p)
{
    int l;
    if (!p) return;
    for (l = 0; l <= o->L; ++l) free(p[l]);
    free(p);
}

/* per refinement level: the finest copied from fine, each coarser cell the
 * area-weighted mean of its 4 children */
static double **level_profile(const octx *o, const double *fine)
{
    int l, T, j;
    double **p;
    if (!fine) return NULL;
    p = (double **)calloc((size_t)o->L + 1, sizeof(double *));
    if (!p) return NULL;
    for (l = 0; l <= o->L; ++l) p[l] = (double *)calloc((size_t)o->grid[l].n_cells, sizeof(double));
    memcpy(p[o->L], fine, (size_t)o->grid[o->L].n_cells * sizeof(double));
    for (l = o->L - 1; l >= 0; --l)
        for (T = 0; T < o->grid[l].n_cells; ++T) {
            double s = 0.0, a = 0.0;
            for (j = 0; j < 4; ++j) {
                const double aj = o->grid[l + 1].area[4 * T + j];
                s += aj * p[l + 1][4 * T + j];
                a += aj;
            }
            p[l][T] = s / a;
        }
    return p;
}

static double *copy_vec(const double *v, int n)
{
    double *c;
    if (!v) return NULL;
    c = (double *)malloc((size_t)n * sizeof(double));
    if (c) memcpy(c, v, (size_t)n * sizeof(double));
    return c;
}

/* General profiles of the problem's operator on the finest level (NULL clears all
 * three; all three must be given otherwise): beta, alpha_S [n_cells][n_r], alpha_r
 * [n_cells][n_r + 1] (faces). */
/* per refinement level, m values per cell: the finest copied, each coarser (cell, j)
 * the area-weighted mean over the 4 children's (cell, j) */
static double **level_profile_cols(const octx *o, const double *fine, int m)
{
    int l, T, c, j;
    double **p = (double **)calloc((size_t)o->L + 1, sizeof(double *));
    if (!p) return NULL;
    for (l = 0; l <= o->L; ++l) p[l] = (double *)calloc((size_t)o->grid[l].n_cells * m, sizeof(double));
    memcpy(p[o->L], fine, (size_t)o->grid[o->L].n_cells * m * sizeof(double));
    for (l = o->L - 1; l >= 0; --l)
        for (T = 0; T < o->grid[l].n_cells; ++T)
            for (j = 0; j < m; ++j) {
                double s = 0.0, a = 0.0;
                for (c = 0; c < 4; ++c) {
                    const double ac = o->grid[l + 1].area[4 * T + c];
                    s += ac * p[l + 1][(size_t)(4 * T + c) * m + j];
                    a += ac;
                }
                p[l][(size_t)T * m + j] = s / a;
            }
    return p;
}

/* xi [n_cells][n_r + 1] (faces), or NULL: the problem's vertical advection, with the
 * general profiles only. */
void oracle_set_outer_profiles(void *h, const double *beta, const double *ar, const double *aS, const double *xi)
{
    octx *o = (octx *)h;
    const size_t n = (size_t)mg_grid(o, o->n_levels - 1)->n_cells;
    free(o->pf_beta); free(o->pf_ar); free(o->pf_aS); free(o->pf_xi);
    free_level_profile(o, o->pl_beta);
    free_level_profile(o, o->pl_ar);
    free_level_profile(o, o->pl_aS);
    free_level_profile(o, o->pl_xi);
    o->pf_beta = o->pf_ar = o->pf_aS = o->pf_xi = NULL;
    o->pl_beta = o->pl_ar = o->pl_aS = o->pl_xi = NULL;
    if (!beta || !ar || !aS) return;
    o->pf_beta = copy_vec(beta, (int)(n * o->n_r));
    o->pf_ar = copy_vec(ar, (int)(n * (o->n_r + 1)));
    o->pf_aS = copy_vec(aS, (int)(n * o->n_r));
    o->pl_beta = level_profile_cols(o, beta, o->n_r);
    o->pl_ar = level_profile_cols(o, ar, o->n_r + 1);
    o->pl_aS = level_profile_cols(o, aS, o->n_r);
    if (xi) {
        o->pf_xi = copy_vec(xi, (int)(n * (o->n_r + 1)));
        o->pl_xi = level_profile_cols(o, xi, o->n_r + 1);
    }
}

/* on != 0: the V-cycle's operators use the general profiles too (TPMG^full) */
void oracle_set_vcycle_full(void *h, int on) { ((octx *)h)->vc_full = on != 0; }

/* on != 0: the V-cycle's operators take alpha_r from the general profiles and beta,
 * alpha_S from the factorised ones (partial factorisation TPMG^partial, Sec. 5.3) */
void oracle_set_vcycle_partial(void *h, int on) { ((octx *)h)->vc_full = on != 0 ? 2 : 0; }

/* y = A x with the problem's operator (oracle_apply gives the V-cycle's level operators). */
int oracle_apply_outer(void *h, const double *x, double *y)
{
    apply_outer((octx *)h, x, y);
    return 0;
}

/* Factorised profiles (NULL = 1): vertical beta^r, alpha_S^r at the n_r cell
 * centres, alpha_r^r at the n_r + 1 faces; horizontal beta^S, alpha_r^S,
 * alpha_S^S on the cells of the finest level; the advection xi_r^r (faces) and
 * xi_r^S (cells), both NULL for none. */
void oracle_set_profiles(void *h, const double *beta_r, const double *aS_r, const double *ar_r, const double *beta_s,
                         const double *ar_s, const double *aS_s, const double *xi_r, const double *xi_s)
{
    octx *o = (octx *)h;
    free(o->pr_beta); free(o->pr_aS); free(o->pr_ar); free(o->pr_xi);
    free_level_profile(o, o->ps_beta);
    free_level_profile(o, o->ps_ar);
    free_level_profile(o, o->ps_aS);
    free_level_profile(o, o->ps_xi);
    o->pr_beta = copy_vec(beta_r, o->n_r);
    o->pr_aS = copy_vec(aS_r, o->n_r);
    o->pr_ar = copy_vec(ar_r, o->n_r + 1);
    o->pr_xi = copy_vec(xi_r, o->n_r + 1);
    o->ps_beta = level_profile(o, beta_s);
    o->ps_ar = level_profile(o, ar_s);
    o->ps_aS = level_profile(o, aS_s);
    o->ps_xi = level_profile(o, xi_s);
}

void oracle_destroy(void *h)
{
    octx *o = (octx *)h;
    int l;
    if (!o) return;
    if (o->grid)
        for (l = 0; l <= o->L; ++l) grid_free(&o->grid[l]);
    free(o->grid);
    free(o->zeta); free(o->r); free(o->dr); free(o->vol); free(o->arv);
    if (o->mg_f)
        for (l = 0; l < o->n_levels; ++l) { free(o->mg_f[l]); free(o->mg_u[l]); free(o->mg_r[l]); }
    free(o->mg_f); free(o->mg_u); free(o->mg_r);
    free(o->col_ws);
    free(o->pr_beta); free(o->pr_aS); free(o->pr_ar); free(o->pr_xi);
    free_level_profile(o, o->ps_beta);
    free_level_profile(o, o->ps_ar);
    free_level_profile(o, o->ps_aS);
    free_level_profile(o, o->ps_xi);
    free(o->pf_beta); free(o->pf_ar); free(o->pf_aS); free(o->pf_xi);
    free_level_profile(o, o->pl_beta);
    free_level_profile(o, o->pl_ar);
    free_level_profile(o, o->pl_aS);
    free_level_profile(o, o->pl_xi);
    free(o);
}

/* omega2 > 0 is used as given; otherwise omega^2 = courant_c * h_min^2 with
 * h_min the smallest distance between neighbouring fine-level centres
 * (Sec. 2: the Courant number omega/h uses the smallest spacing; Reading C1). */
void *oracle_create(int refinement, int n_levels, int n_r, double H, double grading, double omega2,
                    double courant_c, int nu_pre, int nu_post, int nu_coarse, int smoother, double relax,
                    int centre_kind)
{
    octx *o;
    int l, k, T, e;
    if (refinement < 0 || refinement > 10 || n_levels < 1 || n_levels > refinement + 1 || n_r < 1 ||
        !(H > 0.0) || !(grading > 0.0) || nu_pre < 0 || nu_post < 0 || nu_coarse < 0 ||
        (smoother != 0 && smoother != 1) || (centre_kind != 0 && centre_kind != 1))
        return NULL;
    o = (octx *)calloc(1, sizeof(octx));
    if (!o) return NULL;
    o->L = refinement; o->n_levels = n_levels; o->n_r = n_r; o->H = H; o->grading = grading;
    o->nu_pre = nu_pre; o->nu_post = nu_post; o->nu_coarse = nu_coarse;
    o->smoother = smoother; o->relax = relax; o->centre_kind = centre_kind;
    o->grid = (ogrid *)calloc((size_t)refinement + 1, sizeof(ogrid));
    if (!o->grid || build_icosahedron(&o->grid[0]) || match_edges(&o->grid[0])) goto fail;
    for (l = 1; l <= refinement; ++l)
        if (refine(&o->grid[l - 1], &o->grid[l]) || match_edges(&o->grid[l])) goto fail;
    for (l = 0; l <= refinement; ++l) {
        compute_geometry(&o->grid[l], centre_kind);
        if (dsatur_colour(&o->grid[l])) goto fail;
    }
    /* smallest centre distance on the finest level */
    {
        const ogrid *G = &o->grid[refinement];
        o->h_min = HUGE_VAL;
        for (T = 0; T < G->n_cells; ++T)
            for (e = 0; e < 3; ++e) {
                double d = v_norm(v_sub(G->centre[G->nbr[3 * T + e]], G->centre[T]));
                if (d < o->h_min) o->h_min = d;
            }
    }
    o->omega2 = omega2 > 0.0 ? omega2 : courant_c * o->h_min * o->h_min;
    if (!(o->omega2 > 0.0)) goto fail;

    /* Vertical grid (Appendix A; Reading C7: geometric grading, finest at the
     * ground).  Heights zeta_k = r_k - 1 carry full relative precision. */
    o->zeta = (double *)calloc((size_t)n_r + 1, sizeof(double));
    o->r = (double *)calloc((size_t)n_r + 1, sizeof(double));
    o->dr = (double *)calloc((size_t)n_r, sizeof(double));
    o->vol = (double *)calloc((size_t)n_r, sizeof(double));
    o->arv = (double *)calloc((size_t)n_r + 1, sizeof(double));
    if (!o->zeta || !o->r || !o->dr || !o->vol || !o->arv) goto fail;
    for (k = 0; k <= n_r; ++k) {
        if (grading == 1.0) o->zeta[k] = H * (double)k / (double)n_r;
        else o->zeta[k] = H * (pow(grading, (double)k) - 1.0) / (pow(grading, (double)n_r) - 1.0);
    }
    o->zeta[0] = 0.0;
    o->zeta[n_r] = H;
    for (k = 0; k <= n_r; ++k) o->r[k] = 1.0 + o->zeta[k];
    for (k = 0; k < n_r; ++k) {
        o->dr[k] = o->zeta[k + 1] - o->zeta[k];
        /* v_k = (r_{k+1}^3 - r_k^3)/3 in factored form (Reading C8) */
        o->vol[k] = o->dr[k] * (o->r[k + 1] * o->r[k + 1] + o->r[k + 1] * o->r[k] + o->r[k] * o->r[k]) / 3.0;
    }
    /* Neumann: sigma_0 = sigma_{n_r} = 0 (eq. VerticalDiffusion) */
    for (k = 0; k <= n_r; ++k)
        o->arv[k] = (k == 0 || k == n_r) ? 0.0 : 2.0 * o->r[k] * o->r[k] / (o->zeta[k + 1] - o->zeta[k - 1]);

    o->mg_f = (double **)calloc((size_t)n_levels, sizeof(double *));
    o->mg_u = (double **)calloc((size_t)n_levels, sizeof(double *));
    o->mg_r = (double **)calloc((size_t)n_levels, sizeof(double *));
    if (!o->mg_f || !o->mg_u || !o->mg_r) goto fail;
    for (l = 0; l < n_levels; ++l) {
        size_t N = (size_t)mg_grid(o, l)->n_cells * n_r;
        o->mg_f[l] = (double *)calloc(N, sizeof(double));
        o->mg_u[l] = (double *)calloc(N, sizeof(double));
        o->mg_r[l] = (double *)calloc(N, sizeof(double));
        if (!o->mg_f[l] || !o->mg_u[l] || !o->mg_r[l]) goto fail;
    }
    if (ensure_ws(o)) goto fail;
    return o;
fail:
    oracle_destroy(o);
    return NULL;
}

/* scalars: [omega2, h_min, H, grading]; ints: [L, n_levels, n_r] */
void oracle_info(const void *h, double *scalars, int *ints)
{
    const octx *o = (const octx *)h;
    scalars[0] = o->omega2; scalars[1] = o->h_min; scalars[2] = o->H; scalars[3] = o->grading;
    ints[0] = o->L; ints[1] = o->n_levels; ints[2] = o->n_r;
}

/* Per refinement level: n_cells, n_verts, n_edges, n_colours. */
int oracle_grid_sizes(const void *h, int ref, int *out4)
{
    const octx *o = (const octx *)h;
    if (ref < 0 || ref > o->L) return -1;
    out4[0] = o->grid[ref].n_cells; out4[1] = o->grid[ref].n_verts;
    out4[2] = o->grid[ref].n_edges; out4[3] = o->grid[ref].n_colours;
    return 0;
}

/* Any output pointer may be NULL.  centre [n][3], area [n], nbr [n][3],
 * g [n][3], colour [n], corners [n][3][3] (vertex positions of each cell). */
int oracle_export_grid(const void *h, int ref, double *centre, double *area, int *nbr, double *g, int *colour,
                       double *corners)
{
    const octx *o = (const octx *)h;
    const ogrid *G;
    int T, e;
    if (ref < 0 || ref > o->L) return -1;
    G = &o->grid[ref];
    for (T = 0; T < G->n_cells; ++T) {
        if (centre) { centre[3 * T] = G->centre[T].x; centre[3 * T + 1] = G->centre[T].y; centre[3 * T + 2] = G->centre[T].z; }
        if (area) area[T] = G->area[T];
        if (colour) colour[T] = G->colour[T];
        for (e = 0; e < 3; ++e) {
            if (nbr) nbr[3 * T + e] = G->nbr[3 * T + e];
            if (g) g[3 * T + e] = G->g[3 * T + e];
            if (corners) {
                vec3 v = G->vert[G->cv[3 * T + e]];
                corners[9 * T + 3 * e] = v.x; corners[9 * T + 3 * e + 1] = v.y; corners[9 * T + 3 * e + 2] = v.z;
            }
        }
    }
    return 0;
}

/* r_faces [n_r+1], dr [n_r], vol [n_r]; any may be NULL. */
void oracle_export_vertical(const void *h, double *r_faces, double *dr, double *vol)
{
    const octx *o = (const octx *)h;
    int k;
    for (k = 0; k <= o->n_r; ++k) if (r_faces) r_faces[k] = o->r[k];
    for (k = 0; k < o->n_r; ++k) { if (dr) dr[k] = o->dr[k]; if (vol) vol[k] = o->vol[k]; }
}

/* Multigrid level l (0 = coarsest) -> number of cells, or -1. */
int oracle_level_cells(const void *h, int l)
{
    const octx *o = (const octx *)h;
    if (l < 0 || l >= o->n_levels) return -1;
    return mg_grid(o, l)->n_cells;
}

int oracle_apply(void *h, int l, const double *x, double *y)
{
    octx *o = (octx *)h;
    if (l < 0 || l >= o->n_levels) return -1;
    apply_level(o, l, x, y);
    return 0;
}

/* Diagonal blocks of the column equation on level l: sub, diag, sup [n_cells][n_r]. */
int oracle_column_blocks(void *h, int l, double *sub, double *diag, double *sup)
{
    octx *o = (octx *)h;
    const ogrid *G;
    int T;
    if (l < 0 || l >= o->n_levels) return -1;
    G = mg_grid(o, l);
    for (T = 0; T < G->n_cells; ++T)
        column_matrix(o, G, T, sub + (size_t)T * o->n_r, diag + (size_t)T * o->n_r, sup + (size_t)T * o->n_r);
    return 0;
}

/* Column data of the flux form on level l, [n_cells][n_r]: coupling c to the
 * level below (face k; c[.][0] = 0) and diagonal excess m = beta_hat + sum alphaS_hat. */
int oracle_column_couplings(void *h, int l, double *c, double *m)
{
    octx *o = (octx *)h;
    const ogrid *G;
    int T, k, e, n;
    if (l < 0 || l >= o->n_levels) return -1;
    G = mg_grid(o, l);
    n = o->n_r;
    for (T = 0; T < G->n_cells; ++T)
        for (k = 0; k < n; ++k) {
            double hs = 0.0;
            for (e = 0; e < 3; ++e) hs += alphaS_hat(o, G, T, e, k);
            c[(size_t)T * n + k] = alphar_hat(o, G, T, k);
            m[(size_t)T * n + k] = beta_hat(o, G, T, k) + hs;
        }
    return 0;
}

/* With vertical advection: each row's coupling to the row below (cd) and above (cu),
 * [n_cells][n_r], and the excess m. */
int oracle_column_couplings2(void *h, int l, double *cd, double *cu, double *m)
{
    octx *o = (octx *)h;
    const ogrid *G;
    int T, k, e, n;
    if (l < 0 || l >= o->n_levels) return -1;
    G = mg_grid(o, l);
    n = o->n_r;
    for (T = 0; T < G->n_cells; ++T)
        for (k = 0; k < n; ++k) {
            double hs = 0.0;
            for (e = 0; e < 3; ++e) hs += alphaS_hat(o, G, T, e, k);
            cd[(size_t)T * n + k] = k > 0 ? vert_down(o, G, T, k) : 0.0;
            cu[(size_t)T * n + k] = k < n - 1 ? vert_up(o, G, T, k) : 0.0;
            m[(size_t)T * n + k] = beta_hat(o, G, T, k) + hs;
        }
    return 0;
}

/* sweeps of the smoother on level l; dir = +1, -1 or 0 (symmetric). */
int oracle_smooth(void *h, int l, const double *f, double *u, int sweeps, int dir)
{
    octx *o = (octx *)h;
    if (l < 0 || l >= o->n_levels) return -1;
    smooth(o, l, f, u, sweeps, dir);
    return 0;
}

int oracle_restrict(void *h, int l_fine, const double *rf, double *fc)
{
    octx *o = (octx *)h;
    if (l_fine < 1 || l_fine >= o->n_levels) return -1;
    restrict_sum(o, l_fine, rf, fc);
    return 0;
}

int oracle_prolong_add(void *h, int l_fine, const double *uc, double *uf)
{
    octx *o = (octx *)h;
    if (l_fine < 1 || l_fine >= o->n_levels) return -1;
    prolong_add(o, l_fine, uc, uf);
    return 0;
}

/* One V-cycle on the finest level from a zero initial guess: z = B r.  With
 * vc_bf16 set, every hat coefficient the V-cycle uses (operator, column
 * blocks, coarse levels) is rounded to bfloat16 first: the preconditioner of
 * the mixed-precision form, here in FP64 arithmetic. */
int oracle_vcycle(void *h, const double *r, double *z)
{
    octx *o = (octx *)h;
    int l = o->n_levels - 1;
    memset(z, 0, (size_t)mg_grid(o, l)->n_cells * o->n_r * sizeof(double));
    o->bf16_now = o->vc_bf16;
    vcycle_level(o, l, r, z);
    o->bf16_now = 0;
    return 0;
}

/* Replace the coarsest-level solve of the V-cycle by fn followed by one
 * block-Jacobi line relaxation (NULL restores the nu_coarse sweeps): the
 * learned form, where a network predicts the coarse solution. */
void oracle_set_coarse_solve(void *h, coarse_solve_fn fn) { ((octx *)h)->coarse_cb = fn; }

/* Select the V-cycle of the mixed-precision form (on != 0) or the plain one. */
void oracle_set_vcycle_bf16(void *h, int on) { ((octx *)h)->vc_bf16 = on != 0; }

static double dot(size_t N, const double *a, const double *b)
{
    double s = 0.0;
    size_t i;
    for (i = 0; i < N; ++i) s += a[i] * b[i];
    return s;
}

/* Preconditioned conjugate gradients (the outer solver for the symmetric
 * positive definite constant-profile operator), preconditioner B = one
 * V-cycle.  u holds the initial guess on entry.  Stops when
 * ||r_k||_2 <= rtol ||r_0||_2 on the recursively updated residual (Sec. 5:
 * residual reduced by five orders of magnitude for rtol = 1e-5).
 * iters = number of operator products q = A p.  hist (nullable, max_iter+1)
 * receives ||r_k|| / ||r_0||.  true_rel (nullable) receives ||f - A u|| / ||r_0||.
 * Returns 0 converged, 1 not converged, -3 breakdown (p.Ap <= 0 or non-finite). */
int oracle_pcg(void *h, const double *f, double *u, double rtol, int max_iter, int *iters, double *rel_resid,
               double *hist, double *true_rel)
{
    octx *o = (octx *)h;
    int lf = o->n_levels - 1, it, status = 1;
    size_t N = (size_t)mg_grid(o, lf)->n_cells * o->n_r, i;
    double *r = (double *)malloc(N * sizeof(double));
    double *z = (double *)malloc(N * sizeof(double));
    double *p = (double *)malloc(N * sizeof(double));
    double *q = (double *)malloc(N * sizeof(double));
    double rz, rnorm0, rnorm;
    if (!r || !z || !p || !q) { free(r); free(z); free(p); free(q); return -2; }
    apply_outer(o, u, q);
    for (i = 0; i < N; ++i) r[i] = f[i] - q[i];
    rnorm0 = sqrt(dot(N, r, r));
    *iters = 0;
    *rel_resid = 1.0;
    if (hist) hist[0] = 1.0;
    if (!isfinite(rnorm0)) { status = -3; goto done; }
    if (rnorm0 == 0.0) { *rel_resid = 0.0; status = 0; goto done; }
    oracle_vcycle(h, r, z);
    memcpy(p, z, N * sizeof(double));
    rz = dot(N, r, z);
    for (it = 0; it < max_iter; ++it) {
        double pq, alpha, rz_new, beta;
        apply_outer(o, p, q);
        pq = dot(N, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { status = -3; break; }
        alpha = rz / pq;
        for (i = 0; i < N; ++i) { u[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        rnorm = sqrt(dot(N, r, r));
        *iters = it + 1;
        *rel_resid = rnorm / rnorm0;
        if (hist) hist[it + 1] = *rel_resid;
        if (rnorm <= rtol * rnorm0) { status = 0; break; }
        oracle_vcycle(h, r, z);
        rz_new = dot(N, r, z);
        beta = rz_new / rz;
        rz = rz_new;
        for (i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
done:
    if (true_rel) {
        apply_outer(o, u, q);
        for (i = 0; i < N; ++i) q[i] = f[i] - q[i];
        *true_rel = rnorm0 > 0.0 ? sqrt(dot(N, q, q)) / rnorm0 : 0.0;
    }
    free(r); free(z); free(p); free(q);
    return status;
}

/* Flexible conjugate gradients for a preconditioner that is not exactly
 * symmetric (the FP32 / BF16 V-cycle of the mixed-precision form): as
 * oracle_pcg, but with the Polak-Ribiere coefficient
 *     beta_k = <r_{k+1}, z_{k+1} - z_k> / <r_k, z_k>,
 * which equals the Fletcher-Reeves coefficient of plain PCG when B is
 * symmetric (then <r_{k+1}, z_k> = 0).  Same stopping rule, counts and returns. */
int oracle_fcg(void *h, const double *f, double *u, double rtol, int max_iter, int *iters, double *rel_resid,
               double *hist, double *true_rel)
{
    octx *o = (octx *)h;
    int lf = o->n_levels - 1, it, status = 1;
    size_t N = (size_t)mg_grid(o, lf)->n_cells * o->n_r, i;
    double *r = (double *)malloc(N * sizeof(double));
    double *z = (double *)malloc(N * sizeof(double));
    double *p = (double *)malloc(N * sizeof(double));
    double *q = (double *)malloc(N * sizeof(double));
    double rz, rnorm0, rnorm;
    if (!r || !z || !p || !q) { free(r); free(z); free(p); free(q); return -2; }
    apply_outer(o, u, q);
    for (i = 0; i < N; ++i) r[i] = f[i] - q[i];
    rnorm0 = sqrt(dot(N, r, r));
    *iters = 0;
    *rel_resid = 1.0;
    if (hist) hist[0] = 1.0;
    if (!isfinite(rnorm0)) { status = -3; goto done; }
    if (rnorm0 == 0.0) { *rel_resid = 0.0; status = 0; goto done; }
    oracle_vcycle(h, r, z);
    memcpy(p, z, N * sizeof(double));
    rz = dot(N, r, z);
    for (it = 0; it < max_iter; ++it) {
        double pq, alpha, rz_old_new, rz_new, beta;
        apply_outer(o, p, q);
        pq = dot(N, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { status = -3; break; }
        alpha = rz / pq;
        for (i = 0; i < N; ++i) { u[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        rnorm = sqrt(dot(N, r, r));
        *iters = it + 1;
        *rel_resid = rnorm / rnorm0;
        if (hist) hist[it + 1] = *rel_resid;
        if (rnorm <= rtol * rnorm0) { status = 0; break; }
        rz_old_new = dot(N, r, z);          /* <r_{k+1}, z_k> before z is overwritten */
        oracle_vcycle(h, r, z);
        rz_new = dot(N, r, z);
        beta = (rz_new - rz_old_new) / rz;
        rz = rz_new;
        for (i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
done:
    if (true_rel) {
        apply_outer(o, u, q);
        for (i = 0; i < N; ++i) q[i] = f[i] - q[i];
        *true_rel = rnorm0 > 0.0 ? sqrt(dot(N, q, q)) / rnorm0 : 0.0;
    }
    free(r); free(z); free(p); free(q);
    return status;
}

/* Preconditioned Richardson iteration u <- u + B (f - A u), n_iter steps
 * (Sec. 3.2.2).  hist (nullable, n_iter+1) receives ||f - A u_k||_2. */
/* BiCGStab (van der Vorst 1992) preconditioned from the right with one V-cycle
 * per preconditioner application (the paper's Sec. 5 alternative to
 * Richardson): with r^ = r_0,
 *   rho = <r^, r>,  beta = (rho / rho_prev)(alpha / omega),  p = r + beta (p - omega v),
 *   y = B p,  v = A y,  alpha = rho / <r^, v>,  s = r - alpha v,
 *   z = B s,  t = A z,  omega = <t, s> / <t, t>,
 *   u = u + alpha y + omega z,  r = s - omega t,
 * stopping when ||r_k|| <= rtol ||r_0|| (recursively updated residual).  Returns 0
 * (converged), 1 (max_iter), -3 (breakdown: rho, <r^, v> or <t, t> zero or not finite). */
int oracle_bicgstab(void *h, const double *f, double *u, double rtol, int max_iter, int *iters, double *rel_resid,
                    double *hist)
{
    octx *o = (octx *)h;
    int lf = o->n_levels - 1, it, status = 1;
    size_t N = (size_t)mg_grid(o, lf)->n_cells * o->n_r, i;
    double *r = (double *)calloc(N, sizeof(double)), *rh = (double *)calloc(N, sizeof(double));
    double *p = (double *)calloc(N, sizeof(double)), *v = (double *)calloc(N, sizeof(double));
    double *y = (double *)calloc(N, sizeof(double)), *sv = (double *)calloc(N, sizeof(double));
    double *z = (double *)calloc(N, sizeof(double)), *t = (double *)calloc(N, sizeof(double));
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0, rnorm0;
    *iters = 0;
    *rel_resid = 1.0;
    if (!r || !rh || !p || !v || !y || !sv || !z || !t) { status = -2; goto done; }
    apply_outer(o, u, t);
    for (i = 0; i < N; ++i) r[i] = f[i] - t[i];
    memcpy(rh, r, N * sizeof(double));
    rnorm0 = sqrt(dot(N, r, r));
    if (hist) hist[0] = 1.0;
    if (!isfinite(rnorm0)) { status = -3; goto done; }
    if (rnorm0 == 0.0) { *rel_resid = 0.0; status = 0; goto done; }
    for (it = 0; it < max_iter; ++it) {
        double rho = dot(N, rh, r), beta, rv, tt, rel;
        if (!(rho != 0.0) || !isfinite(rho)) { status = -3; break; }
        beta = (rho / rho_prev) * (alpha / omega);
        for (i = 0; i < N; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        oracle_vcycle(h, p, y);
        apply_outer(o, y, v);
        rv = dot(N, rh, v);
        if (!(rv != 0.0) || !isfinite(rv)) { status = -3; break; }
        alpha = rho / rv;
        for (i = 0; i < N; ++i) sv[i] = r[i] - alpha * v[i];
        oracle_vcycle(h, sv, z);
        apply_outer(o, z, t);
        tt = dot(N, t, t);
        if (!(tt > 0.0) || !isfinite(tt)) { status = -3; break; }
        omega = dot(N, t, sv) / tt;
        for (i = 0; i < N; ++i) {
            u[i] += alpha * y[i] + omega * z[i];
            r[i] = sv[i] - omega * t[i];
        }
        rho_prev = rho;
        rel = sqrt(dot(N, r, r)) / rnorm0;
        *iters = it + 1;
        *rel_resid = rel;
        if (hist) hist[it + 1] = rel;
        if (!isfinite(rel)) { status = -3; break; }
        if (rel <= rtol) { status = 0; break; }
    }
done:
    free(r); free(rh); free(p); free(v); free(y); free(sv); free(z); free(t);
    return status;
}

int oracle_richardson(void *h, const double *f, double *u, int n_iter, double *hist)
{
    octx *o = (octx *)h;
    int lf = o->n_levels - 1, it;
    size_t N = (size_t)mg_grid(o, lf)->n_cells * o->n_r, i;
    double *r = (double *)malloc(N * sizeof(double));
    double *z = (double *)malloc(N * sizeof(double));
    if (!r || !z) { free(r); free(z); return -2; }
    for (it = 0; it <= n_iter; ++it) {
        apply_outer(o, u, r);
        for (i = 0; i < N; ++i) r[i] = f[i] - r[i];
        if (hist) hist[it] = sqrt(dot(N, r, r));
        if (it == n_iter) break;
        oracle_vcycle(h, r, z);
        for (i = 0; i < N; ++i) u[i] += z[i];
    }
    free(r); free(z);
    return 0;
}
