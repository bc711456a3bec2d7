// Host construction of the icosahedral grid hierarchy, its geometry and the
// vertical grid (Dedner, Mueller & Scheichl, arXiv:1408.2981, Sec. 4.1-4.2 and
// Appendix A).  Run once in tpmg_setup; nothing here is on the solve path.
//
// Cell order (shared with every user of the library): level 0 is the regular
// icosahedron with vertices the cyclic permutations of (0, +-1, +-phi) in the
// order index = 4p + 2[s1 > 0] + [s2 > 0] (cyclic shift p of (0, s1, s2 phi)),
// faces (i, j, k) with i the smallest vertex id, counter-clockwise seen from
// outside, sorted lexicographically.  Refining cell T with corners (v0, v1, v2)
// and arc midpoints m_ab = normalize(v_a + v_b) gives cells 4T + j:
//   j = 0: (m01, m12, m20), 1: (v0, m01, m20), 2: (m01, v1, m12), 3: (m20, m12, v2).
// Neighbour slot e of a cell is the cell across its edge (corner e, corner e+1).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <functional>
#include <queue>

#include "tpmg_internal.h"

namespace tpmg {
namespace {

struct V3 {
    double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double len(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 unit(V3 a) { return (1.0 / len(a)) * a; }

inline V3 corner_of(const HostLevel &L, int T, int c)
{
    const double *p = &L.corner[9 * (size_t)T + 3 * c];
    return {p[0], p[1], p[2]};
}
inline void set_corner(HostLevel &L, int T, int c, V3 v)
{
    double *p = &L.corner[9 * (size_t)T + 3 * c];
    p[0] = v.x; p[1] = v.y; p[2] = v.z;
}

// Great-circle distance from the chord: 2 asin(|q - p| / 2), accurate for short arcs.
inline double arc(V3 p, V3 q) { return 2.0 * std::asin(0.5 * len(q - p)); }

bool build_level0(HostLevel &L, std::string &err)
{
    const double phi = 0.5 * (1.0 + std::sqrt(5.0));
    std::array<V3, 12> raw;
    for (int p = 0; p < 3; ++p)
        for (int s1 = 0; s1 < 2; ++s1)
            for (int s2 = 0; s2 < 2; ++s2) {
                const double a = 0.0, b = s1 ? 1.0 : -1.0, c = s2 ? phi : -phi;
                const double t[3] = {a, b, c};
                // cyclic shift p: component m of the vertex is t[(m - p) mod 3]
                raw[4 * p + 2 * s1 + s2] = {t[(3 - p) % 3], t[(4 - p) % 3], t[(5 - p) % 3]};
            }
    // Faces from the vertex stars: the 5 neighbours of vertex i sorted by angle
    // around i (counter-clockwise seen from outside); consecutive pairs close a face.
    std::vector<std::array<int, 3>> faces;
    for (int i = 0; i < 12; ++i) {
        const V3 n = unit(raw[i]);
        std::vector<std::pair<double, int>> star;
        V3 t1 = {0, 0, 0};
        for (int j = 0; j < 12; ++j) {
            if (j == i) continue;
            const V3 d = raw[j] - raw[i];
            if (std::fabs(dot(d, d) - 4.0) > 1e-9) continue;
            if (dot(t1, t1) == 0.0) t1 = unit(d - dot(d, n) * n);
            const V3 t2 = cross(n, t1);
            star.push_back({std::atan2(dot(d, t2), dot(d, t1)), j});
        }
        if (star.size() != 5) { err = "icosahedron: vertex star is not of size 5"; return false; }
        std::sort(star.begin(), star.end());
        for (int m = 0; m < 5; ++m) {
            const int j = star[m].second, k = star[(m + 1) % 5].second;
            if (i < j && i < k) faces.push_back({i, j, k});
        }
    }
    std::sort(faces.begin(), faces.end());
    if (faces.size() != 20) { err = "icosahedron: expected 20 faces"; return false; }
    L.ref = 0;
    L.n = 20;
    L.corner.assign(9 * 20, 0.0);
    L.nbr.assign(3 * 20, -1);
    for (int T = 0; T < 20; ++T)
        for (int c = 0; c < 3; ++c) set_corner(L, T, c, unit(raw[faces[T][c]]));
    // neighbours: the face holding the reversed edge
    for (int T = 0; T < 20; ++T)
        for (int e = 0; e < 3; ++e) {
            const int a = faces[T][e], b = faces[T][(e + 1) % 3];
            for (int U = 0; U < 20; ++U)
                for (int f = 0; f < 3; ++f)
                    if (faces[U][f] == b && faces[U][(f + 1) % 3] == a) L.nbr[3 * T + e] = U;
            if (L.nbr[3 * T + e] < 0) { err = "icosahedron: open edge"; return false; }
        }
    return true;
}

// Slot of U that points back to T.
inline int back_slot(const HostLevel &L, int U, int T)
{
    for (int f = 0; f < 3; ++f)
        if (L.nbr[3 * U + f] == T) return f;
    return -1;
}

bool refine(const HostLevel &P, HostLevel &C, std::string &err)
{
    C.ref = P.ref + 1;
    C.n = 4 * P.n;
    C.corner.assign(9 * (size_t)C.n, 0.0);
    C.nbr.assign(3 * (size_t)C.n, -1);
    for (int T = 0; T < P.n; ++T) {
        const V3 v0 = corner_of(P, T, 0), v1 = corner_of(P, T, 1), v2 = corner_of(P, T, 2);
        const V3 m01 = unit(v0 + v1), m12 = unit(v1 + v2), m20 = unit(v2 + v0);
        const int c = 4 * T;
        set_corner(C, c + 0, 0, m01); set_corner(C, c + 0, 1, m12); set_corner(C, c + 0, 2, m20);
        set_corner(C, c + 1, 0, v0);  set_corner(C, c + 1, 1, m01); set_corner(C, c + 1, 2, m20);
        set_corner(C, c + 2, 0, m01); set_corner(C, c + 2, 1, v1);  set_corner(C, c + 2, 2, m12);
        set_corner(C, c + 3, 0, m20); set_corner(C, c + 3, 1, m12); set_corner(C, c + 3, 2, v2);
        // interior edges: centre child against the corner children
        C.nbr[3 * (c + 0) + 0] = c + 2; C.nbr[3 * (c + 2) + 2] = c + 0;
        C.nbr[3 * (c + 0) + 1] = c + 3; C.nbr[3 * (c + 3) + 0] = c + 0;
        C.nbr[3 * (c + 0) + 2] = c + 1; C.nbr[3 * (c + 1) + 1] = c + 0;
        // boundary edges: parent edge e is split between the corner children at
        // corner e (child 1+e) and corner e+1 (child 1+(e+1)%3), both in slot e.
        // Across it, the neighbour N holds the same edge reversed in slot f, so its
        // corner f+1 is our corner e and its corner f is our corner e+1.
        for (int e = 0; e < 3; ++e) {
            const int N = P.nbr[3 * T + e];
            const int f = back_slot(P, N, T);
            if (f < 0) { err = "refine: neighbour relation not symmetric"; return false; }
            C.nbr[3 * (c + 1 + e) + e] = 4 * N + 1 + (f + 1) % 3;
            C.nbr[3 * (c + 1 + (e + 1) % 3) + e] = 4 * N + 1 + f;
        }
    }
    return true;
}

void geometry(HostLevel &L, int centre_kind)
{
    L.centre.assign(3 * (size_t)L.n, 0.0);
    L.area.assign(L.n, 0.0);
    L.g.assign(3 * (size_t)L.n, 0.0);
    for (int T = 0; T < L.n; ++T) {
        const V3 a = corner_of(L, T, 0), b = corner_of(L, T, 1), c = corner_of(L, T, 2);
        // L'Huilier: tan(E/4) = sqrt(tan(s/2) tan((s-A)/2) tan((s-B)/2) tan((s-C)/2))
        const double A = arc(b, c), B = arc(c, a), Cc = arc(a, b);
        const double s = 0.5 * (A + B + Cc);
        const double t = std::tan(0.5 * s) * std::tan(0.5 * (s - A)) * std::tan(0.5 * (s - B)) *
                         std::tan(0.5 * (s - Cc));
        L.area[T] = 4.0 * std::atan(std::sqrt(std::max(t, 0.0)));
        V3 cen;
        if (centre_kind == TPMG_CENTRE_CIRCUM)
            cen = unit(cross(b - a, c - a));   // normal of the corner plane = point equidistant from a, b, c
        else
            cen = unit((a + b) + c);
        L.centre[3 * (size_t)T] = cen.x; L.centre[3 * (size_t)T + 1] = cen.y; L.centre[3 * (size_t)T + 2] = cen.z;
    }
    for (int T = 0; T < L.n; ++T)
        for (int e = 0; e < 3; ++e) {
            const int U = L.nbr[3 * T + e];
            if (U < T) continue;   // once per edge, from the smaller id; copied to the other side
            const V3 p = corner_of(L, T, e), q = corner_of(L, T, (e + 1) % 3);
            const double S = arc(p, q);
            V3 n = unit(cross(p, q - p));   // normal of the great circle through p, q
            const V3 cT = {L.centre[3 * (size_t)T], L.centre[3 * (size_t)T + 1], L.centre[3 * (size_t)T + 2]};
            const V3 cU = {L.centre[3 * (size_t)U], L.centre[3 * (size_t)U + 1], L.centre[3 * (size_t)U + 2]};
            const V3 d = cU - cT;
            double nd = dot(n, d);
            if (nd < 0.0) nd = -nd;
            const double gv = S * nd / dot(d, d);
            L.g[3 * (size_t)T + e] = gv;
            L.g[3 * (size_t)U + back_slot(L, U, T)] = gv;
        }
}

// Colouring for the multicolour block-SOR: Brelaz's saturation-degree
// order (DSATUR).  The next cell coloured is, among the uncoloured ones, one
// whose coloured neighbours show the most distinct colours (the lowest cell id
// among those), and it takes the lowest colour its neighbours do not have.
// With 3 neighbours per cell at most 4 colours occur; the refined icosahedra
// need 3, i.e. 3 sequential passes per sweep.
void colour_dsatur(HostLevel &L)
{
    L.colour.assign(L.n, -1);
    L.n_colours = 0;
    std::vector<int> sat(L.n, 0);
    using MinHeap = std::priority_queue<int, std::vector<int>, std::greater<int>>;
    MinHeap cand[4];   // cell ids by saturation; stale entries are skipped
    for (int T = 0; T < L.n; ++T) cand[0].push(T);
    auto colours_around = [&](int T) {
        unsigned m = 0;
        for (int e = 0; e < 3; ++e) {
            const int c = L.colour[L.nbr[3 * T + e]];
            if (c >= 0) m |= 1u << c;
        }
        return m;
    };
    for (int done = 0; done < L.n; ++done) {
        int T = -1;
        for (int s = 3; s >= 0 && T < 0; --s)
            while (!cand[s].empty()) {
                const int v = cand[s].top();
                cand[s].pop();
                if (L.colour[v] < 0 && sat[v] == s) { T = v; break; }
            }
        const unsigned used = colours_around(T);
        int c = 0;
        while (used & (1u << c)) ++c;
        L.colour[T] = c;
        L.n_colours = std::max(L.n_colours, c + 1);
        for (int e = 0; e < 3; ++e) {
            const int U = L.nbr[3 * T + e];
            if (L.colour[U] >= 0) continue;
            const int su = __builtin_popcount(colours_around(U));
            if (su > sat[U]) {
                sat[U] = su;
                cand[su].push(U);
            }
        }
    }
}

}  // namespace

bool build_host_grid(const tpmg_params &p, HostGrid &G, std::string &err)
{
    G.lev.assign(p.refinement + 1, HostLevel());
    if (!build_level0(G.lev[0], err)) return false;
    for (int l = 1; l <= p.refinement; ++l)
        if (!refine(G.lev[l - 1], G.lev[l], err)) return false;
    const int lc = p.refinement - p.n_levels + 1;
    for (int l = 0; l <= p.refinement; ++l) {
        if (l < lc) {   // only the multigrid levels need geometry
            continue;
        }
        geometry(G.lev[l], p.centre);
        colour_dsatur(G.lev[l]);
        if (G.lev[l].n_colours > 4) { err = "colouring needed more than 4 colours"; return false; }
        for (int T = 0; T < G.lev[l].n; ++T)
            for (int e = 0; e < 3; ++e)
                if (!(G.lev[l].g[3 * (size_t)T + e] > 0.0)) { err = "non-positive flux factor"; return false; }
    }
    // smallest neighbour-centre distance on the finest level (Courant number uses the smallest spacing)
    const HostLevel &F = G.lev[p.refinement];
    double h = HUGE_VAL;
    for (int T = 0; T < F.n; ++T)
        for (int e = 0; e < 3; ++e) {
            const int U = F.nbr[3 * T + e];
            const double dx = F.centre[3 * (size_t)U] - F.centre[3 * (size_t)T];
            const double dy = F.centre[3 * (size_t)U + 1] - F.centre[3 * (size_t)T + 1];
            const double dz = F.centre[3 * (size_t)U + 2] - F.centre[3 * (size_t)T + 2];
            h = std::min(h, std::sqrt(dx * dx + dy * dy + dz * dz));
        }
    G.h_min = h;
    G.omega2 = p.omega2 > 0.0 ? p.omega2 : p.courant_c * h * h;
    if (!(G.omega2 > 0.0) || !std::isfinite(G.omega2)) { err = "omega^2 must be positive"; return false; }

    // vertical grid: heights zeta_k = H (g^k - 1)/(g^n - 1) (uniform for g = 1)
    const int n = p.n_r;
    G.zeta.assign(n + 1, 0.0);
    for (int k = 1; k < n; ++k)
        G.zeta[k] = p.grading == 1.0 ? p.H * (double)k / (double)n
                                     : p.H * (std::pow(p.grading, (double)k) - 1.0) / (std::pow(p.grading, (double)n) - 1.0);
    G.zeta[n] = p.H;
    G.r.assign(n + 1, 0.0);
    for (int k = 0; k <= n; ++k) G.r[k] = 1.0 + G.zeta[k];
    G.dr.assign(n, 0.0);
    G.vol.assign(n, 0.0);
    for (int k = 0; k < n; ++k) {
        const double d = G.zeta[k + 1] - G.zeta[k];
        if (!(d > 0.0)) { err = "vertical grid is not increasing"; return false; }
        G.dr[k] = d;
        const double r0 = G.r[k], r1 = G.r[k + 1];
        G.vol[k] = d * (r1 * r1 + r1 * r0 + r0 * r0) / 3.0;   // (r1^3 - r0^3)/3 without cancellation
    }
    G.face.assign(n + 1, 0.0);   // sigma_0 = sigma_n = 0: zero-flux top and bottom
    for (int k = 1; k < n; ++k) G.face[k] = 2.0 * G.r[k] * G.r[k] / (G.zeta[k + 1] - G.zeta[k - 1]);
    return true;
}

}  // namespace tpmg
