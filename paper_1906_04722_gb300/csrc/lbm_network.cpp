// lbm_network.cpp -- the pore network of a sphere packing and quasi-static
// drainage on it (host code).
//
//   * Pore-space decomposition (Sec. 2.2.1): the regular triangulation of the
//     sphere centres, each weighted by its squared radius, built by
//     Bowyer-Watson insertion.  Every tetrahedron is a pore body, every facet a
//     pore throat between the three spheres at its corners.  For equal radii it
//     is the Delaunay tetrahedralisation.
//   * The network of a lattice sample: each interior void lattice cell belongs
//     to the tetrahedron that contains its centre (cells outside the convex hull
//     of the centres join the nearest pore through the void, by a breadth-first
//     flood), which gives every pore its lattice volume; throats are the facets
//     shared by two tetrahedra; pores with cells next to the non-wetting
//     reservoir or next to the wetting reservoir (membrane) are linked to it.
//   * Drainage (Sec. 2.2.2, Sec. 3.1.1): the capillary pressure rises through a
//     ladder of levels; at each level the non-wetting fluid passes every throat
//     whose entry pressure p_c^e lies below the level, from a non-wetting pore
//     (or the reservoir) into a wetting pore, the lowest entry pressure first
//     (invasion percolation, the quasi-static order).  Wetting fluid that has
//     lost every path to the wetting reservoir stays where it is ("disconnected
//     regions remain saturated"): such pores are trapped and never invaded.
//     The membrane lets no non-wetting fluid into the wetting reservoir.
//   * The incircle estimate of a throat's entry pressure (Sec. 1 cites it as an
//     alternative to solving the meniscus): the circle in the plane of the three
//     centres that touches the three sphere sections, p_c^e = 2 sigma cos(theta)
//     / r_i for a meniscus of that radius.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <new>
#include <numeric>
#include <queue>
#include <string>
#include <vector>

#include "lbm_internal.h"

namespace lbmk {

namespace {

struct V3 {
    double x, y, z;
};
inline V3 sub(const V3& a, const V3& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline double dot(const V3& a, const V3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(const V3& a, const V3& b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double orient(const V3& a, const V3& b, const V3& c, const V3& d) {
    return dot(sub(b, a), cross(sub(c, a), sub(d, a)));
}

struct Tet {
    int v[4];
    int nb[4];   // neighbour across the face opposite v[i], -1 on the outer hull
    V3 oc;       // centre of the orthogonal sphere
    double or2;  // its squared radius: |p_i - oc|^2 - w_i for every corner i
    bool alive;
};

// Bowyer-Watson insertion of weighted points (w = r^2).  Finite tetrahedra are
// positively oriented and carry their orthogonal sphere (centre oc, squared
// radius or2 with |p_i - oc|^2 - w_i = or2 at every corner); a new point q
// conflicts with one when it has negative power with respect to it,
// |q - oc|^2 - w_q < or2.  The convex hull is closed by "infinite" tetrahedra
// (a, b, c, INF) on its faces, (a, b, c) ordered so that the hull's interior
// lies on the negative side: q conflicts with one when it lies beyond that face
// (or on its plane, inside the power circle of a, b, c).  The cavity of
// conflicting tetrahedra is removed and refilled by joining q to its boundary.
class Regular {
  public:
    std::vector<V3> p;
    std::vector<double> w;
    std::vector<Tet> t;
    int INF = -1;  // index of the vertex at infinity (n)
    V3 inside{0, 0, 0};
    int last = 0;
    int skipped = 0;

    bool is_inf(const Tet& T) const { return T.v[3] == INF; }

    bool ortho(Tet& T) const {
        const V3& a = p[T.v[0]];
        // 2 (p_i - p_0) . c = |p_i|^2 - |p_0|^2 - (w_i - w_0), i = 1..3 (Cramer's rule)
        double M[3][3], r[3];
        for (int i = 1; i <= 3; ++i) {
            const V3 d = sub(p[T.v[i]], a);
            M[i - 1][0] = 2 * d.x;
            M[i - 1][1] = 2 * d.y;
            M[i - 1][2] = 2 * d.z;
            r[i - 1] = dot(p[T.v[i]], p[T.v[i]]) - dot(a, a) - (w[T.v[i]] - w[T.v[0]]);
        }
        auto det3 = [](const double A[3][3]) {
            return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                   A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
        };
        const double det = det3(M);
        if (!(std::fabs(det) > 0)) return false;
        double X[3];
        for (int c = 0; c < 3; ++c) {
            double A[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) A[i][j] = (j == c) ? r[i] : M[i][j];
            X[c] = det3(A) / det;
        }
        T.oc = {X[0], X[1], X[2]};
        const V3 d = sub(a, T.oc);
        T.or2 = dot(d, d) - w[T.v[0]];
        return true;
    }
    // power of q with respect to the orthogonal circle of the face (a, b, c), in
    // its plane: negative inside
    double face_power(int a, int b, int c, int q) const {
        const V3 e1 = sub(p[b], p[a]), e2 = sub(p[c], p[a]);
        // centre = p_a + s e1 + u e2 with 2 e_i . (centre - p_a) = |e_i|^2 - (w_i - w_a)
        const double A11 = 2 * dot(e1, e1), A12 = 2 * dot(e1, e2), A22 = 2 * dot(e2, e2);
        const double b1 = dot(e1, e1) - (w[b] - w[a]), b2 = dot(e2, e2) - (w[c] - w[a]);
        const double det = A11 * A22 - A12 * A12;
        if (!(std::fabs(det) > 0)) return 0.0;
        const double sc = (b1 * A22 - A12 * b2) / det, uc = (A11 * b2 - A12 * b1) / det;
        const V3 cen{p[a].x + sc * e1.x + uc * e2.x, p[a].y + sc * e1.y + uc * e2.y, p[a].z + sc * e1.z + uc * e2.z};
        const V3 da = sub(p[a], cen), dq = sub(p[q], cen);
        return (dot(dq, dq) - w[q]) - (dot(da, da) - w[a]);
    }
    bool conflict(const Tet& T, int q) const {
        if (is_inf(T)) {
            const double o = orient(p[T.v[0]], p[T.v[1]], p[T.v[2]], p[q]);
            if (o > 0) return true;
            if (o < 0) return false;
            return face_power(T.v[0], T.v[1], T.v[2], q) < 0;
        }
        const V3 d = sub(p[q], T.oc);
        return dot(d, d) - w[q] < T.or2;
    }

    // a new tetrahedron from three vertices (one may be INF) and q; false for a
    // flat finite tetrahedron (degenerate input)
    bool make(int a, int b, int c, int q, Tet& T) {
        for (int i = 0; i < 4; ++i) T.nb[i] = -1;
        T.alive = true;
        int f[3] = {a, b, c};
        int k = -1;
        for (int i = 0; i < 3; ++i)
            if (f[i] == INF) k = i;
        if (k < 0) {
            T.v[0] = a;
            T.v[1] = b;
            T.v[2] = c;
            T.v[3] = q;
            double o = orient(p[a], p[b], p[c], p[q]);
            if (o < 0) {
                std::swap(T.v[0], T.v[1]);
                o = -o;
            }
            return o > 0 && ortho(T);
        }
        // infinite: finite face (the other two and q), interior on its negative side
        int g[3], m = 0;
        for (int i = 0; i < 3; ++i)
            if (i != k) g[m++] = f[i];
        g[2] = q;
        if (orient(p[g[0]], p[g[1]], p[g[2]], inside) > 0) std::swap(g[0], g[1]);
        T.v[0] = g[0];
        T.v[1] = g[1];
        T.v[2] = g[2];
        T.v[3] = INF;
        return true;
    }

    bool build(const double* spheres, int n) {
        INF = n;
        for (int i = 0; i < n; ++i) {
            p.push_back({spheres[4 * i], spheres[4 * i + 1], spheres[4 * i + 2]});
            w.push_back(spheres[4 * i + 3] * spheres[4 * i + 3]);
        }
        // first tetrahedron: four affinely independent centres (relative to the
        // extent of the set, so that rounding is not taken for independence)
        double ext = 0.0;
        for (int i = 1; i < n; ++i) {
            const V3 d = sub(p[i], p[0]);
            ext = std::max(ext, std::sqrt(dot(d, d)));
        }
        if (!(ext > 0)) return false;
        const double tol = 1e-9;
        int i0 = 0, i1 = -1, i2 = -1, i3 = -1;
        for (int i = 1; i < n && i1 < 0; ++i) {
            const V3 d = sub(p[i], p[i0]);
            if (std::sqrt(dot(d, d)) > tol * ext) i1 = i;
        }
        for (int i = 1; i < n && i1 >= 0 && i2 < 0; ++i) {
            if (i == i1) continue;
            const V3 c = cross(sub(p[i1], p[i0]), sub(p[i], p[i0]));
            if (std::sqrt(dot(c, c)) > tol * ext * ext) i2 = i;
        }
        for (int i = 1; i < n && i2 >= 0 && i3 < 0; ++i) {
            if (i == i1 || i == i2) continue;
            if (std::fabs(orient(p[i0], p[i1], p[i2], p[i])) > tol * ext * ext * ext) i3 = i;
        }
        if (i3 < 0) return false;
        inside = {(p[i0].x + p[i1].x + p[i2].x + p[i3].x) / 4, (p[i0].y + p[i1].y + p[i2].y + p[i3].y) / 4,
                  (p[i0].z + p[i1].z + p[i2].z + p[i3].z) / 4};
        Tet T0;
        if (!make(i0, i1, i2, i3, T0)) return false;
        t.push_back(T0);
        // its four faces, each closed by an infinite tetrahedron
        for (int f = 0; f < 4; ++f) {
            int g[3], m = 0;
            for (int j = 0; j < 4; ++j)
                if (j != f) g[m++] = t[0].v[j];
            Tet I;
            make(g[0], g[1], INF, g[2], I);
            const int id = (int)t.size();
            t.push_back(I);
            t[0].nb[f] = id;
            t[id].nb[3] = 0;
        }
        // infinite tetrahedra meet along the hull edges
        link_all(1, (int)t.size());
        for (int i = 0; i < n; ++i) {
            if (i == i0 || i == i1 || i == i2 || i == i3) continue;
            if (!insert(i)) return false;
        }
        return true;
    }

    // links the faces through a shared edge among tetrahedra [from, to) whose
    // neighbour slots are still open
    void link_all(int from, int to) {
        std::map<std::array<int, 3>, std::pair<int, int>> open;
        for (int id = from; id < to; ++id)
            for (int i = 0; i < 4; ++i) {
                if (t[id].nb[i] >= 0) continue;
                std::array<int, 3> key;
                int m = 0;
                for (int j = 0; j < 4; ++j)
                    if (j != i) key[m++] = t[id].v[j];
                std::sort(key.begin(), key.end());
                auto it = open.find(key);
                if (it == open.end()) {
                    open[key] = {id, i};
                } else {
                    t[id].nb[i] = it->second.first;
                    t[it->second.first].nb[it->second.second] = id;
                    open.erase(it);
                }
            }
    }

    int locate(int q) {
        // visibility walk over finite tetrahedra from the last new one; stepping
        // onto an infinite tetrahedron means q lies beyond the hull there
        int cur = -1;
        if (last < (int)t.size() && t[last].alive && !is_inf(t[last])) cur = last;
        if (cur < 0)
            for (int i = (int)t.size() - 1; i >= 0; --i)
                if (t[i].alive && !is_inf(t[i])) { cur = i; break; }
        for (int steps = 0; cur >= 0 && steps < 1000000; ++steps) {
            const Tet& T = t[cur];
            if (is_inf(T)) return cur;
            int next = -1;
            for (int i = 0; i < 4 && next < 0; ++i) {
                V3 c[4] = {p[T.v[0]], p[T.v[1]], p[T.v[2]], p[T.v[3]]};
                c[i] = p[q];
                if (orient(c[0], c[1], c[2], c[3]) < 0) next = T.nb[i];
            }
            if (next < 0) return cur;
            cur = next;
        }
        return -1;
    }

    bool insert(int q) {
        int start = locate(q);
        if (start < 0 || !conflict(t[start], q)) {
            start = -1;
            for (int i = 0; i < (int)t.size(); ++i)
                if (t[i].alive && conflict(t[i], q)) { start = i; break; }
        }
        if (start < 0) {  // a redundant weighted point: its power cell is empty
            ++skipped;
            return true;
        }
        std::vector<int> cav{start};
        std::vector<char> in(t.size(), 0);
        in[start] = 1;
        for (size_t h = 0; h < cav.size(); ++h) {
            const Tet& T = t[cav[h]];
            for (int i = 0; i < 4; ++i) {
                const int nb = T.nb[i];
                if (nb >= 0 && !in[nb] && conflict(t[nb], q)) {
                    in[nb] = 1;
                    cav.push_back(nb);
                }
            }
        }
        struct Face {
            int a, b, c, outside;
        };
        std::vector<Face> faces;
        for (int ti : cav)
            for (int i = 0; i < 4; ++i) {
                const int nb = t[ti].nb[i];
                if (nb >= 0 && in[nb]) continue;
                int f[3], m = 0;
                for (int j = 0; j < 4; ++j)
                    if (j != i) f[m++] = t[ti].v[j];
                faces.push_back({f[0], f[1], f[2], nb});
            }
        for (int ti : cav) t[ti].alive = false;
        const int base = (int)t.size();
        for (const Face& F : faces) {
            Tet T;
            if (!make(F.a, F.b, F.c, q, T)) return false;
            // the slot opposite q faces the old neighbour
            int qi = -1;
            for (int i = 0; i < 4; ++i)
                if (T.v[i] == q) qi = i;
            T.nb[qi] = F.outside;
            const int id = (int)t.size();
            t.push_back(T);
            if (F.outside >= 0) {
                Tet& O = t[F.outside];
                for (int i = 0; i < 4; ++i) {
                    const int ov = O.v[i];
                    if (ov != F.a && ov != F.b && ov != F.c) O.nb[i] = id;
                }
            }
        }
        link_all(base, (int)t.size());
        last = base;
        return true;
    }
};

// Inscribed circle of a throat: in the plane of the three centres, the largest
// clearance f(p) = min_i (|p - c_i| - r_i) over points p of their triangle (the
// widest circle centred in the triangle that the three sphere sections leave
// free).  Along a curve where two clearances are equal f grows away from their
// centres, so its maximum is either the point where all three are equal (the
// circle touching the three sections, |c - c_i| = r + r_i, when its centre lies
// in the triangle) or lies on an edge.  Subtracting the first tangency equation
// from the others makes c linear in r, the first is then a quadratic in r; each
// edge is sampled and the best sample refined by golden-section search.
// Returns 0 when the spheres close the throat (no positive clearance).
double incircle3(const double* s3) {
    V3 c[3];
    double r[3];
    for (int i = 0; i < 3; ++i) {
        c[i] = {s3[4 * i], s3[4 * i + 1], s3[4 * i + 2]};
        r[i] = s3[4 * i + 3];
    }
    const V3 a = sub(c[1], c[0]), b = sub(c[2], c[0]);
    const double la = std::sqrt(dot(a, a));
    if (!(la > 0)) return 0;
    const V3 e1{a.x / la, a.y / la, a.z / la};
    V3 n = cross(a, b);
    const double ln = std::sqrt(dot(n, n));
    if (!(ln > 0)) return 0;
    n = {n.x / ln, n.y / ln, n.z / ln};
    const V3 e2 = cross(n, e1);
    const double P[3][2] = {{0, 0}, {la, 0}, {dot(b, e1), dot(b, e2)}};
    auto clearance = [&](double x, double y) {
        double m = std::numeric_limits<double>::infinity();
        for (int i = 0; i < 3; ++i) m = std::min(m, std::hypot(x - P[i][0], y - P[i][1]) - r[i]);
        return m;
    };
    auto inside = [&](double x, double y) {
        auto side = [&](int i, int j) {
            return (P[j][0] - P[i][0]) * (y - P[i][1]) - (P[j][1] - P[i][1]) * (x - P[i][0]);
        };
        const double s0 = side(0, 1), s1 = side(1, 2), s2 = side(2, 0);
        return (s0 >= 0 && s1 >= 0 && s2 >= 0) || (s0 <= 0 && s1 <= 0 && s2 <= 0);
    };
    double best = -std::numeric_limits<double>::infinity();
    // 1. the circle touching the three sections: c = g + h r
    double A[2][2], u[2], v[2];
    for (int i = 1; i <= 2; ++i) {
        A[i - 1][0] = 2 * (P[i][0] - P[0][0]);
        A[i - 1][1] = 2 * (P[i][1] - P[0][1]);
        u[i - 1] = P[i][0] * P[i][0] + P[i][1] * P[i][1] - P[0][0] * P[0][0] - P[0][1] * P[0][1] -
                   (r[i] * r[i] - r[0] * r[0]);
        v[i - 1] = -2 * (r[i] - r[0]);
    }
    const double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    if (std::fabs(det) > 0) {
        const double g0 = (u[0] * A[1][1] - A[0][1] * u[1]) / det, g1 = (A[0][0] * u[1] - u[0] * A[1][0]) / det;
        const double h0 = (v[0] * A[1][1] - A[0][1] * v[1]) / det, h1 = (A[0][0] * v[1] - v[0] * A[1][0]) / det;
        // |g + h r - P0|^2 = (r + r0)^2
        const double dx = g0 - P[0][0], dy = g1 - P[0][1];
        const double qa = h0 * h0 + h1 * h1 - 1.0;
        const double qb = 2 * (dx * h0 + dy * h1) - 2 * r[0];
        const double qc = dx * dx + dy * dy - r[0] * r[0];
        double roots[2];
        int nr = 0;
        if (std::fabs(qa) < 1e-14) {
            if (std::fabs(qb) > 0) roots[nr++] = -qc / qb;
        } else {
            const double disc = qb * qb - 4 * qa * qc;
            if (disc >= 0) {
                const double sq = std::sqrt(disc);
                roots[nr++] = (-qb - sq) / (2 * qa);
                roots[nr++] = (-qb + sq) / (2 * qa);
            }
        }
        for (int k = 0; k < nr; ++k) {
            const double rr = roots[k];
            if (!std::isfinite(rr) || rr + std::max({r[0], r[1], r[2]}) < 0) continue;
            const double cx = g0 + h0 * rr, cy = g1 + h1 * rr;
            if (inside(cx, cy)) best = std::max(best, clearance(cx, cy));
        }
    }
    // 2. the edges
    for (int e = 0; e < 3; ++e) {
        const double* p0 = P[e];
        const double* p1 = P[(e + 1) % 3];
        auto at = [&](double t) { return clearance(p0[0] + t * (p1[0] - p0[0]), p0[1] + t * (p1[1] - p0[1])); };
        const int M = 512;
        int bi = 0;
        double bv = at(0.0);
        for (int i = 1; i <= M; ++i) {
            const double fv = at((double)i / M);
            if (fv > bv) { bv = fv; bi = i; }
        }
        double lo = std::max(0.0, (bi - 1.0) / M), hi = std::min(1.0, (bi + 1.0) / M);
        const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
        double x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
        double f1 = at(x1), f2 = at(x2);
        for (int it = 0; it < 80; ++it) {
            if (f1 < f2) { lo = x1; x1 = x2; f1 = f2; x2 = lo + gr * (hi - lo); f2 = at(x2); }
            else { hi = x2; x2 = x1; f2 = f1; x1 = hi - gr * (hi - lo); f1 = at(x1); }
        }
        best = std::max({best, bv, f1, f2});
    }
    return best > 0 ? best : 0.0;
}

}  // namespace

double throat_incircle(const double* s3) { return incircle3(s3); }

}  // namespace lbmk

using namespace lbmk;

extern "C" {

int lbm_regular_triangulation(const double* spheres, int n, int* tets_out, int capacity, int* n_tets) {
    if (!spheres || n < 4 || !n_tets || capacity < 0 || (capacity > 0 && !tets_out)) {
        set_error("lbm_regular_triangulation: NULL argument, fewer than 4 spheres or capacity < 0");
        return LBM_ERR_ARG;
    }
    for (int i = 0; i < 4 * n; ++i)
        if (!std::isfinite(spheres[i]) || (i % 4 == 3 && spheres[i] < 0)) {
            set_error("lbm_regular_triangulation: sphere entries must be finite with r >= 0");
            return LBM_ERR_ARG;
        }
    try {
        Regular R;
        if (!R.build(spheres, n)) {
            set_error("lbm_regular_triangulation: degenerate input (flat or coplanar configuration)");
            return LBM_ERR_ARG;
        }
        std::vector<std::array<int, 4>> out;
        for (const Tet& T : R.t) {
            if (!T.alive) continue;
            bool real = true;
            for (int i = 0; i < 4; ++i) real = real && T.v[i] != R.INF;
            if (real) out.push_back({T.v[0], T.v[1], T.v[2], T.v[3]});
        }
        *n_tets = (int)out.size();
        if (capacity < (int)out.size()) {
            if (capacity > 0) {
                set_error("lbm_regular_triangulation: capacity too small (*n_tets holds the count)");
                return LBM_ERR_ARG;
            }
            return LBM_OK;
        }
        for (size_t i = 0; i < out.size(); ++i)
            for (int j = 0; j < 4; ++j) tets_out[4 * i + j] = out[i][j];
        return LBM_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
}

int lbm_packing_throats(const double* spheres, int n, double max_edge, int* facets_out, int capacity,
                        int* n_facets) {
    if (!n_facets || capacity < 0 || (capacity > 0 && !facets_out) || !(max_edge > 0)) {
        set_error("lbm_packing_throats: NULL argument, capacity < 0 or max_edge <= 0");
        return LBM_ERR_ARG;
    }
    int nt = 0;
    int rc = lbm_regular_triangulation(spheres, n, nullptr, 0, &nt);
    if (rc) return rc;
    try {
        std::vector<int> tets((size_t)nt * 4);
        rc = lbm_regular_triangulation(spheres, n, tets.data(), nt, &nt);
        if (rc) return rc;
        // facets shared by two tetrahedra, as sorted sphere triples
        std::vector<std::array<int, 3>> all;
        all.reserve((size_t)nt * 4);
        for (int t = 0; t < nt; ++t)
            for (int f = 0; f < 4; ++f) {
                std::array<int, 3> key;
                int m = 0;
                for (int j = 0; j < 4; ++j)
                    if (j != f) key[m++] = tets[4 * (size_t)t + j];
                std::sort(key.begin(), key.end());
                all.push_back(key);
            }
        std::sort(all.begin(), all.end());
        std::vector<std::array<int, 3>> out;
        for (size_t i = 0; i + 1 < all.size(); ++i) {
            if (all[i] != all[i + 1]) continue;
            const std::array<int, 3>& k = all[i];
            double e = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = a + 1; b < 3; ++b) {
                    const double* p = spheres + 4 * (size_t)k[a];
                    const double* q = spheres + 4 * (size_t)k[b];
                    e = std::max(e, std::sqrt((p[0] - q[0]) * (p[0] - q[0]) + (p[1] - q[1]) * (p[1] - q[1]) +
                                              (p[2] - q[2]) * (p[2] - q[2])));
                }
            if (e < max_edge) out.push_back(k);
            ++i;  // a facet appears at most twice
        }
        *n_facets = (int)out.size();
        if (capacity < (int)out.size()) {
            if (capacity > 0) {
                set_error("lbm_packing_throats: capacity too small (*n_facets holds the count)");
                return LBM_ERR_ARG;
            }
            return LBM_OK;
        }
        for (size_t i = 0; i < out.size(); ++i)
            for (int j = 0; j < 3; ++j) facets_out[3 * i + j] = out[i][j];
        return LBM_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
}

int lbm_throat_incircle(const double* throats, int n, double* r_out) {
    if (!throats || !r_out || n < 0) {
        set_error("lbm_throat_incircle: NULL argument or n < 0");
        return LBM_ERR_ARG;
    }
    for (int i = 0; i < n; ++i) r_out[i] = incircle3(throats + 12 * (size_t)i);
    return LBM_OK;
}

int lbm_throat_pce_incircle(const double* throats, int n, double sigma, double cos_theta, double* pce_out) {
    if (!throats || !pce_out || n < 0 || !std::isfinite(sigma) || !std::isfinite(cos_theta)) {
        set_error("lbm_throat_pce_incircle: NULL argument, n < 0 or non-finite sigma / cos_theta");
        return LBM_ERR_ARG;
    }
    for (int i = 0; i < n; ++i) {
        const double r = incircle3(throats + 12 * (size_t)i);
        pce_out[i] = r > 0 ? 2.0 * sigma * cos_theta / r : INFINITY;  // a closed throat is never passed
    }
    return LBM_OK;
}

int lbm_pn_build(const double* spheres, int n_spheres, const int* tets, int n_tets, const unsigned char* mask,
                 const int box[3], double* pore_volume, int* n_throats, int* throat_pores, int* throat_spheres,
                 int capacity) {
    if (!spheres || !tets || n_tets < 1 || !mask || !box || !pore_volume || !n_throats || capacity < 0 ||
        (capacity > 0 && (!throat_pores || !throat_spheres))) {
        set_error("lbm_pn_build: NULL argument, no tetrahedra or capacity < 0");
        return LBM_ERR_ARG;
    }
    const int nx = box[0], ny = box[1], nz = box[2];
    if (nx < 1 || ny < 1 || nz < 1) { set_error("lbm_pn_build: bad box"); return LBM_ERR_ARG; }
    for (int i = 0; i < 4 * n_tets; ++i)
        if (tets[i] < 0 || tets[i] >= n_spheres) { set_error("lbm_pn_build: tetrahedron corner out of range"); return LBM_ERR_ARG; }
    try {
        const long long N = (long long)nx * ny * nz;
        const long long nxy = (long long)nx * ny;
        auto interior = [&](long long c) { return mask[c] == 0; };  // void, not a reservoir or membrane layer
        std::vector<int> owner((size_t)N, -1);
        // 1. cells whose centre lies in a tetrahedron (the first tetrahedron wins on shared faces)
        for (int ti = 0; ti < n_tets; ++ti) {
            V3 v[4];
            double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
            for (int j = 0; j < 4; ++j) {
                const double* s = spheres + 4 * tets[4 * ti + j];
                v[j] = {s[0], s[1], s[2]};
                for (int d = 0; d < 3; ++d) {
                    lo[d] = std::min(lo[d], s[d]);
                    hi[d] = std::max(hi[d], s[d]);
                }
            }
            const double o = orient(v[0], v[1], v[2], v[3]);
            if (!(std::fabs(o) > 0)) continue;
            const int x0 = std::max(0, (int)std::ceil(lo[0])), x1 = std::min(nx - 1, (int)std::floor(hi[0]));
            const int y0 = std::max(0, (int)std::ceil(lo[1])), y1 = std::min(ny - 1, (int)std::floor(hi[1]));
            const int z0 = std::max(0, (int)std::ceil(lo[2])), z1 = std::min(nz - 1, (int)std::floor(hi[2]));
            for (int z = z0; z <= z1; ++z)
                for (int y = y0; y <= y1; ++y)
                    for (int x = x0; x <= x1; ++x) {
                        const long long c = z * nxy + (long long)y * nx + x;
                        if (owner[(size_t)c] >= 0 || !interior(c)) continue;
                        const V3 q{(double)x, (double)y, (double)z};
                        bool in = true;
                        for (int f = 0; f < 4 && in; ++f) {
                            V3 w4[4] = {v[0], v[1], v[2], v[3]};
                            w4[f] = q;
                            const double of = orient(w4[0], w4[1], w4[2], w4[3]);
                            in = (o > 0) ? (of >= 0) : (of <= 0);
                        }
                        if (in) owner[(size_t)c] = ti;
                    }
        }
        // 2. the remaining interior void cells join the nearest owned cell through the void
        {
            std::vector<long long> frontier;
            for (long long c = 0; c < N; ++c)
                if (owner[(size_t)c] >= 0) frontier.push_back(c);
            std::vector<long long> next;
            while (!frontier.empty()) {
                next.clear();
                for (long long c : frontier) {
                    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / nxy);
                    const int d6[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
                    for (const auto& d : d6) {
                        const int X = x + d[0], Y = y + d[1], Z = z + d[2];
                        if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
                        const long long e = Z * nxy + (long long)Y * nx + X;
                        if (owner[(size_t)e] >= 0 || !interior(e)) continue;
                        owner[(size_t)e] = owner[(size_t)c];
                        next.push_back(e);
                    }
                }
                frontier.swap(next);
            }
        }
        for (int ti = 0; ti < n_tets; ++ti) pore_volume[ti] = 0.0;
        // reservoir links: a pore with a cell next to the inlet layer, or next to
        // the first layer below the interior (membrane or outlet)
        std::vector<char> to_in(n_tets, 0), to_out(n_tets, 0);
        for (long long c = 0; c < N; ++c) {
            const int o = owner[(size_t)c];
            if (o < 0) continue;
            pore_volume[o] += 1.0;
            const int z = (int)(c / nxy);
            if (z > 0 && (mask[c - nxy] & LBM_MASK_INLET)) to_in[o] = 1;
            if (z + 1 < nz && (mask[c + nxy] & (LBM_MASK_MEMBRANE | LBM_MASK_OUTLET))) to_out[o] = 1;
        }
        // throats: facets shared by two tetrahedra
        std::map<std::array<int, 3>, int> facet;
        std::vector<std::array<int, 5>> th;  // pore a, pore b, three spheres
        for (int ti = 0; ti < n_tets; ++ti)
            for (int f = 0; f < 4; ++f) {
                std::array<int, 3> key;
                int m = 0;
                for (int j = 0; j < 4; ++j)
                    if (j != f) key[m++] = tets[4 * ti + j];
                std::sort(key.begin(), key.end());
                auto it = facet.find(key);
                if (it == facet.end()) {
                    facet[key] = ti;
                } else {
                    th.push_back({it->second, ti, key[0], key[1], key[2]});
                    facet.erase(it);
                }
            }
        for (int ti = 0; ti < n_tets; ++ti) {
            if (to_in[ti]) th.push_back({ti, LBM_PN_INLET, -1, -1, -1});
            if (to_out[ti]) th.push_back({ti, LBM_PN_OUTLET, -1, -1, -1});
        }
        *n_throats = (int)th.size();
        if (capacity < (int)th.size()) {
            if (capacity > 0) {
                set_error("lbm_pn_build: capacity too small (*n_throats holds the count)");
                return LBM_ERR_ARG;
            }
            return LBM_OK;
        }
        for (size_t i = 0; i < th.size(); ++i) {
            throat_pores[2 * i] = th[i][0];
            throat_pores[2 * i + 1] = th[i][1];
            for (int j = 0; j < 3; ++j) throat_spheres[3 * i + j] = th[i][2 + j];
        }
        return LBM_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
}

int lbm_partition_lpt(const double* cost, int n, int parts, int* part_out, double* load_out) {
    if (!cost || !part_out || n < 0 || parts < 1) {
        set_error("lbm_partition_lpt: NULL argument, n < 0 or parts < 1");
        return LBM_ERR_ARG;
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(cost[i]) || cost[i] < 0) { set_error("lbm_partition_lpt: costs must be finite and >= 0"); return LBM_ERR_ARG; }
    try {
        // longest processing time first: items by decreasing cost (ties: lower
        // index), each to the part with the least load so far (ties: lower part)
        std::vector<int> order((size_t)n);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        using P = std::pair<double, int>;
        std::priority_queue<P, std::vector<P>, std::greater<P>> heap;
        for (int q = 0; q < parts; ++q) heap.push({0.0, q});
        std::vector<double> load((size_t)parts, 0.0);
        for (int i : order) {
            P top = heap.top();
            heap.pop();
            part_out[i] = top.second;
            top.first += cost[i];
            load[(size_t)top.second] = top.first;
            heap.push(top);
        }
        if (load_out)
            for (int q = 0; q < parts; ++q) load_out[q] = load[(size_t)q];
        return LBM_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
}

int lbm_pn_drainage(int n_pores, const double* pore_volume, int n_throats, const int* throat_pores,
                    const double* throat_pce, int n_levels, const double* p_c, double* S_w,
                    int* pore_invaded_at, int* pore_trapped_at) {
    if (n_pores < 1 || !pore_volume || n_throats < 0 || (n_throats > 0 && (!throat_pores || !throat_pce)) ||
        n_levels < 1 || !p_c || !S_w) {
        set_error("lbm_pn_drainage: NULL argument or empty network / ladder");
        return LBM_ERR_ARG;
    }
    for (int i = 0; i < n_throats; ++i) {
        const int a = throat_pores[2 * i], b = throat_pores[2 * i + 1];
        const bool ok_a = a >= 0 && a < n_pores, ok_b = (b >= 0 && b < n_pores) || b == LBM_PN_INLET || b == LBM_PN_OUTLET;
        if (!ok_a || !ok_b || a == b) {
            set_error("lbm_pn_drainage: throat pores out of range (pore a must be a pore, b a pore or a reservoir)");
            return LBM_ERR_ARG;
        }
        if (std::isnan(throat_pce[i])) { set_error("lbm_pn_drainage: NaN entry pressure"); return LBM_ERR_ARG; }
    }
    try {
        // adjacency: throat indices per pore
        std::vector<std::vector<int>> adj((size_t)n_pores);
        for (int i = 0; i < n_throats; ++i) {
            adj[(size_t)throat_pores[2 * i]].push_back(i);
            const int b = throat_pores[2 * i + 1];
            if (b >= 0) adj[(size_t)b].push_back(i);
        }
        enum : char { WET = 0, NONWET = 1, TRAPPED = 2 };
        std::vector<char> state((size_t)n_pores, WET);
        std::vector<int> inv((size_t)n_pores, -1), trap((size_t)n_pores, -1);
        double vtot = 0.0;
        for (int i = 0; i < n_pores; ++i) vtot += pore_volume[i];
        auto other = [&](int th, int pore) {
            const int a = throat_pores[2 * th], b = throat_pores[2 * th + 1];
            return a == pore ? b : a;
        };
        // wetting pores that still reach the wetting reservoir through wetting pores
        std::vector<char> seen((size_t)n_pores);
        auto update_trapping = [&](int level) {
            std::fill(seen.begin(), seen.end(), 0);
            std::vector<int> stack;
            for (int i = 0; i < n_throats; ++i)
                if (throat_pores[2 * i + 1] == LBM_PN_OUTLET) {
                    const int a = throat_pores[2 * i];
                    if (state[(size_t)a] == WET && !seen[(size_t)a]) { seen[(size_t)a] = 1; stack.push_back(a); }
                }
            while (!stack.empty()) {
                const int u = stack.back();
                stack.pop_back();
                for (int th : adj[(size_t)u]) {
                    const int v = other(th, u);
                    if (v < 0 || seen[(size_t)v] || state[(size_t)v] != WET) continue;
                    seen[(size_t)v] = 1;
                    stack.push_back(v);
                }
            }
            for (int i = 0; i < n_pores; ++i)
                if (state[(size_t)i] == WET && !seen[(size_t)i]) {
                    state[(size_t)i] = TRAPPED;
                    trap[(size_t)i] = level;
                }
        };
        // candidate throats (entry pressure, throat, wetting pore behind it) that the
        // non-wetting fluid touches
        using Cand = std::pair<double, std::pair<int, int>>;
        std::priority_queue<Cand, std::vector<Cand>, std::greater<Cand>> heap;
        auto push_front = [&](int pore_nw) {  // throats leaving a pore that just turned non-wetting
            for (int th : adj[(size_t)pore_nw]) {
                const int v = other(th, pore_nw);
                if (v >= 0 && state[(size_t)v] == WET) heap.push({throat_pce[th], {th, v}});
            }
        };
        for (int i = 0; i < n_throats; ++i)
            if (throat_pores[2 * i + 1] == LBM_PN_INLET) heap.push({throat_pce[i], {i, throat_pores[2 * i]}});
        update_trapping(0);  // wetting pores cut off from the start count as trapped at level 0
        for (int l = 0; l < n_levels; ++l) {
            while (!heap.empty() && heap.top().first < p_c[l]) {
                const int v = heap.top().second.second;
                heap.pop();
                if (state[(size_t)v] != WET) continue;  // invaded meanwhile, or trapped
                state[(size_t)v] = NONWET;
                inv[(size_t)v] = l;
                push_front(v);
                update_trapping(l);
            }
            double vw = 0.0;
            for (int i = 0; i < n_pores; ++i)
                if (state[(size_t)i] != NONWET) vw += pore_volume[i];
            S_w[l] = vtot > 0 ? vw / vtot : NAN;
        }
        if (pore_invaded_at)
            for (int i = 0; i < n_pores; ++i) pore_invaded_at[i] = inv[(size_t)i];
        if (pore_trapped_at)
            for (int i = 0; i < n_pores; ++i) pore_trapped_at[i] = trap[(size_t)i];
        return LBM_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
}

}  // extern "C"
