// lbm_msp.cpp -- the Mayer-Stowe-Princen (MS-P) estimate of a pore throat's
// entry capillary pressure (host code): the second approximation Sec. 1 cites
// beside the incircle, built here as a baseline for the LBM and the surrogate.
//
// The throat is taken as a prism.  Its cross-section is the triangle T of the
// three sphere centres minus the three sphere sections (circles of the sphere
// radii: the plane passes through the centres); its sides are the neutral walls
// of the lattice throat domain (contact angle 90 degrees).  At a capillary
// pressure p_c the wetting fluid holds the corners between two grains behind
// arc menisci of radius r = sigma / p_c (a prism has no curvature along its
// axis) that meet the grains at the contact angle theta and the walls at 90
// degrees.  Equivalently the non-wetting region N(r) is the part of the section
// covered by discs of radius r whose centres O lie in T at a distance of at
// least rho_i = sqrt(R_i^2 + r^2 + 2 R_i r cos(theta)) from every centre c_i (a
// disc at exactly that distance cuts grain i at the angle theta).  The MS-P
// condition is the energy balance of a small advance of the non-wetting front
// along the prism,
//     p_c A_nw = sigma (L_nw + L_ns cos(theta)),
// A_nw the area of N, L_nw the length of its menisci, L_ns the length of its
// contact with the grains (the walls add cos 90 = 0); so r solves
//     r = A_nw(r) / (L_nw(r) + L_ns(r) cos(theta))
// and p_c^e = sigma / r.
//
// N(r) is computed exactly, for any arrangement.  The allowed-centre set A is
// T minus the three discs |O - c_i| < rho_i; its boundary is found by splitting
// the three edges and the three constraint circles at their intersections and
// keeping the pieces that border A.  The boundary of N lies on the walls, on
// the grain circles and on circles of radius r about the corner points of A
// (the offsets of A's other boundary pieces fall outside T or inside the
// grains).  Each of these curves is split at its intersections with all the
// others; a piece belongs to the boundary of N when a point just to one side of
// it is in N and the point just to the other side is not (x is in N when it
// lies in T, outside the grains and within r of A).  Green's theorem over the
// oriented pieces gives A_nw; the pieces on grain circles give L_ns, those on
// the corner circles L_nw.
#include <algorithm>
#include <cmath>
#include <limits>
#include <string>

#include "lbm_host.h"
#include "lbm_internal.h"

namespace lbmk {

namespace {

constexpr double kPi = 3.14159265358979323846;

struct P2 {
    double x, y;
};

inline double wrap2pi(double a) {
    a = std::fmod(a, 2.0 * kPi);
    return a < 0 ? a + 2.0 * kPi : a;
}

// The throat's section in its own plane: centres counter-clockwise.
struct Section {
    P2 c[3];
    double R[3];
};

bool make_section(const double* s3, Section& s) {
    double c3[3][3];
    for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 3; ++k) c3[i][k] = s3[4 * i + k];
        s.R[i] = s3[4 * i + 3];
    }
    double a[3], b[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = c3[1][k] - c3[0][k];
        b[k] = c3[2][k] - c3[0][k];
    }
    const double la = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    if (!(la > 0)) return false;
    double e1[3] = {a[0] / la, a[1] / la, a[2] / la};
    double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    const double ln = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(ln > 0)) return false;
    for (double& v : n) v /= ln;
    const double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
    s.c[0] = {0, 0};
    s.c[1] = {la, 0};
    s.c[2] = {b[0] * e1[0] + b[1] * e1[1] + b[2] * e1[2], b[0] * e2[0] + b[1] * e2[1] + b[2] * e2[2]};
    return true;
}

enum CurveKind { WALL, GRAIN, MENISCUS, CONSTRAINT };

// A segment a -> b (parameter t in [0, 1]) or a circle (angle t, counter-clockwise).
struct Curve {
    bool circle;
    P2 a, b, c;
    double rad;
    CurveKind kind;
    P2 at(double t) const {
        return circle ? P2{c.x + rad * std::cos(t), c.y + rad * std::sin(t)}
                      : P2{a.x + t * (b.x - a.x), a.y + t * (b.y - a.y)};
    }
    // unit tangent in the direction of increasing t
    P2 tangent(double t) const {
        if (circle) return {-std::sin(t), std::cos(t)};
        const double l = std::hypot(b.x - a.x, b.y - a.y);
        return {(b.x - a.x) / l, (b.y - a.y) / l};
    }
};

struct Piece {
    const Curve* cv;
    double t0, t1;
};

// Parameters on p of the points where p meets q (tangencies within tol count once).
void crossings(const Curve& p, const Curve& q, double tol, std::vector<double>& ts) {
    if (!p.circle && !q.circle) return;  // edges meet only at the triangle's corners
    P2 pts[2];
    int n = 0;
    if (!p.circle || !q.circle) {
        const Curve& sg = p.circle ? q : p;
        const Curve& cc = p.circle ? p : q;
        const P2 D{sg.b.x - sg.a.x, sg.b.y - sg.a.y};
        const double L2 = D.x * D.x + D.y * D.y;
        const double tf = ((cc.c.x - sg.a.x) * D.x + (cc.c.y - sg.a.y) * D.y) / L2;  // foot of the centre
        const double h = std::fabs(D.x * (cc.c.y - sg.a.y) - D.y * (cc.c.x - sg.a.x)) / std::sqrt(L2);
        double tt[2];
        int m = 0;
        if (std::fabs(h - cc.rad) <= tol) tt[m++] = tf;
        else if (h < cc.rad) {
            const double w = std::sqrt(cc.rad * cc.rad - h * h) / std::sqrt(L2);
            tt[m++] = tf - w;
            tt[m++] = tf + w;
        }
        for (int k = 0; k < m; ++k)
            if (tt[k] > 0 && tt[k] < 1) pts[n++] = sg.at(tt[k]);
    } else {
        const double dx = q.c.x - p.c.x, dy = q.c.y - p.c.y, d = std::hypot(dx, dy);
        if (!(d > tol)) return;
        const double base = std::atan2(dy, dx);
        if (std::fabs(d - (p.rad + q.rad)) <= tol) pts[n++] = p.at(base);
        else if (std::fabs(d - std::fabs(p.rad - q.rad)) <= tol) pts[n++] = p.at(p.rad > q.rad ? base : base + kPi);
        else if (d < p.rad + q.rad && d > std::fabs(p.rad - q.rad)) {
            const double x = (d * d + p.rad * p.rad - q.rad * q.rad) / (2 * d);
            const double half = std::acos(std::min(1.0, std::max(-1.0, x / p.rad)));
            pts[n++] = p.at(base - half);
            pts[n++] = p.at(base + half);
        }
    }
    for (int k = 0; k < n; ++k) {
        if (p.circle) ts.push_back(wrap2pi(std::atan2(pts[k].y - p.c.y, pts[k].x - p.c.x)));
        else {
            const P2 D{p.b.x - p.a.x, p.b.y - p.a.y};
            ts.push_back(((pts[k].x - p.a.x) * D.x + (pts[k].y - p.a.y) * D.y) / (D.x * D.x + D.y * D.y));
        }
    }
}

// Splits every curve at its crossings with the others.
std::vector<Piece> split(const std::vector<Curve>& cv, double tol) {
    std::vector<Piece> out;
    std::vector<double> ts;
    for (size_t i = 0; i < cv.size(); ++i) {
        ts.clear();
        for (size_t j = 0; j < cv.size(); ++j)
            if (j != i) crossings(cv[i], cv[j], tol, ts);
        std::sort(ts.begin(), ts.end());
        if (!cv[i].circle) {
            double prev = 0;
            for (double t : ts) {
                if (t > prev) out.push_back({&cv[i], prev, t});
                prev = std::max(prev, t);
            }
            if (prev < 1) out.push_back({&cv[i], prev, 1.0});
        } else if (ts.empty()) {
            out.push_back({&cv[i], 0.0, 2 * kPi});
        } else {
            for (size_t k = 0; k + 1 < ts.size(); ++k)
                if (ts[k + 1] > ts[k]) out.push_back({&cv[i], ts[k], ts[k + 1]});
            out.push_back({&cv[i], ts.back(), ts.front() + 2 * kPi});
        }
    }
    return out;
}

struct Terms {
    const Section& s;
    double rho[3], r, scale;
    std::vector<Curve> acv;  // edges and constraint circles
    std::vector<Piece> abd;  // the pieces of A's boundary

    bool in_T(const P2& x) const {
        for (int i = 0; i < 3; ++i) {
            const P2 p = s.c[i], q = s.c[(i + 1) % 3];
            if ((q.x - p.x) * (x.y - p.y) - (q.y - p.y) * (x.x - p.x) < 0) return false;
        }
        return true;
    }
    bool in_A(const P2& x) const {
        if (!in_T(x)) return false;
        for (int i = 0; i < 3; ++i)
            if (std::hypot(x.x - s.c[i].x, x.y - s.c[i].y) < rho[i]) return false;
        return true;
    }
    double dist_A(const P2& x) const {
        if (in_A(x)) return 0;
        double best = std::numeric_limits<double>::infinity();
        for (const Piece& p : abd) {
            const Curve& c = *p.cv;
            if (!c.circle) {
                const P2 D{c.b.x - c.a.x, c.b.y - c.a.y};
                double t = ((x.x - c.a.x) * D.x + (x.y - c.a.y) * D.y) / (D.x * D.x + D.y * D.y);
                t = std::min(std::max(t, p.t0), p.t1);
                const P2 q = c.at(t);
                best = std::min(best, std::hypot(x.x - q.x, x.y - q.y));
            } else {
                double ang = std::atan2(x.y - c.c.y, x.x - c.c.x);
                ang = p.t0 + wrap2pi(ang - p.t0);
                if (ang <= p.t1) best = std::min(best, std::fabs(std::hypot(x.x - c.c.x, x.y - c.c.y) - c.rad));
                else {
                    const P2 q0 = c.at(p.t0), q1 = c.at(p.t1);
                    best = std::min({best, std::hypot(x.x - q0.x, x.y - q0.y), std::hypot(x.x - q1.x, x.y - q1.y)});
                }
            }
        }
        return best;
    }
    bool in_N(const P2& x) const {
        if (!in_T(x)) return false;
        for (int i = 0; i < 3; ++i)
            if (std::hypot(x.x - s.c[i].x, x.y - s.c[i].y) < s.R[i]) return false;
        return dist_A(x) <= r;
    }

    Terms(const Section& sec, double rr, const double* rh) : s(sec), r(rr) {
        for (int i = 0; i < 3; ++i) rho[i] = rh[i];
        scale = 0;
        for (int i = 0; i < 3; ++i)
            scale = std::max(scale, std::hypot(s.c[(i + 1) % 3].x - s.c[i].x, s.c[(i + 1) % 3].y - s.c[i].y));
    }

    void run(double out[3]) {
        const double tol = 1e-11 * scale, eps = 1e-8 * scale;
        // the boundary of A
        for (int i = 0; i < 3; ++i) acv.push_back({false, s.c[i], s.c[(i + 1) % 3], {0, 0}, 0, WALL});
        for (int i = 0; i < 3; ++i) acv.push_back({true, {0, 0}, {0, 0}, s.c[i], rho[i], CONSTRAINT});
        for (const Piece& p : split(acv, tol)) {
            const P2 m = p.cv->at(0.5 * (p.t0 + p.t1));
            bool keep;
            if (!p.cv->circle) {
                keep = true;
                for (int j = 0; j < 3; ++j)
                    if (std::hypot(m.x - s.c[j].x, m.y - s.c[j].y) < rho[j]) keep = false;
            } else {
                keep = in_T(m);
                const int own = (int)(p.cv - acv.data()) - 3;  // the constraint circle the piece lies on
                for (int j = 0; j < 3; ++j)
                    if (j != own && std::hypot(m.x - s.c[j].x, m.y - s.c[j].y) < rho[j]) keep = false;
            }
            if (keep) abd.push_back(p);
        }
        // corner points of A: ends of its boundary pieces, once each
        std::vector<P2> vert;
        for (const Piece& p : abd)
            for (double t : {p.t0, p.t1}) {
                const P2 q = p.cv->at(t);
                bool seen = false;
                for (const P2& v : vert)
                    if (std::hypot(v.x - q.x, v.y - q.y) <= 1e3 * tol) seen = true;
                if (!seen) vert.push_back(q);
            }
        // candidate boundary curves of N, split at all crossings, each piece kept
        // (oriented with N on its left) when N lies on exactly one side of it
        std::vector<Curve> ncv;
        for (int i = 0; i < 3; ++i) ncv.push_back({false, s.c[i], s.c[(i + 1) % 3], {0, 0}, 0, WALL});
        for (int i = 0; i < 3; ++i) ncv.push_back({true, {0, 0}, {0, 0}, s.c[i], s.R[i], GRAIN});
        for (const P2& v : vert) ncv.push_back({true, {0, 0}, {0, 0}, v, r, MENISCUS});
        double area2 = 0, l_nw = 0, l_ns = 0;
        for (const Piece& p : split(ncv, tol)) {
            const Curve& c = *p.cv;
            const double tm = 0.5 * (p.t0 + p.t1);
            const P2 m = c.at(tm), tg = c.tangent(tm), nl{-tg.y, tg.x};
            const bool left = in_N({m.x + eps * nl.x, m.y + eps * nl.y});
            const bool right = in_N({m.x - eps * nl.x, m.y - eps * nl.y});
            if (left == right) continue;
            const double a0 = left ? p.t0 : p.t1, a1 = left ? p.t1 : p.t0;
            if (!c.circle) {
                const P2 q0 = c.at(a0), q1 = c.at(a1);
                area2 += q0.x * q1.y - q1.x * q0.y;
            } else {
                area2 += c.rad * c.rad * (a1 - a0) +
                         c.rad * (c.c.x * (std::sin(a1) - std::sin(a0)) - c.c.y * (std::cos(a1) - std::cos(a0)));
                const double len = c.rad * (p.t1 - p.t0);
                if (c.kind == GRAIN) l_ns += len;
                else l_nw += len;
            }
        }
        out[0] = 0.5 * area2;
        out[1] = l_nw;
        out[2] = l_ns;
    }
};

// A_nw, L_nw and L_ns of N(r); false for a degenerate throat or r <= 0.
bool msp_terms(const double* s3, double r, double cos_theta, double out[3]) {
    Section s;
    if (!make_section(s3, s) || !(r > 0)) return false;
    double rho[3];
    for (int i = 0; i < 3; ++i) {
        const double q = s.R[i] * s.R[i] + r * r + 2 * s.R[i] * r * cos_theta;
        if (!(q > r * r)) return false;  // contact angles of 90 degrees and beyond
        rho[i] = std::sqrt(q);
    }
    Terms t(s, r, rho);
    t.run(out);
    return true;
}

// The meniscus radius r of the MS-P condition: a scan of r upward from 0 in
// steps of r_ins / 64 (r_ins the throat's incircle) to the first r where
// F(r) = A_nw - r (L_nw + L_ns cos(theta)) is not positive, then bisection.
// (Where F stays positive until A empties, the root is the r at which it
// empties: no non-wetting region fits the section beyond it.)  Returns 0 for a
// closed throat, NaN for a degenerate one or when no root lies below 16 r_ins.
double msp_radius(const double* s3, double cos_theta) {
    const double rin = throat_incircle(s3);
    if (!(rin > 0)) return 0.0;
    auto F = [&](double r, bool& ok) {
        double t[3];
        ok = msp_terms(s3, r, cos_theta, t);
        return ok ? t[0] - r * (t[1] + t[2] * cos_theta) : 0.0;
    };
    const int steps = 64, max_steps = 64 * 16;
    double lo = 0, hi = -1;
    for (int kk = 1; kk <= max_steps; ++kk) {
        const double r = rin * kk / steps;
        bool ok;
        const double f = F(r, ok);
        if (!ok) return std::numeric_limits<double>::quiet_NaN();
        if (f <= 0) {
            hi = r;
            break;
        }
        lo = r;
    }
    if (!(hi > 0)) return std::numeric_limits<double>::quiet_NaN();
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        bool ok;
        const double f = F(mid, ok);
        if (ok && f > 0) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

}  // namespace lbmk

using namespace lbmk;

extern "C" {

int lbm_throat_msp_terms(const double* throat, double r, double cos_theta, double out[3]) {
    if (!throat || !out || !std::isfinite(r) || !std::isfinite(cos_theta)) {
        set_error("lbm_throat_msp_terms: NULL argument or non-finite r / cos_theta");
        return LBM_ERR_ARG;
    }
    if (!msp_terms(throat, r, cos_theta, out)) {
        set_error("lbm_throat_msp_terms: collinear centres, r <= 0 or a contact angle of 90 degrees or more");
        return LBM_ERR_ARG;
    }
    return LBM_OK;
}

int lbm_throat_pce_msp(const double* throats, int n, double sigma, double cos_theta, double* pce_out) {
    if (!throats || !pce_out || n < 0 || !std::isfinite(sigma) || !std::isfinite(cos_theta) || !(cos_theta > 0) ||
        !(cos_theta <= 1)) {
        set_error("lbm_throat_pce_msp: NULL argument, n < 0, non-finite sigma or cos_theta outside (0, 1]");
        return LBM_ERR_ARG;
    }
    const bool ok = host_parallel_for(n, [&](int t) {
        const double r = msp_radius(throats + 12 * (size_t)t, cos_theta);
        pce_out[t] = r == 0.0 ? INFINITY : sigma / r;  // NaN stays NaN
    });
    if (!ok) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
    return LBM_OK;
}

}  // extern "C"
