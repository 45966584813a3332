// lbm_geometry.cpp -- host voxeliser of sphere packings and throat prisms.
//
// Cell (x, y, z) has its centre at (x, y, z) (lattice units).  A cell is grain
// (solid + adhesive) when its centre satisfies |p - c| <= r, evaluated as
// dx*dx + dy*dy + dz*dz <= r*r with every product and sum rounded separately
// (this file is compiled with -ffp-contract=off) so the decision is identical
// on every host.  The throat domain of Sec. 2.2.2 is the triangular prism whose
// three walls stand orthogonal to the plane of the three sphere centres and
// pass through two centres each; cells outside it are neutral walls.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "lbm_host.h"
#include "lbm_internal.h"

namespace lbmk {

namespace {

inline bool ball_contains(double px, double py, double pz, const double* s) {
    const double dx = px - s[0];
    const double dy = py - s[1];
    const double dz = pz - s[2];
    const double d2 = dx * dx + dy * dy + dz * dz;
    return d2 <= s[3] * s[3];
}

inline void sub3(const double* a, const double* b, double* o) {
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}
inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
inline void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Inside the prism of centres a, b, c: on the inner side of the three walls
// (the in-plane normal of edge i is n x (edge i), n = (b - a) x (c - a)); a
// point on a wall counts as inside.
struct Prism {
    double v[3][3] = {};
    double inward[3][3] = {};
    Prism() = default;
    explicit Prism(const double* s0, const double* s1, const double* s2) {
        const double* c[3] = {s0, s1, s2};
        for (int i = 0; i < 3; ++i)
            for (int d = 0; d < 3; ++d) v[i][d] = c[i][d];
        double ab[3], ac[3], n[3];
        sub3(v[1], v[0], ab);
        sub3(v[2], v[0], ac);
        cross3(ab, ac, n);
        for (int i = 0; i < 3; ++i) {
            double edge[3];
            sub3(v[(i + 1) % 3], v[i], edge);
            cross3(n, edge, inward[i]);
        }
    }
    bool contains(const double* p) const {
        for (int i = 0; i < 3; ++i) {
            double rel[3];
            sub3(p, v[i], rel);
            if (dot3(rel, inward[i]) < 0.0) return false;
        }
        return true;
    }
};

}  // namespace

void voxelise_box(int nx, int ny, int nz, const double* spheres, int n_spheres, int prism_clip, int reservoirs,
                  int membrane_layers, uint8_t* mask) {
    const bool clip = prism_clip && n_spheres >= 3 && spheres != nullptr;
    const Prism prism = clip ? Prism(spheres, spheres + 4, spheres + 8) : Prism();
    const size_t nxy = (size_t)nx * ny;
    // one plane per task on the host cores; every cell's value depends on that
    // cell alone, so the result does not depend on the order
    host_parallel_for(nz, [&](int z) {
        uint8_t* m = mask + (size_t)z * nxy;
        std::memset(m, 0, nxy);
        // grain: each sphere's bounding box within this plane
        for (int i = 0; i < n_spheres; ++i) {
            const double* s = spheres + 4 * i;
            const int z0 = (int)std::floor(s[2] - s[3]) - 1, z1 = (int)std::ceil(s[2] + s[3]) + 1;
            if (z < z0 || z > z1) continue;
            const int x0 = std::max(0, (int)std::floor(s[0] - s[3]) - 1), x1 = std::min(nx - 1, (int)std::ceil(s[0] + s[3]) + 1);
            const int y0 = std::max(0, (int)std::floor(s[1] - s[3]) - 1), y1 = std::min(ny - 1, (int)std::ceil(s[1] + s[3]) + 1);
            for (int y = y0; y <= y1; ++y)
                for (int x = x0; x <= x1; ++x)
                    if (ball_contains((double)x, (double)y, (double)z, s))
                        m[(size_t)y * nx + x] = LBM_MASK_SOLID | LBM_MASK_ADHESIVE;
        }
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                uint8_t& c = m[(size_t)y * nx + x];
                if (c) continue;
                if (clip) {
                    const double p[3] = {(double)x, (double)y, (double)z};
                    if (!prism.contains(p)) {
                        c = LBM_MASK_SOLID;
                        continue;
                    }
                }
                if (reservoirs) {
                    if (z == 0) c = LBM_MASK_INLET;
                    else if (z == nz - 1) c = LBM_MASK_OUTLET;
                    else if (z >= nz - 1 - membrane_layers) c = LBM_MASK_MEMBRANE;
                }
            }
    });
}

// Throat frame of Sec. 2.2.2 for centres c0, c1, c2: e1 along c1 - c0, e3 the
// unit normal (c1 - c0) x (c2 - c0), e2 = e3 x e1; the local coordinates of a
// point q are ((q - c0).e1, (q - c0).e2, (q - c0).e3).  The box spans the
// integer bounding box of the centres' local x and y and z in [-ceil(H),
// ceil(H)], H the largest radius; cell (i, j, k) sits at local
// (x0 + i, y0 + j, -ceil(H) + k).
void throat_frame(const double* sph, int dims[3], double origin[3], double local[12]) {
    const double* c0 = sph;
    const double* c1 = sph + 4;
    const double* c2 = sph + 8;
    double a[3], b[3], e1[3], e2[3], e3[3], n3[3];
    sub3(c1, c0, a);
    sub3(c2, c0, b);
    const double la = std::sqrt(dot3(a, a));
    for (int d = 0; d < 3; ++d) e1[d] = a[d] / la;
    cross3(a, b, n3);
    const double ln = std::sqrt(dot3(n3, n3));
    for (int d = 0; d < 3; ++d) e3[d] = n3[d] / ln;
    cross3(e3, e1, e2);
    double H = 0.0, lx[3], ly[3];
    for (int i = 0; i < 3; ++i) {
        const double* ci = sph + 4 * i;
        double rel[3];
        sub3(ci, c0, rel);
        lx[i] = dot3(rel, e1);
        ly[i] = dot3(rel, e2);
        local[4 * i + 0] = lx[i];
        local[4 * i + 1] = ly[i];
        local[4 * i + 2] = dot3(rel, e3);
        local[4 * i + 3] = ci[3];
        if (ci[3] > H) H = ci[3];
    }
    const double xmin = std::min(lx[0], std::min(lx[1], lx[2])), xmax = std::max(lx[0], std::max(lx[1], lx[2]));
    const double ymin = std::min(ly[0], std::min(ly[1], ly[2])), ymax = std::max(ly[0], std::max(ly[1], ly[2]));
    const double x0 = std::floor(xmin), y0 = std::floor(ymin), hz = std::ceil(H);
    dims[0] = (int)(std::ceil(xmax) - x0) + 1;
    dims[1] = (int)(std::ceil(ymax) - y0) + 1;
    dims[2] = 2 * (int)hz + 1;
    origin[0] = x0;
    origin[1] = y0;
    origin[2] = -hz;
}

// Throat box mask: grain inside the spheres, neutral wall outside the prism,
// inlet layer k = 0, outlet layer k = nz - 1.  probe = the fluid cell of plane
// nz - 3 farthest from every sphere surface (max of min_s |p - c_s| - r_s; the
// first in cell order on ties), or (-1, -1, -1) when that plane has no fluid.
void voxelise_throat(const double* sph, uint8_t* mask, int probe[3]) {
    int dims[3];
    double org[3], loc[12];
    throat_frame(sph, dims, org, loc);
    const Prism prism(loc, loc + 4, loc + 8);
    for (int k = 0; k < dims[2]; ++k)
        for (int j = 0; j < dims[1]; ++j)
            for (int i = 0; i < dims[0]; ++i) {
                const long long c = ((long long)k * dims[1] + j) * dims[0] + i;
                const double p[3] = {org[0] + (double)i, org[1] + (double)j, org[2] + (double)k};
                uint8_t m = 0;
                for (int s = 0; s < 3; ++s)
                    if (ball_contains(p[0], p[1], p[2], loc + 4 * s)) { m = LBM_MASK_SOLID | LBM_MASK_ADHESIVE; break; }
                if (!m && !prism.contains(p)) m = LBM_MASK_SOLID;
                if (!m) {
                    if (k == 0) m = LBM_MASK_INLET;
                    else if (k == dims[2] - 1) m = LBM_MASK_OUTLET;
                }
                mask[c] = m;
            }
    probe[0] = probe[1] = probe[2] = -1;
    const int k = dims[2] - 3;
    if (k < 0) return;
    double best = -1e300;
    for (int j = 0; j < dims[1]; ++j)
        for (int i = 0; i < dims[0]; ++i) {
            const long long c = ((long long)k * dims[1] + j) * dims[0] + i;
            if (mask[c] & LBM_MASK_SOLID) continue;
            const double p[3] = {org[0] + (double)i, org[1] + (double)j, org[2] + (double)k};
            double dmin = 1e300;
            for (int s = 0; s < 3; ++s) {
                const double* q = loc + 4 * s;
                const double dx = p[0] - q[0];
                const double dy = p[1] - q[1];
                const double dz = p[2] - q[2];
                const double d = std::sqrt(dx * dx + dy * dy + dz * dz) - q[3];
                if (d < dmin) dmin = d;
            }
            if (dmin > best) {
                best = dmin;
                probe[0] = i;
                probe[1] = j;
                probe[2] = k;
            }
        }
}

}  // namespace lbmk

namespace lbmk {

namespace {

// Squared Euclidean distance transform of one line: d[i] = min_j (f[j] + (i - j)^2),
// by the lower envelope of the parabolas rooted at every j (Felzenszwalb and
// Huttenlocher, "Distance transforms of sampled functions", 2012).  f holds 0
// at background cells and a large finite value (far above any squared distance
// of the plane) elsewhere.  v, zb: scratch of n and n + 1 entries.
void edt_line(const double* f, int n, double* d, int* v, double* zb) {
    int k = 0;
    v[0] = 0;
    zb[0] = -1e300;
    zb[1] = 1e300;
    for (int q = 1; q < n; ++q) {
        double s;
        while (true) {
            const int p = v[k];
            s = ((f[q] + (double)q * q) - (f[p] + (double)p * p)) / (2.0 * (q - p));
            if (s > zb[k]) break;  // zb[0] is below any s: the loop ends at k = 0 at the latest
            --k;
        }
        ++k;
        v[k] = q;
        zb[k] = s;
        zb[k + 1] = 1e300;
    }
    k = 0;
    for (int q = 0; q < n; ++q) {
        while (zb[k + 1] < q) ++k;
        const double dq = (double)(q - v[k]);
        d[q] = dq * dq + f[v[k]];
    }
}

// Largest distance from a non-solid cell of plane (nx x ny, x fastest) to the
// nearest solid cell of that plane; the plane diagonal where it has no solid cell.
double plane_incircle(const uint8_t* m, int nx, int ny) {
    const double big = 1e12;  // "no solid cell yet": far above (2 x 512)^2
    const int nmax = std::max(nx, ny);
    std::vector<double> g((size_t)nx * ny), f((size_t)nmax), d((size_t)nmax), zb((size_t)nmax + 1);
    std::vector<int> v((size_t)nmax);
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) f[(size_t)x] = (m[(size_t)y * nx + x] & LBM_MASK_SOLID) ? 0.0 : big;
        edt_line(f.data(), nx, d.data(), v.data(), zb.data());
        for (int x = 0; x < nx; ++x) g[(size_t)y * nx + x] = d[(size_t)x];
    }
    double best = 0.0;
    for (int x = 0; x < nx; ++x) {
        for (int y = 0; y < ny; ++y) f[(size_t)y] = g[(size_t)y * nx + x];
        edt_line(f.data(), ny, d.data(), v.data(), zb.data());
        for (int y = 0; y < ny; ++y)
            if (!(m[(size_t)y * nx + x] & LBM_MASK_SOLID)) best = std::max(best, d[(size_t)y]);
    }
    const double diag = (double)nx * nx + (double)ny * ny;
    return std::sqrt(std::min(best, diag));
}

void lattice_features(const uint8_t* m, int nx, int ny, int nz, double* o) {
    const size_t nxy = (size_t)nx * ny;
    std::vector<long long> area((size_t)nz, 0);
    long long nonsolid = 0;
    for (int k = 0; k < nz; ++k) {
        long long a = 0;
        for (size_t c = 0; c < nxy; ++c) a += !(m[(size_t)k * nxy + c] & LBM_MASK_SOLID);
        area[(size_t)k] = a;
        nonsolid += a;
    }
    std::vector<int> planes;
    for (int k = nz < 3 ? 0 : 1; k < (nz < 3 ? nz : nz - 1); ++k) planes.push_back(k);
    std::stable_sort(planes.begin(), planes.end(),
                     [&](int a, int b) { return area[(size_t)a] < area[(size_t)b]; });
    const int ks = planes[0];
    const int nsel = std::min<int>(3, (int)planes.size());
    double inc[3] = {0.0, 0.0, 0.0}, amean3 = 0.0, ainner = 0.0;
    for (int i = 0; i < nsel; ++i) {
        inc[i] = plane_incircle(m + (size_t)planes[(size_t)i] * nxy, nx, ny);
        amean3 += (double)area[(size_t)planes[(size_t)i]];
    }
    for (int k : planes) ainner += (double)area[(size_t)k];
    long long perim = 0;
    const uint8_t* p = m + (size_t)ks * nxy;
    auto solid = [&](int x, int y) {
        return x < 0 || y < 0 || x >= nx || y >= ny || (p[(size_t)y * nx + x] & LBM_MASK_SOLID);
    };
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            if (!solid(x, y) && (solid(x - 1, y) || solid(x + 1, y) || solid(x, y - 1) || solid(x, y + 1))) ++perim;
    const double amin = (double)area[(size_t)ks];
    double imax = 0.0, imean = 0.0;
    for (int i = 0; i < nsel; ++i) {
        imax = std::max(imax, inc[i]);
        imean += inc[i] / nsel;
    }
    o[0] = nx;
    o[1] = ny;
    o[2] = nz;
    o[3] = (double)nonsolid / ((double)nxy * nz);
    o[4] = amin;
    o[5] = std::sqrt(amin / 3.14159265358979323846);
    o[6] = ainner / (double)planes.size();
    o[7] = (double)ks / nz;
    o[8] = inc[0];
    o[9] = imax;
    o[10] = imean;
    o[11] = amin / (double)std::max<long long>(perim, 1);
    o[12] = (double)perim;
    o[13] = amean3 / nsel;
}

}  // namespace

}  // namespace lbmk

using namespace lbmk;

extern "C" int lbm_throat_lattice_features(const double* throats, int n, double* out) {
    if (!throats || !out || n < 1) {
        set_error("lbm_throat_lattice_features: NULL argument or empty batch");
        return LBM_ERR_ARG;
    }
    std::vector<int> dims((size_t)3 * n);
    for (int t = 0; t < n; ++t)
        if (int rc = lbm_throat_geometry(throats + 12 * t, dims.data() + 3 * t, nullptr, nullptr)) return rc;
    const bool ok = host_parallel_for(n, [&](int t) {
        const int* d = dims.data() + 3 * t;
        std::vector<uint8_t> mask((size_t)d[0] * d[1] * d[2]);
        int dd[3], probe[3];
        lbm_throat_geometry(throats + 12 * t, dd, mask.data(), probe);
        lattice_features(mask.data(), d[0], d[1], d[2], out + (size_t)LBM_THROAT_LATTICE_FEATURES * t);
    });
    if (!ok) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
    return LBM_OK;
}
