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
    const long long N = (long long)nx * ny * nz;
    std::memset(mask, 0, (size_t)N);
    // grain: visit each sphere's bounding box only
    for (int i = 0; i < n_spheres; ++i) {
        const double* s = spheres + 4 * i;
        const int x0 = std::max(0, (int)std::floor(s[0] - s[3]) - 1), x1 = std::min(nx - 1, (int)std::ceil(s[0] + s[3]) + 1);
        const int y0 = std::max(0, (int)std::floor(s[1] - s[3]) - 1), y1 = std::min(ny - 1, (int)std::ceil(s[1] + s[3]) + 1);
        const int z0 = std::max(0, (int)std::floor(s[2] - s[3]) - 1), z1 = std::min(nz - 1, (int)std::ceil(s[2] + s[3]) + 1);
        for (int z = z0; z <= z1; ++z)
            for (int y = y0; y <= y1; ++y)
                for (int x = x0; x <= x1; ++x)
                    if (ball_contains((double)x, (double)y, (double)z, s))
                        mask[((long long)z * ny + y) * nx + x] = LBM_MASK_SOLID | LBM_MASK_ADHESIVE;
    }
    const bool clip = prism_clip && n_spheres >= 3 && spheres != nullptr;
    const Prism prism = clip ? Prism(spheres, spheres + 4, spheres + 8) : Prism();
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long long c = ((long long)z * ny + y) * nx + x;
                if (mask[c]) continue;
                if (clip) {
                    const double p[3] = {(double)x, (double)y, (double)z};
                    if (!prism.contains(p)) {
                        mask[c] = LBM_MASK_SOLID;
                        continue;
                    }
                }
                if (reservoirs) {
                    if (z == 0) mask[c] = LBM_MASK_INLET;
                    else if (z == nz - 1) mask[c] = LBM_MASK_OUTLET;
                    else if (z >= nz - 1 - membrane_layers) mask[c] = LBM_MASK_MEMBRANE;
                }
            }
}

}  // namespace lbmk
