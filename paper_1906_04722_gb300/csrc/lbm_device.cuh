// lbm_device.cuh -- device-side building blocks shared by the step, density and
// measurement kernels: column coordinates with periodic wrap, and the pull of
// one cell's 2 x 19 populations with half-way bounce-back (Eq. 1, left-hand side).
#pragma once

#include "lbm_internal.h"

namespace lbmk {

// Wrap a coordinate one step beyond the box; ok is cleared when it falls beyond
// a closed edge (the returned value is then clamped and must not be used).
__device__ __forceinline__ int wrap1(int v, int n, int periodic, bool& ok) {
    if (v < 0) {
        if (periodic) return v + n;
        ok = false;
        return 0;
    }
    if (v >= n) {
        if (periodic) return v - n;
        ok = false;
        return n - 1;
    }
    return v;
}

// Neighbour coordinate for a source lookup: wrapped, or clamped into the box
// (a clamped value is only ever used behind a bounce-back bit).
__device__ __forceinline__ int nb1(int v, int n, int periodic) {
    if (v < 0) return periodic ? v + n : 0;
    if (v >= n) return periodic ? v - n : n - 1;
    return v;
}

// The x/y part of a cell's pull addresses.  xo[i] / yo[i] are the (wrapped)
// x offset and y row offset of x - 1 + i / y - 1 + i.
struct Column {
    int xo[3];
    int yo[3];
    bool ok;  // the column exists (inside the box or a periodic image)
};

__device__ __forceinline__ Column make_column(int gx, int gy, const Geom& g) {
    Column c;
    c.ok = true;
    int x = wrap1(gx, g.nx, g.px, c.ok);
    int y = wrap1(gy, g.ny, g.py, c.ok);
    c.xo[0] = nb1(x - 1, g.nx, g.px);
    c.xo[1] = x;
    c.xo[2] = nb1(x + 1, g.nx, g.px);
    c.yo[0] = nb1(y - 1, g.ny, g.py) * g.nx;
    c.yo[1] = y * g.nx;
    c.yo[2] = nb1(y + 1, g.ny, g.py) * g.nx;
    return c;
}

// Pull the populations of one cell whose geometry word w is known:
//   f_k(x) = f*_k(x - e_k)   if x - e_k is fluid for the component,
//   f_k(x) = f*_kbar(x)      otherwise (half-way bounce-back),
// from the post-collision array fin[(s*19 + k) * plane + cell].  zz is the
// cell's (wrapped) plane.  Returns the component densities (0 where a component
// is not fluid): with ILP in four interleaved partial sums, otherwise in k order.
// With KEEP the pulled values are left in f.
template <bool KEEP, bool ILP = false>
__device__ __forceinline__ void pull_known(const float* __restrict__ fin, const uint32_t* __restrict__ nbr_nw,
                                           const Geom& g, const Column& c, int zz, int cell, uint32_t w,
                                           float (&f)[2][Q], float& rw, float& rn) {
    rw = 0.f;
    rn = 0.f;
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    if (cls == CLS_SOLID || cls == CLS_OUTSIDE) return;
    // away from periodic seams the source of direction k is cell - (ex + ey nx + ez nxy)
    const bool seam = (g.px && (c.xo[1] == 0 || c.xo[1] == g.nx - 1)) ||
                      (g.py && (c.yo[1] == 0 || c.yo[1] == (g.ny - 1) * g.nx)) ||
                      (g.pz && (zz == 0 || zz == g.nz - 1));
    int zo[3];
    zo[0] = nb1(zz - 1, g.nz, g.pz) * g.nxy;
    zo[1] = zz * g.nxy;
    zo[2] = nb1(zz + 1, g.nz, g.pz) * g.nxy;
    const uint32_t wn = (cls == CLS_MEMBRANE) ? 0u : ((w & BIT_NW_DIFF) ? __ldg(nbr_nw + cell) : w);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (s == 1 && cls == CLS_MEMBRANE) {
            if (KEEP) {
#pragma unroll
                for (int k = 0; k < Q; ++k) f[1][k] = 0.f;
            }
            break;
        }
        const uint32_t bits = s == 0 ? w : wn;
        const float* fs = fin + (size_t)s * Q * g.plane;
        float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            int src;
            if (!seam) src = cell - (EX(k) + EY(k) * g.nx + EZ(k) * g.nxy);
            else src = zo[1 - EZ(k)] + c.yo[1 - EY(k)] + c.xo[1 - EX(k)];
            const int idx = ((bits >> k) & 1u) ? (OPP(k) * g.plane + cell) : (k * g.plane + src);
            const float v = __ldg(fs + idx);
            if (KEEP) f[s][k] = v;
            if (ILP) a[k & 3] += v;
            else a[0] += v;
        }
        const float r = ILP ? (a[0] + a[1]) + (a[2] + a[3]) : a[0];
        if (s == 0) rw = r;
        else rn = r;
    }
}

// Pull cell (column, z): loads the geometry word, then as pull_known.  Returns
// the word (class CLS_OUTSIDE for a cell beyond a closed edge).
template <bool KEEP>
__device__ __forceinline__ uint32_t pull_cell(const float* __restrict__ fin, const uint32_t* __restrict__ nbr,
                                              const uint32_t* __restrict__ nbr_nw, const Geom& g,
                                              const Column& c, int z, float (&f)[2][Q], float& rw, float& rn,
                                              int& cell_out) {
    rw = 0.f;
    rn = 0.f;
    cell_out = 0;
    bool ok = c.ok;
    const int zz = wrap1(z, g.nz, g.pz, ok);
    if (!ok) return CLS_OUTSIDE << CLS_SHIFT;
    const int cell = zz * g.nxy + c.yo[1] + c.xo[1];
    cell_out = cell;
    const uint32_t w = __ldg(nbr + cell);
    pull_known<KEEP>(fin, nbr_nw, g, c, zz, cell, w, f, rw, rn);
    return w;
}

// Adds one cell's contribution to the measurement sums (definitions in lbm.h):
// mass and sanity per component where it is fluid, Eq. 5 pressure, reservoir
// means, interior counts and bulk-phase pressures.
__device__ __forceinline__ void measure_accumulate(double (&acc)[NMEAS], uint32_t cls, double rw, double rn,
                                                   double G) {
    if (cls == CLS_SOLID || cls == CLS_OUTSIDE) return;
    acc[MS_MASS_W] += rw;
    if (!isfinite(rw)) acc[MS_N_NONFINITE] += 1.0;
    else if (rw < 0.0) acc[MS_N_NEGATIVE] += 1.0;
    if (cls != CLS_MEMBRANE) {
        acc[MS_MASS_NW] += rn;
        if (!isfinite(rn)) acc[MS_N_NONFINITE] += 1.0;
        else if (rn < 0.0) acc[MS_N_NEGATIVE] += 1.0;
    }
    const double p = (rw + rn) / 3.0 + G * rw * rn / 3.0;  // Eq. 5
    if (cls == CLS_INLET) { acc[MS_PIN] += p; acc[MS_N_IN] += 1.0; return; }
    if (cls == CLS_OUTLET) { acc[MS_POUT] += p; acc[MS_N_OUT] += 1.0; return; }
    if (cls == CLS_MEMBRANE) return;
    acc[MS_N_FLUID] += 1.0;
    if (rw > rn) acc[MS_N_W] += 1.0;
    const double phi = (rw - rn) / (rw + rn);
    if (fabs(phi) < 0.5) acc[MS_N_INTERFACE] += 1.0;
    if (phi > 0.9) { acc[MS_PW] += p; acc[MS_N_BULK_W] += 1.0; }
    if (phi < -0.9) { acc[MS_PNW] += p; acc[MS_N_BULK_NW] += 1.0; }
}

}  // namespace lbmk
