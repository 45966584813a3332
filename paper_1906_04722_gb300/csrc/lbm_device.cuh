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

// Pull the populations of cell (column, z) for both components:
//   f_k(x) = f*_k(x - e_k)   if x - e_k is fluid for the component,
//   f_k(x) = f*_kbar(x)      otherwise (half-way bounce-back),
// from the post-collision array fin[(s*19 + k) * plane + cell].  Returns the
// cell's geometry word (class CLS_OUTSIDE for a cell beyond a closed edge) and
// the component densities (0 where a component is not fluid).  With KEEP the
// pulled values are left in f; otherwise only the sums are formed.
template <bool KEEP>
__device__ __forceinline__ uint32_t pull_cell(const float* __restrict__ fin, const uint32_t* __restrict__ nbr,
                                              const uint32_t* __restrict__ nbr_nw, const Geom& g,
                                              const Column& c, int z, float (&f)[2][Q], float& rw, float& rn,
                                              int& cell_out) {
    rw = 0.f;
    rn = 0.f;
    cell_out = 0;
    bool ok = c.ok;
    int zz = wrap1(z, g.nz, g.pz, ok);
    if (!ok) return CLS_OUTSIDE << CLS_SHIFT;
    int zo[3];
    zo[0] = nb1(zz - 1, g.nz, g.pz) * g.nxy;
    zo[1] = zz * g.nxy;
    zo[2] = nb1(zz + 1, g.nz, g.pz) * g.nxy;
    const int cell = zo[1] + c.yo[1] + c.xo[1];
    cell_out = cell;
    const uint32_t w = __ldg(nbr + cell);
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    if (cls == CLS_SOLID) return w;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int src = zo[1 - EZ(k)] + c.yo[1 - EY(k)] + c.xo[1 - EX(k)];
        const bool bb = (w >> k) & 1u;
        const int idx = bb ? (OPP(k) * g.plane + cell) : (k * g.plane + src);
        const float v = __ldg(fin + idx);
        if (KEEP) f[0][k] = v;
        rw += v;
    }
    if (cls != CLS_MEMBRANE) {
        const uint32_t wn = (w & BIT_NW_DIFF) ? __ldg(nbr_nw + cell) : w;
        const float* fin1 = fin + (size_t)Q * g.plane;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int src = zo[1 - EZ(k)] + c.yo[1 - EY(k)] + c.xo[1 - EX(k)];
            const bool bb = (wn >> k) & 1u;
            const int idx = bb ? (OPP(k) * g.plane + cell) : (k * g.plane + src);
            const float v = __ldg(fin1 + idx);
            if (KEEP) f[1][k] = v;
            rn += v;
        }
    } else if (KEEP) {
#pragma unroll
        for (int k = 0; k < Q; ++k) f[1][k] = 0.f;
    }
    return w;
}

}  // namespace lbmk
