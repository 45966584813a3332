// lbm_step_core.cuh -- the fused two-component Shan-Chen D3Q19 step as device
// functions, shared by the single-domain kernel (lbm_step.cu) and the batched
// throat kernel (lbm_batch.cu).
//
//
// One launch advances every cell by one time step:
//   pull streaming with half-way bounce-back (Eq. 1, left-hand side),
//   moments rho_s, j_s (Eqs. 2-3),
//   Shan-Chen cohesion F_s = -G rho_s(x) sum_k w_k rho_sbar(x+e_k) e_k (Eq. 4,
//   psi = rho), wall adhesion -G_ads,s rho_s(x) sum_k w_k s(x+e_k) e_k and the
//   body force rho_s g,
//   common velocity u' = sum_s (j_s/tau_s) / sum_s (rho_s/tau_s), velocity shift
//   u_eq,s = u' + tau_s F_s / rho_s and the BGK relaxation towards
//   f^eq(rho_s, u_eq,s) (Eq. 1, right-hand side; Shan & Chen 1993 forcing),
//   reservoir layers reset to the rest equilibrium of their imposed densities.
//
// The force at x needs rho at the 18 neighbours at the same time level, known
// only after those neighbours have pulled.  Each CTA owns a 30 x (BY-2) column
// of cells and marches along z through a segment of planes.  Its 32 x BY threads
// cover the column plus a one-cell ring; every thread pulls its own cell one
// plane at a time with cp.async (4-byte asynchronous global->shared copies,
// bounce-back decided per copy), three planes in flight per thread in private
// shared-memory slots.  When a plane has landed the thread sums its densities
// into a 4-plane ring buffer visible to the whole CTA; after one barrier the
// interior threads collide the plane before it with all 18 neighbour densities
// at hand while the next planes are still arriving.  The ring cells are pulled
// twice (here and by their owner) and those re-reads are served by L2, so DRAM
// sees each population read once and written once: 2 x 19 x (4 + 4) = 304
// bytes per fluid cell update.
//
// FP32 throughout.  The rest population is set to rho - sum_{k>=1} f*_k so that
// the collision conserves each component's mass to rounding (the FP32 lattice
// weights do not sum to exactly one, which otherwise drifts the mass by about
// 1.5e-8 per step).
#pragma once

#include "lbm_device.cuh"

namespace lbmk {


__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Cell index of this thread's column on plane z (periodic wrap); ok is cleared
// for a plane beyond a closed z edge.
__device__ __forceinline__ int plane_cell(const Geom& g, const Column& c, int z, int& zz, bool& ok) {
    ok = c.ok;
    zz = wrap1(z, g.nz, g.pz, ok);
    return zz * g.nxy + c.yo[1] + c.xo[1];
}

// Queue the pull of this thread's cell (index cell, geometry word w, plane zz)
// into its private stage slots st[(s*19 + k) * NT + tid].  Away from periodic
// seams the source of direction k is cell + poff[k] (a kernel-parameter offset);
// on a seam the wrapped neighbour offsets are used.  Bounce-back is decided per
// copy from the geometry word.
template <int NT>
__device__ __forceinline__ void issue_pull(const float* __restrict__ fin, const uint32_t* __restrict__ nbr_nw,
                                          const Geom& g, const Column& c, int zz, int cell, uint32_t w, float* st,
                                          int tid) {
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    if (cls == CLS_SOLID || cls == CLS_OUTSIDE) return;
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
        if (s == 1 && cls == CLS_MEMBRANE) break;
        const uint32_t bits = s == 0 ? w : wn;
        const float* fs = fin + (size_t)s * Q * g.plane;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            int idx;
            if (!seam) idx = cell + g.poff[k];
            else idx = k * g.plane + zo[1 - EZ(k)] + c.yo[1 - EY(k)] + c.xo[1 - EX(k)];
            if ((bits >> k) & 1u) idx = OPP(k) * g.plane + cell;
            cp_async4(st + (s * Q + k) * NT + tid, fs + idx);
        }
    }
}

// Densities of a landed plane (0 where a component is not fluid), summed in k order.
template <int NT>
__device__ __forceinline__ void plane_density(uint32_t w, const float* st, int tid, float& rw, float& rn) {
    rw = 0.f;
    rn = 0.f;
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    if (cls == CLS_SOLID || cls == CLS_OUTSIDE) return;
    // four interleaved partial sums keep the adds independent
    float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < Q; ++k) a[k & 3] += st[k * NT + tid];
    rw = (a[0] + a[1]) + (a[2] + a[3]);
    if (cls != CLS_MEMBRANE) {
        float b[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < Q; ++k) b[k & 3] += st[(Q + k) * NT + tid];
        rn = (b[0] + b[1]) + (b[2] + b[3]);
    }
}

// Collide one interior fluid cell of plane z (pulled populations f) and hand
// each post-collision value to sink(s, k, v) (component s, direction k).  ring
// holds (rho_w, rho_nw) of planes z-1..z+1 for the CTA's 32 x BY cells:
// ring[slot * 32*BY + row*32 + lane].  Directions come in opposite pairs
// (k, k+1) with e_{k+1} = -e_k, which halves the arithmetic of the moments, the
// force sums and the equilibria (the symmetric and the antisymmetric part of
// f^eq are shared by a pair).  The rest population is rho_s - sum_{k>=1} f*_k.
//
// collide_core is the general form: rho_at(k) returns (rho_w, rho_nw) at x + e_k
// (k = 0: the cell itself), 0 where that cell is not fluid.  TAU1 = true is the
// form for tau = 1 in both components, with omega = 1 and 1 - omega = 0 known
// at compile time: for finite populations it gives the same bits as the
// general form run with tau = 1 (multiplying by 1 and adding 0 times a finite
// value are exact), with the multiplications left out.
template <bool TAU1 = false, class RhoAt, class Sink>
__device__ __forceinline__ void collide_core(const float (&f)[2][Q], uint32_t w, uint32_t a, const Phys& P,
                                             RhoAt&& rho_at, Sink&& sink) {
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    const bool has_nw = cls != CLS_MEMBRANE;

    if (cls == CLS_INLET || cls == CLS_OUTLET) {
        const float r0 = __ldg(P.bc + (cls == CLS_INLET ? 0 : 2));
        const float r1 = __ldg(P.bc + (cls == CLS_INLET ? 1 : 3));
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const float va = WK(k) * r0, vb = WK(k) * r1;
            s0 += va;
            s1 += vb;
            sink(0, k, va);
            sink(1, k, vb);
        }
        sink(0, 0, r0 - s0);
        sink(1, 0, r1 - s1);
        return;
    }

    const float2 r00 = rho_at(0);
    const float rw = r00.x;
    const float rn = r00.y;

    // neighbour density sums over opposite pairs:
    // cw = sum_k w_k rho_nw(x+e_k) e_k (acts on w), cn = sum_k w_k rho_w(x+e_k) e_k
    float cw[3] = {0.f, 0.f, 0.f}, cn[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 1; k < Q; k += 2) {
        const float2 p = rho_at(k), m = rho_at(k + 1);
        const float dn = WK(k) * (p.y - m.y);
        const float dw = WK(k) * (p.x - m.x);
        if (EX(k)) { cw[0] += EX(k) > 0 ? dn : -dn; cn[0] += EX(k) > 0 ? dw : -dw; }
        if (EY(k)) { cw[1] += EY(k) > 0 ? dn : -dn; cn[1] += EY(k) > 0 ? dw : -dw; }
        if (EZ(k)) { cw[2] += EZ(k) > 0 ? dn : -dn; cn[2] += EZ(k) > 0 ? dw : -dw; }
    }
    float ad[3] = {0.f, 0.f, 0.f};
    if (w & BIT_ADH) {
        ad[0] = (float)(int8_t)(a & 0xffu) * (1.0f / 36.0f);
        ad[1] = (float)(int8_t)((a >> 8) & 0xffu) * (1.0f / 36.0f);
        ad[2] = (float)(int8_t)((a >> 16) & 0xffu) * (1.0f / 36.0f);
    }

    // momenta (Eq. 3) over opposite pairs
    float j[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int k = 1; k < Q; k += 2) {
            const float d = f[s][k] - f[s][k + 1];
            if (EX(k)) j[s][0] += EX(k) > 0 ? d : -d;
            if (EY(k)) j[s][1] += EY(k) > 0 ? d : -d;
            if (EZ(k)) j[s][2] += EZ(k) > 0 ? d : -d;
        }

    // common velocity u' = (j_w/tau_w + j_nw/tau_nw) / (rho_w/tau_w + rho_nw/tau_nw)
    float up[3];
    {
        const float om0 = TAU1 ? 1.0f : P.omega[0], om1 = TAU1 ? 1.0f : P.omega[1];
        const float den = rw * om0 + (has_nw ? rn * om1 : 0.f);
        const float inv = den != 0.f ? 1.0f / den : 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) up[d] = (j[0][d] * om0 + (has_nw ? j[1][d] * om1 : 0.f)) * inv;
    }

#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (s == 1 && !has_nw) break;
        const float rs = s == 0 ? rw : rn;
        const float* coh = s == 0 ? cw : cn;
        float ueq[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float F = -P.G * rs * coh[d] - P.Gads[s] * rs * ad[d] + rs * P.g[d];
            ueq[d] = up[d] + (rs != 0.f ? (TAU1 ? F : P.tau[s] * F) / rs : 0.f);
        }
        const float uu = ueq[0] * ueq[0] + ueq[1] * ueq[1] + ueq[2] * ueq[2];
        const float om = TAU1 ? 1.0f : P.omega[s];
        const float keep = TAU1 ? 0.0f : 1.0f - om;
        const float base = rs * (1.0f - 1.5f * uu);
        const float r45 = 4.5f * rs;
        const float r3 = 3.0f * rs;
        float part[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 1; k < Q; k += 2) {
            const float eu = (float)EX(k) * ueq[0] + (float)EY(k) * ueq[1] + (float)EZ(k) * ueq[2];
            // f^eq_k = w rho (1 + 3 eu + 4.5 eu^2 - 1.5 uu), f^eq_{k+1} with -eu
            const float sym = WK(k) * (base + r45 * eu * eu);
            const float asym = WK(k) * (r3 * eu);
            const float v0 = TAU1 ? sym + asym : keep * f[s][k] + om * (sym + asym);
            const float v1 = TAU1 ? sym - asym : keep * f[s][k + 1] + om * (sym - asym);
            part[(k >> 1) % 3] += v0 + v1;
            sink(s, k, v0);
            sink(s, k + 1, v1);
        }
        sink(s, 0, rs - ((part[0] + part[1]) + part[2]));  // rest population: the collision keeps rho_s
    }
}

// A ring of density planes in shared memory: planes RPLANE float2 apart, rows
// RROW apart, (row, lane) the cell's coordinates in them, plane z at z & 3.
template <int RROW, int RPLANE, class Sink>
__device__ __forceinline__ void collide_ring(const float (&f)[2][Q], const float2* ring, uint32_t w, uint32_t a,
                                             int z, int row, int lane, const Phys& P, Sink&& sink) {
    collide_core(f, w, a, P,
                 [&](int k) { return ring[((z + EZ(k)) & 3) * RPLANE + (row + EY(k)) * RROW + (lane + EX(k))]; },
                 static_cast<Sink&&>(sink));
}

// The ring of the staged kernels: planes of 32 x BY cells, one per thread.
template <int BY, class Sink>
__device__ __forceinline__ void collide_generic(const float (&f)[2][Q], const float2* ring, uint32_t w, uint32_t a,
                                                int z, int row, int lane, const Phys& P, Sink&& sink) {
    collide_ring<32, 32 * BY>(f, ring, w, a, z, row, lane, P, static_cast<Sink&&>(sink));
}

// Momentum of component s (Eq. 3) over opposite pairs, in the order of the
// staged kernel.
__device__ __forceinline__ void momentum(const float (&f)[Q], float (&j)[3]) {
    j[0] = j[1] = j[2] = 0.f;
#pragma unroll
    for (int k = 1; k < Q; k += 2) {
        const float d = f[k] - f[k + 1];
        if (EX(k)) j[0] += EX(k) > 0 ? d : -d;
        if (EY(k)) j[1] += EY(k) > 0 ? d : -d;
        if (EZ(k)) j[2] += EZ(k) > 0 ? d : -d;
    }
}

// Collision of component s of one interior cell of plane z, for kernels that
// run one thread per cell and component: the arithmetic of collide_core for one
// component (the same operations in the same order).  f: the pulled populations;
// cls, a: the cell's class and adhesion word; j: this component's momentum; jo:
// the other component's (0 where it is not fluid).  rho holds density planes
// [4][2][RPLANE] (plane z at z & 3, then component, rows RROW apart); rc is the
// cell's index in a plane.  sink(k, v) receives every f*_k; it may overwrite
// f[k] (each f[k] is read before its sink call).
template <int RROW, int RPLANE, class Sink>
__device__ __forceinline__ void collide_component(const float (&f)[Q], uint32_t cls, uint32_t a, int s,
                                                  const float (&j)[3], const float (&jo)[3], const float* rho, int z,
                                                  int rc, const Phys& P, Sink&& sink) {
    if (cls == CLS_INLET || cls == CLS_OUTLET) {
        const float r = __ldg(P.bc + (cls == CLS_INLET ? 0 : 2) + s);  // device array: indexing is fine
        float sum = 0.f;
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const float v = WK(k) * r;
            sum += v;
            sink(k, v);
        }
        sink(0, r - sum);
        return;
    }
    const float* rz = rho + ((z & 3) * 2) * RPLANE;
    const float rw = rz[rc], rn = rz[RPLANE + rc];
    const float rs = s == 0 ? rw : rn;
    const bool has_nw = cls != CLS_MEMBRANE;
    // cohesion sum over the other component's neighbour densities
    float coh[3] = {0.f, 0.f, 0.f};
    {
        const int so = s ^ 1;
#pragma unroll
        for (int k = 1; k < Q; k += 2) {
            const float p = rho[(((z + EZ(k)) & 3) * 2 + so) * RPLANE + rc + EY(k) * RROW + EX(k)];
            const float m = rho[(((z - EZ(k)) & 3) * 2 + so) * RPLANE + rc - EY(k) * RROW - EX(k)];
            const float dd = WK(k) * (p - m);
            if (EX(k)) coh[0] += EX(k) > 0 ? dd : -dd;
            if (EY(k)) coh[1] += EY(k) > 0 ? dd : -dd;
            if (EZ(k)) coh[2] += EZ(k) > 0 ? dd : -dd;
        }
    }
    float ad[3] = {0.f, 0.f, 0.f};
    if (a != 0u) {
        ad[0] = (float)(int8_t)(a & 0xffu) * (1.0f / 36.0f);
        ad[1] = (float)(int8_t)((a >> 8) & 0xffu) * (1.0f / 36.0f);
        ad[2] = (float)(int8_t)((a >> 16) & 0xffu) * (1.0f / 36.0f);
    }
    float up[3];
    {
        const float den = rw * P.omega[0] + (has_nw ? rn * P.omega[1] : 0.f);
        const float inv = den != 0.f ? 1.0f / den : 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float j0 = s == 0 ? j[c] : jo[c];
            const float j1 = s == 0 ? jo[c] : j[c];
            up[c] = (j0 * P.omega[0] + (has_nw ? j1 * P.omega[1] : 0.f)) * inv;
        }
    }
    // the thread's component is a run-time value: select the parameters (an
    // indexed kernel parameter would be copied to local memory)
    const float gads = s == 0 ? P.Gads[0] : P.Gads[1];
    const float tau = s == 0 ? P.tau[0] : P.tau[1];
    float ueq[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float F = -P.G * rs * coh[c] - gads * rs * ad[c] + rs * P.g[c];
        ueq[c] = up[c] + (rs != 0.f ? tau * F / rs : 0.f);
    }
    const float uu = ueq[0] * ueq[0] + ueq[1] * ueq[1] + ueq[2] * ueq[2];
    const float om = s == 0 ? P.omega[0] : P.omega[1];
    const float keep = 1.0f - om;
    const float base = rs * (1.0f - 1.5f * uu);
    const float r45 = 4.5f * rs;
    const float r3 = 3.0f * rs;
    float part[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 1; k < Q; k += 2) {
        const float eu = (float)EX(k) * ueq[0] + (float)EY(k) * ueq[1] + (float)EZ(k) * ueq[2];
        const float sym = WK(k) * (base + r45 * eu * eu);
        const float asym = WK(k) * (r3 * eu);
        const float v0 = keep * f[k] + om * (sym + asym);
        const float v1 = keep * f[k + 1] + om * (sym - asym);
        part[(k >> 1) % 3] += v0 + v1;
        sink(k, v0);
        sink(k + 1, v1);
    }
    const float v = rs - ((part[0] + part[1]) + part[2]);  // rest population: the collision keeps rho_s
    sink(0, v);
}

// FP32 storage: the post-collision values go straight to fout[(s*19 + k) * plane + cell].
template <int BY>
__device__ __forceinline__ void collide_cell(const float (&f)[2][Q], const float2* ring, uint32_t w, uint32_t a,
                                             int cell, int z, int row, int lane, const Phys& P, const Geom& g,
                                             float* __restrict__ fout) {
    float* __restrict__ out0 = fout + cell;
    float* __restrict__ out1 = fout + (size_t)Q * g.plane + cell;
    collide_generic<BY>(f, ring, w, a, z, row, lane, P, [&](int s, int k, float v) {
        (s == 0 ? out0 : out1)[(size_t)k * g.plane] = v;
    });
}

// Pipeline: plane p is queued LEAD iterations before it is collided; plane z+1
// must have landed when plane z is collided (its densities feed the force), so
// LEAD + 1 planes of populations sit in each thread's private stage slots.
// The geometry word of a plane is fetched one iteration before its pull is
// queued, so the queueing never waits on memory.
//
// step_column advances the column (tile tx, ty) of planes [z0, z1) by one step.
// smem holds the stage slots, the density ring and the word slots
// (smem_bytes<BY, LEAD>()).  The caller must separate two calls that share smem
// by a __syncthreads (the ring is read across threads).
template <int BY, int LEAD>
__device__ __forceinline__ void step_column(const float* __restrict__ fin, float* __restrict__ fout,
                                            const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw,
                                            const uint32_t* __restrict__ adh, const Geom& g, const Phys& P, int tx,
                                            int ty, int z0, int z1, float* smem) {
    constexpr int TY = BY - 2;
    constexpr int NT = 32 * BY;
    constexpr int NS = LEAD + 1;  // stages
    float* stage = smem;                                                // [NS][2*Q][NT], private columns
    float2* ring = reinterpret_cast<float2*>(smem + NS * 2 * Q * NT);  // [4][NT] (rho_w, rho_nw)
    uint32_t* words = reinterpret_cast<uint32_t*>(ring + 4 * NT);       // [NS][NT]
    uint32_t* adhw = words + NS * NT;                                   // [NS][NT]
    const int lane = threadIdx.x;
    const int row = threadIdx.y;
    const int tid = row * 32 + lane;
    const int gx = tx * 30 - 1 + lane;
    const int gy = ty * TY - 1 + row;
    const Column col = make_column(gx, gy, g);
    // columns beyond the last halo column are not needed by anyone
    const bool needed = gx <= g.nx && gy <= g.ny;
    const bool interior = lane >= 1 && lane <= 30 && row >= 1 && row <= TY && gx < g.nx && gy < g.ny;
    auto slot = [&](int p) { return (p - z0 + 1) % NS; };  // p >= z0 - 1
    auto st_of = [&](int p) { return stage + slot(p) * (2 * Q * NT); };
    // geometry word of plane p (CLS_OUTSIDE when not needed or beyond a closed edge)
    auto fetch_word = [&](int p) -> uint32_t {
        if (!needed || p > z1) return CLS_OUTSIDE << CLS_SHIFT;
        int zz;
        bool ok;
        const int cell = plane_cell(g, col, p, zz, ok);
        return ok ? __ldg(nbr + cell) : (CLS_OUTSIDE << CLS_SHIFT);
    };
    auto issue = [&](int p, uint32_t w) {
        words[slot(p) * NT + tid] = w;
        if (!needed || p > z1) return;
        int zz;
        bool ok;
        const int cell = plane_cell(g, col, p, zz, ok);
        if (!ok) return;
        issue_pull<NT>(fin, nbr_nw, g, col, zz, cell, w, st_of(p), tid);
        if (w & BIT_ADH)
            cp_async4(reinterpret_cast<float*>(adhw + slot(p) * NT + tid), reinterpret_cast<const float*>(adh + cell));
    };
    auto publish = [&](int p) {
        float rw, rn;
        plane_density<NT>(words[slot(p) * NT + tid], st_of(p), tid, rw, rn);
        ring[(p & 3) * NT + tid] = make_float2(rw, rn);
    };

    // prologue: planes z0-1 .. z0+LEAD-1 queued, z0-1 and z0 published
    uint32_t wnext = fetch_word(z0 - 1);
#pragma unroll
    for (int i = 0; i <= LEAD; ++i) {
        const int p = z0 - 1 + i;
        const uint32_t w = wnext;
        wnext = fetch_word(p + 1);
        issue(p, w);
        cp_async_commit();
    }
    // groups queued: planes z0-1 .. z0+LEAD-1 (LEAD+1 groups); planes z0-1, z0 done
    cp_async_wait<LEAD - 1>();
    publish(z0 - 1);
    publish(z0);
    for (int z = z0; z < z1; ++z) {
        {
            const int p = z + LEAD;
            const uint32_t w = wnext;
            wnext = fetch_word(p + 1);
            issue(p, w);
            cp_async_commit();
        }
        cp_async_wait<LEAD - 1>();  // plane z+1 has landed
        publish(z + 1);
        __syncthreads();
        const uint32_t w0 = words[slot(z) * NT + tid];
        const uint32_t cls = (w0 >> CLS_SHIFT) & CLS_MASK;
        if (interior && cls != CLS_SOLID && cls != CLS_OUTSIDE) {
            int zz;
            bool ok;
            const int cell = plane_cell(g, col, z, zz, ok);
            const float* st = st_of(z);
            const bool has_nw = cls != CLS_MEMBRANE;
            float f[2][Q];
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                f[0][k] = st[k * NT + tid];
                f[1][k] = has_nw ? st[(Q + k) * NT + tid] : 0.f;
            }
            collide_cell<BY>(f, ring, w0, adhw[slot(z) * NT + tid], cell, z, row, lane, P, g, fout);
        }
    }
    cp_async_wait<0>();
}

template <int BY, int LEAD>
size_t smem_bytes() {
    return sizeof(float) * (size_t)((LEAD + 1) * 2 * Q + 4 * 2 + 2 * (LEAD + 1)) * 32 * BY;
}

}  // namespace lbmk
