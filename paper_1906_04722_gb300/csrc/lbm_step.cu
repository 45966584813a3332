// lbm_step.cu -- the fused two-component Shan-Chen D3Q19 time step.
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
#include "lbm_device.cuh"

namespace lbmk {

namespace {

constexpr int STAGES = 3;

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Queue the pull of this thread's cell on plane z into its private stage slots
// st[(s*19 + k) * NT + tid].  Returns the geometry word (CLS_OUTSIDE beyond a
// closed edge) and the cell index.
template <int NT>
__device__ __forceinline__ uint32_t issue_pull(const float* __restrict__ fin, const uint32_t* __restrict__ nbr,
                                               const uint32_t* __restrict__ nbr_nw, const Geom& g,
                                               const Column& c, int z, float* st, int tid, int& cell_out) {
    cell_out = 0;
    bool ok = c.ok;
    const int zz = wrap1(z, g.nz, g.pz, ok);
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
        const int idx = ((w >> k) & 1u) ? (OPP(k) * g.plane + cell) : (k * g.plane + src);
        cp_async4(st + k * NT + tid, fin + idx);
    }
    if (cls != CLS_MEMBRANE) {
        const uint32_t wn = (w & BIT_NW_DIFF) ? __ldg(nbr_nw + cell) : w;
        const float* fin1 = fin + (size_t)Q * g.plane;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int src = zo[1 - EZ(k)] + c.yo[1 - EY(k)] + c.xo[1 - EX(k)];
            const int idx = ((wn >> k) & 1u) ? (OPP(k) * g.plane + cell) : (k * g.plane + src);
            cp_async4(st + (Q + k) * NT + tid, fin1 + idx);
        }
    }
    return w;
}

// Densities of a landed plane (0 where a component is not fluid), summed in k order.
template <int NT>
__device__ __forceinline__ void plane_density(uint32_t w, const float* st, int tid, float& rw, float& rn) {
    rw = 0.f;
    rn = 0.f;
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    if (cls == CLS_SOLID || cls == CLS_OUTSIDE) return;
#pragma unroll
    for (int k = 0; k < Q; ++k) rw += st[k * NT + tid];
    if (cls != CLS_MEMBRANE) {
#pragma unroll
        for (int k = 0; k < Q; ++k) rn += st[(Q + k) * NT + tid];
    }
}

// Collide one interior fluid cell of plane z and store its post-collision values.
template <int BY>
__device__ __forceinline__ void collide_store(const float* st, const float* ring, uint32_t w, int cell, int z,
                                              int row, int lane, const uint32_t* __restrict__ adh, const Phys& P,
                                              const Geom& g, float* __restrict__ fout) {
    constexpr int NT = 32 * BY;
    const int tid = row * 32 + lane;
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    const bool has_nw = cls != CLS_MEMBRANE;
    float* __restrict__ out0 = fout;
    float* __restrict__ out1 = fout + (size_t)Q * g.plane;

    if (cls == CLS_INLET || cls == CLS_OUTLET) {
        const float r0 = cls == CLS_INLET ? P.rho_in[0] : P.rho_out[0];
        const float r1 = cls == CLS_INLET ? P.rho_in[1] : P.rho_out[1];
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const float a = WK(k) * r0, b = WK(k) * r1;
            s0 += a;
            s1 += b;
            out0[k * g.plane + cell] = a;
            out1[k * g.plane + cell] = b;
        }
        out0[cell] = r0 - s0;
        out1[cell] = r1 - s1;
        return;
    }

    // ring[(slot*2 + comp) * NT + row*32 + lane]
    auto rho_at = [&](int k, int comp) {
        const int slot = (z + EZ(k)) & 3;
        return ring[(slot * 2 + comp) * NT + (row + EY(k)) * 32 + (lane + EX(k))];
    };
    const float rw = rho_at(0, 0);
    const float rn = rho_at(0, 1);

    // neighbour density sums: cw = sum_k w_k rho_nw(x+e_k) e_k (acts on w),
    // cn = sum_k w_k rho_w(x+e_k) e_k (acts on nw)
    float cw[3] = {0.f, 0.f, 0.f}, cn[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        const float nrw = rho_at(k, 0);
        const float nrn = rho_at(k, 1);
        const float wk = WK(k);
        if (EX(k)) { cw[0] += wk * nrn * (float)EX(k); cn[0] += wk * nrw * (float)EX(k); }
        if (EY(k)) { cw[1] += wk * nrn * (float)EY(k); cn[1] += wk * nrw * (float)EY(k); }
        if (EZ(k)) { cw[2] += wk * nrn * (float)EZ(k); cn[2] += wk * nrw * (float)EZ(k); }
    }
    float ad[3] = {0.f, 0.f, 0.f};
    if (w & BIT_ADH) {
        const uint32_t a = __ldg(adh + cell);
        ad[0] = (float)(int8_t)(a & 0xffu) * (1.0f / 36.0f);
        ad[1] = (float)(int8_t)((a >> 8) & 0xffu) * (1.0f / 36.0f);
        ad[2] = (float)(int8_t)((a >> 16) & 0xffu) * (1.0f / 36.0f);
    }

    float f[2][Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        f[0][k] = st[k * NT + tid];
        f[1][k] = has_nw ? st[(Q + k) * NT + tid] : 0.f;
    }

    // momenta (Eq. 3)
    float j0[3] = {0.f, 0.f, 0.f}, j1[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        if (EX(k)) { j0[0] += EX(k) > 0 ? f[0][k] : -f[0][k]; j1[0] += EX(k) > 0 ? f[1][k] : -f[1][k]; }
        if (EY(k)) { j0[1] += EY(k) > 0 ? f[0][k] : -f[0][k]; j1[1] += EY(k) > 0 ? f[1][k] : -f[1][k]; }
        if (EZ(k)) { j0[2] += EZ(k) > 0 ? f[0][k] : -f[0][k]; j1[2] += EZ(k) > 0 ? f[1][k] : -f[1][k]; }
    }

    // common velocity u' = (j_w/tau_w + j_nw/tau_nw) / (rho_w/tau_w + rho_nw/tau_nw)
    float up[3];
    {
        const float den = rw * P.omega[0] + (has_nw ? rn * P.omega[1] : 0.f);
        const float inv = den != 0.f ? 1.0f / den : 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) up[d] = (j0[d] * P.omega[0] + (has_nw ? j1[d] * P.omega[1] : 0.f)) * inv;
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
            ueq[d] = up[d] + (rs != 0.f ? P.tau[s] * F / rs : 0.f);
        }
        const float uu = ueq[0] * ueq[0] + ueq[1] * ueq[1] + ueq[2] * ueq[2];
        const float om = P.omega[s];
        float* __restrict__ out = s == 0 ? out0 : out1;
        float sum = 0.f;
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const float eu = (float)EX(k) * ueq[0] + (float)EY(k) * ueq[1] + (float)EZ(k) * ueq[2];
            const float feq = WK(k) * rs * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * uu);
            const float v = f[s][k] - om * (f[s][k] - feq);
            sum += v;
            out[k * g.plane + cell] = v;
        }
        out[cell] = rs - sum;  // rest population: the collision keeps rho_s
    }
}

template <int BY>
__global__ void __launch_bounds__(32 * BY, 1) sc_step_kernel(const float* __restrict__ fin, float* __restrict__ fout,
                                                             const uint32_t* __restrict__ nbr,
                                                             const uint32_t* __restrict__ nbr_nw,
                                                             const uint32_t* __restrict__ adh, Geom g, Phys P,
                                                             int lz) {
    constexpr int TY = BY - 2;
    constexpr int NT = 32 * BY;
    extern __shared__ float smem[];
    float* stage = smem;                         // [STAGES][2*Q][NT], each thread its own column
    float* ring = smem + STAGES * 2 * Q * NT;    // [4][2][NT]
    const int lane = threadIdx.x;
    const int row = threadIdx.y;
    const int tid = row * 32 + lane;
    const int gx = blockIdx.x * 30 - 1 + lane;
    const int gy = blockIdx.y * TY - 1 + row;
    const int z0 = blockIdx.z * lz;
    const int z1 = min(z0 + lz, g.nz);
    const Column col = make_column(gx, gy, g);
    // columns beyond the last halo column are not needed by anyone
    const bool needed = gx <= g.nx && gy <= g.ny;
    const bool interior = lane >= 1 && lane <= 30 && row >= 1 && row <= TY && gx < g.nx && gy < g.ny;
    auto st_of = [&](int p) { return stage + ((p + STAGES) % STAGES) * (2 * Q * NT); };
    auto issue = [&](int p, int& cell) -> uint32_t {
        if (!needed || p > z1) { cell = 0; return CLS_OUTSIDE << CLS_SHIFT; }
        return issue_pull<NT>(fin, nbr, nbr_nw, g, col, p, st_of(p), tid, cell);
    };
    auto publish = [&](int p, uint32_t w) {
        float rw, rn;
        plane_density<NT>(w, st_of(p), tid, rw, rn);
        ring[((p & 3) * 2 + 0) * NT + tid] = rw;
        ring[((p & 3) * 2 + 1) * NT + tid] = rn;
    };

    int cm, c0, c1;
    const uint32_t wm = issue(z0 - 1, cm);
    cp_async_commit();
    uint32_t w0 = issue(z0, c0);
    cp_async_commit();
    uint32_t w1 = issue(z0 + 1, c1);
    cp_async_commit();
    cp_async_wait<1>();
    publish(z0 - 1, wm);
    publish(z0, w0);
    for (int z = z0; z < z1; ++z) {
        int c2;
        const uint32_t w2 = issue(z + 2, c2);
        cp_async_commit();
        cp_async_wait<1>();
        publish(z + 1, w1);
        __syncthreads();
        const uint32_t cls = (w0 >> CLS_SHIFT) & CLS_MASK;
        if (interior && cls != CLS_SOLID && cls != CLS_OUTSIDE)
            collide_store<BY>(st_of(z), ring, w0, c0, z, row, lane, adh, P, g, fout);
        w0 = w1;
        c0 = c1;
        w1 = w2;
        c1 = c2;
    }
    cp_async_wait<0>();
}

template <int BY>
size_t smem_bytes() {
    return sizeof(float) * (size_t)(STAGES * 2 * Q + 4 * 2) * 32 * BY;
}

template <int BY>
cudaError_t launch_by(const float* fin, float* fout, const uint32_t* nbr, const uint32_t* nbr_nw, const uint32_t* adh,
                      const Geom& g, const Phys& p, int lz, cudaStream_t s) {
    constexpr int TY = BY - 2;
    static unsigned long long configured = 0;  // one bit per device: the attribute is per device
    const size_t sm = smem_bytes<BY>();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(sc_step_kernel<BY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    dim3 grid((g.nx + 29) / 30, (g.ny + TY - 1) / TY, (g.nz + lz - 1) / lz);
    dim3 block(32, BY);
    sc_step_kernel<BY><<<grid, block, sm, s>>>(fin, fout, nbr, nbr_nw, adh, g, p, lz);
    return cudaGetLastError();
}

}  // namespace

StepTile default_tile(const Geom& g) {
    StepTile t;
    t.by = 10;
    // z segments: about 4 waves of one CTA per SM on 152 SMs, segments of >= 8 planes
    const long long tiles_xy = (long long)((g.nx + 29) / 30) * ((g.ny + (t.by - 2) - 1) / (t.by - 2));
    const long long want_segments = (4LL * 152 + tiles_xy - 1) / tiles_xy;
    int lz = (int)((g.nz + want_segments - 1) / want_segments);
    if (lz < 8) lz = 8;
    if (lz > g.nz) lz = g.nz;
    t.lz = lz;
    return t;
}

bool tile_supported(int by) { return by == 6 || by == 8 || by == 10 || by == 12; }

cudaError_t launch_step(const float* fin, float* fout, const uint32_t* nbr, const uint32_t* nbr_nw,
                        const uint32_t* adh, const Geom& g, const Phys& p, StepTile tile, cudaStream_t s) {
    if (tile.lz < 1) return cudaErrorInvalidValue;
    switch (tile.by) {
        case 6: return launch_by<6>(fin, fout, nbr, nbr_nw, adh, g, p, tile.lz, s);
        case 8: return launch_by<8>(fin, fout, nbr, nbr_nw, adh, g, p, tile.lz, s);
        case 10: return launch_by<10>(fin, fout, nbr, nbr_nw, adh, g, p, tile.lz, s);
        case 12: return launch_by<12>(fin, fout, nbr, nbr_nw, adh, g, p, tile.lz, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbmk
