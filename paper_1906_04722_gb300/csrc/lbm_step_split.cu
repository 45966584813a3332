// lbm_step_split.cu -- the fused two-component Shan-Chen D3Q19 step (FP32) as
// two launches without shared memory.
//
// The force at x needs the densities of the 18 neighbours at the same time
// level (Eq. 4), which the staged and TMA kernels obtain by pulling a one-cell
// ring around every tile a second time inside the CTA.  Here:
//
//   density_pair_kernel  pulls every cell (Eq. 1 left-hand side, half-way
//                        bounce-back) and stores only (rho_w, rho_nw) (Eq. 2),
//                        0 where a component is not fluid;
//   sc_step_split_kernel pulls every cell again, reads its 18 neighbour
//                        density pairs from that field (through L1/L2), and
//                        collides and stores as the other kernels do
//                        (collide_core: the same arithmetic).
//
// One thread per cell, no barrier, no shared memory: every thread keeps its 38
// loads in flight and the SM holds enough warps to cover DRAM latency.  The
// price is traffic: each population is read twice from DRAM (the population
// buffers are far larger than L2), plus 8 bytes per cell written and read for
// the densities -- about 472 bytes per cell update instead of 304.  It works for
// any box and periodicity.
#include "lbm_step_core.cuh"

namespace lbmk {

namespace {

constexpr int SX = 32, SY = 8;  // threads per block along x and y; one plane per block

__global__ void __launch_bounds__(SX * SY)
    density_pair_kernel(const float* __restrict__ fin, const uint32_t* __restrict__ nbr,
                        const uint32_t* __restrict__ nbr_nw, Geom g, float2* __restrict__ rho2) {
    const int x = blockIdx.x * SX + threadIdx.x, y = blockIdx.y * SY + threadIdx.y, z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int cell = z * g.nxy + y * g.nx + x;
    const uint32_t w = __ldg(nbr + cell);
    const Column col = make_column(x, y, g);
    float unused[2][Q];
    float rw, rn;
    pull_known<false, true>(fin, nbr_nw, g, col, z, cell, w, unused, rw, rn);
    rho2[cell] = make_float2(rw, rn);
}

__global__ void __launch_bounds__(SX * SY, 2)
    sc_step_split_kernel(const float* __restrict__ fin, float* __restrict__ fout, const float2* __restrict__ rho2,
                         const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw,
                         const uint32_t* __restrict__ adh, Geom g, Phys P) {
    const int x = blockIdx.x * SX + threadIdx.x, y = blockIdx.y * SY + threadIdx.y, z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int cell = z * g.nxy + y * g.nx + x;
    const uint32_t w = __ldg(nbr + cell);
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    if (cls == CLS_SOLID || cls == CLS_OUTSIDE) return;
    const Column col = make_column(x, y, g);
    float f[2][Q];
    float rw, rn;
    pull_known<true, true>(fin, nbr_nw, g, col, z, cell, w, f, rw, rn);
    const uint32_t a = (w & BIT_ADH) ? __ldg(adh + cell) : 0u;
    // neighbour cells: wrapped on periodic axes, absent (density 0) beyond a
    // closed edge
    const bool vx[3] = {x > 0 || g.px, true, x < g.nx - 1 || g.px};
    const bool vy[3] = {y > 0 || g.py, true, y < g.ny - 1 || g.py};
    const bool vz[3] = {z > 0 || g.pz, true, z < g.nz - 1 || g.pz};
    int zo[3];
    zo[0] = nb1(z - 1, g.nz, g.pz) * g.nxy;
    zo[1] = z * g.nxy;
    zo[2] = nb1(z + 1, g.nz, g.pz) * g.nxy;
    auto rho_at = [&](int k) {
        if (!(vx[1 + EX(k)] && vy[1 + EY(k)] && vz[1 + EZ(k)])) return make_float2(0.f, 0.f);
        return __ldg(rho2 + zo[1 + EZ(k)] + col.yo[1 + EY(k)] + col.xo[1 + EX(k)]);
    };
    float* __restrict__ out0 = fout + cell;
    float* __restrict__ out1 = fout + (size_t)Q * g.plane + cell;
    collide_core(f, w, a, P, rho_at, [&](int s, int k, float v) { (s == 0 ? out0 : out1)[(size_t)k * g.plane] = v; });
}

}  // namespace

cudaError_t launch_step_split(const float* fin, float* fout, float2* rho2, const uint32_t* nbr,
                              const uint32_t* nbr_nw, const uint32_t* adh, const Geom& g, const Phys& p,
                              cudaStream_t s) {
    const dim3 grid((g.nx + SX - 1) / SX, (g.ny + SY - 1) / SY, g.nz);
    const dim3 block(SX, SY);
    density_pair_kernel<<<grid, block, 0, s>>>(fin, nbr, nbr_nw, g, rho2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sc_step_split_kernel<<<grid, block, 0, s>>>(fin, fout, rho2, nbr, nbr_nw, adh, g, p);
    return cudaGetLastError();
}

}  // namespace lbmk
