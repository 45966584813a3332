// lbm_step.cu -- launchers of the fused two-component Shan-Chen D3Q19 step on a
// single domain (kernels: the staged step of lbm_step_core.cuh, and a
// double-pull variant).
#include "lbm_step_core.cuh"

namespace lbmk {

namespace {

template <int BY, int LEAD>
__global__ void __launch_bounds__(32 * BY, (BY <= 6 && LEAD <= 2) ? 2 : 1)
    sc_step_kernel(const float* __restrict__ fin, float* __restrict__ fout, const uint32_t* __restrict__ nbr,
                   const uint32_t* __restrict__ nbr_nw, const uint32_t* __restrict__ adh, Geom g, Phys P, int lz) {
    extern __shared__ float smem[];
    const int z0 = blockIdx.z * lz;
    step_column<BY, LEAD>(fin, fout, nbr, nbr_nw, adh, g, P, blockIdx.x, blockIdx.y, z0, min(z0 + lz, g.nz), smem);
}

// Double-pull variant: no staging buffers.  Each iteration first pulls plane
// z+1 into registers only to sum its densities into the shared ring (all 32 x BY
// threads), then, after the barrier, the interior threads pull plane z again --
// the same addresses the previous iteration summed, normally still in L1 -- and
// collide it.  Twice the load instructions, a tenth of the shared memory, so
// two to three CTAs share an SM.
template <int BY, int MINB>
__global__ void __launch_bounds__(32 * BY, MINB) sc_step_dp_kernel(const float* __restrict__ fin,
                                                                  float* __restrict__ fout,
                                                                  const uint32_t* __restrict__ nbr,
                                                                  const uint32_t* __restrict__ nbr_nw,
                                                                  const uint32_t* __restrict__ adh, Geom g, Phys P,
                                                                  int lz) {
    constexpr int TY = BY - 2;
    constexpr int NT = 32 * BY;
    __shared__ float2 ring[4 * NT];
    const int lane = threadIdx.x;
    const int row = threadIdx.y;
    const int tid = row * 32 + lane;
    const int gx = blockIdx.x * 30 - 1 + lane;
    const int gy = blockIdx.y * TY - 1 + row;
    const int z0 = blockIdx.z * lz;
    const int z1 = min(z0 + lz, g.nz);
    const Column col = make_column(gx, gy, g);
    const bool needed = gx <= g.nx && gy <= g.ny;
    const bool interior = lane >= 1 && lane <= 30 && row >= 1 && row <= TY && gx < g.nx && gy < g.ny;
    auto word_of = [&](int p) -> uint32_t {
        if (!needed || p > z1) return CLS_OUTSIDE << CLS_SHIFT;
        int zz;
        bool ok;
        const int cell = plane_cell(g, col, p, zz, ok);
        return ok ? __ldg(nbr + cell) : (CLS_OUTSIDE << CLS_SHIFT);
    };
    auto publish = [&](int p, uint32_t w) {
        float rw = 0.f, rn = 0.f;
        int zz;
        bool ok;
        const int cell = plane_cell(g, col, p, zz, ok);
        float dummy[2][Q];
        if (needed && ok) pull_known<false, true>(fin, nbr_nw, g, col, zz, cell, w, dummy, rw, rn);
        ring[(p & 3) * NT + tid] = make_float2(rw, rn);
    };
    uint32_t wm = word_of(z0 - 1);
    uint32_t w0 = word_of(z0);
    uint32_t w1 = word_of(z0 + 1);
    publish(z0 - 1, wm);
    publish(z0, w0);
    for (int z = z0; z < z1; ++z) {
        const uint32_t w2 = word_of(z + 2);  // prefetched for the next iteration
        publish(z + 1, w1);
        __syncthreads();
        const uint32_t cls = (w0 >> CLS_SHIFT) & CLS_MASK;
        if (interior && cls != CLS_SOLID && cls != CLS_OUTSIDE) {
            int zz;
            bool ok;
            const int cell = plane_cell(g, col, z, zz, ok);
            const uint32_t a = (w0 & BIT_ADH) ? __ldg(adh + cell) : 0u;
            float f[2][Q];
            float rw, rn;
            pull_known<true, true>(fin, nbr_nw, g, col, zz, cell, w0, f, rw, rn);
            collide_cell<BY>(f, ring, w0, a, cell, z, row, lane, P, g, fout);
        }
        w0 = w1;
        w1 = w2;
    }
}


// Per-device one-time setting of the kernel's dynamic shared memory limit.
// Done outside any stream capture (see prepare_step).
template <int BY, int LEAD>
cudaError_t configure_by() {
    static unsigned long long configured = 0;  // one bit per device: the attribute is per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(sc_step_kernel<BY, LEAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes<BY, LEAD>());
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    return cudaSuccess;
}

template <int BY, int LEAD>
cudaError_t launch_by(const float* fin, float* fout, const uint32_t* nbr, const uint32_t* nbr_nw, const uint32_t* adh,
                      const Geom& g, const Phys& p, int lz, cudaStream_t s) {
    constexpr int TY = BY - 2;
    dim3 grid((g.nx + 29) / 30, (g.ny + TY - 1) / TY, (g.nz + lz - 1) / lz);
    dim3 block(32, BY);
    sc_step_kernel<BY, LEAD><<<grid, block, smem_bytes<BY, LEAD>(), s>>>(fin, fout, nbr, nbr_nw, adh, g, p, lz);
    return cudaGetLastError();
}

template <int BY, int MINB>
cudaError_t configure_dp() {
    static unsigned long long configured = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        // most of the unified L1/shared storage goes to L1: the second pull reads from it
        e = cudaFuncSetAttribute(sc_step_dp_kernel<BY, MINB>, cudaFuncAttributePreferredSharedMemoryCarveout, 10);
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    return cudaSuccess;
}

template <int BY, int MINB>
cudaError_t launch_dp(const float* fin, float* fout, const uint32_t* nbr, const uint32_t* nbr_nw, const uint32_t* adh,
                      const Geom& g, const Phys& p, int lz, cudaStream_t s) {
    constexpr int TY = BY - 2;
    dim3 grid((g.nx + 29) / 30, (g.ny + TY - 1) / TY, (g.nz + lz - 1) / lz);
    dim3 block(32, BY);
    sc_step_dp_kernel<BY, MINB><<<grid, block, 0, s>>>(fin, fout, nbr, nbr_nw, adh, g, p, lz);
    return cudaGetLastError();
}

__global__ void set_bc_kernel(float* bc, float in_w, float in_nw, float out_w, float out_nw) {
    bc[0] = in_w;
    bc[1] = in_nw;
    bc[2] = out_w;
    bc[3] = out_nw;
}

__global__ void probe_kernel(const float* __restrict__ f, const uint32_t* __restrict__ nbr,
                             const uint32_t* __restrict__ nbr_nw, Geom g, int x, int y, int z, float* out) {
    const Column col = make_column(x, y, g);
    float dummy[2][Q];
    float rw, rn;
    int cell;
    pull_cell<false>(f, nbr, nbr_nw, g, col, z, dummy, rw, rn, cell);
    out[0] = rw;
    out[1] = rn;
}

}  // namespace

StepTile default_tile(const Geom& g) {
    // 32 x 6 threads per CTA (30 x 4 interior columns), two planes queued ahead:
    // two CTAs per SM.  z segments: long enough that the two halo planes a
    // segment pulls twice stay a small share (at most 32 planes), short enough
    // that a small box still gives about two CTAs per SM -- a CTA walks its
    // segment plane after plane, so on a throat-sized box the segment length is
    // the step's latency.
    StepTile t;
    t.by = 6;
    t.lead = 2;
    const int sms = device_sm_count();
    const long long tiles_xy = (long long)((g.nx + 29) / 30) * ((g.ny + (t.by - 2) - 1) / (t.by - 2));
    long long lz = (g.nz * tiles_xy + 2LL * sms - 1) / (2LL * sms);
    if (lz < 2) lz = 2;
    if (lz > 32) lz = 32;
    if (lz > g.nz) lz = g.nz;
    t.lz = (int)lz;
    t.kind = LBM_KERNEL_STAGED;
    t.tma_lz = 0;
    return t;
}

bool tile_supported(int by, int lead) {
    switch (lead) {
        case 0: return by == 6 || by == 8 || by == 10;  // double-pull kernel
        case 1: return by == 6 || by == 8 || by == 10;  // double-pull kernel, one more CTA per SM
        case 2: return by == 6 || by == 8 || by == 10 || by == 12;
        case 3: return by == 6 || by == 8 || by == 10;
        case 4: return by == 6 || by == 8;
        default: return false;
    }
}

#define LBM_TILES(X)                                                                  \
    X(6, 2) X(8, 2) X(10, 2) X(12, 2) X(6, 3) X(8, 3) X(10, 3) X(6, 4) X(8, 4)
#define LBM_DP_TILES(X) X(6, 0, 3) X(8, 0, 2) X(10, 0, 2) X(6, 1, 4) X(8, 1, 3) X(10, 1, 3)

cudaError_t prepare_step(const StepTile& tile) {
    if (tile.lz < 1 || !tile_supported(tile.by, tile.lead)) return cudaErrorInvalidValue;
#define LBM_CFG(BY, LEAD) \
    if (tile.by == BY && tile.lead == LEAD) return configure_by<BY, LEAD>();
#define LBM_CFG_DP(BY, LEAD, MINB) \
    if (tile.by == BY && tile.lead == LEAD) return configure_dp<BY, MINB>();
    LBM_TILES(LBM_CFG)
    LBM_DP_TILES(LBM_CFG_DP)
#undef LBM_CFG
#undef LBM_CFG_DP
    return cudaErrorInvalidValue;
}

cudaError_t launch_step(const float* fin, float* fout, const uint32_t* nbr, const uint32_t* nbr_nw,
                        const uint32_t* adh, const Geom& g, const Phys& p, StepTile tile, cudaStream_t s) {
    if (tile.lz < 1 || !tile_supported(tile.by, tile.lead)) return cudaErrorInvalidValue;
#define LBM_TILE(BY, LEAD) \
    if (tile.by == BY && tile.lead == LEAD) return launch_by<BY, LEAD>(fin, fout, nbr, nbr_nw, adh, g, p, tile.lz, s);
#define LBM_TILE_DP(BY, LEAD, MINB) \
    if (tile.by == BY && tile.lead == LEAD) return launch_dp<BY, MINB>(fin, fout, nbr, nbr_nw, adh, g, p, tile.lz, s);
    LBM_TILES(LBM_TILE)
    LBM_DP_TILES(LBM_TILE_DP)
#undef LBM_TILE
#undef LBM_TILE_DP
    return cudaErrorInvalidValue;
}

cudaError_t launch_set_bc(float* bc, float in_w, float in_nw, float out_w, float out_nw, cudaStream_t s) {
    set_bc_kernel<<<1, 1, 0, s>>>(bc, in_w, in_nw, out_w, out_nw);
    return cudaGetLastError();
}

cudaError_t launch_probe(const float* f, const uint32_t* nbr, const uint32_t* nbr_nw, const Geom& g, int x, int y,
                         int z, float* out, cudaStream_t s) {
    probe_kernel<<<1, 1, 0, s>>>(f, nbr, nbr_nw, g, x, y, z, out);
    return cudaGetLastError();
}

}  // namespace lbmk
