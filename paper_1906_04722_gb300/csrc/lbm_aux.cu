// lbm_aux.cu -- per-domain set-up and read-out kernels: geometry words from the
// mask, the initial populations, the density field and the FP64 measurements.
#include "lbm_device.cuh"

namespace lbmk {

namespace {

__device__ __forceinline__ bool fluid_w(uint8_t m) { return !(m & LBM_MASK_SOLID); }
__device__ __forceinline__ bool fluid_nw(uint8_t m) { return !(m & (LBM_MASK_SOLID | LBM_MASK_MEMBRANE)); }

// Geometry words (layout in lbm_internal.h).  For every direction k the pull
// source x - e_k decides the bounce bit of each component; the neighbour
// x + e_k contributes 36 w_k e_k to the adhesion vector when it is grain.
// One thread per cell: x and y from the block and thread, z from blockIdx.z.
__global__ void __launch_bounds__(256) geometry_kernel(const uint8_t* __restrict__ mask, uint32_t* __restrict__ nbr,
                                                       uint32_t* __restrict__ nbr_nw, uint32_t* __restrict__ adh,
                                                       Geom g) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    {
        const long long c = (long long)z * g.nxy + (long long)y * g.nx + x;
        const uint8_t m = __ldg(mask + c);
        uint32_t cls;
        if (m & LBM_MASK_SOLID) cls = CLS_SOLID;
        else if (m & LBM_MASK_INLET) cls = CLS_INLET;
        else if (m & LBM_MASK_OUTLET) cls = CLS_OUTLET;
        else if (m & LBM_MASK_MEMBRANE) cls = CLS_MEMBRANE;
        else cls = CLS_FLUID;
        uint32_t bw = 0, bn = 0;
        int ax = 0, ay = 0, az = 0;
        for (int k = 1; k < Q; ++k) {
            bool ok = true;
            const int sx = wrap1(x - EX(k), g.nx, g.px, ok);
            const int sy = wrap1(y - EY(k), g.ny, g.py, ok);
            const int sz = wrap1(z - EZ(k), g.nz, g.pz, ok);
            if (!ok) {
                bw |= 1u << k;
                bn |= 1u << k;
            } else {
                const uint8_t ms = __ldg(mask + (long long)sz * g.nxy + (long long)sy * g.nx + sx);
                if (!fluid_w(ms)) bw |= 1u << k;
                if (!fluid_nw(ms)) bn |= 1u << k;
            }
            bool ok2 = true;
            const int tx = wrap1(x + EX(k), g.nx, g.px, ok2);
            const int ty = wrap1(y + EY(k), g.ny, g.py, ok2);
            const int tz = wrap1(z + EZ(k), g.nz, g.pz, ok2);
            if (ok2) {
                const uint8_t mt = __ldg(mask + (long long)tz * g.nxy + (long long)ty * g.nx + tx);
                if ((mt & LBM_MASK_SOLID) && (mt & LBM_MASK_ADHESIVE)) {
                    ax += W36(k) * EX(k);
                    ay += W36(k) * EY(k);
                    az += W36(k) * EZ(k);
                }
            }
        }
        uint32_t word = bw | (cls << CLS_SHIFT);
        if (bn != bw) word |= BIT_NW_DIFF;
        if (ax || ay || az) word |= BIT_ADH;
        nbr[c] = word;
        nbr_nw[c] = bn;
        adh[c] = (uint32_t)(uint8_t)(int8_t)ax | ((uint32_t)(uint8_t)(int8_t)ay << 8) |
                 ((uint32_t)(uint8_t)(int8_t)az << 16);
    }
}

// Stored populations whose pull yields the rest equilibrium w_k rho0(x) at every
// fluid cell: B_j(y) = w_j rho0(y + e_j) when y + e_j is fluid for the component
// (it pulls direction j from y), else w_j rho0(y) (y pulls jbar from itself).
__global__ void init_kernel(const float* __restrict__ rho0, float* __restrict__ f, const uint32_t* __restrict__ nbr,
                            const uint32_t* __restrict__ nbr_nw, Geom g) {
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)c;  // a domain holds fewer than 2^31 cells (lbm_create_domain)
        const int x = ci % g.nx;
        const int y = (ci / g.nx) % g.ny;
        const int z = ci / g.nxy;
        const uint32_t w = nbr[c];
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        for (int s = 0; s < 2; ++s) {
            const bool fl = cls != CLS_SOLID && !(s == 1 && cls == CLS_MEMBRANE);
            const uint32_t bits = s == 0 ? w : nbr_nw[c];
            const float* r = rho0 + (size_t)s * N;
            float* fs = f + (size_t)s * Q * g.plane;
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                float v = 0.f;
                if (fl && j == 0) {
                    // rest value closes the pulled sum on rho0 exactly (sum_j w_j != 1 in FP32)
                    float sum = 0.f;
#pragma unroll
                    for (int i = 1; i < Q; ++i) sum += WK(i) * r[c];
                    v = r[c] - sum;
                } else if (fl) {
                    if ((bits >> OPP(j)) & 1u) {
                        v = WK(j) * r[c];
                    } else {
                        bool ok = true;
                        const int tx = wrap1(x + EX(j), g.nx, g.px, ok);
                        const int ty = wrap1(y + EY(j), g.ny, g.py, ok);
                        const int tz = wrap1(z + EZ(j), g.nz, g.pz, ok);
                        v = WK(j) * r[(long long)tz * g.nxy + (long long)ty * g.nx + tx];
                    }
                }
                fs[(size_t)j * g.plane + c] = v;
            }
        }
    }
}

// rho_s(x, t) = sum_k f_k(x, t) of the pulled populations (Eq. 2).
__global__ void density_kernel(const float* __restrict__ f, float* __restrict__ rho, const uint32_t* __restrict__ nbr,
                               const uint32_t* __restrict__ nbr_nw, Geom g) {
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)c;  // a domain holds fewer than 2^31 cells (lbm_create_domain)
        const int x = ci % g.nx;
        const int y = (ci / g.nx) % g.ny;
        const int z = ci / g.nxy;
        Column col = make_column(x, y, g);
        float dummy[2][Q];
        float rw, rn;
        int cell;
        pull_cell<false>(f, nbr, nbr_nw, g, col, z, dummy, rw, rn, cell);
        rho[c] = rw;
        rho[N + c] = rn;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

constexpr int MEAS_THREADS = 256;

// Measurements of the current state (definitions in lbm.h), one FP64 partial
// per block; a second kernel adds the partials in block order.
__global__ void __launch_bounds__(MEAS_THREADS) measure_kernel(const float* __restrict__ f,
                                                               const uint32_t* __restrict__ nbr,
                                                               const uint32_t* __restrict__ nbr_nw, Geom g,
                                                               double G, double* __restrict__ partials) {
    double acc[NMEAS];
#pragma unroll
    for (int i = 0; i < NMEAS; ++i) acc[i] = 0.0;
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)c;  // a domain holds fewer than 2^31 cells (lbm_create_domain)
        const int x = ci % g.nx;
        const int y = (ci / g.nx) % g.ny;
        const int z = ci / g.nxy;
        Column col = make_column(x, y, g);
        float dummy[2][Q];
        float rwf, rnf;
        int cell;
        const uint32_t w = pull_cell<false>(f, nbr, nbr_nw, g, col, z, dummy, rwf, rnf, cell);
        measure_accumulate(acc, (w >> CLS_SHIFT) & CLS_MASK, (double)rwf, (double)rnf, G);
    }
    __shared__ double red[MEAS_THREADS / 32][NMEAS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NMEAS; ++i) {
        const double v = warp_sum(acc[i]);
        if (lane == 0) red[wid][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < NMEAS) {
        double v = 0.0;
        for (int wv = 0; wv < MEAS_THREADS / 32; ++wv) v += red[wv][threadIdx.x];
        partials[(size_t)blockIdx.x * NMEAS + threadIdx.x] = v;
    }
}

__global__ void finalize_kernel(const double* __restrict__ partials, int nblocks, double* __restrict__ result) {
    const int i = threadIdx.x;
    if (i < NMEAS) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += partials[(size_t)b * NMEAS + i];
        result[i] = v;
    }
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 16LL * device_sm_count();
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int device_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    return sms;
}

cudaError_t launch_geometry(const uint8_t* mask, uint32_t* nbr, uint32_t* nbr_nw, uint32_t* adh, const Geom& g,
                            cudaStream_t s) {
    const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    geometry_kernel<<<grid, dim3(32, 8), 0, s>>>(mask, nbr, nbr_nw, adh, g);
    return cudaGetLastError();
}

cudaError_t launch_init(const float* rho0, float* f, const uint32_t* nbr, const uint32_t* nbr_nw, const Geom& g,
                        cudaStream_t s) {
    const long long N = (long long)g.nxy * g.nz;
    init_kernel<<<grid_for(N, 256), 256, 0, s>>>(rho0, f, nbr, nbr_nw, g);
    return cudaGetLastError();
}

cudaError_t launch_density(const float* f, float* rho, const uint32_t* nbr, const uint32_t* nbr_nw, const Geom& g,
                           cudaStream_t s) {
    const long long N = (long long)g.nxy * g.nz;
    density_kernel<<<grid_for(N, 256), 256, 0, s>>>(f, rho, nbr, nbr_nw, g);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, int nblocks, double* result, cudaStream_t s) {
    finalize_kernel<<<1, 32, 0, s>>>(partials, nblocks, result);
    return cudaGetLastError();
}

int measure_blocks(const Geom& g) {
    const long long N = (long long)g.nxy * g.nz;
    long long b = (N + MEAS_THREADS * 8 - 1) / (MEAS_THREADS * 8);
    const long long cap = 8LL * device_sm_count();
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_measure(const float* f, const uint32_t* nbr, const uint32_t* nbr_nw, const Geom& g, double G,
                           double* partials, int nblocks, double* result, cudaStream_t s) {
    measure_kernel<<<nblocks, MEAS_THREADS, 0, s>>>(f, nbr, nbr_nw, g, G, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finalize_kernel<<<1, 32, 0, s>>>(partials, nblocks, result);
    return cudaGetLastError();
}

}  // namespace lbmk
