// lbm_noalloc.cu -- measurements of a caller-held state without any device
// allocation.
//
// lbm_measure pulls its per-block FP64 partial sums through scratch memory that
// lbm_create_domain allocated.  Some callers must not allocate device memory:
// plug-ins whose host application owns every device byte through its own pool
// (a framework's caching allocator that must account for all memory), and
// control loops that cannot afford the implicit device synchronisation of
// cudaMalloc/cudaFree.  They keep the populations in their own buffers and call
// lbm_measure_state_noalloc, which takes its scratch from the file-scope device
// array below instead.  The call still copies its 16 sums to the host and waits
// for its stream before it returns.
//
// The array is a fixed part of the library image: every GPU that loads the
// library holds it (MAX_BLOCKS x 16 doubles + 16 doubles, about 128 KiB) until
// the process exits.  All calls share it, so calls whose device work overlaps
// (on different streams or host threads) race on it.
#include "lbm_device.cuh"

namespace lbmk {

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 1024;
constexpr long long NA_MAX_CELLS = 56LL * 1000 * 1000;  // 32-bit population indices: 38 x N < 2^31

// Per-block partials followed by the final sums.  Every slot a call reads was
// written earlier by the same call, so nothing has to be cleared in between.
static __device__ __align__(256) double g_noalloc_scratch[(NA_MAX_BLOCKS + 1) * NMEAS];

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Fluid-ness of a pull source for component s, from its raw mask bits (as the
// geometry words decide bounce-back): solid stops both components, membrane
// stops the non-wetting one.
__device__ __forceinline__ bool na_fluid(uint8_t m, int s) {
    if (m & LBM_MASK_SOLID) return false;
    return !(s == 1 && (m & LBM_MASK_MEMBRANE));
}

// Class of a cell from its mask byte, in the priority order the geometry words
// use: solid, then inlet, outlet, membrane, fluid.
__device__ __forceinline__ uint32_t na_class(uint8_t m) {
    if (m & LBM_MASK_SOLID) return CLS_SOLID;
    if (m & LBM_MASK_INLET) return CLS_INLET;
    if (m & LBM_MASK_OUTLET) return CLS_OUTLET;
    if (m & LBM_MASK_MEMBRANE) return CLS_MEMBRANE;
    return CLS_FLUID;
}

// The measurements of lbm_measure, with bounce-back decided from the mask bytes
// of the pull sources instead of precomputed geometry words.  f is laid out
// f[(s*19 + k) * N + cell] (the checkpoint layout of lbm_get_state).
__global__ void __launch_bounds__(NA_THREADS) na_measure_kernel(const float* __restrict__ f,
                                                                const uint8_t* __restrict__ mask, Geom g, double G,
                                                                double* __restrict__ partials) {
    double acc[NMEAS];
#pragma unroll
    for (int i = 0; i < NMEAS; ++i) acc[i] = 0.0;
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const uint8_t m = mask[c];
        const uint32_t cls = na_class(m);
        if (cls == CLS_SOLID) continue;
        const int x = (int)(c % g.nx);
        const int y = (int)((c / g.nx) % g.ny);
        const int z = (int)(c / g.nxy);
        float rho[2] = {0.f, 0.f};
        for (int s = 0; s < 2; ++s) {
            // a membrane cell holds no non-wetting fluid; every other class holds both
            if (s == 1 && cls == CLS_MEMBRANE) continue;
            const float* fs = f + (size_t)s * Q * g.plane;
            float r = 0.f;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                bool ok = true;
                const int sx = wrap1(x - EX(k), g.nx, g.px, ok);
                const int sy = wrap1(y - EY(k), g.ny, g.py, ok);
                const int sz = wrap1(z - EZ(k), g.nz, g.pz, ok);
                long long src = -1;
                if (ok) {
                    src = (long long)sz * g.nxy + (long long)sy * g.nx + sx;
                    if (!na_fluid(mask[src], s)) src = -1;
                }
                r += src >= 0 ? fs[(size_t)k * g.plane + src] : fs[(size_t)OPP(k) * g.plane + c];
            }
            rho[s] = r;
        }
        // the same accumulation as lbm_measure
        measure_accumulate(acc, cls, (double)rho[0], (double)rho[1], G);
    }
    __shared__ double red[NA_THREADS / 32][NMEAS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NMEAS; ++i) {
        const double v = na_warp_sum(acc[i]);
        if (lane == 0) red[wid][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < NMEAS) {
        double v = 0.0;
        for (int wv = 0; wv < NA_THREADS / 32; ++wv) v += red[wv][threadIdx.x];
        partials[(size_t)blockIdx.x * NMEAS + threadIdx.x] = v;
    }
}

__global__ void na_finalize_kernel(const double* __restrict__ partials, int nblocks, double* __restrict__ result) {
    const int i = threadIdx.x;
    if (i < NMEAS) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += partials[(size_t)b * NMEAS + i];
        result[i] = v;
    }
}

// Device address of g_noalloc_scratch on the current device.  The host-side
// name of the array is only a stand-in; its device address is looked up on
// every call (a lookup in the loaded module, no allocation), so that a module
// reloaded into a new context is never reached through a stale address.
int scratch_address(double** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    *out = static_cast<double*>(p);
    return LBM_OK;
}

}  // namespace

}  // namespace lbmk

using namespace lbmk;

extern "C" int lbm_measure_state_noalloc(const lbm_params* params, const int box[3], const float* f_dev,
                                         const unsigned char* mask_dev, void* stream, lbm_measurement* out) {
    if (!params || !box || !f_dev || !mask_dev || !out) {
        set_error("lbm_measure_state_noalloc: a pointer argument is NULL");
        return LBM_ERR_ARG;
    }
    for (int d = 0; d < 3; ++d)
        if (box[d] < 1 || box[d] > 4096) {
            set_error("lbm_measure_state_noalloc: box sizes must be in [1, 4096]");
            return LBM_ERR_ARG;
        }
    const long long N = (long long)box[0] * box[1] * box[2];
    if (N > NA_MAX_CELLS) {
        set_error("lbm_measure_state_noalloc: the state exceeds the 56,000,000-cell maximum of this entry point");
        return LBM_ERR_ARG;
    }
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    Geom g;
    g.nx = box[0];
    g.ny = box[1];
    g.nz = box[2];
    g.nxy = box[0] * box[1];
    g.plane = (int)N;
    g.px = params->periodic[0] ? 1 : 0;
    g.py = params->periodic[1] ? 1 : 0;
    g.pz = params->periodic[2] ? 1 : 0;
    fill_pull_offsets(g);
    long long nb = (N + NA_THREADS * 8 - 1) / (NA_THREADS * 8);
    if (nb > NA_MAX_BLOCKS) nb = NA_MAX_BLOCKS;
    if (nb < 1) nb = 1;
    cudaStream_t s = (cudaStream_t)stream;
    double* partials = scratch;
    double* result = scratch + (size_t)NA_MAX_BLOCKS * NMEAS;
    na_measure_kernel<<<(int)nb, NA_THREADS, 0, s>>>(f_dev, mask_dev, g, params->G, partials);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        na_finalize_kernel<<<1, 32, 0, s>>>(partials, (int)nb, result);
        e = cudaGetLastError();
    }
    double r[NMEAS];
    if (e == cudaSuccess) e = cudaMemcpyAsync(r, result, sizeof(r), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error(std::string("lbm_measure_state_noalloc: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    *out = lbm_measurement{};
    out->mass[0] = r[MS_MASS_W];
    out->mass[1] = r[MS_MASS_NW];
    out->n_fluid = (long long)r[MS_N_FLUID];
    out->n_w = (long long)r[MS_N_W];
    out->n_interface = (long long)r[MS_N_INTERFACE];
    out->n_bulk_w = (long long)r[MS_N_BULK_W];
    out->n_bulk_nw = (long long)r[MS_N_BULK_NW];
    out->n_in = (long long)r[MS_N_IN];
    out->n_out = (long long)r[MS_N_OUT];
    out->n_nonfinite = (long long)r[MS_N_NONFINITE];
    out->n_negative = (long long)r[MS_N_NEGATIVE];
    out->p_w = out->n_bulk_w ? r[MS_PW] / (double)out->n_bulk_w : NAN;
    out->p_nw = out->n_bulk_nw ? r[MS_PNW] / (double)out->n_bulk_nw : NAN;
    out->p_c = out->p_nw - out->p_w;
    out->p_in = out->n_in ? r[MS_PIN] / (double)out->n_in : NAN;
    out->p_out = out->n_out ? r[MS_POUT] / (double)out->n_out : NAN;
    out->p_c_res = out->p_in - out->p_out;
    out->S_w = out->n_fluid ? (double)out->n_w / (double)out->n_fluid : NAN;
    out->status_flags = (out->n_nonfinite ? 1 : 0) | (out->n_negative ? 2 : 0);
    if (out->status_flags) {
        set_error("non-finite or negative densities in the state");
        return LBM_ERR_NONFINITE;
    }
    return LBM_OK;
}
