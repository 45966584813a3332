// lbm_noalloc.cu -- measurements of a caller-held state without any device
// allocation.
//
// lbm_measure pulls its per-block FP64 partial sums through scratch memory that
// lbm_create_domain allocated.  Some callers cannot allocate device memory at
// all: code running while a stream is being captured, plug-ins whose host
// application owns every device byte through its own pool (a framework's
// caching allocator that must account for all memory), or control loops that
// cannot afford the implicit device synchronisation of cudaMalloc/cudaFree.
// They keep the populations in their own buffers and call
// lbm_measure_state_noalloc, which takes its scratch from the file-scope
// device array below instead.
//
// The array is a fixed part of the library image: every GPU that loads the
// library holds it (MAX_BLOCKS x 16 doubles + 16 doubles, about 128 KiB) until
// the process exits.  All calls share it, so calls whose device work overlaps
// (on different streams or host threads) race on it.
#include <mutex>

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

__device__ __forceinline__ bool na_fluid(uint8_t m, int s) {
    if (m & LBM_MASK_SOLID) return false;
    return !(s == 1 && (m & LBM_MASK_MEMBRANE));
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
        if (m & LBM_MASK_SOLID) continue;
        const int x = (int)(c % g.nx);
        const int y = (int)((c / g.nx) % g.ny);
        const int z = (int)(c / g.nxy);
        float rho[2] = {0.f, 0.f};
        for (int s = 0; s < 2; ++s) {
            if (!na_fluid(m, s)) continue;
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
        const double rw = rho[0], rn = rho[1];
        acc[MS_MASS_W] += rw;
        if (!isfinite(rw)) acc[MS_N_NONFINITE] += 1.0;
        else if (rw < 0.0) acc[MS_N_NEGATIVE] += 1.0;
        if (!(m & LBM_MASK_MEMBRANE)) {
            acc[MS_MASS_NW] += rn;
            if (!isfinite(rn)) acc[MS_N_NONFINITE] += 1.0;
            else if (rn < 0.0) acc[MS_N_NEGATIVE] += 1.0;
        }
        const double p = (rw + rn) / 3.0 + G * rw * rn / 3.0;  // Eq. 5
        if (m & LBM_MASK_INLET) { acc[MS_PIN] += p; acc[MS_N_IN] += 1.0; continue; }
        if (m & LBM_MASK_OUTLET) { acc[MS_POUT] += p; acc[MS_N_OUT] += 1.0; continue; }
        if (m & LBM_MASK_MEMBRANE) continue;
        acc[MS_N_FLUID] += 1.0;
        if (rw > rn) acc[MS_N_W] += 1.0;
        const double phi = (rw - rn) / (rw + rn);
        if (fabs(phi) < 0.5) acc[MS_N_INTERFACE] += 1.0;
        if (phi > 0.9) { acc[MS_PW] += p; acc[MS_N_BULK_W] += 1.0; }
        if (phi < -0.9) { acc[MS_PNW] += p; acc[MS_N_BULK_NW] += 1.0; }
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

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (the host-side name of the array is only a stand-in).
std::mutex g_na_mutex;
double* g_na_ptr[64] = {};

int scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    if (dev < 0 || dev >= 64) {
        set_error("lbm_measure_state_noalloc supports devices 0..63");
        return LBM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            return LBM_ERR_CUDA;
        }
        g_na_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_na_ptr[dev];
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
