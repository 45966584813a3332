// lbm_api.cu -- the extern "C" entry points declared in include/lbm.h.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "lbm_internal.h"

namespace lbmk {

namespace {
thread_local std::string g_error;

// Rounds n up to a multiple of 32 floats so that every population plane starts
// on a 128-byte boundary.
long long plane_stride(long long n) { return (n + 31) / 32 * 32; }

#define LBM_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                \
            return e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;          \
        }                                                                                 \
    } while (0)

int check_params(const lbm_params* p) {
    if (!p) { set_error("params is NULL"); return LBM_ERR_ARG; }
    for (int s = 0; s < 2; ++s)
        if (!(p->tau[s] > 0.5) || !std::isfinite(p->tau[s])) { set_error("tau must be finite and > 0.5"); return LBM_ERR_ARG; }
    if (!std::isfinite(p->G) || !std::isfinite(p->G_ads[0]) || !std::isfinite(p->G_ads[1])) {
        set_error("G and G_ads must be finite");
        return LBM_ERR_ARG;
    }
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(p->body_force[d])) { set_error("body_force must be finite"); return LBM_ERR_ARG; }
    if (!(p->rho_major > 0) || !(p->rho_minor >= 0) || !std::isfinite(p->rho_major) || !std::isfinite(p->rho_minor)) {
        set_error("rho_major must be > 0 and rho_minor >= 0");
        return LBM_ERR_ARG;
    }
    if (p->precision < 0 || p->precision > 2) {
        set_error("precision must be 0 (FP32), 1 (FP16 deviations) or 2 (BF16 deviations)");
        return LBM_ERR_ARG;
    }
    if (p->membrane_layers < 0) { set_error("membrane_layers must be >= 0"); return LBM_ERR_ARG; }
    return LBM_OK;
}

int check_box(const int box[3]) {
    if (!box) { set_error("box is NULL"); return LBM_ERR_ARG; }
    for (int d = 0; d < 3; ++d)
        if (box[d] < 1 || box[d] > 4096) { set_error("box sizes must be in [1, 4096]"); return LBM_ERR_ARG; }
    const long long N = (long long)box[0] * box[1] * box[2];
    // population indices are 32-bit: 2 * 19 planes must stay below 2^31 entries
    if (plane_stride(N) * 2 * Q >= (1LL << 31)) {
        set_error("domain too large for one launch (at most ~56 million cells)");
        return LBM_ERR_ARG;
    }
    return LBM_OK;
}

void fill_phys(lbm_domain* d) {
    const lbm_params& p = d->params;
    Phys& ph = d->phys;
    for (int s = 0; s < 2; ++s) {
        ph.tau[s] = (float)p.tau[s];
        ph.omega[s] = (float)(1.0 / p.tau[s]);
        ph.Gads[s] = (float)p.G_ads[s];
    }
    ph.G = (float)p.G;
    for (int k = 0; k < 3; ++k) ph.g[k] = (float)p.body_force[k];
    ph.bc = d->d_bc;
}

// Queue the reservoir densities (inlet: rho_minor / rho_in_nw, outlet:
// rho_out_w / rho_minor) on the domain's stream.
int set_bc(lbm_domain* d, double rho_in_nw, double rho_out_w) {
    d->bc_host[0] = d->params.rho_minor;
    d->bc_host[1] = rho_in_nw;
    d->bc_host[2] = rho_out_w;
    d->bc_host[3] = d->params.rho_minor;
    LBM_CUDA(launch_set_bc(d->d_bc, (float)d->bc_host[0], (float)d->bc_host[1], (float)d->bc_host[2],
                           (float)d->bc_host[3], d->stream));
    return LBM_OK;
}

void drop_graphs(lbm_domain* d) {
    for (int i = 0; i < 2; ++i)
        if (d->graph[i]) {
            cudaGraphExecDestroy(d->graph[i]);
            d->graph[i] = nullptr;
        }
}

// One step from buffer `cur` to buffer cur ^ 1 on stream s.
cudaError_t launch_one(lbm_domain* d, int cur, cudaStream_t s) {
    if (d->params.precision != 0 && d->tile.kind == LBM_KERNEL_PUSH)
        return launch_step16_push(d->params.precision, d->tile.push_shape, d->push16_w[cur], d->push16_r[cur],
                                  reinterpret_cast<uint32_t*>(d->f[cur ^ 1]), d->R[cur ^ 1], d->d_nbr, d->d_nbr_nw,
                                  d->d_adh, d->geom, d->phys, d->tile.push_lz, d->d_err, s);
    if (d->params.precision == 0 && d->tile.kind == LBM_KERNEL_PUSH)
        return launch_step_push(d->tile.push_shape, d->push_maps[cur], d->f[cur ^ 1], d->d_nbr, d->d_nbr_nw, d->d_adh,
                                d->geom, d->phys, d->tile.push_lz, d->tile.push_pf, d->tile.push_order, d->d_err, s);
    if (d->params.precision == 0 && d->tile.kind == LBM_KERNEL_TMA)
        return launch_step_tma(d->tma, cur, d->f[cur], d->f[cur ^ 1], d->d_nbr_nw, d->d_adh, d->geom, d->phys,
                               d->tile.tma_lz, d->d_err, s);
    if (d->params.precision == 0 && d->tile.kind == LBM_KERNEL_STAGED2)
        return launch_step2(d->f[cur], d->f[cur ^ 1], d->d_nbr, d->d_nbr_nw, d->d_adh, d->geom, d->phys, d->tile, s);
    if (d->params.precision == 0 && d->tile.kind == LBM_KERNEL_SPLIT)
        return launch_step_split(d->f[cur], d->f[cur ^ 1], d->d_rho2, d->d_nbr, d->d_nbr_nw, d->d_adh, d->geom,
                                 d->phys, s);
    if (d->params.precision == 0)
        return launch_step(d->f[cur], d->f[cur ^ 1], d->d_nbr, d->d_nbr_nw, d->d_adh, d->geom, d->phys, d->tile, s);
    return launch_step16(d->params.precision, reinterpret_cast<const uint32_t*>(d->f[cur]),
                         reinterpret_cast<uint32_t*>(d->f[cur ^ 1]), d->R[cur], d->R[cur ^ 1], d->d_nbr, d->d_nbr_nw,
                         d->d_adh, d->geom, d->phys, d->tile, s);
}

cudaError_t prepare_one(lbm_domain* d) {
    if (d->params.precision != 0 && d->tile.kind == LBM_KERNEL_PUSH)
        return prepare_step16_push(d->params.precision, d->tile.push_shape);
    if (d->params.precision == 0 && d->tile.kind == LBM_KERNEL_PUSH) return prepare_step_push(d->tile.push_shape);
    if (d->params.precision == 0 && d->tile.kind == LBM_KERNEL_TMA) return prepare_step_tma();
    if (d->params.precision == 0 && d->tile.kind == LBM_KERNEL_SPLIT) return cudaSuccess;
    if (d->params.precision == 0 && d->tile.kind == LBM_KERNEL_STAGED2) return prepare_step2(d->tile);
    return d->params.precision == 0 ? prepare_step(d->tile) : prepare_step16(d->params.precision, d->tile);
}

// The layout the current kernel kind steps on: the push kernels keep the state
// in the push layout (FP32: paired; 16-bit: the pull words, each at its reader),
// every other kernel in the pull layout.
int wanted_layout(const lbm_domain* d) { return d->tile.kind == LBM_KERNEL_PUSH ? 1 : 0; }

// Converts the state into the given layout (into the other buffer, which then
// becomes the current one).  The step counter is unchanged.
int set_layout(lbm_domain* d, int layout) {
    if (d->layout == layout) return LBM_OK;
    if (d->params.precision != 0) {
        const uint32_t* in = reinterpret_cast<const uint32_t*>(d->f[d->cur]);
        uint32_t* out = reinterpret_cast<uint32_t*>(d->f[d->cur ^ 1]);
        if (layout == 1) LBM_CUDA(launch_pull16_to_push16(in, out, d->d_nbr, d->d_nbr_nw, d->geom, d->stream));
        else LBM_CUDA(launch_push16_to_pull16(in, out, d->d_nbr, d->d_nbr_nw, d->geom, d->stream));
        // the density pairs go with the words
        LBM_CUDA(cudaMemcpyAsync(d->R[d->cur ^ 1], d->R[d->cur], sizeof(float2) * (size_t)d->geom.plane,
                                 cudaMemcpyDeviceToDevice, d->stream));
        d->cur ^= 1;
        d->layout = layout;
        return LBM_OK;
    }
    if (layout == 1)
        LBM_CUDA(launch_pull_to_push(d->f[d->cur], d->f[d->cur ^ 1], d->d_nbr, d->d_nbr_nw, d->geom, d->stream));
    else
        LBM_CUDA(launch_push_to_pull(d->f[d->cur], d->f[d->cur ^ 1], d->d_nbr, d->d_nbr_nw, d->geom, d->stream));
    d->cur ^= 1;
    d->layout = layout;
    d->ghosts_ok = false;
    return LBM_OK;
}

// The current FP32 state in the pull layout, for the read-out kernels: f[cur]
// itself, or (paired push layout) its conversion into the other buffer, which
// the next step overwrites anyway.
int pull_view(lbm_domain* d, const float** out) {
    if (d->layout == 0) {
        *out = d->f[d->cur];
        return LBM_OK;
    }
    LBM_CUDA(launch_push_to_pull(d->f[d->cur], d->f[d->cur ^ 1], d->d_nbr, d->d_nbr_nw, d->geom, d->stream));
    *out = d->f[d->cur ^ 1];
    return LBM_OK;
}

// The current 16-bit words in the pull layout, for the read-out kernels: f[cur]
// itself, or (push layout) their conversion into the other buffer, which the
// next step overwrites anyway.  The density pairs are R[cur] either way.
int pull16_view(lbm_domain* d, const uint32_t** out) {
    const uint32_t* in = reinterpret_cast<const uint32_t*>(d->f[d->cur]);
    if (d->layout == 0) {
        *out = in;
        return LBM_OK;
    }
    uint32_t* o = reinterpret_cast<uint32_t*>(d->f[d->cur ^ 1]);
    LBM_CUDA(launch_push16_to_pull16(in, o, d->d_nbr, d->d_nbr_nw, d->geom, d->stream));
    *out = o;
    return LBM_OK;
}

// Tensor maps of the 16-bit words and density pairs of both buffers for the
// 16-bit push kernel's current shape.
int ensure_push16_maps(lbm_domain* d) {
    const int rows = push16_shape_rows(d->tile.push_shape);
    if (d->push16_maps_rows == rows) return LBM_OK;
    cudaError_t e = encode_push16_maps(d->geom, reinterpret_cast<uint32_t*>(d->f[0]),
                                       reinterpret_cast<uint32_t*>(d->f[1]), d->R[0], d->R[1], rows, d->push16_w,
                                       d->push16_r);
    if (e != cudaSuccess) {
        d->push16_maps_rows = 0;
        set_error(std::string("tensor maps of the 16-bit push kernel: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    d->push16_maps_rows = rows;
    return LBM_OK;
}

// Tensor maps of both buffers for the push kernel's current shape.
int ensure_push_maps(lbm_domain* d) {
    const int rows = push_shape_rows(d->tile.push_shape);
    if (d->push_maps_rows == rows) return LBM_OK;
    cudaError_t e = encode_push_maps(d->geom, d->f[0], d->f[1], rows, d->push_maps);
    if (e != cudaSuccess) {
        d->push_maps_rows = 0;
        set_error(std::string("tensor maps of the push kernel: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    d->push_maps_rows = rows;
    return LBM_OK;
}

// Capture GRAPH_STEPS step launches that start from buffer `parity` on the
// domain's private capture stream; the graph is launched on the domain's stream.
int capture_graph(lbm_domain* d, int parity) {
    LBM_CUDA(prepare_one(d));
    if (!d->capture_stream) LBM_CUDA(cudaStreamCreateWithFlags(&d->capture_stream, cudaStreamNonBlocking));
    LBM_CUDA(cudaStreamBeginCapture(d->capture_stream, cudaStreamCaptureModeThreadLocal));
    int cur = parity;
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < GRAPH_STEPS && err == cudaSuccess; ++i) {
        err = launch_one(d, cur, d->capture_stream);
        cur ^= 1;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t end = cudaStreamEndCapture(d->capture_stream, &graph);
    if (err != cudaSuccess || end != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        set_error(std::string("graph capture of the step failed: ") +
                  cudaGetErrorString(err != cudaSuccess ? err : end));
        return LBM_ERR_CUDA;
    }
    cudaError_t inst = cudaGraphInstantiate(&d->graph[parity], graph, 0);
    cudaGraphDestroy(graph);
    if (inst != cudaSuccess) {
        d->graph[parity] = nullptr;
        set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(inst));
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

// n steps: whole chunks replay a captured graph, the remainder is launched one by one.
int run_steps(lbm_domain* d, int n) {
    if (n <= 0) return LBM_OK;
    if (int rc = set_layout(d, wanted_layout(d))) return rc;
    if (d->tile.kind == LBM_KERNEL_PUSH) {
        if (int rc = d->params.precision == 0 ? ensure_push_maps(d) : ensure_push16_maps(d)) return rc;
        d->tma_pending = true;  // the push kernels report a wait that ran out through d_err
    }
    const bool tma = d->params.precision == 0 && d->tile.kind == LBM_KERNEL_TMA;
    if (tma && !d->ghosts_ok) {
        LBM_CUDA(launch_ghost_fill(d->f[d->cur], d->d_nbr, d->d_nbr_nw, d->geom, d->stream));
        d->ghosts_ok = true;
    }
    if (!tma) d->ghosts_ok = false;
    if (tma) d->tma_pending = true;
    while (n >= GRAPH_STEPS) {
        if (!d->graph[d->cur]) {
            int rc = capture_graph(d, d->cur);
            if (rc) return rc;
        }
        LBM_CUDA(cudaGraphLaunch(d->graph[d->cur], d->stream));
        d->step += GRAPH_STEPS;
        n -= GRAPH_STEPS;
    }
    for (int i = 0; i < n; ++i) {
        LBM_CUDA(prepare_one(d));
        LBM_CUDA(launch_one(d, d->cur, d->stream));
        d->cur ^= 1;
        ++d->step;
    }
    return LBM_OK;
}

void free_domain(lbm_domain* d) {
    if (!d) return;
    cudaFree(d->f[0]);
    cudaFree(d->f[1]);
    cudaFree(d->R[0]);
    cudaFree(d->R[1]);
    cudaFree(d->d_mask);
    cudaFree(d->d_nbr);
    cudaFree(d->d_nbr_nw);
    cudaFree(d->d_adh);
    cudaFree(d->d_rho);
    cudaFree(d->d_partials);
    cudaFree(d->d_result);
    cudaFree(d->d_bc);
    cudaFree(d->d_probe);
    cudaFree(d->d_err);
    if (d->h_err) cudaFreeHost(d->h_err);
    cudaFree(d->d_rho2);
    drop_graphs(d);
    if (d->capture_stream) cudaStreamDestroy(d->capture_stream);
    if (d->h_result) cudaFreeHost(d->h_result);
    if (d->done) cudaEventDestroy(d->done);
    delete d;
}

// Bounded wait for the domain's queued work: polls an event for up to 60 s.
int wait_domain(lbm_domain* d) {
    // a TMA step kernel whose bounded wait for its loads ran out leaves a flag:
    // read it on the domain's stream, behind the work being waited for
    const bool check = d->tma_pending;
    if (check) LBM_CUDA(cudaMemcpyAsync(d->h_err, d->d_err, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
    LBM_CUDA(cudaEventRecord(d->done, d->stream));
    const auto t0 = std::chrono::steady_clock::now();
    while (true) {
        cudaError_t e = cudaEventQuery(d->done);
        if (e == cudaSuccess) {
            if (check) {
                d->tma_pending = false;
                if (*d->h_err) {
                    *d->h_err = 0;
                    LBM_CUDA(cudaMemsetAsync(d->d_err, 0, sizeof(int), d->stream));
                    set_error("a step kernel gave up waiting for its population loads");
                    return LBM_ERR_TIMEOUT;
                }
            }
            return LBM_OK;
        }
        if (e != cudaErrorNotReady) {
            set_error(std::string("device work failed: ") + cudaGetErrorString(e));
            return LBM_ERR_CUDA;
        }
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60)) {
            set_error("device work did not finish within 60 s");
            return LBM_ERR_TIMEOUT;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// The default initial densities (2 x N floats): wetting fluid everywhere, the
// non-wetting reservoir on the inlet layer, from the mask on the device.
__global__ void rest_density_kernel(const uint8_t* __restrict__ mask, float* __restrict__ rho, long long N,
                                    float rho_major, float rho_minor) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const bool inlet = mask[c] & LBM_MASK_INLET;
        rho[c] = inlet ? rho_minor : rho_major;
        rho[N + c] = inlet ? rho_major : rho_minor;
    }
}

// Build the stored populations from the densities in d->d_rho.
int init_from_densities(lbm_domain* d) {
    if (d->params.precision == 0) {
        LBM_CUDA(launch_init(d->d_rho, d->f[0], d->d_nbr, d->d_nbr_nw, d->geom, d->stream));
    } else {
        LBM_CUDA(cudaMemsetAsync(d->f[0], 0, sizeof(uint32_t) * (size_t)d->geom.plane * Q, d->stream));
        LBM_CUDA(launch_init16(d->d_rho, d->R[0], d->geom, d->stream));
    }
    d->cur = 0;
    d->step = 0;
    d->ghosts_ok = false;
    d->layout = 0;
    return wait_domain(d);
}

// Upload rest-equilibrium densities (host doubles, 2 x N) and build the stored
// populations from them.
int upload_densities(lbm_domain* d, const double* rho) {
    const long long N = d->N;
    std::vector<float> tmp((size_t)(2 * N));
    for (long long i = 0; i < 2 * N; ++i) tmp[(size_t)i] = (float)rho[i];
    LBM_CUDA(cudaMemcpyAsync(d->d_rho, tmp.data(), sizeof(float) * 2 * N, cudaMemcpyHostToDevice, d->stream));
    return init_from_densities(d);
}

int create_common(const lbm_params* params, const uint8_t* mask_host, const int box[3], void* stream,
                  lbm_domain** out) {
    lbm_domain* d = new (std::nothrow) lbm_domain();
    if (!d) { set_error("host allocation failed"); return LBM_ERR_OOM; }
    std::memset(d, 0, sizeof(*d));
    d->params = *params;
    d->stream = (cudaStream_t)stream;
    Geom& g = d->geom;
    g.nx = box[0];
    g.ny = box[1];
    g.nz = box[2];
    g.nxy = box[0] * box[1];
    d->N = (long long)g.nxy * g.nz;
    g.plane = (int)plane_stride(d->N);
    g.px = params->periodic[0] ? 1 : 0;
    g.py = params->periodic[1] ? 1 : 0;
    g.pz = params->periodic[2] ? 1 : 0;
    fill_pull_offsets(g);
    d->tile = default_tile(g);
    // FP32: shape 1 (6 rows, 3 stages, two CTAs per SM); 16-bit: shape 0 (8 rows, 4 stages)
    d->tile.push_shape = params->precision == 0 ? 1 : 0;
    d->tile.push_lz = params->precision == 0 ? push_default_lz(g, 1) : push16_default_lz(g, 0);
    d->tile.push_pf = 0;
    d->tile.push_order = 0;
    d->layout = 0;
    d->push_maps_rows = 0;
    d->push16_maps_rows = 0;

    auto fail = [&](int rc) { free_domain(d); return rc; };
#define LBM_CUDA_D(call)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA);    \
        }                                                                                 \
    } while (0)
    // FP32: 2 x 19 floats per cell; 16-bit: 19 pair words per cell plus the density pair
    const size_t fbytes = (params->precision == 0 ? sizeof(float) * 2 : sizeof(uint32_t)) * (size_t)g.plane * Q;
    LBM_CUDA_D(cudaEventCreateWithFlags(&d->done, cudaEventDisableTiming));
    LBM_CUDA_D(cudaMalloc(&d->f[0], fbytes));
    LBM_CUDA_D(cudaMalloc(&d->f[1], fbytes));
    if (params->precision != 0) {
        LBM_CUDA_D(cudaMalloc(&d->R[0], sizeof(float2) * (size_t)g.plane));
        LBM_CUDA_D(cudaMalloc(&d->R[1], sizeof(float2) * (size_t)g.plane));
        LBM_CUDA_D(cudaMemsetAsync(d->R[0], 0, sizeof(float2) * (size_t)g.plane, d->stream));
        LBM_CUDA_D(cudaMemsetAsync(d->R[1], 0, sizeof(float2) * (size_t)g.plane, d->stream));
    }
    LBM_CUDA_D(cudaMalloc(&d->d_mask, (size_t)d->N));
    LBM_CUDA_D(cudaMalloc(&d->d_nbr, sizeof(uint32_t) * (size_t)d->N));
    LBM_CUDA_D(cudaMalloc(&d->d_nbr_nw, sizeof(uint32_t) * (size_t)d->N));
    LBM_CUDA_D(cudaMalloc(&d->d_adh, sizeof(uint32_t) * (size_t)d->N));
    LBM_CUDA_D(cudaMalloc(&d->d_rho, sizeof(float) * 2 * (size_t)d->N));
    d->meas_blocks = measure_blocks(g);
    LBM_CUDA_D(cudaMalloc(&d->d_partials, sizeof(double) * NMEAS * (size_t)d->meas_blocks));
    LBM_CUDA_D(cudaMalloc(&d->d_result, sizeof(double) * NMEAS));
    LBM_CUDA_D(cudaMallocHost(&d->h_result, sizeof(double) * NMEAS));
    LBM_CUDA_D(cudaMalloc(&d->d_bc, sizeof(float) * 4));
    LBM_CUDA_D(cudaMalloc(&d->d_probe, sizeof(float) * 2));
    LBM_CUDA_D(cudaMalloc(&d->d_err, sizeof(int)));
    LBM_CUDA_D(cudaMallocHost(&d->h_err, sizeof(int)));
    *d->h_err = 0;
    if (params->precision == 0) LBM_CUDA_D(cudaMalloc(&d->d_rho2, sizeof(float2) * (size_t)d->N));
    LBM_CUDA_D(cudaMemsetAsync(d->d_err, 0, sizeof(int), d->stream));
    fill_phys(d);
    if (int rc = set_bc(d, params->rho_major, params->rho_major)) return fail(rc);
    // the untouched planes between N and the plane stride stay zero
    LBM_CUDA_D(cudaMemsetAsync(d->f[0], 0, fbytes, d->stream));
    LBM_CUDA_D(cudaMemsetAsync(d->f[1], 0, fbytes, d->stream));
    LBM_CUDA_D(cudaMemcpyAsync(d->d_mask, mask_host, (size_t)d->N, cudaMemcpyHostToDevice, d->stream));
    LBM_CUDA_D(launch_geometry(d->d_mask, d->d_nbr, d->d_nbr_nw, d->d_adh, g, d->stream));
#undef LBM_CUDA_D
    // FP32 boxes the TMA kernel can serve get its tensor maps; the staged kernel
    // stays the default (lbm_set_step_kernel and lbm_autotune select the other)
    if (params->precision == 0 && tma_step_applicable(g) &&
        encode_step_maps(g, d->f[0], d->f[1], d->d_nbr, d->tma) == cudaSuccess) {
        d->tma_ok = true;
        d->tile.tma_lz = tma_default_lz(g);
    }
    long long nf = 0;
    for (long long c = 0; c < d->N; ++c)
        if (mask_host[c] == 0) ++nf;
    d->n_fluid = nf;

    // default initial state: wetting fluid everywhere, non-wetting reservoir on the inlet layer
    rest_density_kernel<<<1216, 256, 0, d->stream>>>(d->d_mask, d->d_rho, d->N, (float)params->rho_major,
                                                     (float)params->rho_minor);
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) {
        set_error(std::string("rest_density_kernel: ") + cudaGetErrorString(e));
        return fail(LBM_ERR_CUDA);
    }
    int rc = init_from_densities(d);
    if (rc != LBM_OK) return fail(rc);
    *out = d;
    return LBM_OK;
}

}  // namespace

void set_error(const std::string& msg) { g_error = msg; }

}  // namespace lbmk

using namespace lbmk;

extern "C" {

int lbm_create_domain(const lbm_params* params, const double* spheres, int n_spheres, const int box[3],
                      void* stream, lbm_domain** out) {
    try {
        int rc = check_params(params);
        if (rc) return rc;
        rc = check_box(box);
        if (rc) return rc;
        if (!out) { set_error("out is NULL"); return LBM_ERR_ARG; }
        if (n_spheres < 0 || (n_spheres > 0 && !spheres)) { set_error("bad sphere list"); return LBM_ERR_ARG; }
        for (int i = 0; i < n_spheres; ++i)
            for (int k = 0; k < 4; ++k)
                if (!std::isfinite(spheres[4 * i + k]) || (k == 3 && spheres[4 * i + k] < 0)) {
                    set_error("sphere entries must be finite with r >= 0");
                    return LBM_ERR_ARG;
                }
        if (params->prism_clip && n_spheres < 3) { set_error("prism_clip needs three spheres"); return LBM_ERR_ARG; }
        const long long N = (long long)box[0] * box[1] * box[2];
        std::vector<uint8_t> mask((size_t)N);
        voxelise_box(box[0], box[1], box[2], spheres, n_spheres, params->prism_clip, params->reservoirs,
                     params->membrane_layers, mask.data());
        return create_common(params, mask.data(), box, stream, out);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    } catch (...) {
        set_error("unexpected host exception");
        return LBM_ERR_ARG;
    }
}

int lbm_create_domain_mask(const lbm_params* params, const unsigned char* mask, const int box[3], void* stream,
                           lbm_domain** out) {
    try {
        int rc = check_params(params);
        if (rc) return rc;
        rc = check_box(box);
        if (rc) return rc;
        if (!out || !mask) { set_error("mask or out is NULL"); return LBM_ERR_ARG; }
        return create_common(params, mask, box, stream, out);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    } catch (...) {
        set_error("unexpected host exception");
        return LBM_ERR_ARG;
    }
}

int lbm_set_densities(lbm_domain* d, const double* rho) {
    if (!d || !rho) { set_error("domain or rho is NULL"); return LBM_ERR_ARG; }
    try {
        return upload_densities(d, rho);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
}

int lbm_set_pressure_bc(lbm_domain* d, double rho_in_nw, double rho_out_w) {
    if (!d) { set_error("domain is NULL"); return LBM_ERR_ARG; }
    if (!std::isfinite(rho_in_nw) || !std::isfinite(rho_out_w) || rho_in_nw < 0 || rho_out_w < 0) {
        set_error("reservoir densities must be finite and >= 0");
        return LBM_ERR_ARG;
    }
    return set_bc(d, rho_in_nw, rho_out_w);
}

int lbm_step(lbm_domain* d, int n_steps) {
    if (!d || n_steps < 0) { set_error("domain is NULL or n_steps < 0"); return LBM_ERR_ARG; }
    return run_steps(d, n_steps);
}

int lbm_get_density_at(lbm_domain* d, int x, int y, int z, double rho_out[2]) {
    if (!d || !rho_out) { set_error("domain or rho_out is NULL"); return LBM_ERR_ARG; }
    if (x < 0 || y < 0 || z < 0 || x >= d->geom.nx || y >= d->geom.ny || z >= d->geom.nz) {
        set_error("probe cell outside the box");
        return LBM_ERR_ARG;
    }
    if (d->params.precision == 0 && d->layout == 1) {
        LBM_CUDA(launch_probe_push(d->f[d->cur], d->d_nbr, d->geom, x, y, z, d->d_probe, d->stream));
    } else if (d->params.precision == 0) {
        LBM_CUDA(launch_probe(d->f[d->cur], d->d_nbr, d->d_nbr_nw, d->geom, x, y, z, d->d_probe, d->stream));
    }
    else {
        const uint32_t* w16 = nullptr;
        if (int rc = pull16_view(d, &w16)) return rc;
        LBM_CUDA(launch_probe16(d->params.precision, w16, d->R[d->cur],
                                d->d_nbr, d->d_nbr_nw, d->geom, x, y, z, d->d_probe, d->stream));
    }
    LBM_CUDA(cudaMemcpyAsync(d->h_result, d->d_probe, sizeof(float) * 2, cudaMemcpyDeviceToHost, d->stream));
    int rc = wait_domain(d);
    if (rc) return rc;
    const float* r = reinterpret_cast<const float*>(d->h_result);
    rho_out[0] = r[0];
    rho_out[1] = r[1];
    return LBM_OK;
}

int lbm_run_drainage(lbm_domain* d, const double* rho_in_nw, int n_incr, int n_steps, double rho_out_w,
                     const int probe[3], lbm_increment* rows, double* p_ce, int* invaded_at) {
    if (!d || !rho_in_nw || !probe || !rows || !p_ce || !invaded_at || n_incr < 1 || n_steps < 0) {
        set_error("lbm_run_drainage: NULL argument, n_incr < 1 or n_steps < 0");
        return LBM_ERR_ARG;
    }
    *invaded_at = -1;
    for (int i = 0; i < n_incr; ++i) {
        int rc = lbm_set_pressure_bc(d, rho_in_nw[i], rho_out_w);
        if (rc) return rc;
        rc = run_steps(d, n_steps);
        if (rc) return rc;
        lbm_measurement m;
        rc = lbm_measure(d, &m);
        if (rc && rc != LBM_ERR_NONFINITE) return rc;
        double pr[2];
        int rp = lbm_get_density_at(d, probe[0], probe[1], probe[2], pr);
        if (rp) return rp;
        lbm_increment& r = rows[i];
        r.rho_in_nw = rho_in_nw[i];
        r.p_c = m.p_c;
        r.p_c_res = m.p_c_res;
        r.S_w = m.S_w;
        r.p_w = m.p_w;
        r.p_nw = m.p_nw;
        r.n_interface = m.n_interface;
        r.phi_probe = (pr[0] + pr[1]) != 0.0 ? (pr[0] - pr[1]) / (pr[0] + pr[1]) : 0.0;
        if (*invaded_at < 0 && r.phi_probe < 0.0) *invaded_at = i;
        if (rc == LBM_ERR_NONFINITE) return rc;
    }
    // p_c^e: the largest p_c up to and including the invasion increment (the
    // maximum p_c reached during invasion, Sec. 2.2.2); first maximiser on ties
    if (*invaded_at < 0) {
        *p_ce = INFINITY;
    } else {
        double best = -INFINITY;
        for (int i = 0; i <= *invaded_at; ++i)
            if (rows[i].p_c == rows[i].p_c && rows[i].p_c > best) best = rows[i].p_c;
        *p_ce = best;
    }
    return LBM_OK;
}

int lbm_measure(lbm_domain* d, lbm_measurement* out) {
    if (!d || !out) { set_error("domain or out is NULL"); return LBM_ERR_ARG; }
    if (d->params.precision == 0 && d->layout == 1) {
        LBM_CUDA(launch_measure_push(d->f[d->cur], d->d_nbr, d->geom, d->params.G, d->d_partials, d->meas_blocks,
                                     d->d_result, d->stream));
    } else if (d->params.precision == 0) {
        LBM_CUDA(launch_measure(d->f[d->cur], d->d_nbr, d->d_nbr_nw, d->geom, d->params.G, d->d_partials,
                                d->meas_blocks, d->d_result, d->stream));
    }
    else {
        const uint32_t* w16 = nullptr;
        if (int rc = pull16_view(d, &w16)) return rc;
        LBM_CUDA(launch_measure16(d->params.precision, w16, d->R[d->cur],
                                  d->d_nbr, d->d_nbr_nw, d->geom, d->params.G, d->d_partials, d->meas_blocks,
                                  d->d_result, d->stream));
    }
    LBM_CUDA(cudaMemcpyAsync(d->h_result, d->d_result, sizeof(double) * NMEAS, cudaMemcpyDeviceToHost, d->stream));
    int rc = wait_domain(d);
    if (rc) return rc;
    const double* r = d->h_result;
    std::memset(out, 0, sizeof(*out));
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

int lbm_get_density(lbm_domain* d, double* rho_out) {
    if (!d || !rho_out) { set_error("domain or rho_out is NULL"); return LBM_ERR_ARG; }
    try {
        if (d->params.precision == 0 && d->layout == 1) {
            LBM_CUDA(launch_density_push(d->f[d->cur], d->d_nbr, d->geom, d->d_rho, d->stream));
        } else if (d->params.precision == 0) {
            LBM_CUDA(launch_density(d->f[d->cur], d->d_rho, d->d_nbr, d->d_nbr_nw, d->geom, d->stream));
        }
        else {
            const uint32_t* w16 = nullptr;
            if (int rc = pull16_view(d, &w16)) return rc;
            LBM_CUDA(launch_density16(d->params.precision, w16,
                                      d->R[d->cur], d->d_nbr, d->d_nbr_nw, d->geom, d->d_rho, d->stream));
        }
        std::vector<float> tmp((size_t)(2 * d->N));
        LBM_CUDA(cudaMemcpyAsync(tmp.data(), d->d_rho, sizeof(float) * 2 * d->N, cudaMemcpyDeviceToHost, d->stream));
        int rc = wait_domain(d);
        if (rc) return rc;
        for (long long i = 0; i < 2 * d->N; ++i) rho_out[i] = tmp[(size_t)i];
        return LBM_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
}

int lbm_get_mask(const lbm_domain* d, unsigned char* mask_out) {
    if (!d || !mask_out) { set_error("domain or mask_out is NULL"); return LBM_ERR_ARG; }
    LBM_CUDA(cudaMemcpy(mask_out, d->d_mask, (size_t)d->N, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

int lbm_get_dims(const lbm_domain* d, int dims_out[3], long long* n_fluid_cells) {
    if (!d || !dims_out) { set_error("domain or dims_out is NULL"); return LBM_ERR_ARG; }
    dims_out[0] = d->geom.nx;
    dims_out[1] = d->geom.ny;
    dims_out[2] = d->geom.nz;
    if (n_fluid_cells) *n_fluid_cells = d->n_fluid;
    return LBM_OK;
}

int lbm_get_state(lbm_domain* d, float* f_out, long long* step_out) {
    if (!d || !f_out) { set_error("domain or f_out is NULL"); return LBM_ERR_ARG; }
    if (d->params.precision != 0) { set_error("checkpoints are available for FP32 domains only"); return LBM_ERR_STATE; }
    const long long N = d->N;
    const float* fp = nullptr;
    if (int rc = pull_view(d, &fp)) return rc;
    for (int p = 0; p < 2 * Q; ++p)
        LBM_CUDA(cudaMemcpyAsync(f_out + (size_t)p * N, fp + (size_t)p * d->geom.plane, sizeof(float) * N,
                                 cudaMemcpyDeviceToHost, d->stream));
    int rc = wait_domain(d);
    if (rc) return rc;
    if (step_out) *step_out = d->step;
    return LBM_OK;
}

int lbm_set_state(lbm_domain* d, const float* f_in, long long step) {
    if (!d || !f_in || step < 0) { set_error("domain or f_in is NULL, or step < 0"); return LBM_ERR_ARG; }
    if (d->params.precision != 0) { set_error("checkpoints are available for FP32 domains only"); return LBM_ERR_STATE; }
    const long long N = d->N;
    for (int p = 0; p < 2 * Q; ++p)
        LBM_CUDA(cudaMemcpyAsync(d->f[d->cur] + (size_t)p * d->geom.plane, f_in + (size_t)p * N, sizeof(float) * N,
                                 cudaMemcpyHostToDevice, d->stream));
    d->step = step;
    d->ghosts_ok = false;
    d->layout = 0;
    return wait_domain(d);
}

int lbm_set_tile(lbm_domain* d, int by, int lz, int lead) {
    if (!d) { set_error("domain is NULL"); return LBM_ERR_ARG; }
    if (lz < 1 || !(d->params.precision == 0 ? tile_supported(by, lead) : tile16_supported(by, lead))) {
        set_error("unsupported tile: by in {6,8,10,12}, lz >= 1, lead in {2,3,4} (lead 3: by <= 10, lead 4: by <= 8)");
        return LBM_ERR_ARG;
    }
    d->tile.by = by;
    d->tile.lz = lz > d->geom.nz ? d->geom.nz : lz;
    d->tile.lead = lead;
    d->tile.kind = LBM_KERNEL_STAGED;
    drop_graphs(d);  // captured with the old shape
    return LBM_OK;
}

int lbm_set_step_kernel(lbm_domain* d, int kind, int lz) {
    if (!d) { set_error("domain is NULL"); return LBM_ERR_ARG; }
    if (kind != LBM_KERNEL_STAGED && kind != LBM_KERNEL_TMA && kind != LBM_KERNEL_SPLIT &&
        kind != LBM_KERNEL_STAGED2 && kind != LBM_KERNEL_PUSH) {
        set_error("unknown step kernel");
        return LBM_ERR_ARG;
    }
    if (kind == LBM_KERNEL_PUSH) {
        const bool fp32 = d->params.precision == 0;
        if (fp32 ? !push_step_applicable(d->geom) : !push16_step_applicable(d->geom)) {
            set_error(fp32 ? "the push step kernel needs a box without periodic x or y and with an even nx"
                           : "the 16-bit push step kernel needs a box without periodic x or y and with nx % 4 == 0");
            return LBM_ERR_STATE;
        }
        if (lz > 0) d->tile.push_lz = lz > d->geom.nz ? d->geom.nz : lz;
        d->tile.kind = kind;
        drop_graphs(d);
        return fp32 ? ensure_push_maps(d) : ensure_push16_maps(d);
    }
    if ((kind == LBM_KERNEL_SPLIT || kind == LBM_KERNEL_STAGED2) && d->params.precision != 0) {
        set_error("the two-launch and two-threads-per-cell step kernels need an FP32 domain");
        return LBM_ERR_STATE;
    }
    if (kind == LBM_KERNEL_STAGED2) {
        d->tile.by = tile2_supported(d->tile.by, 2) ? d->tile.by : 6;
        d->tile.lead = 2;
        if (lz > 0) d->tile.lz = lz > d->geom.nz ? d->geom.nz : lz;
    }
    if (kind == LBM_KERNEL_TMA) {
        if (d->params.precision != 0 || !d->tma_ok) {
            set_error("the TMA step kernel needs an FP32 domain without periodic x or y and with nx % 4 == 0");
            return LBM_ERR_STATE;
        }
        d->tile.tma_lz = lz <= 0 ? tma_default_lz(d->geom) : (lz > d->geom.nz ? d->geom.nz : lz);
    }
    d->tile.kind = kind;
    drop_graphs(d);
    return LBM_OK;
}

int lbm_get_step_kernel(const lbm_domain* d, int* kind, int* lz) {
    if (!d || !kind || !lz) { set_error("NULL argument"); return LBM_ERR_ARG; }
    *kind = d->tile.kind;
    *lz = d->tile.kind == LBM_KERNEL_TMA ? d->tile.tma_lz
          : d->tile.kind == LBM_KERNEL_PUSH ? d->tile.push_lz
                                            : d->tile.lz;  // staged kinds: the z segment
    return LBM_OK;
}

int lbm_set_push_shape(lbm_domain* d, int shape, int lz) {
    if (!d) { set_error("domain is NULL"); return LBM_ERR_ARG; }
    const bool fp32 = d->params.precision == 0;
    if (shape < 0 || shape >= (fp32 ? push_shape_count() : push16_shape_count())) {
        set_error("unknown push kernel shape");
        return LBM_ERR_ARG;
    }
    if (fp32 ? !push_step_applicable(d->geom) : !push16_step_applicable(d->geom)) {
        set_error(fp32 ? "the push step kernel needs a box without periodic x or y and with an even nx"
                       : "the 16-bit push step kernel needs a box without periodic x or y and with nx % 4 == 0");
        return LBM_ERR_STATE;
    }
    d->tile.push_shape = shape;
    d->tile.push_lz = lz > 0 ? (lz > d->geom.nz ? d->geom.nz : lz)
                             : (fp32 ? push_default_lz(d->geom, shape) : push16_default_lz(d->geom, shape));
    d->tile.kind = LBM_KERNEL_PUSH;
    drop_graphs(d);
    return fp32 ? ensure_push_maps(d) : ensure_push16_maps(d);
}

int lbm_set_push_prefetch(lbm_domain* d, int planes) {
    if (!d) { set_error("domain is NULL"); return LBM_ERR_ARG; }
    if (planes < 0 || planes > PUSH_MAX_PREFETCH) {
        set_error("push prefetch distance outside [0, 4]");
        return LBM_ERR_ARG;
    }
    d->tile.push_pf = planes;
    drop_graphs(d);
    return LBM_OK;
}

int lbm_set_push_order(lbm_domain* d, int order) {
    if (!d) { set_error("domain is NULL"); return LBM_ERR_ARG; }
    if (order < 0 || order > 1) {
        set_error("push segment order must be 0 or 1");
        return LBM_ERR_ARG;
    }
    d->tile.push_order = order;
    drop_graphs(d);
    return LBM_OK;
}

int lbm_get_tile(const lbm_domain* d, int* by, int* lz, int* lead) {
    if (!d || !by || !lz || !lead) { set_error("NULL argument"); return LBM_ERR_ARG; }
    *by = d->tile.by;
    *lz = d->tile.lz;
    *lead = d->tile.lead;
    return LBM_OK;
}

int lbm_autotune(lbm_domain* d, int trial_steps, lbm_tune_result* out) {
    if (!d || trial_steps < 1) { set_error("domain is NULL or trial_steps < 1"); return LBM_ERR_ARG; }
    int rc = wait_domain(d);
    if (rc) return rc;
    const Geom& g = d->geom;
    const bool fp32 = d->params.precision == 0;
    const size_t fbytes = (fp32 ? sizeof(float) * 2 : sizeof(uint32_t)) * (size_t)g.plane * Q;
    const size_t rbytes = fp32 ? 0 : sizeof(float2) * (size_t)g.plane;
    const StepTile orig = d->tile;
    const int cur = d->cur;
    const long long step = d->step;
    const int layout = d->layout;
    // candidates
    std::vector<StepTile> cand;
    auto add = [&](int kind, int by, int lz, int lead) {
        StepTile t = orig;
        t.kind = kind;
        t.by = by;
        t.lead = lead;
        if (kind == LBM_KERNEL_TMA) t.tma_lz = lz > g.nz ? g.nz : lz;
        else if (kind == LBM_KERNEL_PUSH) t.push_lz = lz > g.nz ? g.nz : lz;
        else t.lz = lz > g.nz ? g.nz : lz;
        cand.push_back(t);
    };
    if (fp32 && push_step_applicable(g))
        for (int sh = 0; sh < push_shape_count(); ++sh)
            for (int lz : {16, 24, 32, 48, 64})
                for (int pf : {0, 2})
                    for (int order : {0}) {  // order 1 was slower on every shape measured
                        StepTile t = orig;
                        t.kind = LBM_KERNEL_PUSH;
                        t.push_shape = sh;
                        t.push_lz = lz > g.nz ? g.nz : lz;
                        t.push_pf = pf;
                        t.push_order = order;
                        cand.push_back(t);
                    }
    if (!fp32 && push16_step_applicable(g))
        for (int sh = 0; sh < push16_shape_count(); ++sh)
            for (int lz : {16, 24, 32, 48}) {
                StepTile t = orig;
                t.kind = LBM_KERNEL_PUSH;
                t.push_shape = sh;
                t.push_lz = lz > g.nz ? g.nz : lz;
                t.push_pf = 0;
                t.push_order = 0;
                cand.push_back(t);
            }
    if (fp32 && d->tma_ok)
        for (int lz : {8, 12, 16, 24, 32, 48}) add(LBM_KERNEL_TMA, orig.by, lz, orig.lead);
    if (fp32) add(LBM_KERNEL_SPLIT, orig.by, orig.lz, orig.lead);
    if (fp32)
        for (int by : {6, 8})
            for (int lz : {8, 16, 32}) add(LBM_KERNEL_STAGED2, by, lz, 2);
    for (int by : {6, 8, 10})
        for (int lead : {0, 1, 2, 3})
            for (int lz : {8, 16, 32}) {
                if (fp32 ? !tile_supported(by, lead) : !tile16_supported(by, lead)) continue;
                add(LBM_KERNEL_STAGED, by, lz, lead);
            }
    void* fsave = nullptr;
    void* rsave = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        cudaFree(fsave);
        cudaFree(rsave);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    auto restore = [&]() -> int {
        LBM_CUDA(cudaMemcpyAsync(d->f[cur], fsave, fbytes, cudaMemcpyDeviceToDevice, d->stream));
        if (rbytes) LBM_CUDA(cudaMemcpyAsync(d->R[cur], rsave, rbytes, cudaMemcpyDeviceToDevice, d->stream));
        d->cur = cur;
        d->step = step;
        d->layout = layout;
        d->ghosts_ok = false;
        return LBM_OK;
    };
    auto fail = [&](int code) {
        d->tile = orig;
        drop_graphs(d);
        if (fsave) restore();
        wait_domain(d);
        cleanup();
        return code;
    };
    cudaError_t e = cudaMalloc(&fsave, fbytes);
    if (e == cudaSuccess && rbytes) e = cudaMalloc(&rsave, rbytes);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        set_error(std::string("lbm_autotune: ") + cudaGetErrorString(e));
        return fail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA);
    }
    e = cudaMemcpyAsync(fsave, d->f[cur], fbytes, cudaMemcpyDeviceToDevice, d->stream);
    if (e == cudaSuccess && rbytes) e = cudaMemcpyAsync(rsave, d->R[cur], rbytes, cudaMemcpyDeviceToDevice, d->stream);
    if (e != cudaSuccess) {
        set_error(std::string("lbm_autotune: ") + cudaGetErrorString(e));
        return fail(LBM_ERR_CUDA);
    }
    double best = 1e300;
    StepTile best_t = orig;
    for (const StepTile& t : cand) {
        d->tile = t;
        drop_graphs(d);
        if ((rc = restore())) return fail(rc);
        if ((rc = run_steps(d, 1))) return fail(rc);  // untimed: kernel set-up, ghost stores
        if (cudaEventRecord(e0, d->stream) != cudaSuccess) return fail(LBM_ERR_CUDA);
        if ((rc = run_steps(d, trial_steps))) return fail(rc);
        if (cudaEventRecord(e1, d->stream) != cudaSuccess) return fail(LBM_ERR_CUDA);
        if ((rc = wait_domain(d))) return fail(rc);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return fail(LBM_ERR_CUDA);
        const double per = ms / trial_steps;
        if (per < best) {
            best = per;
            best_t = t;
        }
    }
    d->tile = best_t;
    drop_graphs(d);
    if ((rc = restore())) return fail(rc);
    rc = wait_domain(d);
    cleanup();
    if (rc) return rc;
    if (out) {
        out->kind = best_t.kind;
        out->by = best_t.kind == LBM_KERNEL_PUSH
                      ? (fp32 ? push_shape_rows(best_t.push_shape) : push16_shape_rows(best_t.push_shape))
                      : best_t.by;
        out->lz = best_t.kind == LBM_KERNEL_TMA ? best_t.tma_lz
                  : best_t.kind == LBM_KERNEL_PUSH ? best_t.push_lz
                                                   : best_t.lz;
        out->lead = best_t.kind == LBM_KERNEL_PUSH
                        ? (fp32 ? push_shape_stages(best_t.push_shape) : push16_shape_stages(best_t.push_shape))
                        : best_t.lead;
        out->ms_per_step = best;
        out->n_candidates = (int)cand.size();
        out->prefetch = best_t.kind == LBM_KERNEL_PUSH ? best_t.push_pf : 0;
        out->shape = best_t.kind == LBM_KERNEL_PUSH ? best_t.push_shape : -1;
        out->order = best_t.kind == LBM_KERNEL_PUSH ? best_t.push_order : 0;
    }
    return LBM_OK;
}

int lbm_selftest_bounded_wait(int limit_us, int* gave_up) {
    if (!gave_up || limit_us < 1 || limit_us > 10000000) {
        set_error("lbm_selftest_bounded_wait: gave_up is NULL or limit_us outside [1, 1e7]");
        return LBM_ERR_ARG;
    }
    int* d_flag = nullptr;
    int h = 0;
    LBM_CUDA(cudaMalloc(&d_flag, sizeof(int)));
    cudaError_t e = cudaMemset(d_flag, 0, sizeof(int));
    if (e == cudaSuccess) e = launch_wait_selftest(1000LL * limit_us, d_flag, 0);
    if (e == cudaSuccess) e = cudaMemcpy(&h, d_flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d_flag);
    if (e != cudaSuccess) {
        set_error(std::string("lbm_selftest_bounded_wait: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    *gave_up = h;
    return LBM_OK;
}

void lbm_destroy(lbm_domain* d) {
    if (!d) return;
    if (d->done) wait_domain(d);
    free_domain(d);
}

const char* lbm_last_error(void) { return g_error.c_str(); }

}  // extern "C"
