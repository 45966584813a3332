// lbm_internal.h -- shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "lbm.h"

namespace lbmk {

constexpr int Q = 19;

// D3Q19 in the ABI order (rest, 6 faces, 12 edges); opposite pairs (1,2), (3,4), ...
__host__ __device__ constexpr int EX(int k) {
    constexpr int a[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return a[k];
}
__host__ __device__ constexpr int EY(int k) {
    constexpr int a[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return a[k];
}
__host__ __device__ constexpr int EZ(int k) {
    constexpr int a[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return a[k];
}
__host__ __device__ constexpr int OPP(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }
// lattice weights: 1/3 rest, 1/18 faces, 1/36 edges (cs^2 = 1/3)
__host__ __device__ constexpr float WK(int k) { return k == 0 ? (1.0f / 3.0f) : (k <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f)); }
// 36 * w_k for k >= 1: 2 on faces, 1 on edges (adhesion vectors are stored in these units)
__host__ __device__ constexpr int W36(int k) { return k == 0 ? 12 : (k <= 6 ? 2 : 1); }

// Per-cell geometry word (uint32), built once per domain from the mask:
//   bit k (1..18)  pulling direction k at this cell bounces back (x - e_k is not
//                  fluid for the wetting component or lies beyond a closed edge)
//   bits 19..21    cell class (below)
//   bit 22         the non-wetting component bounces differently (membrane
//                  nearby): its bits are in the second word array
//   bit 23         an adhesive grain cell is among the 18 neighbours: the
//                  adhesion vector sum_k 36 w_k s(x+e_k) e_k is in the third array
//                  (three int8 in the low bytes)
constexpr int CLS_SHIFT = 19;
constexpr uint32_t CLS_MASK = 7u;
enum : uint32_t { CLS_FLUID = 0, CLS_SOLID = 1, CLS_INLET = 2, CLS_OUTLET = 3, CLS_MEMBRANE = 4, CLS_OUTSIDE = 5 };
constexpr uint32_t BIT_NW_DIFF = 1u << 22;
constexpr uint32_t BIT_ADH = 1u << 23;

struct Geom {
    int nx, ny, nz;
    int nxy;
    int plane;  // stride between population planes (>= N, multiple of 32)
    int px, py, pz;
    // poff[k] = k * plane - (ex_k + ey_k nx + ez_k nxy): from a cell's index to
    // its pull source of direction k in population plane k (kernel parameters
    // live in the constant bank, so these cost no registers)
    int poff[Q];
};

inline void fill_pull_offsets(Geom& g) {
    for (int k = 0; k < Q; ++k) g.poff[k] = k * g.plane - (EX(k) + EY(k) * g.nx + EZ(k) * g.nxy);
}

struct Phys {
    float tau[2];
    float omega[2];
    float G;
    float Gads[2];
    float g[3];
    // device pointer to the reservoir densities (inlet w, inlet nw, outlet w,
    // outlet nw): kept in device memory so that a captured graph of steps stays
    // valid when the pressure ladder moves on
    const float* bc;
};

// Number of doubles in one measurement partial.
constexpr int NMEAS = 16;
enum {
    MS_MASS_W = 0, MS_MASS_NW, MS_PW, MS_PNW, MS_PIN, MS_POUT,
    MS_N_FLUID, MS_N_W, MS_N_INTERFACE, MS_N_BULK_W, MS_N_BULK_NW, MS_N_IN, MS_N_OUT,
    MS_N_NONFINITE, MS_N_NEGATIVE, MS_SPARE
};

// ---------------------------------------------------------------- launchers
// Streaming multiprocessors of the current device (1 when the query fails:
// grid-stride kernels stay correct with any grid).
int device_sm_count();
struct StepTile {
    int by;    // block rows including the two halo rows (6, 8, 10 or 12)
    int lz;    // z-segment length per CTA
    int lead;  // planes queued ahead of the collided plane (2, 3 or 4)
    int kind;  // LBM_KERNEL_STAGED, _TMA, _SPLIT, _STAGED2 or _PUSH
    int tma_lz;  // z-segment length of the TMA kernel
    int push_shape;  // shape index of the push kernel (push_shape_rows / _stages)
    int push_lz;     // z-segment length of the push kernel
    int push_pf;     // planes the push kernel prefetches into L2 beyond its loads (0 .. PUSH_MAX_PREFETCH)
    int push_order;  // 0: segments march +z in x-y-z launch order; 1: a column's segments together, alternating
};

// Tensor maps of the TMA step kernel (lbm_step_tma.cu): the two population
// buffers as 4-D tensors (x, y, z, array) and the geometry words (x, y, z).
struct TmaMaps {
    CUtensorMap f[2];
    CUtensorMap w;
};

cudaError_t launch_geometry(const uint8_t* mask, uint32_t* nbr, uint32_t* nbr_nw, uint32_t* adh, const Geom& g,
                            cudaStream_t s);
cudaError_t launch_init(const float* rho0, float* f, const uint32_t* nbr, const uint32_t* nbr_nw, const Geom& g,
                        cudaStream_t s);
cudaError_t launch_step(const float* fin, float* fout, const uint32_t* nbr, const uint32_t* nbr_nw,
                        const uint32_t* adh, const Geom& g, const Phys& p, StepTile tile, cudaStream_t s);
cudaError_t launch_density(const float* f, float* rho, const uint32_t* nbr, const uint32_t* nbr_nw, const Geom& g,
                           cudaStream_t s);
int measure_blocks(const Geom& g);
cudaError_t launch_measure(const float* f, const uint32_t* nbr, const uint32_t* nbr_nw, const Geom& g, double G,
                           double* partials, int nblocks, double* result, cudaStream_t s);
cudaError_t prepare_step(const StepTile& tile);
cudaError_t launch_set_bc(float* bc, float in_w, float in_nw, float out_w, float out_nw, cudaStream_t s);
cudaError_t launch_probe(const float* f, const uint32_t* nbr, const uint32_t* nbr_nw, const Geom& g, int x, int y,
                         int z, float* out, cudaStream_t s);
cudaError_t launch_finalize(const double* partials, int nblocks, double* result, cudaStream_t s);
// 16-bit storage (precision 1 = FP16, 2 = BF16 deviations; lbm_step16.cu)
bool tile16_supported(int by, int lead);
cudaError_t prepare_step16(int precision, const StepTile& t);
cudaError_t launch_step16(int precision, const uint32_t* win, uint32_t* wout, const float2* Rin, float2* Rout,
                          const uint32_t* nbr, const uint32_t* nbr_nw, const uint32_t* adh, const Geom& g,
                          const Phys& p, StepTile t, cudaStream_t s);
cudaError_t launch_init16(const float* rho0, float2* R, const Geom& g, cudaStream_t s);
cudaError_t launch_density16(int precision, const uint32_t* w, const float2* R, const uint32_t* nbr,
                             const uint32_t* nbr_nw, const Geom& g, float* rho, cudaStream_t s);
cudaError_t launch_measure16(int precision, const uint32_t* w, const float2* R, const uint32_t* nbr,
                             const uint32_t* nbr_nw, const Geom& g, double G, double* partials, int nblocks,
                             double* result, cudaStream_t s);
cudaError_t launch_probe16(int precision, const uint32_t* w, const float2* R, const uint32_t* nbr,
                           const uint32_t* nbr_nw, const Geom& g, int x, int y, int z, float* out, cudaStream_t s);
StepTile default_tile(const Geom& g);
bool tile_supported(int by, int lead);
// TMA step kernel (FP32; no periodic x / y, nx % 4 == 0)
bool tma_step_applicable(const Geom& g);
int tma_default_lz(const Geom& g);
cudaError_t encode_step_maps(const Geom& g, float* f0, float* f1, const uint32_t* nbr, TmaMaps& m);
cudaError_t prepare_step_tma();
cudaError_t launch_step_tma(const TmaMaps& m, int cur, const float* fin, float* fout, const uint32_t* nbr_nw,
                            const uint32_t* adh, const Geom& g, const Phys& p, int lz, int* err, cudaStream_t s);
// staged step with two threads per cell, one per component (lbm_step2.cu)
bool tile2_supported(int by, int lead);
cudaError_t prepare_step2(const StepTile& t);
cudaError_t launch_step2(const float* fin, float* fout, const uint32_t* nbr, const uint32_t* nbr_nw,
                         const uint32_t* adh, const Geom& g, const Phys& p, const StepTile& t, cudaStream_t s);
// two-launch step: densities first, then pull + collide reading the neighbour
// densities from rho2 (lbm_step_split.cu)
cudaError_t launch_step_split(const float* fin, float* fout, float2* rho2, const uint32_t* nbr,
                              const uint32_t* nbr_nw, const uint32_t* adh, const Geom& g, const Phys& p,
                              cudaStream_t s);
// paired push-form step (lbm_step_push.cu): float2 F[19][plane] of the current
// time level; TMA box loads of whole planes (no periodic x / y, nx even)
// Inscribed circle of a throat (3 x (cx, cy, cz, r)): the largest clearance
// over the triangle of the centres, 0 when the spheres close it.
double throat_incircle(const double* s3);

constexpr int PUSH_MAX_PREFETCH = 4;

// The push kernel of 16-bit storage (lbm_step16_push.cu) and the conversions
// of a 16-bit state between the pull and push layouts (lbm_step16.cu).
int push16_shape_count();
int push16_shape_rows(int shape);
int push16_shape_stages(int shape);
bool push16_step_applicable(const Geom& g);
int push16_default_lz(const Geom& g, int shape);
cudaError_t encode_push16_maps(const Geom& g, uint32_t* w0, uint32_t* w1, float2* r0, float2* r1, int by,
                               CUtensorMap (&mw)[2], CUtensorMap (&mr)[2]);
cudaError_t prepare_step16_push(int precision, int shape);
cudaError_t launch_step16_push(int precision, int shape, const CUtensorMap& tw, const CUtensorMap& tr,
                               uint32_t* wout, float2* Rout, const uint32_t* nbr, const uint32_t* nbr_nw,
                               const uint32_t* adh, const Geom& g, const Phys& p, int lz, int* err, cudaStream_t s);
cudaError_t launch_pull16_to_push16(const uint32_t* win, uint32_t* wout, const uint32_t* nbr, const uint32_t* nbr_nw,
                                    const Geom& g, cudaStream_t s);
cudaError_t launch_push16_to_pull16(const uint32_t* win, uint32_t* wout, const uint32_t* nbr, const uint32_t* nbr_nw,
                                    const Geom& g, cudaStream_t s);
int push_shape_count();
int push_shape_rows(int shape);
int push_shape_stages(int shape);
int push_shape_ctas(int shape);
bool push_shape_resident(int shape);
bool push_step_applicable(const Geom& g);
int push_default_lz(const Geom& g, int shape);
cudaError_t encode_push_maps(const Geom& g, float* f0, float* f1, int by, CUtensorMap (&maps)[2]);
cudaError_t prepare_step_push(int shape);
cudaError_t launch_step_push(int shape, const CUtensorMap& tm_in, float* fout, const uint32_t* nbr,
                             const uint32_t* nbr_nw, const uint32_t* adh, const Geom& g, const Phys& p, int lz,
                             int pf, int order, int* err, cudaStream_t s);
cudaError_t launch_pull_to_push(const float* fin, float* F, const uint32_t* nbr, const uint32_t* nbr_nw,
                                const Geom& g, cudaStream_t s);
cudaError_t launch_push_to_pull(const float* F, float* fout, const uint32_t* nbr, const uint32_t* nbr_nw,
                                const Geom& g, cudaStream_t s);
// read-outs straight from the paired push layout (a cell's densities are the
// sums of its own pairs; the same bits as the pull read-outs)
cudaError_t launch_measure_push(const float* F, const uint32_t* nbr, const Geom& g, double G, double* partials,
                               int nblocks, double* result, cudaStream_t s);
cudaError_t launch_density_push(const float* F, const uint32_t* nbr, const Geom& g, float* rho, cudaStream_t s);
cudaError_t launch_probe_push(const float* F, const uint32_t* nbr, const Geom& g, int x, int y, int z, float* out,
                              cudaStream_t s);
// one CTA waiting, bounded, on an mbarrier that nothing completes (self-test)
cudaError_t launch_wait_selftest(long long limit_ns, int* gave_up, cudaStream_t s);
// ghost stores (the reflected populations the TMA kernel pulls from wall cells) of a state
cudaError_t launch_ghost_fill(float* f, const uint32_t* nbr, const uint32_t* nbr_nw, const Geom& g, cudaStream_t s);

// host geometry (lbm_geometry.cpp)
void voxelise_box(int nx, int ny, int nz, const double* spheres, int n_spheres, int prism_clip, int reservoirs,
                  int membrane_layers, uint8_t* mask);

void throat_frame(const double* spheres3, int dims[3], double origin[3], double local[12]);
void voxelise_throat(const double* spheres3, uint8_t* mask, int probe[3]);

// thread-local error text
void set_error(const std::string& msg);

}  // namespace lbmk

// The opaque domain handle of the ABI.
struct lbm_domain {
    lbm_params params;
    lbmk::Geom geom;
    lbmk::Phys phys;
    lbmk::StepTile tile;
    long long N;
    long long n_fluid;
    float* f[2];       // populations (FP32) or 16-bit deviation pairs (uint32 words)
    float2* R[2];      // 16-bit storage: densities of the previous time level
    int cur;
    long long step;
    uint8_t* d_mask;
    uint32_t* d_nbr;
    uint32_t* d_nbr_nw;
    uint32_t* d_adh;
    float* d_rho;
    double* d_partials;
    double* d_result;
    double* h_result;  // pinned
    int meas_blocks;
    cudaStream_t stream;
    cudaEvent_t done;
    float* d_bc;        // reservoir densities (4 floats)
    float* d_probe;     // density at a probe cell (2 floats)
    double bc_host[4];  // last reservoir densities set
    // captured chunks of GRAPH_STEPS steps, one per starting buffer
    cudaGraphExec_t graph[2];
    cudaStream_t capture_stream;
    lbmk::TmaMaps tma;  // valid when tma_ok
    bool tma_ok;
    bool ghosts_ok;     // the current FP32 state holds the TMA kernel's ghost stores
    int* d_err;         // set by a step kernel whose bounded wait ran out
    int* h_err;         // pinned copy of d_err, read after a wait
    bool tma_pending;   // a TMA step ran since d_err was last read
    float2* d_rho2;     // FP32 domains: (rho_w, rho_nw) per cell for the two-launch step
    int layout;         // FP32 state in f[cur]: 0 = pull layout, 1 = paired push layout
    CUtensorMap push_maps[2];  // tensor maps of f[0], f[1] for the push kernel's shape
    CUtensorMap push16_w[2];   // 16-bit storage: tensor maps of the words of f[0], f[1]
    CUtensorMap push16_r[2];   // and of the density pairs R[0], R[1]
    int push16_maps_rows;      // box rows the 16-bit push maps were encoded for (0: none)
    int push_maps_rows;        // box rows the push maps were encoded for (0: none)
};

constexpr int GRAPH_STEPS = 64;  // steps per captured graph (even: the buffer parity is unchanged)
