// lbm_batch.cu -- many pore throats per call (lbm_run_throat_batch), in four
// forms that give the same rows bit for bit.
//
// The hybrid method runs one small LBM simulation per pore throat (Sec. 2.2.2)
// and the paper assigns one throat per CPU core (Sec. 4).  Here all throats of
// a batch run together on the GPU, each with its own box, geometry words and
// reservoir ladder, found through a record table.
//
// Cell list (the default).  A throat box is mostly grain: it is the bounding box
// of a triangular prism whose corners the spheres fill.  This form stores the
// populations of the non-solid cells only, compactly and after streaming, and
// runs two launches per time step over that list: densities, then the
// collision, which pushes every value to the cell it streams to.  A measurement
// launch (a CTA per slice of a throat box) ends each increment.
//
// March.  The same cell list in one launch per time step: a CTA per chunk of a
// throat's planes sums the densities of a plane and steps the plane below it.
//
// Tiles.  One launch per time step over a work list of (throat, active tile,
// z segment) items of the box layout, the step_column of the single-domain
// staged kernel; the kernel boundary orders the steps.
//
// Persistent.  One launch per increment: a CTA takes a whole throat off a work
// counter (largest first) and runs the increment's steps on its box tile by
// tile, with a CTA barrier between steps, then measures it.  A batch of few
// throats leaves most SMs idle in this form and waits on its largest throat.
//
// In the cell-list and tile forms one increment is captured as a CUDA graph and
// relaunched, the increment index living in device memory; the persistent form
// captures all increments in one graph.
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "lbm_host.h"
#include "lbm_step_core.cuh"

namespace lbmk {

namespace {

struct ThroatRec {
    Geom g;
    long long f_off;  // offset of the throat's populations in each population arena (floats)
    long long c_off;  // offset of its cells in the per-cell arenas
    int probe;        // probe cell index in the box, -1 if none
    int tile_begin;   // this throat's active tiles in the tile list
    int tile_count;
};

constexpr int BATCH_BY = 6;
constexpr int BATCH_LEAD = 2;
constexpr int BATCH_THREADS = 32 * BATCH_BY;

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.y * 32 + threadIdx.x;
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < BATCH_THREADS / 32; ++w) s += red[w];
    return s;  // valid in thread 0
}

// Measurements of a throat box (definitions of lbm_measure).  The box's cells
// are cut into slices of MEAS_SLICE cells; a slice's sums are the CTA sum
// (block_sum) of per-thread sums, thread t adding cells t, t + BATCH_THREADS, ...
// of the slice in that order; a throat's sums are its slices' sums added in
// slice order.  Every form computes exactly these sums: the box forms slice by
// slice in one CTA, the cell-list form one CTA per slice.
constexpr int MEAS_SLICE = 32 * BATCH_THREADS;

// The sums of box cells c0 .. c1 - 1 (valid in thread 0).  state(c, rw, rn)
// returns the geometry word of box cell c (class CLS_SOLID for grain) and its
// densities after streaming, summed in k order.
template <class CellState>
__device__ void measure_slice(int c0, int c1, double G, double* red, CellState&& state, double (&tot)[NMEAS]) {
    double acc[NMEAS];
#pragma unroll
    for (int i = 0; i < NMEAS; ++i) acc[i] = 0.0;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    // a thread's cells are c0 + tid, c0 + tid + BATCH_THREADS, ...: read MEAS_AHEAD
    // of them at a time (their loads in flight together), then add them up in
    // that order
    constexpr int MEAS_AHEAD = 4;
    for (int cb = c0 + tid; cb < c1; cb += MEAS_AHEAD * BATCH_THREADS) {
        float rwf[MEAS_AHEAD], rnf[MEAS_AHEAD];
        uint32_t wv[MEAS_AHEAD];
#pragma unroll
        for (int u = 0; u < MEAS_AHEAD; ++u) {
            const int c = cb + u * BATCH_THREADS;
            rwf[u] = rnf[u] = 0.f;
            wv[u] = c < c1 ? state(c, rwf[u], rnf[u]) : (uint32_t)CLS_SOLID << CLS_SHIFT;
        }
#pragma unroll
        for (int u = 0; u < MEAS_AHEAD; ++u) {
            const uint32_t cls = (wv[u] >> CLS_SHIFT) & CLS_MASK;
            if (cls == CLS_SOLID) continue;
            const double rw = rwf[u], rn = rnf[u];
            acc[MS_MASS_W] += rw;
            acc[MS_MASS_NW] += rn;
            if (!isfinite(rw) || !isfinite(rn)) acc[MS_N_NONFINITE] += 1.0;
            const double x = rw - rn, y = rw + rn;
            const double p = (y + G * rw * rn) * (1.0 / 3.0);  // Eq. 5
            if (cls == CLS_INLET) { acc[MS_PIN] += p; acc[MS_N_IN] += 1.0; continue; }
            if (cls == CLS_OUTLET) { acc[MS_POUT] += p; acc[MS_N_OUT] += 1.0; continue; }
            acc[MS_N_FLUID] += 1.0;
            if (rw > rn) acc[MS_N_W] += 1.0;
            // phi = x / y against 0.5 and 0.9 without the division: for y > 0,
            // |phi| < 0.5 is |x| < 0.5 y exactly (the scaling is exact and no
            // quotient of doubles lies within half an ulp below 0.5); the product
            // 0.9 y is rounded, so a cell within 1e-12 of that threshold is decided
            // by the division itself, as is every cell with y <= 0 or not finite
            bool in_if, bulk_w, bulk_nw;
            const double t9 = 0.9 * y;
            if (y > 0.0 && fabs(fabs(x) - t9) > 1e-12 * y) {
                in_if = fabs(x) < 0.5 * y;
                bulk_w = x > t9;
                bulk_nw = x < -t9;
            } else {
                const double phi = x / y;
                in_if = fabs(phi) < 0.5;
                bulk_w = phi > 0.9;
                bulk_nw = phi < -0.9;
            }
            if (in_if) acc[MS_N_INTERFACE] += 1.0;
            if (bulk_w) { acc[MS_PW] += p; acc[MS_N_BULK_W] += 1.0; }
            if (bulk_nw) { acc[MS_PNW] += p; acc[MS_N_BULK_NW] += 1.0; }
        }
    }
#pragma unroll
    for (int i = 0; i < NMEAS; ++i) tot[i] = block_sum(acc[i], red);
}

// The increment's row from a throat's sums and its probe densities.
__device__ void measure_row(const double (&tot)[NMEAS], double rho_in_nw, int probe, float pw, float pn,
                            lbm_increment* row) {
    lbm_increment r;
    r.rho_in_nw = rho_in_nw;
    r.p_w = tot[MS_N_BULK_W] > 0 ? tot[MS_PW] / tot[MS_N_BULK_W] : NAN;
    r.p_nw = tot[MS_N_BULK_NW] > 0 ? tot[MS_PNW] / tot[MS_N_BULK_NW] : NAN;
    r.p_c = r.p_nw - r.p_w;
    const double pin = tot[MS_N_IN] > 0 ? tot[MS_PIN] / tot[MS_N_IN] : NAN;
    const double pout = tot[MS_N_OUT] > 0 ? tot[MS_POUT] / tot[MS_N_OUT] : NAN;
    r.p_c_res = pin - pout;
    r.S_w = tot[MS_N_FLUID] > 0 ? tot[MS_N_W] / tot[MS_N_FLUID] : NAN;
    const double a = pw, b = pn;
    r.phi_probe = probe >= 0 && (a + b) != 0.0 ? (a - b) / (a + b) : 0.0;
    r.n_interface = (long long)tot[MS_N_INTERFACE];
    *row = r;
}

// Measurements of one throat box in one CTA, slice by slice, into row.
template <class CellState>
__device__ void measure_cells(const Geom& g, double G, int probe, double rho_in_nw, double* red, lbm_increment* row,
                              CellState&& state) {
    const int N = g.nxy * g.nz;
    double tot[NMEAS];
#pragma unroll
    for (int i = 0; i < NMEAS; ++i) tot[i] = 0.0;
    for (int c0 = 0; c0 < N; c0 += MEAS_SLICE) {
        double part[NMEAS];
        measure_slice(c0, min(N, c0 + MEAS_SLICE), G, red, state, part);
#pragma unroll
        for (int i = 0; i < NMEAS; ++i) tot[i] += part[i];
    }
    const int tid = threadIdx.y * 32 + threadIdx.x;
    if (tid == 0) {
        float pr[2] = {0.f, 0.f};
        if (probe >= 0) state(probe, pr[0], pr[1]);
        measure_row(tot, rho_in_nw, probe, pr[0], pr[1], row);
    }
}

// The same on the box layout: densities pulled from the post-collision arrays.
__device__ void measure_throat(const float* __restrict__ f, const uint32_t* __restrict__ nbr,
                               const uint32_t* __restrict__ nbr_nw, const Geom& g, double G, int probe,
                               double rho_in_nw, double* red, lbm_increment* row) {
    measure_cells(g, G, probe, rho_in_nw, red, row, [&](int c, float& rw, float& rn) {
        const int x = c % g.nx;
        const int y = (c / g.nx) % g.ny;
        const int z = c / g.nxy;
        const Column col = make_column(x, y, g);
        float dummy[2][Q];
        int cell;
        return pull_cell<false>(f, nbr, nbr_nw, g, col, z, dummy, rw, rn, cell);
    });
}

template <int BY, int LEAD>
__global__ void __launch_bounds__(32 * BY, 2)
    throat_batch_kernel(const ThroatRec* __restrict__ recs, const int* __restrict__ order, int n,
                        int* __restrict__ counter, const int* __restrict__ tiles, float* arena0, float* arena1,
                        const uint32_t* __restrict__ nbr,
                        const uint32_t* __restrict__ nbr_nw, const uint32_t* __restrict__ adh, Phys P, int n_steps,
                        int parity, double G, const float* __restrict__ bc_all, const double* __restrict__ rin_all,
                        int ladder_stride, lbm_increment* __restrict__ rows, int incr, int n_incr) {
    extern __shared__ float smem[];
    __shared__ int s_t;
    __shared__ double red[32];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    while (true) {
        if (tid == 0) s_t = atomicAdd(counter, 1);
        __syncthreads();
        const int t = s_t;
        __syncthreads();
        if (t >= n) break;
        const int id = order[t];
        const Geom g = recs[id].g;
        const long long f_off = recs[id].f_off, c_off = recs[id].c_off;
        const int probe = recs[id].probe;
        const int tb = recs[id].tile_begin, tc = recs[id].tile_count;
        // this throat's reservoir densities of this increment (its own ladder,
        // or the shared one when ladder_stride is 0)
        const size_t li = (size_t)id * ladder_stride + incr;
        Phys Pt = P;
        Pt.bc = bc_all + 4 * li;
        const double rho_in_nw = rin_all[li];
        float* buf[2] = {arena0 + f_off, arena1 + f_off};
        const uint32_t* tn = nbr + c_off;
        const uint32_t* tnn = nbr_nw + c_off;
        const uint32_t* ta = adh + c_off;
        int cur = parity;
        for (int s = 0; s < n_steps; ++s) {
            // only tiles whose columns hold a non-solid cell: a throat box is
            // the bounding box of a triangular prism, and the columns outside
            // the triangle are solid from end to end
            for (int i = 0; i < tc; ++i) {
                const int packed = __ldg(tiles + tb + i);
                step_column<BY, LEAD>(buf[cur], buf[cur ^ 1], tn, tnn, ta, g, Pt, packed & 0xffff, packed >> 16, 0,
                                      g.nz, smem);
                __syncthreads();
            }
            cur ^= 1;
        }
        measure_throat(buf[cur], tn, tnn, g, G, probe, rho_in_nw, red, rows + (size_t)id * n_incr + incr);
        __syncthreads();
    }
}

// One time step of the work item blockIdx.x (throat, tile, z range) of the batch;
// fin / fout are the population arenas of this step.
template <int BY, int LEAD>
__global__ void __launch_bounds__(32 * BY, 2)
    throat_item_step_kernel(const ThroatRec* __restrict__ recs, const int4* __restrict__ items,
                            const float* __restrict__ fin, float* __restrict__ fout,
                            const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw,
                            const uint32_t* __restrict__ adh, Phys P, const float* __restrict__ bc_all,
                            int ladder_stride, const int* __restrict__ incr_now) {
    extern __shared__ float smem[];
    const int4 it = items[blockIdx.x];  // (throat, tx | ty << 16, z0, z1)
    const int id = it.x;
    const Geom g = recs[id].g;
    const long long f_off = recs[id].f_off, c_off = recs[id].c_off;
    Phys Pt = P;
    Pt.bc = bc_all + 4 * ((size_t)id * ladder_stride + *incr_now);
    step_column<BY, LEAD>(fin + f_off, fout + f_off, nbr + c_off, nbr_nw + c_off, adh + c_off, g, Pt, it.y & 0xffff,
                          it.y >> 16, it.z, it.w, smem);
}

// Measurements of throat blockIdx.x at the end of increment *incr_now, then
// (last CTA to finish) the increment index moves on.
__global__ void __launch_bounds__(BATCH_THREADS)
    throat_item_measure_kernel(const ThroatRec* __restrict__ recs, int n, const float* __restrict__ f,
                               const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw, double G,
                               const double* __restrict__ rin_all, int ladder_stride, lbm_increment* __restrict__ rows,
                               int n_incr, int* incr_now, int* done) {
    __shared__ double red[32];
    const int id = blockIdx.x;
    const int incr = *incr_now;
    const Geom g = recs[id].g;
    measure_throat(f + recs[id].f_off, nbr + recs[id].c_off, nbr_nw + recs[id].c_off, g, G, recs[id].probe,
                   rin_all[(size_t)id * ladder_stride + incr], red, rows + (size_t)id * n_incr + incr);
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        __threadfence();
        if (atomicAdd(done, 1) == n - 1) {  // every CTA has read the index
            *done = 0;
            *incr_now = incr + 1;
        }
    }
}

// The cell-list form.  A list item is (throat, x | y << 10 | z << 20) of a
// non-solid cell of that throat's box; boxes are at most 512 cells along an axis.
// Items are ordered by throat and, inside a throat, in memory order, so that the
// +x neighbour of item i, when it is not grain, is item i + 1.
//
// Storage is compact: population (s, k) of item i lives at fc[(s Q + k) cp + i]
// (cp: item count rounded up to 32), and the stored value is the population
// after streaming -- what the pull of Eq. 1 would deliver to the cell.  Both
// passes of a step read a cell's own values only; the collision pushes each
// post-collision value f*_k to the slot (k) of the cell x + e_k, or, where
// x + e_k is not fluid for the component, back into the cell's own slot
// (opposite k) -- half-way bounce-back, decided by the bits the pull uses (bit
// k' of a word: x - e_k' is not fluid).  Every slot is written exactly once.
struct CellAt {
    int id, x, y, z, cell;
};
__device__ __forceinline__ CellAt decode_cell(int2 it, const Geom& g) {
    CellAt c;
    c.id = it.x;
    c.x = it.y & 1023;
    c.y = (it.y >> 10) & 1023;
    c.z = it.y >> 20;
    c.cell = c.z * g.nxy + c.y * g.nx + c.x;
    return c;
}

constexpr int CELL_THREADS = 256;
constexpr int NB_DIRS = Q - 3;  // directions 3..18 leave the x row; 1 and 2 are +x and -x

// Push-table entries: NB = int holds the item itself (-1: none), NB = int16_t
// its offset from the item that reads it (INT16_MIN: none), half the bytes;
// the host picks int16_t when every throat's items lie within 32767 of their
// neighbours (items follow memory order inside a throat, so a neighbour is at
// most nx ny + nx + 1 items away).
__device__ __forceinline__ int nb_encode(int item, int self, int) { return item; }
__device__ __forceinline__ int16_t nb_encode(int item, int self, int16_t) {
    return item < 0 ? (int16_t)INT16_MIN : (int16_t)(item - self);
}
__device__ __forceinline__ int nb_decode(int v, int) { return v; }
__device__ __forceinline__ int nb_decode(int16_t v, int self) { return v == INT16_MIN ? -1 : self + v; }

// Compact copies of the geometry words and the push table: nbp[(k - 3) cp + i]
// is the item of x + e_k (encoded as NB), none where that cell is grain or
// beyond the box.
template <class NB>
__global__ void __launch_bounds__(CELL_THREADS)
    cell_gather_kernel(const ThroatRec* __restrict__ recs, const int2* __restrict__ items, int n_items, int cp,
                       const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw,
                       const uint32_t* __restrict__ adh, const int* __restrict__ box_to_item,
                       uint32_t* __restrict__ wc, uint32_t* __restrict__ wnc, uint32_t* __restrict__ adhc,
                       NB* __restrict__ nbp) {
    const int i = blockIdx.x * CELL_THREADS + threadIdx.x;
    if (i >= n_items) return;
    const int2 it = items[i];
    const ThroatRec& r = recs[it.x];
    const Geom g = r.g;
    const CellAt c = decode_cell(it, g);
    const long long c_off = r.c_off;
    const uint32_t w = nbr[c_off + c.cell];
    wc[i] = w;
    wnc[i] = (w & BIT_NW_DIFF) ? nbr_nw[c_off + c.cell] : w;
    adhc[i] = (w & BIT_ADH) ? adh[c_off + c.cell] : 0u;
#pragma unroll
    for (int k = 3; k < Q; ++k) {
        const int x = c.x + EX(k), y = c.y + EY(k), z = c.z + EZ(k);
        const bool in = x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz;
        nbp[(size_t)(k - 3) * cp + i] =
            nb_encode(in ? box_to_item[c_off + (long long)z * g.nxy + y * g.nx + x] : -1, i, NB());
    }
}

// Rest equilibrium at the start (as throat_init_kernel: wetting fluid
// everywhere, the non-wetting fluid on the inlet layer), stored after streaming
// as pairs: fc[k cp + i] = (f_k^w, f_k^nw) of item i.
__global__ void __launch_bounds__(CELL_THREADS)
    cell_init_kernel(const uint32_t* __restrict__ wc, int n_items, int cp, float2* __restrict__ fc, float rho_major,
                     float rho_minor) {
    const int i = blockIdx.x * CELL_THREADS + threadIdx.x;
    if (i >= n_items) return;
    const uint32_t cls = (wc[i] >> CLS_SHIFT) & CLS_MASK;
    const bool inlet = cls == CLS_INLET;
    float v[2][Q];
    for (int s = 0; s < 2; ++s) {
        const bool fl = !(s == 1 && cls == CLS_MEMBRANE);
        const float r = !fl ? 0.f : s == 0 ? (inlet ? rho_minor : rho_major) : (inlet ? rho_major : rho_minor);
        float sum = 0.f;
        for (int k = 1; k < Q; ++k) sum += WK(k) * r;
        v[s][0] = fl ? r - sum : 0.f;
        for (int k = 1; k < Q; ++k) v[s][k] = fl ? WK(k) * r : 0.f;
    }
    for (int k = 0; k < Q; ++k) fc[(size_t)k * cp + i] = make_float2(v[0][k], v[1][k]);
}

// (rho_w, rho_nw) of item i (Eq. 2), in four interleaved partial sums as the
// staged kernel sums its density ring; 0 for the non-wetting fluid on a membrane.
__device__ __forceinline__ void cell_density_item(int i, const uint32_t* __restrict__ wc, int cp,
                                                  const float2* __restrict__ fc, float2* __restrict__ rho2) {
    const uint32_t cls = (__ldg(wc + i) >> CLS_SHIFT) & CLS_MASK;
    float a[4] = {0.f, 0.f, 0.f, 0.f}, b[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const float2 v = __ldg(fc + (size_t)k * cp + i);
        a[k & 3] += v.x;
        b[k & 3] += v.y;
    }
    const float rn = cls == CLS_MEMBRANE ? 0.f : (b[0] + b[1]) + (b[2] + b[3]);
    rho2[i] = make_float2((a[0] + a[1]) + (a[2] + a[3]), rn);
}

// The densities of every item.
__global__ void __launch_bounds__(CELL_THREADS)
    cell_density_kernel(const uint32_t* __restrict__ wc, int n_items, int cp, const float2* __restrict__ fc,
                        float2* __restrict__ rho2) {
    const int i = blockIdx.x * CELL_THREADS + threadIdx.x;
    if (i < n_items) cell_density_item(i, wc, cp, fc, rho2);
}

// One time step of every item: own population pairs, neighbour densities of the
// density pass (0 where x + e_k is not fluid for the wetting component, i.e.
// grain or beyond the box), collide_core (the compile-time tau = 1 form when
// TAU1), push: one 8-byte store per direction where both components stream
// alike, separate stores where a membrane makes them differ.  The bounce-back
// choice selects an address rather than a branch: one store instruction per
// value for the whole warp, whichever way each lane goes.
template <bool TAU1, class NB>
__device__ __forceinline__ void cell_step_item(int i, const int2* __restrict__ items, int cp,
                                               const float2* __restrict__ fin, float2* __restrict__ fout,
                                               const float2* __restrict__ rho2, const uint32_t* __restrict__ wc,
                                               const uint32_t* __restrict__ wnc, const uint32_t* __restrict__ adhc,
                                               const NB* __restrict__ nbp, const Phys& P,
                                               const float* __restrict__ bc_all, int ladder_stride,
                                               const int* __restrict__ incr_now) {
    const uint32_t w = __ldg(wc + i);
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    const bool has_nw = cls != CLS_MEMBRANE;
    float f[2][Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const float2 v = __ldg(fin + (size_t)k * cp + i);
        f[0][k] = v.x;
        f[1][k] = has_nw ? v.y : 0.f;
    }
    const uint32_t wn = (w & BIT_NW_DIFF) ? __ldg(wnc + i) : w;  // read only next to a membrane
    const uint32_t a = (w & BIT_ADH) ? __ldg(adhc + i) : 0u;
    int dst[Q];  // item of x + e_k
#pragma unroll
    for (int k = 1; k < Q; ++k)
        dst[k] = k == 1 ? i + 1 : k == 2 ? i - 1 : nb_decode(__ldg(nbp + (size_t)(k - 3) * cp + i), i);
    auto rho_at = [&](int k) {
        if (k == 0) return __ldg(rho2 + i);
        const bool wall = (w >> OPP(k)) & 1u;
        const float2 v = __ldg(rho2 + (wall ? i : dst[k]));
        return wall ? make_float2(0.f, 0.f) : v;
    };
    Phys Pt = P;
    if (cls == CLS_INLET || cls == CLS_OUTLET)  // the reservoir pair of the throat's current increment
        Pt.bc = bc_all + 4 * ((size_t)__ldg(&items[i].x) * ladder_stride + *incr_now);
    float o[2][Q];
    collide_core<TAU1>(f, w, a, Pt, rho_at, [&](int s, int k, float v) { o[s][k] = v; });
    auto addr = [&](int k, uint32_t bits) {
        return ((bits >> OPP(k)) & 1u) ? (size_t)OPP(k) * cp + i : (size_t)k * cp + dst[k];
    };
    float* fo = reinterpret_cast<float*>(fout);
    if (!has_nw) {
        fo[2 * (size_t)i] = o[0][0];
#pragma unroll
        for (int k = 1; k < Q; ++k) fo[2 * addr(k, w)] = o[0][k];
    } else if (w & BIT_NW_DIFF) {
        fout[i] = make_float2(o[0][0], o[1][0]);
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            fo[2 * addr(k, w)] = o[0][k];
            fo[2 * addr(k, wn) + 1] = o[1][k];
        }
    } else {
        fout[i] = make_float2(o[0][0], o[1][0]);
#pragma unroll
        for (int k = 1; k < Q; ++k) fout[addr(k, w)] = make_float2(o[0][k], o[1][k]);
    }
}

// four CTAs of 256 per SM (64 registers a thread, a few spilled): 32 warps hide
// more of the neighbour-density and push-table latency than 24 or 16 (427, 424
// and 402 throats/s on the 1024-throat batch)
template <bool TAU1, class NB>
__global__ void __launch_bounds__(CELL_THREADS, 4)
    cell_step_kernel(const int2* __restrict__ items, int n_items, int cp, const float2* __restrict__ fin,
                     float2* __restrict__ fout, const float2* __restrict__ rho2, const uint32_t* __restrict__ wc,
                     const uint32_t* __restrict__ wnc, const uint32_t* __restrict__ adhc, const NB* __restrict__ nbp,
                     Phys P, const float* __restrict__ bc_all, int ladder_stride, const int* __restrict__ incr_now) {
    const int i = blockIdx.x * CELL_THREADS + threadIdx.x;
    if (i < n_items)
        cell_step_item<TAU1, NB>(i, items, cp, fin, fout, rho2, wc, wnc, adhc, nbp, P, bc_all, ladder_stride,
                                 incr_now);
}

// One time step of the cell list in one launch, a CTA per chunk of a throat's
// planes.  Chunk (b, nz, z0, z1): plane_item[b + z] is the first item of plane
// z of its throat (items follow memory order inside a throat), plane_item[b + nz]
// its end.  The CTA computes the densities of planes z0 - 1 .. z1 (those in the
// box) plane by plane and steps each plane of [z0, z1) right after the density
// of the plane above it: density(z), barrier, step(z - 1).  A plane's pairs are
// read for its density and again for its step one plane later, from cache
// rather than DRAM.  Chunks of one throat compute the densities of their shared
// boundary planes twice, with the same values.
// MT threads a CTA, MINB CTAs an SM (which caps a thread's registers).
template <int MT, int MINB, bool TAU1, class NB>
__global__ void __launch_bounds__(MT, MINB)
    cell_march_kernel(const int4* __restrict__ chunks, const int* __restrict__ plane_item,
                      const int2* __restrict__ items, int cp, const float2* __restrict__ fin, float2* __restrict__ fout,
                      float2* __restrict__ rho2, const uint32_t* __restrict__ wc, const uint32_t* __restrict__ wnc,
                      const uint32_t* __restrict__ adhc, const NB* __restrict__ nbp, Phys P,
                      const float* __restrict__ bc_all, int ladder_stride, const int* __restrict__ incr_now) {
    const int4 ch = chunks[blockIdx.x];
    const int* pl = plane_item + ch.x;
    const int nz = ch.y, z0 = ch.z, z1 = ch.w;
    auto step_plane = [&](int z) {
#pragma unroll 1
        for (int i = __ldg(pl + z) + (int)threadIdx.x; i < __ldg(pl + z + 1); i += MT)
            cell_step_item<TAU1, NB>(i, items, cp, fin, fout, rho2, wc, wnc, adhc, nbp, P, bc_all, ladder_stride,
                                     incr_now);
    };
    const int zs = max(z0 - 1, 0), ze = min(z1, nz - 1);
    for (int z = zs; z <= ze; ++z) {
#pragma unroll 1
        for (int i = __ldg(pl + z) + (int)threadIdx.x; i < __ldg(pl + z + 1); i += MT)
            cell_density_item(i, wc, cp, fin, rho2);
        __syncthreads();  // densities of plane z visible to every thread of the CTA
        if (z - 1 >= z0 && z - 1 < z1) step_plane(z - 1);
    }
    if (z1 == nz) step_plane(nz - 1);  // no plane above the top one
}

// One marching step with MT threads a CTA over n_chunks chunks.
template <int MT, int MINB>
cudaError_t launch_march_mt(bool t1, bool nb16, int n_chunks, cudaStream_t s, const int4* chunks,
                            const int* plane_item, const int2* items, int cp, const float2* fin, float2* fout,
                            float2* rho2, const uint32_t* wc, const uint32_t* wnc, const uint32_t* adhc,
                            const void* nbp, const Phys& P, const float* bc, int ls, const int* incr) {
    const int16_t* n16 = static_cast<const int16_t*>(nbp);
    const int* n32 = static_cast<const int*>(nbp);
    if (t1 && nb16)
        cell_march_kernel<MT, MINB, true, int16_t><<<n_chunks, MT, 0, s>>>(chunks, plane_item, items, cp, fin, fout,
                                                                         rho2, wc, wnc, adhc, n16, P, bc, ls, incr);
    else if (t1)
        cell_march_kernel<MT, MINB, true, int><<<n_chunks, MT, 0, s>>>(chunks, plane_item, items, cp, fin, fout, rho2,
                                                                     wc, wnc, adhc, n32, P, bc, ls, incr);
    else if (nb16)
        cell_march_kernel<MT, MINB, false, int16_t><<<n_chunks, MT, 0, s>>>(chunks, plane_item, items, cp, fin, fout,
                                                                          rho2, wc, wnc, adhc, n16, P, bc, ls, incr);
    else
        cell_march_kernel<MT, MINB, false, int><<<n_chunks, MT, 0, s>>>(chunks, plane_item, items, cp, fin, fout,
                                                                      rho2, wc, wnc, adhc, n32, P, bc, ls, incr);
    return cudaGetLastError();
}

cudaError_t launch_march(int mt, bool t1, bool nb16, int n_chunks, cudaStream_t s, const int4* chunks,
                         const int* plane_item, const int2* items, int cp, const float2* fin, float2* fout,
                         float2* rho2, const uint32_t* wc, const uint32_t* wnc, const uint32_t* adhc, const void* nbp,
                         const Phys& P, const float* bc, int ls, const int* incr) {
    switch (mt) {
        case 128:
            return launch_march_mt<128, 4>(t1, nb16, n_chunks, s, chunks, plane_item, items, cp, fin, fout, rho2, wc,
                                           wnc, adhc, nbp, P, bc, ls, incr);
        case 256:
            return launch_march_mt<256, 2>(t1, nb16, n_chunks, s, chunks, plane_item, items, cp, fin, fout, rho2, wc,
                                           wnc, adhc, nbp, P, bc, ls, incr);
        case 384:
            return launch_march_mt<384, 1>(t1, nb16, n_chunks, s, chunks, plane_item, items, cp, fin, fout, rho2, wc,
                                           wnc, adhc, nbp, P, bc, ls, incr);
        case 512:
            return launch_march_mt<512, 1>(t1, nb16, n_chunks, s, chunks, plane_item, items, cp, fin, fout, rho2, wc,
                                           wnc, adhc, nbp, P, bc, ls, incr);
    }
    return cudaErrorInvalidValue;
}

// Measurements of the cell-list form from the compact populations, one CTA per
// slice of a throat box: slice (throat, first box cell, end box cell, index of
// the throat's first slice), walked in the box order of the box-layout forms
// through the box -> item map (the same sums, the same rounding).  The last CTA
// of a throat to finish adds its slices' sums in slice order and writes the
// row; the last CTA of all advances the increment index.
__global__ void __launch_bounds__(BATCH_THREADS)
    cell_measure_kernel(const ThroatRec* __restrict__ recs, const int4* __restrict__ slices, int n_slices,
                        const int* __restrict__ box_to_item, int cp, const float2* __restrict__ fc,
                        const uint32_t* __restrict__ wc, double G, const double* __restrict__ rin_all,
                        int ladder_stride, lbm_increment* __restrict__ rows, int n_incr, double* partials,
                        int* throat_done, int* incr_now, int* done) {
    __shared__ double red[32];
    __shared__ int s_last;
    const int4 S = slices[blockIdx.x];
    const int id = S.x;
    const int incr = *incr_now;
    const Geom g = recs[id].g;
    const int* map = box_to_item + recs[id].c_off;
    auto state = [&](int c, float& rw, float& rn) {
        rw = 0.f;
        rn = 0.f;
        const int j = map[c];
        if (j < 0) return (uint32_t)CLS_SOLID << CLS_SHIFT;
        const uint32_t w = wc[j];
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        for (int k = 0; k < Q; ++k) rw += fc[(size_t)k * cp + j].x;
        if (cls != CLS_MEMBRANE)
            for (int k = 0; k < Q; ++k) rn += fc[(size_t)k * cp + j].y;
        return w;
    };
    double part[NMEAS];
    measure_slice(S.y, S.z, G, red, state, part);
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int n_sl = (g.nxy * g.nz + MEAS_SLICE - 1) / MEAS_SLICE;
    if (tid == 0) {
        for (int i = 0; i < NMEAS; ++i) partials[(size_t)blockIdx.x * NMEAS + i] = part[i];
        __threadfence();
        s_last = atomicAdd(throat_done + id, 1) == n_sl - 1;
    }
    __syncthreads();
    if (tid == 0) {
        if (s_last) {  // every slice of this throat has stored its sums
            __threadfence();
            throat_done[id] = 0;
            double tot[NMEAS];
            for (int i = 0; i < NMEAS; ++i) tot[i] = 0.0;
            for (int q = 0; q < n_sl; ++q)
                for (int i = 0; i < NMEAS; ++i) tot[i] += __ldcg(partials + (size_t)(S.w + q) * NMEAS + i);
            const int probe = recs[id].probe;
            float pr[2] = {0.f, 0.f};
            if (probe >= 0) state(probe, pr[0], pr[1]);
            measure_row(tot, rin_all[(size_t)id * ladder_stride + incr], probe, pr[0], pr[1],
                        rows + (size_t)id * n_incr + incr);
        }
        __threadfence();
        if (atomicAdd(done, 1) == n_slices - 1) {  // every CTA has read the index
            *done = 0;
            *incr_now = incr + 1;
        }
    }
}

// Rest-equilibrium start of every throat: wetting fluid (rho_major, rho_minor)
// everywhere, (rho_minor, rho_major) on the inlet layer; stored so that the first
// pull yields exactly that (as init_kernel).
__global__ void throat_init_kernel(const ThroatRec* __restrict__ recs, int n, float* arena,
                                   const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw,
                                   float rho_major, float rho_minor) {
    const int id = blockIdx.x;
    if (id >= n) return;
    const Geom g = recs[id].g;
    float* f = arena + recs[id].f_off;
    const uint32_t* tn = nbr + recs[id].c_off;
    const uint32_t* tnn = nbr_nw + recs[id].c_off;
    const int N = g.nxy * g.nz;
    auto rho_of = [&](int c, int s) {
        const uint32_t cls = (tn[c] >> CLS_SHIFT) & CLS_MASK;
        const bool inlet = cls == CLS_INLET;
        return s == 0 ? (inlet ? rho_minor : rho_major) : (inlet ? rho_major : rho_minor);
    };
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        const int x = c % g.nx, y = (c / g.nx) % g.ny, z = c / g.nxy;
        const uint32_t w = tn[c];
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        for (int s = 0; s < 2; ++s) {
            const bool fl = cls != CLS_SOLID && !(s == 1 && cls == CLS_MEMBRANE);
            const uint32_t bits = s == 0 ? w : tnn[c];
            float* fs = f + (size_t)s * Q * g.plane;
            const float r = fl ? rho_of(c, s) : 0.f;
            float sum = 0.f;
            for (int i = 1; i < Q; ++i) sum += WK(i) * r;
            for (int j = 0; j < Q; ++j) {
                float v = 0.f;
                if (fl && j == 0) {
                    v = r - sum;
                } else if (fl) {
                    if ((bits >> OPP(j)) & 1u) {
                        v = WK(j) * r;
                    } else {
                        bool ok = true;
                        const int tx = wrap1(x + EX(j), g.nx, g.px, ok);
                        const int ty = wrap1(y + EY(j), g.ny, g.py, ok);
                        const int tz = wrap1(z + EZ(j), g.nz, g.pz, ok);
                        v = WK(j) * rho_of(tz * g.nxy + ty * g.nx + tx, s);
                    }
                }
                fs[(size_t)j * g.plane + c] = v;
            }
        }
    }
}

size_t batch_smem() {
    return sizeof(float) * (size_t)((BATCH_LEAD + 1) * 2 * Q + 4 * 2 + 2 * (BATCH_LEAD + 1)) * BATCH_THREADS;
}

int fail_cuda(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

}  // namespace

}  // namespace lbmk

using namespace lbmk;

extern "C" int lbm_throat_geometry(const double* spheres3, int dims_out[3], unsigned char* mask_out,
                                   int probe_out[3]) {
    if (!spheres3 || !dims_out) {
        set_error("lbm_throat_geometry: NULL argument");
        return LBM_ERR_ARG;
    }
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(spheres3[i])) {
            set_error("lbm_throat_geometry: non-finite sphere entry");
            return LBM_ERR_ARG;
        }
    double a[3], b[3], n[3];
    for (int d = 0; d < 3; ++d) {
        a[d] = spheres3[4 + d] - spheres3[d];
        b[d] = spheres3[8 + d] - spheres3[d];
    }
    n[0] = a[1] * b[2] - a[2] * b[1];
    n[1] = a[2] * b[0] - a[0] * b[2];
    n[2] = a[0] * b[1] - a[1] * b[0];
    if (n[0] * n[0] + n[1] * n[1] + n[2] * n[2] <= 1e-12) {
        set_error("lbm_throat_geometry: the three centres are collinear");
        return LBM_ERR_ARG;
    }
    double org[3], loc[12];
    throat_frame(spheres3, dims_out, org, loc);
    if (dims_out[0] > 512 || dims_out[1] > 512 || dims_out[2] > 512) {
        set_error("lbm_throat_geometry: throat box larger than 512 cells along an axis");
        return LBM_ERR_ARG;
    }
    if (mask_out) {
        int probe[3];
        voxelise_throat(spheres3, mask_out, probe);
        if (probe_out) std::memcpy(probe_out, probe, sizeof(probe));
    }
    return LBM_OK;
}

extern "C" int lbm_run_throat_batch(const double* throats, int n, const lbm_params* params,
                                    const lbm_schedule* sched, lbm_throat_result* results, lbm_increment* rows,
                                    void* stream_ptr) {
    if (!throats || n < 1 || !params || !sched || !results || !rows || !sched->rho_in_nw || sched->n_incr < 1 ||
        sched->n_steps < 0 || (sched->per_throat != 0 && sched->per_throat != 1) || sched->batch_form < 0 ||
        sched->batch_form > LBM_BATCH_MARCH) {
        set_error("lbm_run_throat_batch: NULL argument or empty batch/schedule");
        return LBM_ERR_ARG;
    }
    for (int s = 0; s < 2; ++s)
        if (!(params->tau[s] > 0.5)) {
            set_error("lbm_run_throat_batch: tau must be > 0.5");
            return LBM_ERR_ARG;
        }
    const int march_threads = sched->march_threads ? sched->march_threads : LBM_MARCH_THREADS;
    const int march_planes = sched->march_planes ? sched->march_planes : LBM_MARCH_PLANES;
    if ((march_threads != 128 && march_threads != 256 && march_threads != 384 && march_threads != 512) ||
        march_planes < 1 || march_planes > 64) {
        set_error("lbm_run_throat_batch: march_threads must be 0, 128, 256, 384 or 512 and march_planes 0 .. 64");
        return LBM_ERR_ARG;
    }
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    const int I = sched->n_incr;
    try {
        const int form = sched->batch_form == LBM_BATCH_AUTO ? LBM_BATCH_CELLS : sched->batch_form;
        const bool cell_list = form == LBM_BATCH_CELLS || form == LBM_BATCH_MARCH;
        const bool box_layout = !cell_list;  // the cell-list forms keep compact arenas only
        // host geometry: frames and sizes first (validation, on this thread), then
        // masks, probes and per-throat lists on all host cores
        std::vector<ThroatRec> recs((size_t)n);
        std::vector<std::vector<uint8_t>> masks((size_t)n);
        std::vector<std::array<int, 3>> dims((size_t)n), probes((size_t)n);
        for (int t = 0; t < n; ++t) {
            int rc = lbm_throat_geometry(throats + 12 * t, dims[t].data(), nullptr, nullptr);
            if (rc) return rc;
        }
        std::vector<std::vector<int>> tiles_of((size_t)n), cells_of((size_t)n);
        if (!host_parallel_for(n, [&](int t) {
                const int nx = dims[t][0], ny = dims[t][1], nz = dims[t][2];
                const size_t nxy = (size_t)nx * ny;
                masks[t].resize(nxy * nz);
                int d[3];
                lbm_throat_geometry(throats + 12 * t, d, masks[t].data(), probes[t].data());
                const uint8_t* m = masks[t].data();
                long long nf = 0;
                for (size_t c = 0; c < masks[t].size(); ++c) nf += m[c] == 0;
                results[t].n_fluid = nf;
                if (!box_layout) {
                    // non-solid cells in memory order: x | y << 10 | z << 20
                    std::vector<int>& cl = cells_of[t];
                    for (int z = 0; z < nz; ++z)
                        for (int y = 0; y < ny; ++y)
                            for (int x = 0; x < nx; ++x)
                                if (!(m[(size_t)z * nxy + (size_t)y * nx + x] & LBM_MASK_SOLID))
                                    cl.push_back(x | (y << 10) | (z << 20));
                    return;
                }
                // active tiles: the (30 x 4)-column tiles of the step kernel that
                // hold a non-solid cell at some height
                std::vector<uint8_t> col(nxy, 0);
                for (int z = 0; z < nz; ++z)
                    for (size_t c = 0; c < nxy; ++c)
                        if (!(m[(size_t)z * nxy + c] & LBM_MASK_SOLID)) col[c] = 1;
                const int TYB = BATCH_BY - 2;
                for (int ty = 0; ty * TYB < ny; ++ty)
                    for (int tx = 0; tx * 30 < nx; ++tx) {
                        bool any = false;
                        for (int y = ty * TYB; y < std::min(ny, ty * TYB + TYB) && !any; ++y)
                            for (int x = tx * 30; x < std::min(nx, tx * 30 + 30); ++x)
                                if (col[(size_t)y * nx + x]) { any = true; break; }
                        if (any) tiles_of[t].push_back(tx | (ty << 16));
                    }
            })) {
            set_error("host allocation failed");
            return LBM_ERR_OOM;
        }
        long long f_tot = 0, c_tot = 0;
        std::vector<int> tiles;
        for (int t = 0; t < n; ++t) {
            const int* dm = dims[t].data();
            const int* probe = probes[t].data();
            const long long N = (long long)dm[0] * dm[1] * dm[2];
            Geom& g = recs[t].g;
            std::memset(&g, 0, sizeof(g));
            g.nx = dm[0];
            g.ny = dm[1];
            g.nz = dm[2];
            g.nxy = dm[0] * dm[1];
            g.plane = (int)((N + 31) / 32 * 32);
            fill_pull_offsets(g);
            recs[t].f_off = f_tot;
            recs[t].c_off = c_tot;
            recs[t].probe = probe[0] < 0 ? -1 : (probe[2] * dm[1] + probe[1]) * dm[0] + probe[0];
            f_tot += (long long)g.plane * 2 * Q;
            c_tot += N;
            recs[t].tile_begin = (int)tiles.size();
            tiles.insert(tiles.end(), tiles_of[t].begin(), tiles_of[t].end());
            recs[t].tile_count = (int)tiles_of[t].size();
            lbm_throat_result& r = results[t];
            r.dims[0] = dm[0];
            r.dims[1] = dm[1];
            r.dims[2] = dm[2];
            std::memcpy(r.probe, probe, sizeof(int) * 3);
        }
        // most work first (active tiles x planes; non-solid cells in the cell-list form)
        std::vector<int> order((size_t)n);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            if (!box_layout) return cells_of[a].size() > cells_of[b].size();
            return (long long)recs[a].tile_count * recs[a].g.nz > (long long)recs[b].tile_count * recs[b].g.nz;
        });

        float *a0 = nullptr, *a1 = nullptr, *d_bc = nullptr;
        uint8_t* d_mask = nullptr;
        uint32_t *d_nbr = nullptr, *d_nbr_nw = nullptr, *d_adh = nullptr;
        ThroatRec* d_recs = nullptr;
        int *d_order = nullptr, *d_counter = nullptr, *d_tiles = nullptr, *d_incr = nullptr;
        int4* d_items = nullptr;
        int2* d_cells = nullptr;
        float2* d_rho2 = nullptr;
        int* d_map = nullptr;
        void* d_nbp = nullptr;
        int* d_plane_item = nullptr;
        int4* d_chunks = nullptr;
        int4* d_slices = nullptr;
        double* d_partials = nullptr;
        int* d_throat_done = nullptr;
        uint32_t* d_wc = nullptr;
        cudaGraphExec_t exec2[2] = {nullptr, nullptr};
        double* d_rin = nullptr;
        lbm_increment* d_rows = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaStream_t cap = nullptr;
        auto cleanup = [&]() {
            cudaFree(a0); cudaFree(a1); cudaFree(d_bc); cudaFree(d_mask); cudaFree(d_nbr); cudaFree(d_nbr_nw);
            cudaFree(d_adh); cudaFree(d_recs); cudaFree(d_order); cudaFree(d_counter); cudaFree(d_rows);
            cudaFree(d_tiles);
            cudaFree(d_rin);
            cudaFree(d_incr);
            cudaFree(d_items);
            cudaFree(d_cells);
            cudaFree(d_rho2);
            cudaFree(d_map);
            cudaFree(d_nbp);
            cudaFree(d_plane_item);
            cudaFree(d_chunks);
            cudaFree(d_slices);
            cudaFree(d_partials);
            cudaFree(d_throat_done);
            cudaFree(d_wc);
            if (exec) cudaGraphExecDestroy(exec);
            for (cudaGraphExec_t& e : exec2)
                if (e) cudaGraphExecDestroy(e);
            if (cap) cudaStreamDestroy(cap);
        };
#define BATCH_CUDA(call)                               \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) {                       \
            cleanup();                                 \
            return fail_cuda(e_, #call);               \
        }                                              \
    } while (0)
        if (box_layout) {
            BATCH_CUDA(cudaMalloc(&a0, sizeof(float) * (size_t)f_tot));
            BATCH_CUDA(cudaMalloc(&a1, sizeof(float) * (size_t)f_tot));
        }
        BATCH_CUDA(cudaMalloc(&d_mask, (size_t)c_tot));
        BATCH_CUDA(cudaMalloc(&d_nbr, sizeof(uint32_t) * (size_t)c_tot));
        BATCH_CUDA(cudaMalloc(&d_nbr_nw, sizeof(uint32_t) * (size_t)c_tot));
        BATCH_CUDA(cudaMalloc(&d_adh, sizeof(uint32_t) * (size_t)c_tot));
        BATCH_CUDA(cudaMalloc(&d_recs, sizeof(ThroatRec) * (size_t)n));
        BATCH_CUDA(cudaMalloc(&d_order, sizeof(int) * (size_t)n));
        BATCH_CUDA(cudaMalloc(&d_tiles, sizeof(int) * std::max<size_t>(1, tiles.size())));
        BATCH_CUDA(cudaMalloc(&d_counter, sizeof(int) * (size_t)I));
        BATCH_CUDA(cudaMalloc(&d_rows, sizeof(lbm_increment) * (size_t)n * I));
        const int L = sched->per_throat ? n : 1;  // ladders
        BATCH_CUDA(cudaMalloc(&d_bc, sizeof(float) * 4 * (size_t)I * L));
        BATCH_CUDA(cudaMalloc(&d_rin, sizeof(double) * (size_t)I * L));
        if (box_layout) {
            BATCH_CUDA(cudaMemsetAsync(a0, 0, sizeof(float) * (size_t)f_tot, stream));
            BATCH_CUDA(cudaMemsetAsync(a1, 0, sizeof(float) * (size_t)f_tot, stream));
        }
        {
            std::vector<uint8_t> all((size_t)c_tot);
            for (int t = 0; t < n; ++t) std::memcpy(all.data() + recs[t].c_off, masks[t].data(), masks[t].size());
            BATCH_CUDA(cudaMemcpyAsync(d_mask, all.data(), (size_t)c_tot, cudaMemcpyHostToDevice, stream));
            for (int t = 0; t < n; ++t)
                BATCH_CUDA(launch_geometry(d_mask + recs[t].c_off, d_nbr + recs[t].c_off, d_nbr_nw + recs[t].c_off,
                                           d_adh + recs[t].c_off, recs[t].g, stream));
            BATCH_CUDA(cudaMemcpyAsync(d_recs, recs.data(), sizeof(ThroatRec) * (size_t)n, cudaMemcpyHostToDevice,
                                       stream));
            BATCH_CUDA(cudaMemcpyAsync(d_order, order.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, stream));
            if (!tiles.empty())
                BATCH_CUDA(cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice,
                                           stream));
            std::vector<float> bc((size_t)4 * I * L);
            for (size_t i = 0; i < (size_t)I * L; ++i) {
                bc[4 * i + 0] = (float)params->rho_minor;
                bc[4 * i + 1] = (float)sched->rho_in_nw[i];
                bc[4 * i + 2] = (float)sched->rho_out_w;
                bc[4 * i + 3] = (float)params->rho_minor;
            }
            BATCH_CUDA(cudaMemcpyAsync(d_bc, bc.data(), sizeof(float) * bc.size(), cudaMemcpyHostToDevice, stream));
            BATCH_CUDA(cudaMemcpyAsync(d_rin, sched->rho_in_nw, sizeof(double) * (size_t)I * L,
                                       cudaMemcpyHostToDevice, stream));
            if (box_layout)
                throat_init_kernel<<<n, 256, 0, stream>>>(d_recs, n, a0, d_nbr, d_nbr_nw, (float)params->rho_major,
                                                      (float)params->rho_minor);
            BATCH_CUDA(cudaGetLastError());
            BATCH_CUDA(cudaStreamSynchronize(stream));  // host staging buffers go out of scope
        }
        Phys P;
        P.bc = d_bc;  // per throat and increment inside the kernel
        for (int s = 0; s < 2; ++s) {
            P.tau[s] = (float)params->tau[s];
            P.omega[s] = (float)(1.0 / params->tau[s]);
            P.Gads[s] = (float)params->G_ads[s];
        }
        P.G = (float)params->G;
        for (int d = 0; d < 3; ++d) P.g[d] = (float)params->body_force[d];

        auto kern = throat_batch_kernel<BATCH_BY, BATCH_LEAD>;
        const size_t smem = batch_smem();
        BATCH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0, dev = 0, sms = 0;
        BATCH_CUDA(cudaGetDevice(&dev));
        BATCH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        BATCH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BATCH_THREADS, smem));
        const int grid = std::max(1, std::min(n, sms * std::max(1, per_sm)));
        BATCH_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));

        if (cell_list) {
            // every non-solid cell of every throat (largest throats first,
            // memory order inside a throat), and the box -> item map
            std::vector<long long> item0((size_t)n);
            long long n_items = 0;
            for (int t : order) {
                item0[t] = n_items;
                n_items += (long long)cells_of[t].size();
            }
            if (n_items > (long long)INT_MAX - 64) {
                cleanup();
                set_error("lbm_run_throat_batch: too many cells for the cell-list form");
                return LBM_ERR_ARG;
            }
            std::vector<int2> cells((size_t)n_items);
            std::vector<int> box_to_item((size_t)c_tot);
            host_parallel_for(n, [&](int t) {
                const Geom& g = recs[t].g;
                int* map = box_to_item.data() + recs[t].c_off;
                std::fill(map, map + (size_t)g.nxy * g.nz, -1);
                const std::vector<int>& cl = cells_of[t];
                for (size_t j = 0; j < cl.size(); ++j) {
                    const int v = cl[j];
                    const int item = (int)(item0[t] + (long long)j);
                    cells[(size_t)item] = make_int2(t, v);
                    map[(size_t)(v >> 20) * g.nxy + (size_t)((v >> 10) & 1023) * g.nx + (v & 1023)] = item;
                }
            });
            const int n_cells = (int)cells.size();
            const int cp = (n_cells + 31) / 32 * 32;
            // marching form: the first item of every plane of every throat, and
            // chunks of at most march_planes planes, largest throats first
            int n_chunks = 0;
            if (form == LBM_BATCH_MARCH) {
                std::vector<int> plane_item;
                std::vector<int4> chunks;
                for (int t : order) {
                    const int nz = recs[t].g.nz, base = (int)plane_item.size();
                    const std::vector<int>& cl = cells_of[t];
                    size_t j = 0;
                    for (int z = 0; z <= nz; ++z) {
                        while (j < cl.size() && (cl[j] >> 20) < z) ++j;
                        plane_item.push_back((int)(item0[t] + (long long)j));
                    }
                    for (int z0 = 0; z0 < nz; z0 += march_planes)
                        chunks.push_back(make_int4(base, nz, z0, std::min(nz, z0 + march_planes)));
                }
                n_chunks = (int)chunks.size();
                BATCH_CUDA(cudaMalloc(&d_plane_item, sizeof(int) * std::max<size_t>(1, plane_item.size())));
                BATCH_CUDA(cudaMalloc(&d_chunks, sizeof(int4) * std::max<size_t>(1, chunks.size())));
                BATCH_CUDA(cudaMemcpyAsync(d_plane_item, plane_item.data(), sizeof(int) * plane_item.size(),
                                           cudaMemcpyHostToDevice, stream));
                if (n_chunks)
                    BATCH_CUDA(cudaMemcpyAsync(d_chunks, chunks.data(), sizeof(int4) * chunks.size(),
                                               cudaMemcpyHostToDevice, stream));
            }
            // measurement slices of every throat box
            std::vector<int4> slices;
            for (int t = 0; t < n; ++t) {
                const int N = recs[t].g.nxy * recs[t].g.nz, first = (int)slices.size();
                for (int c0 = 0; c0 < N; c0 += MEAS_SLICE)
                    slices.push_back(make_int4(t, c0, std::min(N, c0 + MEAS_SLICE), first));
            }
            const int n_slices = (int)slices.size();
            BATCH_CUDA(cudaMalloc(&d_slices, sizeof(int4) * std::max<size_t>(1, slices.size())));
            BATCH_CUDA(cudaMalloc(&d_partials, sizeof(double) * NMEAS * std::max<size_t>(1, slices.size())));
            BATCH_CUDA(cudaMalloc(&d_throat_done, sizeof(int) * (size_t)n));
            BATCH_CUDA(cudaMemsetAsync(d_throat_done, 0, sizeof(int) * (size_t)n, stream));
            if (n_slices)
                BATCH_CUDA(cudaMemcpyAsync(d_slices, slices.data(), sizeof(int4) * slices.size(),
                                           cudaMemcpyHostToDevice, stream));
            const size_t fc_floats = (size_t)2 * Q * std::max(cp, 32);
            BATCH_CUDA(cudaMalloc(&d_cells, sizeof(int2) * std::max<size_t>(1, cells.size())));
            BATCH_CUDA(cudaMalloc(&d_map, sizeof(int) * (size_t)std::max<long long>(1, c_tot)));
            BATCH_CUDA(cudaMalloc(&d_rho2, sizeof(float2) * (size_t)std::max(cp, 32)));
            BATCH_CUDA(cudaMalloc(&d_wc, sizeof(uint32_t) * 3 * (size_t)std::max(cp, 32)));
            // 16-bit push-table offsets where every throat's neighbours lie within reach
            long long reach = 0;
            for (const ThroatRec& r : recs) reach = std::max(reach, (long long)r.g.nxy + r.g.nx + 1);
            const bool nb16 = reach <= 32767;
            BATCH_CUDA(cudaMalloc(&d_nbp, (nb16 ? sizeof(int16_t) : sizeof(int)) * (size_t)NB_DIRS * std::max(cp, 32)));
            BATCH_CUDA(cudaMalloc(&a0, sizeof(float) * fc_floats));
            BATCH_CUDA(cudaMalloc(&a1, sizeof(float) * fc_floats));
            BATCH_CUDA(cudaMalloc(&d_incr, sizeof(int) * 2));
            BATCH_CUDA(cudaMemsetAsync(d_incr, 0, sizeof(int) * 2, stream));
            uint32_t* d_wnc = d_wc + std::max(cp, 32);
            uint32_t* d_adhc = d_wnc + std::max(cp, 32);
            if (c_tot)
                BATCH_CUDA(cudaMemcpyAsync(d_map, box_to_item.data(), sizeof(int) * box_to_item.size(),
                                           cudaMemcpyHostToDevice, stream));
            const unsigned blocks = (unsigned)((n_cells + CELL_THREADS - 1) / CELL_THREADS);
            if (n_cells) {
                BATCH_CUDA(cudaMemcpyAsync(d_cells, cells.data(), sizeof(int2) * cells.size(), cudaMemcpyHostToDevice,
                                           stream));
                if (nb16)
                    cell_gather_kernel<int16_t><<<blocks, CELL_THREADS, 0, stream>>>(
                        d_recs, d_cells, n_cells, cp, d_nbr, d_nbr_nw, d_adh, d_map, d_wc, d_wnc, d_adhc,
                        static_cast<int16_t*>(d_nbp));
                else
                    cell_gather_kernel<int><<<blocks, CELL_THREADS, 0, stream>>>(d_recs, d_cells, n_cells, cp, d_nbr,
                                                                                d_nbr_nw, d_adh, d_map, d_wc, d_wnc,
                                                                                d_adhc, static_cast<int*>(d_nbp));
                BATCH_CUDA(cudaGetLastError());
                cell_init_kernel<<<blocks, CELL_THREADS, 0, stream>>>(d_wc, n_cells, cp, reinterpret_cast<float2*>(a0),
                                                                     (float)params->rho_major,
                                                                     (float)params->rho_minor);
                BATCH_CUDA(cudaGetLastError());
            }
            BATCH_CUDA(cudaStreamSynchronize(stream));  // host lists go out of scope
            const int n_graphs = (sched->n_steps & 1) ? 2 : 1;
            for (int gi = 0; gi < n_graphs; ++gi) {
                BATCH_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
                cudaError_t cerr = cudaSuccess;
                for (int st = 0; st < sched->n_steps && cerr == cudaSuccess && n_cells; ++st) {
                    const int c = (gi + st) & 1;
                    const float2* fin = reinterpret_cast<const float2*>(c ? a1 : a0);
                    float2* fout = reinterpret_cast<float2*>(c ? a0 : a1);
                    const bool t1 = P.tau[0] == 1.0f && P.tau[1] == 1.0f;
                    const int ls = sched->per_throat ? I : 0;
                    const int16_t* nb16p = static_cast<const int16_t*>(d_nbp);
                    const int* nb32p = static_cast<const int*>(d_nbp);
                    if (form == LBM_BATCH_MARCH) {
                        if (n_chunks)
                            cerr = launch_march(march_threads, t1, nb16, n_chunks, cap, d_chunks, d_plane_item,
                                                d_cells, cp, fin, fout, d_rho2, d_wc, d_wnc, d_adhc, d_nbp, P, d_bc,
                                                ls, d_incr);
                        else
                            cerr = cudaGetLastError();
                        continue;
                    }
                    cell_density_kernel<<<blocks, CELL_THREADS, 0, cap>>>(d_wc, n_cells, cp, fin, d_rho2);
                    cerr = cudaGetLastError();
                    if (cerr != cudaSuccess) break;
                    if (t1 && nb16)
                        cell_step_kernel<true, int16_t><<<blocks, CELL_THREADS, 0, cap>>>(
                            d_cells, n_cells, cp, fin, fout, d_rho2, d_wc, d_wnc, d_adhc, nb16p, P, d_bc, ls, d_incr);
                    else if (t1)
                        cell_step_kernel<true, int><<<blocks, CELL_THREADS, 0, cap>>>(
                            d_cells, n_cells, cp, fin, fout, d_rho2, d_wc, d_wnc, d_adhc, nb32p, P, d_bc, ls, d_incr);
                    else if (nb16)
                        cell_step_kernel<false, int16_t><<<blocks, CELL_THREADS, 0, cap>>>(
                            d_cells, n_cells, cp, fin, fout, d_rho2, d_wc, d_wnc, d_adhc, nb16p, P, d_bc, ls, d_incr);
                    else
                        cell_step_kernel<false, int><<<blocks, CELL_THREADS, 0, cap>>>(
                            d_cells, n_cells, cp, fin, fout, d_rho2, d_wc, d_wnc, d_adhc, nb32p, P, d_bc, ls, d_incr);
                    cerr = cudaGetLastError();
                }
                if (cerr == cudaSuccess) {
                    const int c = (gi + sched->n_steps) & 1;
                    cell_measure_kernel<<<n_slices, dim3(32, BATCH_BY), 0, cap>>>(
                        d_recs, d_slices, n_slices, d_map, cp, reinterpret_cast<const float2*>(c ? a1 : a0), d_wc,
                        params->G, d_rin, sched->per_throat ? I : 0, d_rows, I, d_partials, d_throat_done, d_incr,
                        d_incr + 1);
                    cerr = cudaGetLastError();
                }
                cudaGraph_t graph = nullptr;
                cudaError_t eend = cudaStreamEndCapture(cap, &graph);
                if (cerr != cudaSuccess || eend != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    cleanup();
                    return fail_cuda(cerr != cudaSuccess ? cerr : eend, "capture of the throat batch");
                }
                cudaError_t einst = cudaGraphInstantiate(&exec2[gi], graph, 0);
                cudaGraphDestroy(graph);
                if (einst != cudaSuccess) {
                    exec2[gi] = nullptr;
                    cleanup();
                    return fail_cuda(einst, "cudaGraphInstantiate");
                }
            }
            for (int i = 0; i < I; ++i)
                BATCH_CUDA(cudaGraphLaunch(exec2[(int)(((long long)i * sched->n_steps) & 1) % n_graphs], stream));
        } else if (form == LBM_BATCH_PER_STEP) {
            // work list: every active tile of every throat, its column cut into
            // z segments of at most 32 planes (largest throats first)
            std::vector<int4> items;
            for (int t : order) {
                const int nz = recs[t].g.nz, nseg = (nz + 31) / 32;
                for (int i = 0; i < recs[t].tile_count; ++i)
                    for (int sgi = 0; sgi < nseg; ++sgi)
                        items.push_back(make_int4(t, tiles[(size_t)recs[t].tile_begin + i], (int)((long long)nz * sgi / nseg),
                                                  (int)((long long)nz * (sgi + 1) / nseg)));
            }
            auto ikern = throat_item_step_kernel<BATCH_BY, BATCH_LEAD>;
            BATCH_CUDA(cudaFuncSetAttribute(ikern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            BATCH_CUDA(cudaMalloc(&d_items, sizeof(int4) * std::max<size_t>(1, items.size())));
            BATCH_CUDA(cudaMalloc(&d_incr, sizeof(int) * 2));  // increment index, finished-CTA count
            BATCH_CUDA(cudaMemsetAsync(d_incr, 0, sizeof(int) * 2, stream));
            if (!items.empty())
                BATCH_CUDA(cudaMemcpyAsync(d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice,
                                           stream));
            BATCH_CUDA(cudaStreamSynchronize(stream));
            // one increment per graph; with an odd number of steps the arenas
            // swap roles from one increment to the next: two graphs
            const int n_graphs = (sched->n_steps & 1) ? 2 : 1;
            for (int gi = 0; gi < n_graphs; ++gi) {
                BATCH_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
                cudaError_t cerr = cudaSuccess;
                for (int st = 0; st < sched->n_steps && cerr == cudaSuccess && !items.empty(); ++st) {
                    const int c = (gi + st) & 1;
                    ikern<<<(unsigned)items.size(), dim3(32, BATCH_BY), smem, cap>>>(
                        d_recs, d_items, c ? a1 : a0, c ? a0 : a1, d_nbr, d_nbr_nw, d_adh, P, d_bc,
                        sched->per_throat ? I : 0, d_incr);
                    cerr = cudaGetLastError();
                }
                if (cerr == cudaSuccess) {
                    const int c = (gi + sched->n_steps) & 1;
                    throat_item_measure_kernel<<<n, dim3(32, BATCH_BY), 0, cap>>>(
                        d_recs, n, c ? a1 : a0, d_nbr, d_nbr_nw, params->G, d_rin, sched->per_throat ? I : 0, d_rows,
                        I, d_incr, d_incr + 1);
                    cerr = cudaGetLastError();
                }
                cudaGraph_t graph = nullptr;
                cudaError_t eend = cudaStreamEndCapture(cap, &graph);
                if (cerr != cudaSuccess || eend != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    cleanup();
                    return fail_cuda(cerr != cudaSuccess ? cerr : eend, "capture of the throat batch");
                }
                cudaError_t einst = cudaGraphInstantiate(&exec2[gi], graph, 0);
                cudaGraphDestroy(graph);
                if (einst != cudaSuccess) {
                    exec2[gi] = nullptr;
                    cleanup();
                    return fail_cuda(einst, "cudaGraphInstantiate");
                }
            }
            for (int i = 0; i < I; ++i)
                BATCH_CUDA(cudaGraphLaunch(exec2[(int)(((long long)i * sched->n_steps) & 1) % n_graphs], stream));
        } else {
        // one launch per increment, all captured in one graph
        BATCH_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t cerr = cudaMemsetAsync(d_counter, 0, sizeof(int) * (size_t)I, cap);
        for (int i = 0; i < I && cerr == cudaSuccess; ++i) {
            const int parity = (int)(((long long)i * sched->n_steps) & 1);
            kern<<<grid, dim3(32, BATCH_BY), smem, cap>>>(d_recs, d_order, n, d_counter + i, d_tiles, a0, a1, d_nbr,
                                                          d_nbr_nw, d_adh, P, sched->n_steps, parity, params->G, d_bc,
                                                          d_rin, sched->per_throat ? I : 0, d_rows, i, I);
            cerr = cudaGetLastError();
        }
        cudaGraph_t graph = nullptr;
        cudaError_t eend = cudaStreamEndCapture(cap, &graph);
        if (cerr != cudaSuccess || eend != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cleanup();
            return fail_cuda(cerr != cudaSuccess ? cerr : eend, "capture of the throat batch");
        }
        cudaError_t einst = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (einst != cudaSuccess) {
            exec = nullptr;
            cleanup();
            return fail_cuda(einst, "cudaGraphInstantiate");
        }
        BATCH_CUDA(cudaGraphLaunch(exec, stream));
        }
        BATCH_CUDA(cudaMemcpyAsync(rows, d_rows, sizeof(lbm_increment) * (size_t)n * I, cudaMemcpyDeviceToHost,
                                   stream));
        BATCH_CUDA(cudaStreamSynchronize(stream));
        cleanup();
#undef BATCH_CUDA
        // invasion and p_c^e per throat (the rule of lbm_run_drainage)
        for (int t = 0; t < n; ++t) {
            const lbm_increment* r = rows + (size_t)t * I;
            int inv = -1;
            for (int i = 0; i < I; ++i)
                if (r[i].phi_probe < 0.0) { inv = i; break; }
            double best = INFINITY;
            if (inv >= 0) {
                best = -INFINITY;
                for (int i = 0; i <= inv; ++i)
                    if (r[i].p_c == r[i].p_c && r[i].p_c > best) best = r[i].p_c;
            }
            results[t].invaded_at = inv;
            results[t].p_ce = best;
        }
        return LBM_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LBM_ERR_OOM;
    }
}
