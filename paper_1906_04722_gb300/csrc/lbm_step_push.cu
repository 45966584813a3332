// lbm_step_push.cu -- the fused two-component Shan-Chen D3Q19 step (FP32) on
// paired push-form storage, with population planes loaded by the tensor memory
// accelerator.
//
// Storage ("paired push" layout, a domain's alternative to the pull layout of
// the other FP32 kernels): float2 F[nz][ny][19][nx], F[z][y][k][x] =
// (f_k^w, f_k^nw) of cell (x, y, z) at the current time level, i.e. the
// populations after streaming and before collision.  The 19 slots of a row of
// cells follow one another, so that a box load reads 19 row segments within one
// stretch of memory per row of cells instead of one segment in each of 19
// arrays far apart (a plain-load streaming probe of this access pattern ran
// 12 % faster in this layout; the step kernel's TMA loads gained 1.5-2 %).  A cell's own 19 pairs are all it needs for its moments
// (Eqs. 2-3); streaming with half-way bounce-back (Eq. 1, left-hand side)
// happens at the store: the post-collision f*_k of cell x goes to slot k of
// x + e_k, or, when x + e_k is not fluid for the component, to slot kbar of x
// itself.  Nothing is ever stored into a solid cell or into the non-wetting
// half of a membrane cell; those slots are never read either (they may hold
// values of the pull layout the buffer held before), the densities being taken
// as zero there from the cell's class.
//
// Data movement.  A CTA of 32 x BY threads owns a box of 32 x BY columns whose
// interior, 28 x (BY - 2) columns, it advances; it marches along z through a
// segment of planes.  For every plane one thread issues a single 4-D TMA box
// load (x as 64 floats, k, y, z: all 19 slots at once, BY x 19 x 256 bytes)
// into one of NS stage buffers, completing on that stage's mbarrier.
// The box starts two cells left of the interior so that its x coordinate stays
// 16-byte aligned; the cells two columns out are loaded and not used.  When a
// plane has landed every thread sums its cell's two densities (four interleaved
// partial sums, as the staged kernel; its geometry word, loaded a plane ahead,
// zeroes a component that is not fluid there) into a 4-plane density ring.  After one
// CTA barrier per plane the interior threads collide the plane behind with the
// 18 neighbour densities at hand (collide_core, the arithmetic of the staged
// kernel, so the results are the staged kernel's bit for bit) and store the
// pairs to global memory: one 8-byte store per direction where both components
// stream alike, separate stores next to a membrane.  The loads of the next
// NS - 2 planes are in flight meanwhile.
//
// DRAM sees each population read once (whole boxes: grain columns of a tile
// ride along) and written once; the box halos, re-read by neighbouring tiles
// that march in step, are served by L2, and the boundary planes of a z
// segment, re-read by the next segment later, are loaded with an evict-last
// policy.
//
// Waits on the mbarriers are bounded in time: a wait that runs out sets *err,
// waits (bounded again) for the copies in flight and ends the CTA.
//
// Requirements (checked on the host): no periodic x or y axis, nx even (the
// tensor map's row pitch must be a multiple of 16 bytes).  z may be periodic.
#include <cuda.h>

#include "lbm_push_tma.cuh"
#include "lbm_step_core.cuh"

namespace lbmk {

namespace {

constexpr int PX = 32;        // box columns (x)
constexpr int PXI = 28;       // interior columns: box lanes 2 .. 29
template <int BY>
constexpr uint32_t stage_bytes() {
    return (uint32_t)(Q * BY * PX * sizeof(float2));
}
template <int BY, int NS>
constexpr size_t push_smem_bytes() {
    return (size_t)NS * stage_bytes<BY>() + sizeof(float2) * 4 * BY * PX + sizeof(uint64_t) * NS;
}

// RR: each interior thread keeps its cell's 19 pairs in registers from the
// density pass to its collision a plane later, so that a stage is free for the
// next load as soon as every thread has summed its densities (all NS stages in
// flight instead of NS - 2; populations read from shared memory once).
template <int BY, int NS, int MINB, bool TAU1, bool RR>
__global__ void __launch_bounds__(PX * BY, MINB)
    sc_step_push_kernel(const __grid_constant__ CUtensorMap tm, float2* __restrict__ fout,
                        const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw,
                        const uint32_t* __restrict__ adh, Geom g, Phys P, int lz, int pf, int order,
                        int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    // an earlier launch or CTA gave up: the whole CTA leaves (one decision for all its threads)
    if (__syncthreads_or(*reinterpret_cast<volatile int*>(err) != 0)) return;
    constexpr int TY = BY - 2;
    constexpr int NT = PX * BY;
    float2* stages = reinterpret_cast<float2*>(smem);  // [NS][BY][Q][PX]
    float2* ring = reinterpret_cast<float2*>(smem + NS * stage_bytes<BY>());  // [4][BY][PX]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NS * stage_bytes<BY>() + sizeof(float2) * 4 * NT);
    const int lane = threadIdx.x, row = threadIdx.y;
    const int tid = row * PX + lane;
    // order 0: the grid is (x tiles, y tiles, z segments) and every segment
    // marches towards +z.  Order 1: the grid is (z segments, x tiles, y tiles),
    // so that all segments of a tile column run together, and even segments
    // march towards -z: two neighbouring segments start (or end) at the plane
    // they share at the same time, and the second reads its halo planes from L2.
    const int tile_x = order ? blockIdx.y : blockIdx.x, tile_y = order ? blockIdx.z : blockIdx.y;
    const int seg = order ? blockIdx.x : blockIdx.z;
    const int xb = tile_x * PXI - 2;  // box column of lane 0
    const int yb = tile_y * TY - 1;   // box row of row 0
    const int gx = xb + lane, gy = yb + row;
    const int z0 = seg * lz;
    const int z1 = min(z0 + lz, g.nz);
    const int n = z1 - z0;  // planes collided
    const int dir = (order && !(seg & 1)) ? -1 : 1;
    const int start = dir > 0 ? z0 - 1 : z1;  // plane of sequence index 0: the halo before the first
    // the segment's planes in marching order: j = 0 the halo plane before the
    // first collided plane, j = 1 .. n the collided planes, j = n + 1 the halo after
    auto plane = [&](int j) { return start + dir * j; };
    const bool interior = lane >= 2 && lane < 2 + PXI && row >= 1 && row <= TY && gx < g.nx && gy < g.ny;
    const int col = gy * g.nx + gx;  // valid for interior threads

    auto slot = [&](int j) { return j % NS; };
    auto parity = [&](int j) { return (uint32_t)((j / NS) & 1); };
    // plane j of every pair array into its stage; a plane beyond a closed z
    // face is not loaded (its densities are zero) and only completes the phase
    auto issue = [&](int j) {
        uint64_t* b = bar + slot(j);
        int zc = plane(j);
        if (zc < 0 || zc >= g.nz) {
            if (!g.pz) {
                p_mbar_arrive(b);
                return;
            }
            zc = zc < 0 ? zc + g.nz : zc - g.nz;
        }
        p_mbar_arrive_expect_tx(b, stage_bytes<BY>());
        // the segment's two boundary planes are also read by the neighbouring
        // segment, a wave of CTAs later: kept in L2 in preference to the rest
        if (j == 0 || j == n + 1)
            p_tma_load_4d_hint(stages + (size_t)slot(j) * (Q * NT), &tm, 2 * xb, 0, yb, zc, b, p_policy_evict_last());
        else
            p_tma_load_4d(stages + (size_t)slot(j) * (Q * NT), &tm, 2 * xb, 0, yb, zc, b);
    };
    // plane p into L2 ahead of its load (pf planes beyond the loads in flight);
    // the box is moved inside the tensor where it sticks out, so that every
    // coordinate is in range (the hint then covers a few other columns)
    const int pfx = max(0, min(2 * xb, 2 * g.nx - 2 * PX));
    const int pfy = max(0, min(yb, g.ny - BY));
    auto prefetch = [&](int j) {
        if (j > n + 1) return;
        int zc = plane(j);
        if (zc < 0 || zc >= g.nz) {
            if (!g.pz) return;
            zc = zc < 0 ? zc + g.nz : zc - g.nz;
        }
        p_tma_prefetch_4d(&tm, pfx, 0, pfy, zc);
    };
    // geometry word of this thread's box cell on plane j (class CLS_OUTSIDE
    // beyond the box, the segment or a closed z face)
    const bool in_xy = gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny;
    auto word = [&](int j) -> uint32_t {
        if (!in_xy || j > n + 1) return CLS_OUTSIDE << CLS_SHIFT;
        int zc = plane(j);
        if (zc < 0 || zc >= g.nz) {
            if (!g.pz) return CLS_OUTSIDE << CLS_SHIFT;
            zc = zc < 0 ? zc + g.nz : zc - g.nz;
        }
        return __ldg(nbr + (size_t)zc * g.nxy + col);
    };
    // the two densities of this thread's box cell on plane j (geometry word wp)
    // into the ring: 0 where a component is not fluid, whatever the slots hold
    // (a buffer's grain slots may hold another layout's values)
    // (RR: the interior threads keep the pairs in `keep`)
    auto publish = [&](int j, uint32_t wp, float (&keep)[2][Q]) {
        float2 r = make_float2(0.f, 0.f);
        const uint32_t c = (wp >> CLS_SHIFT) & CLS_MASK;
        if (c != CLS_SOLID && c != CLS_OUTSIDE) {
            const float2* st = stages + (size_t)slot(j) * (Q * NT) + row * (Q * PX) + lane;
            float a[4] = {0.f, 0.f, 0.f, 0.f}, b[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const float2 v = st[k * PX];
                a[k & 3] += v.x;
                b[k & 3] += v.y;
                if constexpr (RR) {
                    keep[0][k] = v.x;
                    keep[1][k] = v.y;
                }
            }
            r.x = (a[0] + a[1]) + (a[2] + a[3]);
            if (c != CLS_MEMBRANE) r.y = (b[0] + b[1]) + (b[2] + b[3]);
        }
        ring[(plane(j) & 3) * NT + tid] = r;
    };

    if (tid == 0) {
        for (int i = 0; i < NS; ++i) p_mbar_init(bar + i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    int next = min(NS, n + 2);  // the first sequence index not yet issued (thread 0)
    if (tid == 0) {
        for (int j = 0; j < next; ++j) issue(j);
        for (int j = next; j < next + pf; ++j) prefetch(j);
    }

    // geometry words of sequence planes 0 .. 2, then one plane further per
    // iteration; the adhesion and non-wetting bounce words of an interior cell a
    // plane ahead of its collision
    const uint32_t w_m = word(0);
    uint32_t w_0 = word(1), w_1 = word(2);
    auto extra = [&](int j, uint32_t wp, uint32_t& ap, uint32_t& np) {
        ap = 0u;
        np = 0u;
        if (!interior || j < 1 || j > n) return;
        const int p = plane(j);
        if (wp & BIT_ADH) ap = __ldg(adh + (size_t)p * g.nxy + col);
        if (wp & BIT_NW_DIFF) np = __ldg(nbr_nw + (size_t)p * g.nxy + col);
    };
    uint32_t a_0, nwb_0;
    extra(1, w_0, a_0, nwb_0);

    float fc[2][Q], fn[2][Q];  // RR: pairs of the plane to collide and of the next plane
    bool ok = p_mbar_wait_bounded(bar + slot(0), parity(0));
    if (ok) publish(0, w_m, fn);
    ok = ok && p_mbar_wait_bounded(bar + slot(1), parity(1));
    if (ok) publish(1, w_0, fc);
    // a failed wait here is reported by the first iteration's barrier below
    for (int j = 1; j <= n; ++j) {
        const int z = plane(j);
        const uint32_t w = w_0, a = a_0, nwb = nwb_0;
        const uint32_t w_2 = word(j + 2);  // for the next iteration's publish
        extra(j + 1, w_1, a_0, nwb_0);     // for the next iteration's collision
        const bool okz = ok && p_mbar_wait_bounded(bar + slot(j + 1), parity(j + 1));
        if (okz) publish(j + 1, w_1, fn);
        if (__syncthreads_or(!okz)) {
            if (tid == 0) {
                atomicOr(err, 1);
                // bounded waits for every copy still in flight
                for (int q = max(0, next - NS); q < next; ++q) p_mbar_wait_bounded(bar + slot(q), parity(q));
            }
            __syncthreads();
            return;
        }
        if (tid == 0) {
            // stages read by everyone before the barrier: RR frees the stages of
            // sequence planes up to j + 1, the other form those up to j - 1
            const int last = RR ? j + 1 + NS : j + NS - 1;
            if (next <= n + 1 && next <= last) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            for (; next <= n + 1 && next <= last; ++next) {
                issue(next);
                if (pf > 0) prefetch(next + pf);
            }
        }
        w_0 = w_1;
        w_1 = w_2;
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        if (interior && cls != CLS_SOLID && cls != CLS_OUTSIDE) {
            const float2* st = stages + (size_t)slot(j) * (Q * NT) + row * (Q * PX) + lane;
            float f[2][Q];
            const bool has_nw = cls != CLS_MEMBRANE;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                if constexpr (RR) {
                    f[0][k] = fc[0][k];
                    f[1][k] = has_nw ? fc[1][k] : 0.f;
                } else {
                    const float2 v = st[k * PX];
                    f[0][k] = v.x;
                    f[1][k] = has_nw ? v.y : 0.f;
                }
            }
            float o[2][Q];
            collide_core<TAU1>(
                f, w, a, P,
                [&](int k) { return ring[((z + EZ(k)) & 3) * NT + (row + EY(k)) * PX + (lane + EX(k))]; },
                [&](int s, int k, float v) { o[s][k] = v; });
            // push streaming with half-way bounce-back
            // slot k of the cell in row r = z ny + y at x is pair (r Q + k) nx + x
            const int zz = z;  // z in [0, nz): the plane itself needs no wrap
            const int rowq = Q * g.nx;  // pairs per (y, z) row
            const int dzp = (zz == g.nz - 1) ? (1 - g.nz) * g.ny * rowq : g.ny * rowq;
            const int dzm = (zz == 0) ? (g.nz - 1) * g.ny * rowq : -g.ny * rowq;
            const int cell = (zz * g.ny + gy) * rowq + gx;  // slot 0 of this cell
            const uint32_t pw = p_swap_pairs(w & PUSH_BOUNCE_BITS);
            auto dst = [&](int k, uint32_t bits) -> int {
                const int off = EX(k) + EY(k) * rowq + (EZ(k) > 0 ? dzp : (EZ(k) < 0 ? dzm : 0));
                return ((bits >> k) & 1u) ? (cell + OPP(k) * g.nx) : (cell + k * g.nx + off);
            };
            if (cls == CLS_MEMBRANE) {
                // the wetting fluid only; the non-wetting half of every slot stays zero
                float* fo = reinterpret_cast<float*>(fout);
                fo[2 * (size_t)cell] = o[0][0];
#pragma unroll
                for (int k = 1; k < Q; ++k) fo[2 * (size_t)dst(k, pw)] = o[0][k];
            } else if (w & BIT_NW_DIFF) {
                const uint32_t pn = p_swap_pairs(nwb & PUSH_BOUNCE_BITS);
                float* fo = reinterpret_cast<float*>(fout);
                fout[cell] = make_float2(o[0][0], o[1][0]);
#pragma unroll
                for (int k = 1; k < Q; ++k) {
                    fo[2 * (size_t)dst(k, pw)] = o[0][k];
                    fo[2 * (size_t)dst(k, pn) + 1] = o[1][k];
                }
            } else {
                fout[cell] = make_float2(o[0][0], o[1][0]);
#pragma unroll
                for (int k = 1; k < Q; ++k) fout[dst(k, pw)] = make_float2(o[0][k], o[1][k]);
            }
        }
        if constexpr (RR) {
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                fc[0][k] = fn[0][k];
                fc[1][k] = fn[1][k];
            }
        }
    }
}

// Pair index of slot k of cell c (c = (z ny + y) nx + x) in the paired push
// layout: the 19 slots of a (y, z) row of cells follow one another, each a row
// of nx pairs, so that a tile's box of all 19 slots is 19 consecutive segments
// per row of cells.
__device__ __forceinline__ size_t push_slot(const Geom& g, int k, long long c) {
    const long long r = c / g.nx, x = c - r * g.nx;
    return (size_t)((r * Q + k) * g.nx + x);
}

// Pull layout -> paired push layout: F_k(x) = the pull of x (source x - e_k if
// it is fluid for the component, else the cell's own slot kbar); zero where a
// component is not fluid.
__global__ void pull_to_push_kernel(const float* __restrict__ fin, float2* __restrict__ F,
                                    const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw, Geom g) {
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)c;
        const int x = ci % g.nx, y = (ci / g.nx) % g.ny, z = ci / g.nxy;
        const Column colm = make_column(x, y, g);
        float f[2][Q];
        float rw, rn;
        int cell;
        const uint32_t w = pull_cell<true>(fin, nbr, nbr_nw, g, colm, z, f, rw, rn, cell);
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        const bool fw = cls != CLS_SOLID && cls != CLS_OUTSIDE;
        const bool fn = fw && cls != CLS_MEMBRANE;
#pragma unroll
        for (int k = 0; k < Q; ++k) F[push_slot(g, k, ci)] = make_float2(fw ? f[0][k] : 0.f, fn ? f[1][k] : 0.f);
    }
}

// Paired push layout -> pull layout: slot k of cell y holds what y + e_k pulls
// from it, F_k(y + e_k), when y + e_k is fluid for the component and pulls from
// y; otherwise what y pulls from itself in direction kbar, F_kbar(y).  Zero
// where the component is not fluid.
__global__ void push_to_pull_kernel(const float2* __restrict__ F, float* __restrict__ fout,
                                    const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw, Geom g) {
    const long long N = (long long)g.nxy * g.nz;
    const float* Fs = reinterpret_cast<const float*>(F);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)c;
        const int x = ci % g.nx, y = (ci / g.nx) % g.ny, z = ci / g.nxy;
        const uint32_t w = nbr[ci];
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        for (int s = 0; s < 2; ++s) {
            const bool fl = cls != CLS_SOLID && !(s == 1 && cls == CLS_MEMBRANE);
            // push bits: bit k set when y + e_k is not fluid for s (or beyond a closed face)
            const uint32_t bits = s == 0 ? w : ((w & BIT_NW_DIFF) ? nbr_nw[ci] : w);
            const uint32_t pb = p_swap_pairs(bits & PUSH_BOUNCE_BITS);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                float v = 0.f;
                if (fl) {
                    if (k == 0 || ((pb >> k) & 1u)) {
                        v = Fs[2 * push_slot(g, OPP(k), ci) + s];  // OPP(0) = 0: the rest slot
                    } else {
                        bool okk = true;
                        const int tx = wrap1(x + EX(k), g.nx, g.px, okk);
                        const int ty = wrap1(y + EY(k), g.ny, g.py, okk);
                        const int tz = wrap1(z + EZ(k), g.nz, g.pz, okk);
                        v = Fs[2 * push_slot(g, k, (long long)tz * g.nxy + (long long)ty * g.nx + tx) + s];
                    }
                }
                fout[((size_t)s * Q + k) * g.plane + ci] = v;
            }
        }
    }
}

// Densities of cell c from its own pairs, summed in k order (the order of the
// pull read-outs, so the same bits); 0 where a component is not fluid.
__device__ __forceinline__ uint32_t push_cell_density(const float* __restrict__ Fs, const uint32_t* __restrict__ nbr,
                                                      const Geom& g, long long c, float& rw, float& rn) {
    rw = 0.f;
    rn = 0.f;
    const uint32_t w = __ldg(nbr + c);
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    if (cls == CLS_SOLID || cls == CLS_OUTSIDE) return w;
    const float2* F2 = reinterpret_cast<const float2*>(Fs);
    float a = 0.f, b = 0.f;
    for (int k = 0; k < Q; ++k) {
        const float2 v = __ldg(F2 + push_slot(g, k, c));
        a += v.x;
        b += v.y;
    }
    rw = a;
    if (cls != CLS_MEMBRANE) rn = b;
    return w;
}

constexpr int PUSH_MEAS_THREADS = 256;

// lbm_measure on the paired push layout: per-block FP64 partials (a second
// kernel adds them in block order).
__global__ void __launch_bounds__(PUSH_MEAS_THREADS)
    push_measure_kernel(const float* __restrict__ Fs, const uint32_t* __restrict__ nbr, Geom g, double G,
                        double* __restrict__ partials) {
    double acc[NMEAS];
#pragma unroll
    for (int i = 0; i < NMEAS; ++i) acc[i] = 0.0;
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        float rw, rn;
        const uint32_t w = push_cell_density(Fs, nbr, g, c, rw, rn);
        measure_accumulate(acc, (w >> CLS_SHIFT) & CLS_MASK, (double)rw, (double)rn, G);
    }
    __shared__ double red[PUSH_MEAS_THREADS / 32][NMEAS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NMEAS; ++i) {
        double v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < NMEAS) {
        double v = 0.0;
        for (int wv = 0; wv < PUSH_MEAS_THREADS / 32; ++wv) v += red[wv][threadIdx.x];
        partials[(size_t)blockIdx.x * NMEAS + threadIdx.x] = v;
    }
}

__global__ void push_density_kernel(const float* __restrict__ Fs, const uint32_t* __restrict__ nbr, Geom g,
                                    float* __restrict__ rho) {
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        float rw, rn;
        push_cell_density(Fs, nbr, g, c, rw, rn);
        rho[c] = rw;
        rho[N + c] = rn;
    }
}

__global__ void push_probe_kernel(const float* __restrict__ Fs, const uint32_t* __restrict__ nbr, Geom g,
                                  long long c, float* __restrict__ out) {
    float rw, rn;
    push_cell_density(Fs, nbr, g, c, rw, rn);
    out[0] = rw;
    out[1] = rn;
}

typedef CUresult (*PushEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PushEncodeFn push_encode_fn() {
    static PushEncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PushEncodeFn>(p);
    }
    return fn;
}

template <int BY, int NS, int MINB, bool TAU1, bool RR>
cudaError_t configure_push() {
    static unsigned long long configured = 0;  // one bit per device: the attribute is per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(sc_step_push_kernel<BY, NS, MINB, TAU1, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)push_smem_bytes<BY, NS>());
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    return cudaSuccess;
}

template <int BY, int NS, int MINB, bool TAU1, bool RR>
cudaError_t launch_push_shape(const CUtensorMap& tm, float2* fout, const uint32_t* nbr, const uint32_t* nbr_nw,
                              const uint32_t* adh, const Geom& g, const Phys& p, int lz, int pf, int order, int* err,
                              cudaStream_t s) {
    constexpr int TY = BY - 2;
    const unsigned tx = (g.nx + PXI - 1) / PXI, ty = (g.ny + TY - 1) / TY, sz = (g.nz + lz - 1) / lz;
    const dim3 grid = order ? dim3(sz, tx, ty) : dim3(tx, ty, sz);
    sc_step_push_kernel<BY, NS, MINB, TAU1, RR><<<grid, dim3(PX, BY), push_smem_bytes<BY, NS>(), s>>>(
        tm, fout, nbr, nbr_nw, adh, g, p, lz, pf, order, err);
    return cudaGetLastError();
}

// tau = 1 in both components selects the compile-time tau = 1 collision
bool tau_one(const Phys& p) { return p.tau[0] == 1.0f && p.tau[1] == 1.0f; }

// Shapes of the push kernel by index: box rows BY, plane stages NS, CTAs per SM
// (MINB, which also caps the registers a thread), register-resident pairs (RR).
struct PushShapeInfo {
    int by, ns, minb;
    bool rr;
};
constexpr PushShapeInfo kPushShapes[] = {
    {8, 4, 1, false}, {6, 3, 2, false}, {10, 3, 1, false}, {7, 3, 2, false}, {10, 4, 1, false}, {12, 3, 1, false},
    {6, 3, 2, true},  {10, 4, 1, true}, {12, 3, 1, true},  {5, 4, 2, true},  {8, 4, 1, true},  {7, 3, 2, true},
};
constexpr int N_PUSH_SHAPES = (int)(sizeof(kPushShapes) / sizeof(kPushShapes[0]));

template <int I>
cudaError_t configure_shape() {
    constexpr PushShapeInfo S = kPushShapes[I];
    cudaError_t e = configure_push<S.by, S.ns, S.minb, false, S.rr>();
    return e == cudaSuccess ? configure_push<S.by, S.ns, S.minb, true, S.rr>() : e;
}

template <int I>
cudaError_t launch_shape(bool t1, const CUtensorMap& tm, float2* fo, const uint32_t* nbr, const uint32_t* nbr_nw,
                         const uint32_t* adh, const Geom& g, const Phys& p, int lz, int pf, int order, int* err,
                         cudaStream_t s) {
    constexpr PushShapeInfo S = kPushShapes[I];
    return t1 ? launch_push_shape<S.by, S.ns, S.minb, true, S.rr>(tm, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s)
              : launch_push_shape<S.by, S.ns, S.minb, false, S.rr>(tm, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err,
                                                                   s);
}

}  // namespace

int push_shape_count() { return N_PUSH_SHAPES; }

bool push_step_applicable(const Geom& g) { return !g.px && !g.py && g.nx % 2 == 0; }

cudaError_t encode_push_maps(const Geom& g, float* f0, float* f1, int by, CUtensorMap (&maps)[2]) {
    if (!push_step_applicable(g)) return cudaErrorInvalidValue;
    PushEncodeFn enc = push_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    // (component-interleaved x as floats, direction, y, z): the slots of a row of
    // cells are consecutive rows of nx pairs
    const cuuint64_t dims[4] = {(cuuint64_t)2 * g.nx, (cuuint64_t)Q, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 8, (cuuint64_t)Q * g.nx * 8, (cuuint64_t)g.ny * Q * g.nx * 8};
    const cuuint32_t box[4] = {2 * PX, (cuuint32_t)Q, (cuuint32_t)by, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    float* bufs[2] = {f0, f1};
    for (int i = 0; i < 2; ++i)
        if (enc(&maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, bufs[i], dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    return cudaSuccess;
}

int push_shape_rows(int shape) { return (shape >= 0 && shape < N_PUSH_SHAPES) ? kPushShapes[shape].by : 0; }

int push_shape_stages(int shape) { return (shape >= 0 && shape < N_PUSH_SHAPES) ? kPushShapes[shape].ns : 0; }

int push_shape_ctas(int shape) { return (shape >= 0 && shape < N_PUSH_SHAPES) ? kPushShapes[shape].minb : 0; }

bool push_shape_resident(int shape) { return shape >= 0 && shape < N_PUSH_SHAPES && kPushShapes[shape].rr; }

int push_default_lz(const Geom& g, int shape) {
    // Short z segments keep neighbouring tiles on the same planes, so that the
    // box halos they share are re-read from L2; small boxes get enough segments
    // to give every SM a CTA.
    const int ty = push_shape_rows(shape) - 2;
    if (ty <= 0) return 1;
    const long long tiles = (long long)((g.nx + PXI - 1) / PXI) * ((g.ny + ty - 1) / ty);
    long long segs = device_sm_count() / tiles;
    if (segs < 1) segs = 1;
    int lz = (int)((g.nz + segs - 1) / segs);
    if (lz > 32) lz = 32;
    if (lz < 4) lz = 4;
    if (lz > g.nz) lz = g.nz;
    return lz;
}

cudaError_t prepare_step_push(int shape) {
    static_assert(N_PUSH_SHAPES == 12, "one case per shape below");
    switch (shape) {
        case 0: return configure_shape<0>();
        case 1: return configure_shape<1>();
        case 2: return configure_shape<2>();
        case 3: return configure_shape<3>();
        case 4: return configure_shape<4>();
        case 5: return configure_shape<5>();
        case 6: return configure_shape<6>();
        case 7: return configure_shape<7>();
        case 8: return configure_shape<8>();
        case 9: return configure_shape<9>();
        case 10: return configure_shape<10>();
        case 11: return configure_shape<11>();
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_push(int shape, const CUtensorMap& tm_in, float* fout, const uint32_t* nbr,
                             const uint32_t* nbr_nw, const uint32_t* adh, const Geom& g, const Phys& p, int lz,
                             int pf, int order, int* err, cudaStream_t s) {
    if (lz < 1 || pf < 0 || pf > PUSH_MAX_PREFETCH || order < 0 || order > 1) return cudaErrorInvalidValue;
    float2* fo = reinterpret_cast<float2*>(fout);
    const bool t1 = tau_one(p);
    switch (shape) {
        case 0: return launch_shape<0>(t1, tm_in, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s);
        case 1: return launch_shape<1>(t1, tm_in, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s);
        case 2: return launch_shape<2>(t1, tm_in, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s);
        case 3: return launch_shape<3>(t1, tm_in, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s);
        case 4: return launch_shape<4>(t1, tm_in, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s);
        case 5: return launch_shape<5>(t1, tm_in, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s);
        case 6: return launch_shape<6>(t1, tm_in, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s);
        case 7: return launch_shape<7>(t1, tm_in, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s);
        case 8: return launch_shape<8>(t1, tm_in, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s);
        case 9: return launch_shape<9>(t1, tm_in, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s);
        case 10: return launch_shape<10>(t1, tm_in, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s);
        case 11: return launch_shape<11>(t1, tm_in, fo, nbr, nbr_nw, adh, g, p, lz, pf, order, err, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_measure_push(const float* F, const uint32_t* nbr, const Geom& g, double G, double* partials,
                               int nblocks, double* result, cudaStream_t s) {
    push_measure_kernel<<<nblocks, PUSH_MEAS_THREADS, 0, s>>>(F, nbr, g, G, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_finalize(partials, nblocks, result, s);
}

cudaError_t launch_density_push(const float* F, const uint32_t* nbr, const Geom& g, float* rho, cudaStream_t s) {
    const long long N = (long long)g.nxy * g.nz;
    long long blocks = (N + 255) / 256;
    const long long cap = 16LL * device_sm_count();
    if (blocks > cap) blocks = cap;
    push_density_kernel<<<(int)blocks, 256, 0, s>>>(F, nbr, g, rho);
    return cudaGetLastError();
}

cudaError_t launch_probe_push(const float* F, const uint32_t* nbr, const Geom& g, int x, int y, int z, float* out,
                              cudaStream_t s) {
    const long long c = ((long long)z * g.ny + y) * g.nx + x;
    push_probe_kernel<<<1, 1, 0, s>>>(F, nbr, g, c, out);
    return cudaGetLastError();
}

cudaError_t launch_pull_to_push(const float* fin, float* F, const uint32_t* nbr, const uint32_t* nbr_nw,
                                const Geom& g, cudaStream_t s) {
    const long long N = (long long)g.nxy * g.nz;
    long long blocks = (N + 255) / 256;
    const long long cap = 16LL * device_sm_count();
    if (blocks > cap) blocks = cap;
    pull_to_push_kernel<<<(int)blocks, 256, 0, s>>>(fin, reinterpret_cast<float2*>(F), nbr, nbr_nw, g);
    return cudaGetLastError();
}

cudaError_t launch_push_to_pull(const float* F, float* fout, const uint32_t* nbr, const uint32_t* nbr_nw,
                                const Geom& g, cudaStream_t s) {
    const long long N = (long long)g.nxy * g.nz;
    long long blocks = (N + 255) / 256;
    const long long cap = 16LL * device_sm_count();
    if (blocks > cap) blocks = cap;
    push_to_pull_kernel<<<(int)blocks, 256, 0, s>>>(reinterpret_cast<const float2*>(F), fout, nbr, nbr_nw, g);
    return cudaGetLastError();
}

}  // namespace lbmk
