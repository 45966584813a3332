// lbm_step_tma.cu -- the fused two-component Shan-Chen D3Q19 step (FP32) with
// the population planes brought into shared memory by the tensor memory
// accelerator.
//
// Same arithmetic as the staged kernel of lbm_step_core.cuh (pull streaming with
// half-way bounce-back, Eqs. 1-4 with the Shan & Chen 1993 velocity shift, the
// reservoir override), different data movement:
//
//   * A CTA of 256 threads owns an interior tile of 32 x 8 columns and marches
//     along z.  For every destination plane d one elected thread issues one TMA
//     box load per population array (2 x 19 arrays, box 40 x 12 cells: the tile,
//     a two-cell halo in y and the 16-byte aligned halo in x) plus one box of
//     geometry words, all completing on one mbarrier.  Array (s, k) of plane d
//     is read from one source plane only, d - ez_k, so two slots (destination
//     plane parity) suffice and the loads of plane d + 2 fly while planes d + 1
//     and d are handled.
//   * Bounce-back needs no second plane: a cell whose neighbour x + e_k is not
//     fluid for component s also stores f*_k into that neighbour's slot of array
//     kbar, where its own pull of direction kbar finds it next step (a "ghost"
//     store; the slot belongs to a grain or membrane cell, which nothing else
//     reads).  Only sources beyond a closed box face are bounced explicitly.
//     ghost_fill_kernel writes the ghosts of a state another kernel produced.
//   * Every thread pulls its own interior cell from shared memory into
//     registers (kept until the next iteration collides it) and publishes the
//     cell's two densities into a 4-plane density ring; 84 threads also pull one
//     cell of the one-cell ring around the tile, for its densities only.
//   * After one CTA barrier per plane the threads collide plane d - 1 with the
//     18 neighbour densities at hand and store the post-collision populations
//     straight to global memory (solid cells are not written).
//
// DRAM sees each population read once and written once (304 bytes per fluid
// cell update) plus the ghost stores next to walls; the halo re-reads of
// neighbouring tiles, which march in step, are served by L2.  Shared memory:
// 160 KB, one CTA per SM.
//
// Waits on the mbarrier are bounded in time: a wait that runs out sets *err,
// waits (bounded again) for the copies in flight and ends the CTA.
//
// Requirements (checked on the host): no periodic x or y axis, nx a multiple of
// 4 (16-byte row pitch for the tensor maps).  z may be periodic; nz >= 3.
#include <cuda.h>

#include "lbm_step_core.cuh"

namespace lbmk {

namespace {

constexpr int TT_X = 32;                        // interior columns along x
constexpr int TT_Y = 8;                         // interior rows
constexpr int TT_CELLS = TT_X * TT_Y;           // 256 interior cells
constexpr int TT_THREADS = 2 * TT_CELLS;        // 512: warp w runs component w & 1 of tile row w >> 1
constexpr int BOX_W = 40;                       // population box columns x0-4 .. x0+35
constexpr int BOX_H = TT_Y + 4;                 // rows y0-2 .. y0+TT_Y+1
constexpr int BOX = BOX_W * BOX_H;              // floats per box (1920 bytes)
constexpr int WBOX_H = TT_Y + 2;                // word box rows y0-1 .. y0+TT_Y
constexpr int WBOX = BOX_W * WBOX_H;            // words per box (1600 bytes)
constexpr int WBOX_PAD = 416;                   // word slot stride (1664 bytes, 128-byte multiple)
constexpr int RHO_W = TT_X + 2;                 // density planes: x0-1 .. x0+32
constexpr int RHO_H = TT_Y + 2;                 //                 y0-1 .. y0+TT_Y
constexpr int RHO_PLANE = RHO_W * RHO_H;        // 340 cells
constexpr int N_RING = RHO_PLANE - TT_CELLS;    // 84 ring cells
constexpr int RING_PER_WARP = 21;               // ring cells of one component: lanes 0..20 of 4 warps
constexpr int ARR = 2 * Q;                      // population arrays

constexpr size_t SM_POP = 0;                                            // [2][ARR][BOX] float
constexpr size_t SM_WORDS = SM_POP + sizeof(float) * 2 * ARR * BOX;     // [2][WBOX_PAD] uint32
constexpr size_t SM_RHO = SM_WORDS + sizeof(uint32_t) * 2 * WBOX_PAD;   // [4][2][RHO_PLANE] float
constexpr size_t SM_XCH = SM_RHO + sizeof(float) * 4 * 2 * RHO_PLANE;   // [2][3][TT_CELLS] float (momenta)
constexpr size_t SM_BAR = SM_XCH + sizeof(float) * 2 * 3 * TT_CELLS;    // 2 mbarriers
constexpr size_t SM_TOTAL = SM_BAR + 2 * sizeof(uint64_t);

static_assert(N_RING == 4 * RING_PER_WARP, "ring cells must match the ring lanes");
static_assert(SM_WORDS % 128 == 0 && SM_RHO % 128 == 0 && SM_BAR % 8 == 0, "TMA destinations are 128-byte aligned");
static_assert((BOX * sizeof(float)) % 128 == 0 && (WBOX_PAD * sizeof(uint32_t)) % 128 == 0, "slot strides");

constexpr uint32_t POP_BOX_BYTES = BOX * sizeof(float);
constexpr uint32_t WORD_BOX_BYTES = WBOX * sizeof(uint32_t);
constexpr long long WAIT_LIMIT_NS = 2000000000LL;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity, for at most limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long limit_ns = WAIT_LIMIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if ((long long)(global_ns() - t0) > limit_ns) return false;
    }
}

// Self-test of the bounded wait: an mbarrier that nothing ever completes.  The
// wait must give up after limit_ns and say so; no copy is in flight.
__global__ void wait_selftest_kernel(long long limit_ns, int* gave_up) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) *gave_up = 1;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

constexpr uint32_t BOUNCE_BITS = 0x7fffeu;  // bits 1..18

// Exchanges the bits of each opposite pair (1,2), (3,4), ..., (17,18): a mask
// over pull directions k becomes the mask over the directions kbar.
__device__ __forceinline__ uint32_t swap_pairs(uint32_t m) {
    return ((m & 0x2aaaau) << 1) | ((m & 0x55554u) >> 1);
}

// Directions whose pull source lies beyond a closed face of the box, for the
// cell (gx, gy, z) with z unwrapped (a periodic z axis has no faces).
__device__ __forceinline__ uint32_t outside_dirs(const Geom& g, int gx, int gy, int z) {
    uint32_t m = 0u;
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        const int sx = gx - EX(k), sy = gy - EY(k), sz = z - EZ(k);
        if (sx < 0 || sx >= g.nx || sy < 0 || sy >= g.ny || (!g.pz && (sz < 0 || sz >= g.nz))) m |= 1u << k;
    }
    return m;
}

// Pull of component s of one cell from slot sl, which holds for every array
// (s, k) the plane d - ez_k of destination plane d; pb is the cell's index
// inside a population box.  Direction k streams from array (s, k) at
// pb - ey_k BOX_W - ex_k.  Half-way bounce-back against a grain or the membrane
// needs no test: the slot of a neighbour that is not fluid for s holds the
// reflected population, stored there by the cell itself in the previous step
// (the ghost store after the collision).  Only a source beyond a closed box face
// (bit k of outside) takes f*_kbar of the cell explicitly: from the slot when
// ez_k = 0 (array kbar of plane d is there), else from global memory.  Returns
// the density, summed in four interleaved partial sums (k & 3) as the staged
// kernel does.
template <bool KEEP>
__device__ __forceinline__ float slot_pull(const float* sl, int s, int pb, uint32_t outside,
                                           const float* __restrict__ fin, int cell, int plane, float (&f)[Q]) {
    const float* base = sl + s * (Q * BOX) + pb;
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    if (outside == 0u) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const float v = base[k * BOX - EY(k) * BOX_W - EX(k)];
            if (KEEP) f[k] = v;
            a[k & 3] += v;
        }
    } else {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            float v;
            if ((outside >> k) & 1u)
                v = EZ(k) == 0 ? base[OPP(k) * BOX] : __ldg(fin + (s * Q + OPP(k)) * plane + cell);
            else
                v = base[k * BOX - EY(k) * BOX_W - EX(k)];
            if (KEEP) f[k] = v;
            a[k & 3] += v;
        }
    }
    return (a[0] + a[1]) + (a[2] + a[3]);
}

// What one thread carries from the pull of its cell's component to its collision.
struct Held {
    float f[Q];      // pulled populations, then the post-collision ones
    uint32_t bits;   // bounce bits of this component
    uint32_t a;      // adhesion word
    uint32_t cls;    // cell class
    int cell;
    int zz;          // wrapped plane
    bool edge;       // on a face of the box
    bool live;       // collided (fluid for the component, inside the segment)
};

// Component s of the cell at density coordinates (rx, ry) on plane d (global
// column gx, gy).  Returns false (density 0) for a cell beyond the box, a solid
// cell, or a membrane cell for the non-wetting component.
template <bool KEEP>
__device__ __forceinline__ bool cell_pull(const float* sl, const uint32_t* wsl, const float* __restrict__ fin,
                                          const Geom& g, int s, int gx, int gy, int d, int rx, int ry, float (&f)[Q],
                                          float& r, uint32_t& w, int& cell, int& zz, bool& edge) {
    r = 0.f;
    w = CLS_OUTSIDE << CLS_SHIFT;
    cell = 0;
    zz = 0;
    edge = false;
    if (gx < 0 || gx >= g.nx || gy < 0 || gy >= g.ny) return false;
    zz = d;
    if (zz < 0 || zz >= g.nz) {
        if (!g.pz) return false;
        zz = zz < 0 ? zz + g.nz : zz - g.nz;
    }
    w = wsl[ry * BOX_W + rx + 3];
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    if (cls == CLS_SOLID || cls == CLS_OUTSIDE || (s == 1 && cls == CLS_MEMBRANE)) return false;
    cell = zz * g.nxy + gy * g.nx + gx;
    edge = gx == 0 || gx == g.nx - 1 || gy == 0 || gy == g.ny - 1 || zz == 0 || zz == g.nz - 1;
    const uint32_t outside = edge ? outside_dirs(g, gx, gy, d) : 0u;
    r = slot_pull<KEEP>(sl, s, (ry + 1) * BOX_W + rx + 3, outside, fin, cell, g.plane, f);
    return true;
}


__global__ void __launch_bounds__(TT_THREADS, 1)
    sc_step_tma_kernel(const __grid_constant__ CUtensorMap tm_f, const __grid_constant__ CUtensorMap tm_w,
                       const float* __restrict__ fin, float* __restrict__ fout, const uint32_t* __restrict__ nbr_nw,
                       const uint32_t* __restrict__ adh, Geom g, Phys P, int lz, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    // an earlier launch or CTA gave up: the whole CTA leaves (one decision for all its threads)
    if (__syncthreads_or(*reinterpret_cast<volatile int*>(err) != 0)) return;
    float* pop = reinterpret_cast<float*>(smem + SM_POP);
    uint32_t* words = reinterpret_cast<uint32_t*>(smem + SM_WORDS);
    float* rho = reinterpret_cast<float*>(smem + SM_RHO);
    float* xch = reinterpret_cast<float*>(smem + SM_XCH);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM_BAR);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int s = warp & 1;       // component of this thread
    const int row = warp >> 1;    // tile row
    const int t = row * 32 + lane;  // interior cell of the tile
    const int rc = (row + 1) * RHO_W + lane + 1;
    const int x0 = blockIdx.x * TT_X, y0 = blockIdx.y * TT_Y;
    const int z0 = blockIdx.z * lz;
    const int z1 = min(z0 + lz, g.nz);
    const int gx = x0 + lane, gy = y0 + row;
    // ring duty: lanes 0..20 of warps 0..7, one ring cell of this thread's component each
    const bool ring = warp < 8 && lane < RING_PER_WARP;
    int rrx = 0, rry = 0;
    {
        const int r = (warp >> 1) * RING_PER_WARP + lane;
        if (r < RHO_W) { rrx = r; rry = 0; }
        else if (r < 2 * RHO_W) { rrx = r - RHO_W; rry = RHO_H - 1; }
        else if (r < 2 * RHO_W + TT_Y) { rrx = 0; rry = r - 2 * RHO_W + 1; }
        else { rrx = RHO_W - 1; rry = r - 2 * RHO_W - TT_Y + 1; }
    }

    // Loads (by the producer thread) of the planes of destination plane q into
    // slot q & 1: plane q - ez_k of every array (s, k) (5 + 9 + 5 arrays per
    // component from planes q + 1, q, q - 1) and plane q of the geometry words.
    auto issue = [&](int q) {
        auto in_box = [&](int p) { return g.pz != 0 || (p >= 0 && p < g.nz); };
        auto wrap = [&](int p) { return p < 0 ? p + g.nz : (p >= g.nz ? p - g.nz : p); };
        const bool in_m = in_box(q - 1), in_0 = in_box(q), in_p = in_box(q + 1);
        const int zm = wrap(q - 1), z0w = wrap(q), zp = wrap(q + 1);
        uint64_t* b = bar + (q & 1);
        const uint32_t bytes = (in_0 ? WORD_BOX_BYTES + 2 * 9 * POP_BOX_BYTES : 0u) +
                               (in_m ? 2 * 5 * POP_BOX_BYTES : 0u) + (in_p ? 2 * 5 * POP_BOX_BYTES : 0u);
        mbar_arrive_expect_tx(b, bytes);
        if (in_0) tma_load_3d(words + (q & 1) * WBOX_PAD, &tm_w, x0 - 4, y0 - 1, z0w, b);
        float* slot = pop + (q & 1) * (ARR * BOX);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const bool in = EZ(k) > 0 ? in_m : (EZ(k) < 0 ? in_p : in_0);
            const int zs = EZ(k) > 0 ? zm : (EZ(k) < 0 ? zp : z0w);
            if (!in) continue;
#pragma unroll
            for (int c = 0; c < 2; ++c) tma_load_4d(slot + (c * Q + k) * BOX, &tm_f, x0 - 4, y0 - 2, zs, c * Q + k, b);
        }
    };
    constexpr int PRODUCER = TT_THREADS - 32;  // lane 0 of the last warp (no ring duty)
    auto parity_of = [&](int d) { return (uint32_t)(((d - z0 + 1) >> 1) & 1); };

    if (tid == 0) {
        mbar_init(bar + 0, 1);
        mbar_init(bar + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    if (tid == PRODUCER) {
        issue(z0 - 1);
        issue(z0);
    }

    // Iteration d: wait for the planes of destination plane d; pull this
    // thread's component of its interior cell (into cur) and of its ring cell
    // (density only); publish the densities; one CTA barrier; queue the planes of
    // d + 2 into the slot just read; collide plane d - 1 (prev): momentum,
    // exchange with the other component's thread of the cell (named barrier of
    // the row's two warps), common velocity, force, relaxation, stores.
    Held cur, prev;
    prev.live = false;
    prev.cls = CLS_OUTSIDE;
    for (int d = z0 - 1; d <= z1; ++d) {
        const bool ok = mbar_wait_bounded(bar + (d & 1), parity_of(d));
        const float* sl = pop + (d & 1) * (ARR * BOX);
        const uint32_t* wsl = words + (d & 1) * WBOX_PAD;
        {
            float r;
            uint32_t w;
            const bool fl = cell_pull<true>(sl, wsl, fin, g, s, gx, gy, d, lane + 1, row + 1, cur.f, r, w, cur.cell,
                                            cur.zz, cur.edge);
            rho[((d & 3) * 2 + s) * RHO_PLANE + rc] = r;
            cur.live = fl && d >= z0 && d < z1;
            cur.cls = (w >> CLS_SHIFT) & CLS_MASK;
            uint32_t bits = 0u;
            if (cur.live) bits = (s == 1 && (w & BIT_NW_DIFF)) ? __ldg(nbr_nw + cur.cell) : w;
            cur.bits = bits & BOUNCE_BITS;
            cur.a = (cur.live && (w & BIT_ADH)) ? __ldg(adh + cur.cell) : 0u;
        }
        if (ring) {
            float unused[Q];
            float r;
            uint32_t w;
            int cell, zz;
            bool edge;
            cell_pull<false>(sl, wsl, fin, g, s, x0 - 1 + rrx, y0 - 1 + rry, d, rrx, rry, unused, r, w, cell, zz,
                             edge);
            rho[((d & 3) * 2 + s) * RHO_PLANE + rry * RHO_W + rrx] = r;
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(err, 1);
            // bounded waits for the copies still in flight (planes d and d + 1)
            mbar_wait_bounded(bar + (d & 1), parity_of(d));
            if (d + 1 <= z1) mbar_wait_bounded(bar + ((d + 1) & 1), parity_of(d + 1));
            return;
        }
        if (tid == PRODUCER && d + 2 <= z1) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            issue(d + 2);
        }
        // collision of plane d - 1
        float j[3] = {0.f, 0.f, 0.f};
        if (prev.live) momentum(prev.f, j);
#pragma unroll
        for (int c = 0; c < 3; ++c) xch[(s * 3 + c) * TT_CELLS + t] = j[c];
        asm volatile("bar.sync %0, %1;\n" ::"r"(1 + row), "r"(64) : "memory");
        if (prev.live) {
            float jo[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) jo[c] = xch[((s ^ 1) * 3 + c) * TT_CELLS + t];
            const int pl = g.plane;
            float* __restrict__ o = fout + s * (Q * pl) + prev.cell;
            collide_component<RHO_W, RHO_PLANE>(prev.f, prev.cls, prev.a, s, j, jo, rho, d - 1, rc, P,
                                                [&](int k, float v) {
                                                    o[k * pl] = v;
                                                    prev.f[k] = v;  // for the ghost stores below
                                                });
            // ghost stores: where x + e_k (inside the box) is not fluid for this
            // component, f*_k goes to that cell's slot of array kbar
            uint32_t gm = swap_pairs(prev.bits);
            if (prev.edge) gm &= ~swap_pairs(outside_dirs(g, gx, gy, d - 1));
            if (gm) {
                const int zp = (prev.zz == g.nz - 1) ? (1 - g.nz) * g.nxy : g.nxy;  // periodic z wrap
                const int zm = (prev.zz == 0) ? (g.nz - 1) * g.nxy : -g.nxy;
#pragma unroll
                for (int k = 1; k < Q; ++k) {
                    const int off = EX(k) + EY(k) * g.nx + (EZ(k) > 0 ? zp : (EZ(k) < 0 ? zm : 0));
                    if ((gm >> k) & 1u) o[OPP(k) * pl + off] = prev.f[k];
                }
            }
        }
        prev = cur;
    }
}

// Ghost stores for a state written by another kernel: for every cell x fluid
// for component s and every direction j whose neighbour x + e_j inside the box
// is not fluid for s, f[s][jbar] at x + e_j = f[s][j] at x.
__global__ void ghost_fill_kernel(float* __restrict__ f, const uint32_t* __restrict__ nbr,
                                  const uint32_t* __restrict__ nbr_nw, Geom g) {
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int cell = (int)c;
        const uint32_t w = nbr[cell];
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        if (cls == CLS_SOLID || cls == CLS_OUTSIDE) continue;
        const int x = cell % g.nx, y = (cell / g.nx) % g.ny, z = cell / g.nxy;
        for (int s = 0; s < 2; ++s) {
            if (s == 1 && cls == CLS_MEMBRANE) break;
            const uint32_t bits = s == 0 ? w : ((w & BIT_NW_DIFF) ? nbr_nw[cell] : w);
#pragma unroll
            for (int j = 1; j < Q; ++j) {
                if (!((bits >> OPP(j)) & 1u)) continue;
                const int tx = x + EX(j), ty = y + EY(j);
                int tz = z + EZ(j);
                if (tx < 0 || tx >= g.nx || ty < 0 || ty >= g.ny) continue;
                if (tz < 0 || tz >= g.nz) {
                    if (!g.pz) continue;
                    tz = tz < 0 ? tz + g.nz : tz - g.nz;
                }
                f[(s * Q + OPP(j)) * g.plane + tz * g.nxy + ty * g.nx + tx] = f[(s * Q + j) * g.plane + cell];
            }
        }
    }
}

}  // namespace

bool tma_step_applicable(const Geom& g) { return !g.px && !g.py && g.nx % 4 == 0 && g.nz >= 3; }

int tma_default_lz(const Geom& g) {
    // Short z segments: CTAs run in waves over the x-y tiles, so neighbouring
    // tiles work on the same planes and their halo re-reads hit L2 (a CTA that
    // marched a whole column would drift away from its neighbours).  Small
    // boxes get enough segments to fill the SMs.
    const int sms = device_sm_count();
    const long long tiles = (long long)((g.nx + TT_X - 1) / TT_X) * ((g.ny + TT_Y - 1) / TT_Y);
    long long segs = sms / tiles;
    if (segs < 1) segs = 1;
    int lz = (int)((g.nz + segs - 1) / segs);
    if (lz > 16) lz = 16;
    if (lz < 4) lz = 4;
    if (lz > g.nz) lz = g.nz;
    return lz;
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

cudaError_t encode_step_maps(const Geom& g, float* f0, float* f1, const uint32_t* nbr, TmaMaps& m) {
    if (!tma_step_applicable(g)) return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)ARR};
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nxy * 4, (cuuint64_t)g.plane * 4};
    const cuuint32_t box[4] = {BOX_W, BOX_H, 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    float* bufs[2] = {f0, f1};
    for (int i = 0; i < 2; ++i)
        if (enc(&m.f[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, bufs[i], dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    const cuuint64_t wdims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t wstrides[2] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nxy * 4};
    const cuuint32_t wbox[3] = {BOX_W, WBOX_H, 1};
    if (enc(&m.w, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<uint32_t*>(nbr), wdims, wstrides, wbox, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t prepare_step_tma() {
    static unsigned long long configured = 0;  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(sc_step_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_TOTAL);
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    return cudaSuccess;
}

cudaError_t launch_step_tma(const TmaMaps& m, int cur, const float* fin, float* fout, const uint32_t* nbr_nw,
                            const uint32_t* adh, const Geom& g, const Phys& p, int lz, int* err, cudaStream_t s) {
    if (lz < 1) return cudaErrorInvalidValue;
    dim3 grid((g.nx + TT_X - 1) / TT_X, (g.ny + TT_Y - 1) / TT_Y, (g.nz + lz - 1) / lz);
    sc_step_tma_kernel<<<grid, TT_THREADS, SM_TOTAL, s>>>(m.f[cur], m.w, fin, fout, nbr_nw, adh, g, p, lz, err);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(long long limit_ns, int* gave_up, cudaStream_t s) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(limit_ns, gave_up);
    return cudaGetLastError();
}

cudaError_t launch_ghost_fill(float* f, const uint32_t* nbr, const uint32_t* nbr_nw, const Geom& g, cudaStream_t s) {
    const long long N = (long long)g.nxy * g.nz;
    long long blocks = (N + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    ghost_fill_kernel<<<(int)blocks, 256, 0, s>>>(f, nbr, nbr_nw, g);
    return cudaGetLastError();
}

}  // namespace lbmk
