// lbm_step16.cu -- the fused step with the populations stored in 16 bits
// (FP16 or BF16) as deviations, all collision arithmetic in FP32.
//
// Storage.  One 32-bit word per (direction k, cell) holds the pair
// (h_w, h_nw) of both components -- one 4-byte copy pulls both -- and every cell
// keeps its density of the previous time level, R(x) = (rho_w, rho_nw) in FP32.
// The stored deviation is taken against the density of the cell that will read
// the value in the next step:
//     h_s,k(y) = f*_s,k(y) - w_k rho_s(D, t),  D = y + e_k, or y itself when that
//     neighbour is a wall for component s (it comes back by bounce-back),
// so the reader reconstructs every pulled value as
//     f_s,k(x) = h_s,k(source) + w_k R_s(x),
// with R its own density of the previous level.  The writer finds rho(D, t) in
// the shared density ring it already holds for the force.  The deviations are
// the velocity and density-change parts of the populations, a few per cent of
// them, which the 11-bit (FP16) or 8-bit (BF16) significand then resolves.
// The rounding error of the 18 moving directions is fed into the rest value, so
// the stored pairs of a cell add up to its density up to one rounding.
// Bytes per fluid-cell update: 19 x 4 read + 19 x 4 written + 8 + 8 = 168.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "lbm_pair16.cuh"
#include "lbm_step_core.cuh"

namespace lbmk {

namespace {

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}

// Source index of direction k for cell (column c, plane zz) of component bits
// (bounce-back to the opposite slot of the cell itself).
__device__ __forceinline__ int src_index(const Geom& g, const Column& c, int zz, const int (&zo)[3], bool seam,
                                         int cell, uint32_t bits, int k) {
    int idx;
    if (!seam) idx = cell + g.poff[k];
    else idx = k * g.plane + zo[1 - EZ(k)] + c.yo[1 - EY(k)] + c.xo[1 - EX(k)];
    if ((bits >> k) & 1u) idx = OPP(k) * g.plane + cell;
    return idx;
}

__device__ __forceinline__ bool seam_of(const Geom& g, const Column& c, int zz) {
    return (g.px && (c.xo[1] == 0 || c.xo[1] == g.nx - 1)) || (g.py && (c.yo[1] == 0 || c.yo[1] == (g.ny - 1) * g.nx)) ||
           (g.pz && (zz == 0 || zz == g.nz - 1));
}

// Densities of one cell of a 16-bit state (0 where a component is not fluid).
template <class H2>
__device__ __forceinline__ uint32_t pull16_density(const uint32_t* __restrict__ win, const float2* __restrict__ Rin,
                                                   const uint32_t* __restrict__ nbr,
                                                   const uint32_t* __restrict__ nbr_nw, const Geom& g,
                                                   const Column& c, int z, float& rw, float& rn) {
    rw = 0.f;
    rn = 0.f;
    bool ok = c.ok;
    const int zz = wrap1(z, g.nz, g.pz, ok);
    if (!ok) return CLS_OUTSIDE << CLS_SHIFT;
    const int cell = zz * g.nxy + c.yo[1] + c.xo[1];
    const uint32_t w = __ldg(nbr + cell);
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    if (cls == CLS_SOLID) return w;
    const uint32_t wn = (cls == CLS_MEMBRANE) ? w : ((w & BIT_NW_DIFF) ? __ldg(nbr_nw + cell) : w);
    const bool seam = seam_of(g, c, zz);
    int zo[3];
    zo[0] = nb1(zz - 1, g.nz, g.pz) * g.nxy;
    zo[1] = zz * g.nxy;
    zo[2] = nb1(zz + 1, g.nz, g.pz) * g.nxy;
    const float2 R = __ldg(Rin + cell);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const float hw = Pair<H2>::unpack(__ldg(win + src_index(g, c, zz, zo, seam, cell, w, k))).x;
        rw += hw + WK(k) * R.x;
        if (cls != CLS_MEMBRANE) {
            const float hn = Pair<H2>::unpack(__ldg(win + src_index(g, c, zz, zo, seam, cell, wn, k))).y;
            rn += hn + WK(k) * R.y;
        }
    }
    return w;
}

template <int BY, int LEAD>
size_t smem16_bytes() {
    // per thread: (LEAD+1) stages of 19 words + an R pair, the ring pair x 4, words and adhesion x (LEAD+1)
    return (size_t)32 * BY * ((LEAD + 1) * (Q * 4 + 8) + 4 * 8 + 2 * 4 * (LEAD + 1));
}

template <class H2, int BY, int LEAD>
__device__ __forceinline__ void step_column16(const uint32_t* __restrict__ win, uint32_t* __restrict__ wout,
                                              const float2* __restrict__ Rin, float2* __restrict__ Rout,
                                              const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw,
                                              const uint32_t* __restrict__ adh, const Geom& g, const Phys& P, int tx,
                                              int ty, int z0, int z1, unsigned char* smem) {
    constexpr int TY = BY - 2;
    constexpr int NT = 32 * BY;
    constexpr int NS = LEAD + 1;
    uint32_t* stage = reinterpret_cast<uint32_t*>(smem);                 // [NS][Q][NT]
    float2* stR = reinterpret_cast<float2*>(stage + NS * Q * NT);        // [NS][NT]
    float2* ring = stR + NS * NT;                                        // [4][NT]
    uint32_t* words = reinterpret_cast<uint32_t*>(ring + 4 * NT);        // [NS][NT]
    uint32_t* adhw = words + NS * NT;                                    // [NS][NT]
    const int lane = threadIdx.x;
    const int row = threadIdx.y;
    const int tid = row * 32 + lane;
    const int gx = tx * 30 - 1 + lane;
    const int gy = ty * TY - 1 + row;
    const Column col = make_column(gx, gy, g);
    const bool needed = gx <= g.nx && gy <= g.ny;
    const bool interior = lane >= 1 && lane <= 30 && row >= 1 && row <= TY && gx < g.nx && gy < g.ny;
    auto slot = [&](int p) { return (p - z0 + 1) % NS; };
    auto fetch_word = [&](int p) -> uint32_t {
        if (!needed || p > z1) return CLS_OUTSIDE << CLS_SHIFT;
        int zz;
        bool ok;
        const int cell = plane_cell(g, col, p, zz, ok);
        return ok ? __ldg(nbr + cell) : (CLS_OUTSIDE << CLS_SHIFT);
    };
    auto issue = [&](int p, uint32_t w) {
        const int sl = slot(p);
        words[sl * NT + tid] = w;
        if (!needed || p > z1) return;
        int zz;
        bool ok;
        const int cell = plane_cell(g, col, p, zz, ok);
        if (!ok) return;
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        if (cls == CLS_SOLID) return;
        const bool seam = seam_of(g, col, zz);
        int zo[3];
        zo[0] = nb1(zz - 1, g.nz, g.pz) * g.nxy;
        zo[1] = zz * g.nxy;
        zo[2] = nb1(zz + 1, g.nz, g.pz) * g.nxy;
        uint32_t* st = stage + sl * Q * NT;
        if (cls == CLS_MEMBRANE || !(w & BIT_NW_DIFF)) {
#pragma unroll
            for (int k = 0; k < Q; ++k)
                cp_async4(reinterpret_cast<float*>(st + k * NT + tid),
                          reinterpret_cast<const float*>(win + src_index(g, col, zz, zo, seam, cell, w, k)));
        } else {
            // the two components bounce differently next to a membrane: assemble each
            // pair from two words (rare; plain loads)
            const uint32_t wn = __ldg(nbr_nw + cell);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const uint32_t a = __ldg(win + src_index(g, col, zz, zo, seam, cell, w, k));
                const uint32_t b = __ldg(win + src_index(g, col, zz, zo, seam, cell, wn, k));
                st[k * NT + tid] = (a & 0xffffu) | (b & 0xffff0000u);
            }
        }
        cp_async8(stR + sl * NT + tid, Rin + cell);
        if (w & BIT_ADH)
            cp_async4(reinterpret_cast<float*>(adhw + sl * NT + tid), reinterpret_cast<const float*>(adh + cell));
    };
    auto reconstruct = [&](int p, uint32_t w, float (&f)[2][Q]) {
        const int sl = slot(p);
        const uint32_t* st = stage + sl * Q * NT;
        const float2 R = stR[sl * NT + tid];
        const bool has_nw = ((w >> CLS_SHIFT) & CLS_MASK) != CLS_MEMBRANE;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const float2 h = Pair<H2>::unpack(st[k * NT + tid]);
            f[0][k] = h.x + WK(k) * R.x;
            f[1][k] = has_nw ? h.y + WK(k) * R.y : 0.f;
        }
    };
    auto publish = [&](int p) {
        const uint32_t w = words[slot(p) * NT + tid];
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        float rw = 0.f, rn = 0.f;
        if (cls != CLS_SOLID && cls != CLS_OUTSIDE) {
            float f[2][Q];
            reconstruct(p, w, f);
            float a[4] = {0.f, 0.f, 0.f, 0.f}, b[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                a[k & 3] += f[0][k];
                b[k & 3] += f[1][k];
            }
            rw = (a[0] + a[1]) + (a[2] + a[3]);
            rn = (b[0] + b[1]) + (b[2] + b[3]);
        }
        ring[(p & 3) * NT + tid] = make_float2(rw, rn);
        if (interior && p >= z0 && p < z1) {
            int zz;
            bool ok;
            const int cell = plane_cell(g, col, p, zz, ok);
            Rout[cell] = make_float2(rw, rn);
        }
    };

    uint32_t wnext = fetch_word(z0 - 1);
#pragma unroll
    for (int i = 0; i <= LEAD; ++i) {
        const int p = z0 - 1 + i;
        const uint32_t w = wnext;
        wnext = fetch_word(p + 1);
        issue(p, w);
        cp_async_commit();
    }
    cp_async_wait<LEAD - 1>();
    publish(z0 - 1);
    publish(z0);
    for (int z = z0; z < z1; ++z) {
        {
            const int p = z + LEAD;
            const uint32_t w = wnext;
            wnext = fetch_word(p + 1);
            issue(p, w);
            cp_async_commit();
        }
        cp_async_wait<LEAD - 1>();
        publish(z + 1);
        __syncthreads();
        const uint32_t w0 = words[slot(z) * NT + tid];
        const uint32_t cls = (w0 >> CLS_SHIFT) & CLS_MASK;
        if (interior && cls != CLS_SOLID && cls != CLS_OUTSIDE) {
            int zz;
            bool ok;
            const int cell = plane_cell(g, col, z, zz, ok);
            const bool has_nw = cls != CLS_MEMBRANE;
            const uint32_t wn = has_nw && (w0 & BIT_NW_DIFF) ? __ldg(nbr_nw + cell) : w0;
            float f[2][Q];
            reconstruct(z, w0, f);
            float out[2][Q];
            collide_generic<BY>(f, ring, w0, adhw[slot(z) * NT + tid], z, row, lane, P,
                                [&](int s, int k, float v) { out[s][k] = v; });
            if (!has_nw) {
#pragma unroll
                for (int k = 0; k < Q; ++k) out[1][k] = 0.f;
            }
            // deviation against the density of the cell that reads the value next step
            auto rho_at = [&](int k) {
                return ring[((z + EZ(k)) & 3) * NT + (row + EY(k)) * 32 + (lane + EX(k))];
            };
            const float2 self = rho_at(0);
            float err[2] = {0.f, 0.f};
#pragma unroll
            for (int k = 1; k < Q; ++k) {
                // the reader through direction k is x + e_k unless that is a wall (bit OPP(k))
                const float2 nb = rho_at(k);
                const float dw = ((w0 >> OPP(k)) & 1u) ? self.x : nb.x;
                const float dn = ((wn >> OPP(k)) & 1u) ? self.y : nb.y;
                const float ew = out[0][k] - WK(k) * dw;
                const float en = has_nw ? out[1][k] - WK(k) * dn : 0.f;
                const float rw = Pair<H2>::round1(ew), rn = Pair<H2>::round1(en);
                err[0] += ew - rw;
                err[1] += en - rn;
                wout[(size_t)k * g.plane + cell] = Pair<H2>::pack(rw, rn);
            }
            const float e0w = out[0][0] - WK(0) * self.x + err[0];
            const float e0n = has_nw ? out[1][0] - WK(0) * self.y + err[1] : 0.f;
            wout[cell] = Pair<H2>::pack(e0w, e0n);
        }
    }
    cp_async_wait<0>();
}

template <class H2, int BY, int LEAD>
__global__ void __launch_bounds__(32 * BY, 2)
    sc_step16_kernel(const uint32_t* __restrict__ win, uint32_t* __restrict__ wout, const float2* __restrict__ Rin,
                     float2* __restrict__ Rout, const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw,
                     const uint32_t* __restrict__ adh, Geom g, Phys P, int lz) {
    extern __shared__ __align__(16) unsigned char smem16[];
    const int z0 = blockIdx.z * lz;
    step_column16<H2, BY, LEAD>(win, wout, Rin, Rout, nbr, nbr_nw, adh, g, P, blockIdx.x, blockIdx.y, z0,
                                min(z0 + lz, g.nz), smem16);
}

template <class H2>
__global__ void density16_kernel(const uint32_t* __restrict__ win, const float2* __restrict__ Rin,
                                 const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw, Geom g,
                                 float* __restrict__ rho) {
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % g.nx), y = (int)((c / g.nx) % g.ny), z = (int)(c / g.nxy);
        float rw, rn;
        pull16_density<H2>(win, Rin, nbr, nbr_nw, g, make_column(x, y, g), z, rw, rn);
        rho[c] = rw;
        rho[N + c] = rn;
    }
}

template <class H2>
__global__ void __launch_bounds__(256) measure16_kernel(const uint32_t* __restrict__ win,
                                                        const float2* __restrict__ Rin,
                                                        const uint32_t* __restrict__ nbr,
                                                        const uint32_t* __restrict__ nbr_nw, Geom g, double G,
                                                        double* __restrict__ partials) {
    double acc[NMEAS];
#pragma unroll
    for (int i = 0; i < NMEAS; ++i) acc[i] = 0.0;
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % g.nx), y = (int)((c / g.nx) % g.ny), z = (int)(c / g.nxy);
        float rw, rn;
        const uint32_t w = pull16_density<H2>(win, Rin, nbr, nbr_nw, g, make_column(x, y, g), z, rw, rn);
        measure_accumulate(acc, (w >> CLS_SHIFT) & CLS_MASK, (double)rw, (double)rn, G);
    }
    __shared__ double red[8][NMEAS];
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
        for (int wv = 0; wv < 8; ++wv) v += red[wv][threadIdx.x];
        partials[(size_t)blockIdx.x * NMEAS + threadIdx.x] = v;
    }
}

template <class H2>
__global__ void probe16_kernel(const uint32_t* __restrict__ win, const float2* __restrict__ Rin,
                               const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw, Geom g, int x,
                               int y, int z, float* out) {
    float rw, rn;
    pull16_density<H2>(win, Rin, nbr, nbr_nw, g, make_column(x, y, g), z, rw, rn);
    out[0] = rw;
    out[1] = rn;
}

// Pull layout -> push layout of a 16-bit state: W[k][D] = the word D pulls in
// direction k, each half from its own component's source (D - e_k where that is
// fluid for the component, else D's own slot kbar); 0 where D is grain and in the
// non-wetting half of a membrane cell.  The deviations stay as they are: in
// both layouts a value is held against the density of the cell that reads it.
__global__ void pull16_to_push16_kernel(const uint32_t* __restrict__ win, uint32_t* __restrict__ wout,
                                        const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw, Geom g) {
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)c;
        const int x = ci % g.nx, y = (ci / g.nx) % g.ny, z = ci / g.nxy;
        const uint32_t w = nbr[ci];
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        if (cls == CLS_SOLID) {
            for (int k = 0; k < Q; ++k) wout[(size_t)k * g.plane + ci] = 0u;
            continue;
        }
        const bool has_nw = cls != CLS_MEMBRANE;
        const uint32_t wn = !has_nw ? w : ((w & BIT_NW_DIFF) ? nbr_nw[ci] : w);
        const Column col = make_column(x, y, g);
        const bool seam = seam_of(g, col, z);
        int zo[3];
        zo[0] = nb1(z - 1, g.nz, g.pz) * g.nxy;
        zo[1] = z * g.nxy;
        zo[2] = nb1(z + 1, g.nz, g.pz) * g.nxy;
        for (int k = 0; k < Q; ++k) {
            const uint32_t a = win[src_index(g, col, z, zo, seam, ci, w, k)];
            const uint32_t b = has_nw ? win[src_index(g, col, z, zo, seam, ci, wn, k)] : 0u;
            wout[(size_t)k * g.plane + ci] = (a & 0xffffu) | (b & 0xffff0000u);
        }
    }
}

// Push layout -> pull layout of a 16-bit state: half s of slot k of cell y holds
// what y + e_k pulls from y, half s of W[k][y + e_k], where y + e_k is fluid for
// component s; otherwise what y pulls from itself in direction kbar, half s of
// W[kbar][y].  0 where the component is not fluid.
__global__ void push16_to_pull16_kernel(const uint32_t* __restrict__ win, uint32_t* __restrict__ wout,
                                        const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ nbr_nw, Geom g) {
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)c;
        const int x = ci % g.nx, y = (ci / g.nx) % g.ny, z = ci / g.nxy;
        const uint32_t w = nbr[ci];
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        uint32_t out[Q];
        for (int k = 0; k < Q; ++k) out[k] = 0u;
        for (int s = 0; s < 2; ++s) {
            if (cls == CLS_SOLID || (s == 1 && cls == CLS_MEMBRANE)) continue;
            const uint32_t bits = s == 0 ? w : ((w & BIT_NW_DIFF) ? nbr_nw[ci] : w);
            for (int k = 0; k < Q; ++k) {
                // bit kbar of the pull bits: y + e_k is not fluid for component s
                size_t src;
                if (k == 0 || ((bits >> OPP(k)) & 1u)) {
                    src = (size_t)OPP(k) * g.plane + ci;  // OPP(0) = 0: the rest slot
                } else {
                    bool ok = true;
                    const int tx = wrap1(x + EX(k), g.nx, g.px, ok);
                    const int ty = wrap1(y + EY(k), g.ny, g.py, ok);
                    const int tz = wrap1(z + EZ(k), g.nz, g.pz, ok);
                    src = (size_t)k * g.plane + (size_t)tz * g.nxy + (size_t)ty * g.nx + tx;
                }
                const uint32_t half = s == 0 ? (win[src] & 0xffffu) : (win[src] & 0xffff0000u);
                out[k] |= half;
            }
        }
        for (int k = 0; k < Q; ++k) wout[(size_t)k * g.plane + ci] = out[k];
    }
}

// Start of a 16-bit state: every deviation 0 and R = rho0, so the first pull
// yields w_k rho0(x) exactly (the rest equilibrium of the given densities).
__global__ void init16_kernel(const float* __restrict__ rho0, float2* __restrict__ R, Geom g) {
    const long long N = (long long)g.nxy * g.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        R[c] = make_float2(rho0[c], rho0[N + c]);
}

template <class H2, int BY, int LEAD>
cudaError_t configure16() {
    static unsigned long long configured = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(sc_step16_kernel<H2, BY, LEAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem16_bytes<BY, LEAD>());
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    return cudaSuccess;
}

int grid_cells(long long n) {
    long long b = (n + 255) / 256;
    const long long cap = 16LL * device_sm_count();
    if (b > cap) b = cap;
    return (int)std::max(1LL, b);
}

}  // namespace

// Tiles of the 16-bit step: 32 x by threads (by in {6, 8, 10}), lead 2.
bool tile16_supported(int by, int lead) { return lead == 2 && (by == 6 || by == 8 || by == 10); }

cudaError_t prepare_step16(int precision, const StepTile& t) {
    if (!tile16_supported(t.by, t.lead)) return cudaErrorInvalidValue;
#define LBM_C16(H2, BY) \
    if (t.by == BY) return configure16<H2, BY, 2>();
    if (precision == 1) { LBM_C16(__half2, 6) LBM_C16(__half2, 8) LBM_C16(__half2, 10) }
    if (precision == 2) { LBM_C16(__nv_bfloat162, 6) LBM_C16(__nv_bfloat162, 8) LBM_C16(__nv_bfloat162, 10) }
#undef LBM_C16
    return cudaErrorInvalidValue;
}

cudaError_t launch_step16(int precision, const uint32_t* win, uint32_t* wout, const float2* Rin, float2* Rout,
                          const uint32_t* nbr, const uint32_t* nbr_nw, const uint32_t* adh, const Geom& g,
                          const Phys& p, StepTile t, cudaStream_t s) {
    if (t.lz < 1 || !tile16_supported(t.by, t.lead)) return cudaErrorInvalidValue;
    const int ty = t.by - 2;
    dim3 grid((g.nx + 29) / 30, (g.ny + ty - 1) / ty, (g.nz + t.lz - 1) / t.lz);
    dim3 block(32, t.by);
#define LBM_L16(H2, BY)                                                                                         \
    if (t.by == BY) {                                                                                           \
        sc_step16_kernel<H2, BY, 2><<<grid, block, smem16_bytes<BY, 2>(), s>>>(win, wout, Rin, Rout, nbr, nbr_nw, \
                                                                               adh, g, p, t.lz);                \
        return cudaGetLastError();                                                                              \
    }
    if (precision == 1) { LBM_L16(__half2, 6) LBM_L16(__half2, 8) LBM_L16(__half2, 10) }
    if (precision == 2) { LBM_L16(__nv_bfloat162, 6) LBM_L16(__nv_bfloat162, 8) LBM_L16(__nv_bfloat162, 10) }
#undef LBM_L16
    return cudaErrorInvalidValue;
}

cudaError_t launch_init16(const float* rho0, float2* R, const Geom& g, cudaStream_t s) {
    init16_kernel<<<grid_cells((long long)g.nxy * g.nz), 256, 0, s>>>(rho0, R, g);
    return cudaGetLastError();
}

cudaError_t launch_density16(int precision, const uint32_t* w, const float2* R, const uint32_t* nbr,
                             const uint32_t* nbr_nw, const Geom& g, float* rho, cudaStream_t s) {
    const int b = grid_cells((long long)g.nxy * g.nz);
    if (precision == 1) density16_kernel<__half2><<<b, 256, 0, s>>>(w, R, nbr, nbr_nw, g, rho);
    else density16_kernel<__nv_bfloat162><<<b, 256, 0, s>>>(w, R, nbr, nbr_nw, g, rho);
    return cudaGetLastError();
}

cudaError_t launch_measure16(int precision, const uint32_t* w, const float2* R, const uint32_t* nbr,
                             const uint32_t* nbr_nw, const Geom& g, double G, double* partials, int nblocks,
                             double* result, cudaStream_t s) {
    if (precision == 1) measure16_kernel<__half2><<<nblocks, 256, 0, s>>>(w, R, nbr, nbr_nw, g, G, partials);
    else measure16_kernel<__nv_bfloat162><<<nblocks, 256, 0, s>>>(w, R, nbr, nbr_nw, g, G, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_finalize(partials, nblocks, result, s);
}

cudaError_t launch_probe16(int precision, const uint32_t* w, const float2* R, const uint32_t* nbr,
                           const uint32_t* nbr_nw, const Geom& g, int x, int y, int z, float* out, cudaStream_t s) {
    if (precision == 1) probe16_kernel<__half2><<<1, 1, 0, s>>>(w, R, nbr, nbr_nw, g, x, y, z, out);
    else probe16_kernel<__nv_bfloat162><<<1, 1, 0, s>>>(w, R, nbr, nbr_nw, g, x, y, z, out);
    return cudaGetLastError();
}

cudaError_t launch_pull16_to_push16(const uint32_t* win, uint32_t* wout, const uint32_t* nbr, const uint32_t* nbr_nw,
                                    const Geom& g, cudaStream_t s) {
    pull16_to_push16_kernel<<<grid_cells((long long)g.nxy * g.nz), 256, 0, s>>>(win, wout, nbr, nbr_nw, g);
    return cudaGetLastError();
}

cudaError_t launch_push16_to_pull16(const uint32_t* win, uint32_t* wout, const uint32_t* nbr, const uint32_t* nbr_nw,
                                    const Geom& g, cudaStream_t s) {
    push16_to_pull16_kernel<<<grid_cells((long long)g.nxy * g.nz), 256, 0, s>>>(win, wout, nbr, nbr_nw, g);
    return cudaGetLastError();
}

}  // namespace lbmk
