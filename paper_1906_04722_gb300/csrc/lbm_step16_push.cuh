// lbm_step16_push.cuh -- the step with the populations stored in 16 bits (FP16 or
// BF16 deviations, all arithmetic in FP32) on push-form storage, with population
// planes loaded by the tensor memory accelerator.
//
// Storage (the push layout of a 16-bit state): uint32 W[19][plane], W[k][cell] =
// the pair (h_w, h_nw) of the cell at the current time level, after streaming
// and before collision, so that f_k(cell) = h_k + w_k R(cell) with R the cell's
// FP32 density pair of the previous time level -- the deviations and R of the
// pull form (lbm_step16.cu), each word stored at the cell that reads it instead
// of at the cell that wrote it.  The writer takes every deviation against the
// density of the cell that will hold it (x + e_k, or x itself where the value
// bounces back), which it finds in its density ring, and feeds the rounding of
// the 18 moving values into the rest value, as the pull kernel does: the results
// equal the pull kernel's bit for bit.  Grain slots and the non-wetting half of
// a membrane cell's words are never written; densities take the cell class from
// its geometry word.
//
// Data movement, per plane: one 4-D box load of the words (36 columns from
// 28 tx - 4, so that the box starts on a 16-byte boundary; BY rows; all 19
// directions) and one 3-D box load of the R pairs of the same cells, into one
// of NS stages completing on that stage's mbarrier; the two densities of every
// box cell into a 4-plane ring; one barrier per plane; the collision of the
// plane behind (collide_core, the pull kernel's arithmetic, in its compile-time
// tau = 1 form where both tau are 1: the same bits) and the pushed
// stores: one 32-bit store per direction where both components stream alike,
// separate 16-bit stores next to a membrane.  The interior threads write their
// cell's new density pair to R out.  A z segment's two boundary planes are
// loaded with an evict-last L2 policy.  Waits are bounded (2 s): one that runs
// out sets *err, waits (bounded) for the copies in flight and ends the CTA.
//
// Requirements (checked on the host): no periodic x or y axis, nx a multiple
// of 4 (the word rows' pitch must be a multiple of 16 bytes).
#pragma once

#include <cuda.h>

#include "lbm_pair16.cuh"
#include "lbm_push_tma.cuh"
#include "lbm_step_core.cuh"

namespace lbmk {

namespace {

constexpr int P16X = 32;   // threads per row: box cells 28 tx - 2 + lane
constexpr int P16XI = 28;  // interior columns: lanes 2 .. 29
constexpr int P16BX = 36;  // box columns loaded: 28 tx - 4 .. 28 tx + 31

// bytes of a plane's word box and R box, and the 128-byte multiples a stage
// reserves for them (every box lands on a 128-byte boundary)
template <int BY>
constexpr uint32_t words16_bytes() {
    return (uint32_t)(Q * BY * P16BX * sizeof(uint32_t));
}
template <int BY>
constexpr uint32_t r16_bytes() {
    return (uint32_t)(BY * P16BX * sizeof(float2));
}
constexpr uint32_t pad128(uint32_t b) { return (b + 127u) / 128u * 128u; }
template <int BY, int NS>
constexpr size_t push16_smem_bytes() {
    return (size_t)NS * (pad128(words16_bytes<BY>()) + pad128(r16_bytes<BY>())) + sizeof(float2) * 4 * BY * P16X +
           sizeof(uint64_t) * NS;
}

// one cell's 19 pair words and its R pair
struct CellWords {
    uint32_t w[Q];
    float2 R;
};

// RR: each interior thread keeps its cell's words in registers from the density
// pass to its collision, so a stage is free once its plane's densities are in
// the ring and all NS stages are in flight; otherwise the collision reads the
// words from the stage again and NS - 2 stages load ahead.  TAU1: the
// compile-time tau = 1 form of the collision (the same bits as the general form
// run with tau = 1).
template <class H2, int BY, int NS, int MINB, bool RR, bool TAU1>
__global__ void __launch_bounds__(P16X * BY, MINB)
    sc_step16_push_kernel(const __grid_constant__ CUtensorMap tw, const __grid_constant__ CUtensorMap tr,
                          uint32_t* __restrict__ wout, float2* __restrict__ Rout, const uint32_t* __restrict__ nbr,
                          const uint32_t* __restrict__ nbr_nw, const uint32_t* __restrict__ adh, Geom g, Phys P,
                          int lz, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    // an earlier launch or CTA gave up: the whole CTA leaves (one decision for all its threads)
    if (__syncthreads_or(*reinterpret_cast<volatile int*>(err) != 0)) return;
    constexpr int TY = BY - 2;
    constexpr int NT = P16X * BY;
    constexpr uint32_t WP = pad128(words16_bytes<BY>()), RP = pad128(r16_bytes<BY>());
    unsigned char* stw = smem;                           // NS word boxes [Q][BY][36], WP bytes apart
    unsigned char* str = smem + NS * WP;                 // NS R boxes [BY][36], RP bytes apart
    float2* ring = reinterpret_cast<float2*>(smem + NS * (WP + RP));  // [4][BY][32]
    uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(ring) + sizeof(float2) * 4 * NT);
    const int lane = threadIdx.x, row = threadIdx.y;
    const int tid = row * P16X + lane;
    const int xb = blockIdx.x * P16XI - 2;  // box column of lane 0
    const int yb = blockIdx.y * TY - 1;     // box row of row 0
    const int gx = xb + lane, gy = yb + row;
    const int z0 = blockIdx.z * lz;
    const int z1 = min(z0 + lz, g.nz);
    const int n = z1 - z0;
    // sequence index j: plane z0 - 1 + j (j = 0 and n + 1 the halo planes)
    auto plane = [&](int j) { return z0 - 1 + j; };
    const bool interior = lane >= 2 && lane < 2 + P16XI && row >= 1 && row <= TY && gx < g.nx && gy < g.ny;
    const int col = gy * g.nx + gx;  // valid for interior threads
    const int sc = row * P16BX + lane + 2;  // this thread's cell in a stage row block

    auto slot = [&](int j) { return j % NS; };
    auto parity = [&](int j) { return (uint32_t)((j / NS) & 1); };
    // plane j's words and R pairs into its stage; a plane beyond a closed z face
    // is not loaded (its densities are zero) and only completes the phase
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
        p_mbar_arrive_expect_tx(b, words16_bytes<BY>() + r16_bytes<BY>());
        unsigned char* dw = stw + (size_t)slot(j) * WP;
        unsigned char* dr = str + (size_t)slot(j) * RP;
        if (j == 0 || j == n + 1) {  // read again by the neighbouring segment later: kept in L2
            const uint64_t pol = p_policy_evict_last();
            p_tma_load_4d_hint(dw, &tw, xb - 2, yb, zc, 0, b, pol);
            p_tma_load_3d_hint(dr, &tr, 2 * (xb - 2), yb, zc, b, pol);
        } else {
            p_tma_load_4d(dw, &tw, xb - 2, yb, zc, 0, b);
            p_tma_load_3d(dr, &tr, 2 * (xb - 2), yb, zc, b);
        }
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
    // the pair words and the R pair of this thread's box cell on plane j
    auto fetch = [&](int j, CellWords& c) {
        const uint32_t* ws = reinterpret_cast<const uint32_t*>(stw + (size_t)slot(j) * WP) + sc;
#pragma unroll
        for (int k = 0; k < Q; ++k) c.w[k] = ws[k * (BY * P16BX)];
        c.R = reinterpret_cast<const float2*>(str + (size_t)slot(j) * RP)[sc];
    };
    // the populations of a cell from its words and R pair (the pull kernel's
    // reconstruction; 0 for the non-wetting fluid on a membrane, whatever that
    // half of the words holds)
    auto reconstruct = [&](const CellWords& c, bool has_nw, float (&f)[2][Q]) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const float2 h = Pair<H2>::unpack(c.w[k]);
            f[0][k] = h.x + WK(k) * c.R.x;
            f[1][k] = has_nw ? h.y + WK(k) * c.R.y : 0.f;
        }
    };
    // densities of the box cell on plane j into the ring (0 where not fluid; a
    // buffer's grain slots may hold anything), and into R out for the interior
    // (RR: the words stay in `keep` for the collision)
    auto publish = [&](int j, uint32_t wp, CellWords& keep) {
        const uint32_t c = (wp >> CLS_SHIFT) & CLS_MASK;
        float rw = 0.f, rn = 0.f;
        if (c != CLS_SOLID && c != CLS_OUTSIDE) {
            float f[2][Q];
            fetch(j, keep);
            reconstruct(keep, c != CLS_MEMBRANE, f);
            float a[4] = {0.f, 0.f, 0.f, 0.f}, b[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                a[k & 3] += f[0][k];
                b[k & 3] += f[1][k];
            }
            rw = (a[0] + a[1]) + (a[2] + a[3]);
            rn = (b[0] + b[1]) + (b[2] + b[3]);
        }
        ring[(plane(j) & 3) * NT + tid] = make_float2(rw, rn);
        if (interior && j >= 1 && j <= n) Rout[(size_t)plane(j) * g.nxy + col] = make_float2(rw, rn);
    };
    // the adhesion and non-wetting bounce words of an interior cell, a plane ahead
    auto extra = [&](int j, uint32_t wp, uint32_t& ap, uint32_t& np) {
        ap = 0u;
        np = 0u;
        if (!interior || j < 1 || j > n) return;
        const int p = plane(j);
        if (wp & BIT_ADH) ap = __ldg(adh + (size_t)p * g.nxy + col);
        if (wp & BIT_NW_DIFF) np = __ldg(nbr_nw + (size_t)p * g.nxy + col);
    };

    if (tid == 0) {
        for (int i = 0; i < NS; ++i) p_mbar_init(bar + i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    int next = min(NS, n + 2);  // the first sequence index not yet issued (thread 0)
    if (tid == 0)
        for (int j = 0; j < next; ++j) issue(j);
    const uint32_t w_m = word(0);
    uint32_t w_0 = word(1), w_1 = word(2);
    uint32_t a_0, nwb_0;
    extra(1, w_0, a_0, nwb_0);
    CellWords cur, nxt;  // RR: words of the plane to collide and of the next plane
    bool ok = p_mbar_wait_bounded(bar + slot(0), parity(0));
    if (ok) publish(0, w_m, nxt);
    ok = ok && p_mbar_wait_bounded(bar + slot(1), parity(1));
    if (ok) publish(1, w_0, cur);
    // a failed wait here is reported by the first iteration's barrier below
    for (int j = 1; j <= n; ++j) {
        const int z = plane(j);
        const uint32_t w = w_0, a = a_0, nwb = nwb_0;
        const uint32_t w_2 = word(j + 2);  // for the next iteration's publish
        extra(j + 1, w_1, a_0, nwb_0);     // for the next iteration's collision
        const bool okz = ok && p_mbar_wait_bounded(bar + slot(j + 1), parity(j + 1));
        if (okz) publish(j + 1, w_1, nxt);
        if (__syncthreads_or(!okz)) {
            if (tid == 0) {
                atomicOr(err, 1);
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
            for (; next <= n + 1 && next <= last; ++next) issue(next);
        }
        w_0 = w_1;
        w_1 = w_2;
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        if (!interior || cls == CLS_SOLID || cls == CLS_OUTSIDE) {
            if constexpr (RR) cur = nxt;
            continue;
        }
        const bool has_nw = cls != CLS_MEMBRANE;
        const uint32_t wn = has_nw && (w & BIT_NW_DIFF) ? nwb : w;
        float f[2][Q];
        if constexpr (RR) {
            reconstruct(cur, has_nw, f);
            cur = nxt;
        } else {
            CellWords c;
            fetch(j, c);
            reconstruct(c, has_nw, f);
        }
        float out[2][Q];
        collide_core<TAU1>(
            f, w, a, P, [&](int k) { return ring[((z + EZ(k)) & 3) * NT + (row + EY(k)) * P16X + (lane + EX(k))]; },
            [&](int s, int k, float v) { out[s][k] = v; });
        if (!has_nw) {
#pragma unroll
            for (int k = 0; k < Q; ++k) out[1][k] = 0.f;
        }
        // each value as a deviation against the density of the cell that will
        // hold it: x + e_k, or x itself where the component bounces back (pull
        // bit kbar: x + e_k is not fluid for it); pushed to that cell's slot k,
        // or to x's own slot kbar
        auto rho_at = [&](int k) { return ring[((z + EZ(k)) & 3) * NT + (row + EY(k)) * P16X + (lane + EX(k))]; };
        const float2 self = rho_at(0);
        const int dzp = (z == g.nz - 1) ? (1 - g.nz) * g.nxy : g.nxy;
        const int dzm = (z == 0) ? (g.nz - 1) * g.nxy : -g.nxy;
        const int cell = z * g.nxy + col;
        auto dst = [&](int k, uint32_t bits) -> size_t {
            const int off = EX(k) + EY(k) * g.nx + (EZ(k) > 0 ? dzp : (EZ(k) < 0 ? dzm : 0));
            return ((bits >> OPP(k)) & 1u) ? (size_t)OPP(k) * g.plane + cell : (size_t)k * g.plane + cell + off;
        };
        const bool alike = has_nw && !(w & BIT_NW_DIFF);
        unsigned short* wo16 = reinterpret_cast<unsigned short*>(wout);
        float e[2] = {0.f, 0.f};
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const float2 nb = rho_at(k);
            const float dw = ((w >> OPP(k)) & 1u) ? self.x : nb.x;
            const float dn = ((wn >> OPP(k)) & 1u) ? self.y : nb.y;
            const float ew = out[0][k] - WK(k) * dw;
            const float en = has_nw ? out[1][k] - WK(k) * dn : 0.f;
            // both halves rounded to nearest in one conversion; their exact
            // values feed the rounding error into the rest value
            const uint32_t u = Pair<H2>::pack(ew, en);
            const float2 r = Pair<H2>::unpack(u);
            e[0] += ew - r.x;
            e[1] += en - r.y;
            if (alike) {
                wout[dst(k, w)] = u;
            } else {
                wo16[2 * dst(k, w)] = (unsigned short)(u & 0xffffu);
                if (has_nw) wo16[2 * dst(k, wn) + 1] = (unsigned short)(u >> 16);
            }
        }
        const float e0w = out[0][0] - WK(0) * self.x + e[0];
        const float e0n = has_nw ? out[1][0] - WK(0) * self.y + e[1] : 0.f;
        wout[cell] = Pair<H2>::pack(e0w, e0n);
    }
}

template <class H2, int BY, int NS, int MINB, bool RR, bool TAU1>
cudaError_t configure_push16() {
    static unsigned long long configured = 0;  // one bit per device: the attribute is per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(sc_step16_push_kernel<H2, BY, NS, MINB, RR, TAU1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)push16_smem_bytes<BY, NS>());
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    return cudaSuccess;
}

template <class H2, int BY, int NS, int MINB, bool RR, bool TAU1>
cudaError_t launch_push16_shape(const CUtensorMap& tw, const CUtensorMap& tr, uint32_t* wout, float2* Rout,
                                const uint32_t* nbr, const uint32_t* nbr_nw, const uint32_t* adh, const Geom& g,
                                const Phys& p, int lz, int* err, cudaStream_t s) {
    constexpr int TY = BY - 2;
    const dim3 grid((g.nx + P16XI - 1) / P16XI, (g.ny + TY - 1) / TY, (g.nz + lz - 1) / lz);
    sc_step16_push_kernel<H2, BY, NS, MINB, RR, TAU1><<<grid, dim3(P16X, BY), push16_smem_bytes<BY, NS>(), s>>>(
        tw, tr, wout, Rout, nbr, nbr_nw, adh, g, p, lz, err);
    return cudaGetLastError();
}

// Shapes by index: box rows BY, plane stages NS, CTAs per SM (which also caps a
// thread's registers), register-resident words (RR).
struct Push16ShapeInfo {
    int by, ns, minb;
    bool rr;
};
constexpr Push16ShapeInfo kPush16Shapes[] = {{8, 4, 2, false}, {6, 4, 2, false}, {7, 4, 2, false},
                                             {10, 3, 2, false}, {6, 4, 2, true},  {8, 4, 2, true},
                                             {9, 3, 2, false},  {7, 3, 3, false}, {6, 3, 3, false},
                                             {11, 3, 2, false}, {12, 3, 1, true}, {8, 3, 2, true}};
constexpr int N_PUSH16_SHAPES = (int)(sizeof(kPush16Shapes) / sizeof(kPush16Shapes[0]));

// both collision forms of shape I
template <int I, class H2>
cudaError_t configure16_shape() {
    constexpr Push16ShapeInfo S = kPush16Shapes[I];
    cudaError_t e = configure_push16<H2, S.by, S.ns, S.minb, S.rr, true>();
    return e != cudaSuccess ? e : configure_push16<H2, S.by, S.ns, S.minb, S.rr, false>();
}

// tau1: tau = 1 in both components (the compile-time tau = 1 collision)
template <int I, class H2>
cudaError_t launch16_shape(bool tau1, const CUtensorMap& tw, const CUtensorMap& tr, uint32_t* wout, float2* Rout,
                           const uint32_t* nbr, const uint32_t* nbr_nw, const uint32_t* adh, const Geom& g,
                           const Phys& p, int lz, int* err, cudaStream_t s) {
    constexpr Push16ShapeInfo S = kPush16Shapes[I];
    return tau1 ? launch_push16_shape<H2, S.by, S.ns, S.minb, S.rr, true>(tw, tr, wout, Rout, nbr, nbr_nw, adh, g, p,
                                                                         lz, err, s)
                : launch_push16_shape<H2, S.by, S.ns, S.minb, S.rr, false>(tw, tr, wout, Rout, nbr, nbr_nw, adh, g, p,
                                                                          lz, err, s);
}

// the 16-bit push step of shape `shape` with the 16-bit type H2 (one case per
// shape; the two translation units instantiate one type each)
template <class H2>
cudaError_t prepare16_any(int shape) {
    static_assert(N_PUSH16_SHAPES == 12, "one case per shape below");
    switch (shape) {
        case 0: return configure16_shape<0, H2>();
        case 1: return configure16_shape<1, H2>();
        case 2: return configure16_shape<2, H2>();
        case 3: return configure16_shape<3, H2>();
        case 4: return configure16_shape<4, H2>();
        case 5: return configure16_shape<5, H2>();
        case 6: return configure16_shape<6, H2>();
        case 7: return configure16_shape<7, H2>();
        case 8: return configure16_shape<8, H2>();
        case 9: return configure16_shape<9, H2>();
        case 10: return configure16_shape<10, H2>();
        case 11: return configure16_shape<11, H2>();
    }
    return cudaErrorInvalidValue;
}

template <class H2>
cudaError_t launch16_any(int shape, const CUtensorMap& tw, const CUtensorMap& tr, uint32_t* wout, float2* Rout,
                         const uint32_t* nbr, const uint32_t* nbr_nw, const uint32_t* adh, const Geom& g, const Phys& p,
                         int lz, int* err, cudaStream_t s) {
    if (lz < 1) return cudaErrorInvalidValue;
    const bool t1 = p.tau[0] == 1.0f && p.tau[1] == 1.0f;
#define LBM_P16(I) \
    case I: return launch16_shape<I, H2>(t1, tw, tr, wout, Rout, nbr, nbr_nw, adh, g, p, lz, err, s);
    switch (shape) {
        LBM_P16(0)
        LBM_P16(1)
        LBM_P16(2)
        LBM_P16(3)
        LBM_P16(4)
        LBM_P16(5)
        LBM_P16(6)
        LBM_P16(7)
        LBM_P16(8)
        LBM_P16(9)
        LBM_P16(10)
        LBM_P16(11)
    }
#undef LBM_P16
    return cudaErrorInvalidValue;
}

}  // namespace

// the BF16 instantiations, compiled in a translation unit of their own
cudaError_t prepare_step16_push_bf16(int shape);
cudaError_t launch_step16_push_bf16(int shape, const CUtensorMap& tw, const CUtensorMap& tr, uint32_t* wout,
                                    float2* Rout, const uint32_t* nbr, const uint32_t* nbr_nw, const uint32_t* adh,
                                    const Geom& g, const Phys& p, int lz, int* err, cudaStream_t s);

}  // namespace lbmk
