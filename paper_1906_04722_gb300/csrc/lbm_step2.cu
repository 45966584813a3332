// lbm_step2.cu -- the staged FP32 step with two threads per cell, one per
// fluid component.
//
// Same data movement as step_column (lbm_step_core.cuh): a CTA owns 30 x (BY-2)
// columns plus a one-cell ring and marches a z segment; every thread queues its
// pulls as 4-byte cp.async copies LEAD planes ahead into private shared-memory
// slots.  The difference is the thread mapping: the block is 32 x BY x 2, the
// second half running the non-wetting component of the same cells.  A thread
// pulls 19 populations instead of 38 and holds 19 in registers, so twice as
// many warps share an SM at the same shared memory per cell -- the step is
// bound by instruction issue and latency, not by DRAM, and more warps hide more
// of it.  The two threads of a cell exchange their momenta through shared
// memory (a named barrier of the row's two warps) for the common velocity; the
// collision is collide_component, the arithmetic of the other kernels.
#include "lbm_step_core.cuh"

namespace lbmk {

namespace {

// Queue the pull of component s of this thread's cell (see issue_pull).
template <int NT>
__device__ __forceinline__ void issue_pull1(const float* __restrict__ fin, const uint32_t* __restrict__ nbr_nw,
                                           const Geom& g, const Column& c, int zz, int cell, uint32_t w, int s,
                                           float* st, int tid) {
    const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
    if (cls == CLS_SOLID || cls == CLS_OUTSIDE || (s == 1 && cls == CLS_MEMBRANE)) return;
    const bool seam = (g.px && (c.xo[1] == 0 || c.xo[1] == g.nx - 1)) ||
                      (g.py && (c.yo[1] == 0 || c.yo[1] == (g.ny - 1) * g.nx)) ||
                      (g.pz && (zz == 0 || zz == g.nz - 1));
    int zo[3];
    zo[0] = nb1(zz - 1, g.nz, g.pz) * g.nxy;
    zo[1] = zz * g.nxy;
    zo[2] = nb1(zz + 1, g.nz, g.pz) * g.nxy;
    const uint32_t bits = (s == 1 && (w & BIT_NW_DIFF)) ? __ldg(nbr_nw + cell) : w;
    const float* fs = fin + (size_t)s * Q * g.plane;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        int idx;
        if (!seam) idx = cell + g.poff[k];
        else idx = k * g.plane + zo[1 - EZ(k)] + c.yo[1 - EY(k)] + c.xo[1 - EX(k)];
        if ((bits >> k) & 1u) idx = OPP(k) * g.plane + cell;
        cp_async4(st + k * NT + tid, fs + idx);
    }
}

template <int BY, int LEAD>
constexpr size_t step2_smem_floats() {
    // stages [NS][2][Q][NT], density ring [4][2][NT], words and adhesion words
    // [NS][2][NT] each, momentum exchange [2][3][NT]
    return (size_t)(LEAD + 1) * 2 * Q * 32 * BY + 8 * 32 * BY + 4 * (LEAD + 1) * 32 * BY + 6 * 32 * BY;
}

template <int BY, int LEAD>
__global__ void __launch_bounds__(64 * BY, 2)
    sc_step2_kernel(const float* __restrict__ fin, float* __restrict__ fout, const uint32_t* __restrict__ nbr,
                    const uint32_t* __restrict__ nbr_nw, const uint32_t* __restrict__ adh, Geom g, Phys P, int lz) {
    constexpr int TY = BY - 2;
    constexpr int NT = 32 * BY;
    constexpr int NS = LEAD + 1;
    extern __shared__ float smem[];
    float* stage = smem;                                              // [NS][2][Q][NT]
    float* ring = stage + NS * 2 * Q * NT;                            // [4][2][NT]
    uint32_t* words = reinterpret_cast<uint32_t*>(ring + 8 * NT);     // [NS][2][NT]
    uint32_t* adhw = words + NS * 2 * NT;                             // [NS][2][NT]
    float* xch = reinterpret_cast<float*>(adhw + NS * 2 * NT);        // [2][3][NT]
    const int lane = threadIdx.x, row = threadIdx.y, s = threadIdx.z;
    const int tid = row * 32 + lane;
    const int z0 = blockIdx.z * lz;
    const int z1 = min(z0 + lz, g.nz);
    const int gx = blockIdx.x * 30 - 1 + lane;
    const int gy = blockIdx.y * TY - 1 + row;
    const Column col = make_column(gx, gy, g);
    const bool needed = gx <= g.nx && gy <= g.ny;
    const bool interior = lane >= 1 && lane <= 30 && row >= 1 && row <= TY && gx < g.nx && gy < g.ny;
    auto slot = [&](int p) { return (p - z0 + 1) % NS; };
    auto st_of = [&](int p) { return stage + (slot(p) * 2 + s) * (Q * NT); };
    auto word_at = [&](int p) -> uint32_t& { return words[(slot(p) * 2 + s) * NT + tid]; };
    auto fetch_word = [&](int p) -> uint32_t {
        if (!needed || p > z1) return CLS_OUTSIDE << CLS_SHIFT;
        int zz;
        bool ok;
        const int cell = plane_cell(g, col, p, zz, ok);
        return ok ? __ldg(nbr + cell) : (CLS_OUTSIDE << CLS_SHIFT);
    };
    auto issue = [&](int p, uint32_t w) {
        word_at(p) = w;
        if (!needed || p > z1) return;
        int zz;
        bool ok;
        const int cell = plane_cell(g, col, p, zz, ok);
        if (!ok) return;
        issue_pull1<NT>(fin, nbr_nw, g, col, zz, cell, w, s, st_of(p), tid);
        if (w & BIT_ADH)
            cp_async4(reinterpret_cast<float*>(adhw + (slot(p) * 2 + s) * NT + tid),
                      reinterpret_cast<const float*>(adh + cell));
    };
    auto publish = [&](int p) {
        const uint32_t w = word_at(p);
        const uint32_t cls = (w >> CLS_SHIFT) & CLS_MASK;
        float r = 0.f;
        if (!(cls == CLS_SOLID || cls == CLS_OUTSIDE || (s == 1 && cls == CLS_MEMBRANE))) {
            const float* st = st_of(p);
            float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < Q; ++k) a[k & 3] += st[k * NT + tid];
            r = (a[0] + a[1]) + (a[2] + a[3]);
        }
        ring[((p & 3) * 2 + s) * NT + tid] = r;
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
        cp_async_wait<LEAD - 1>();  // plane z+1 has landed
        publish(z + 1);
        __syncthreads();
        const uint32_t w0 = word_at(z);
        const uint32_t cls = (w0 >> CLS_SHIFT) & CLS_MASK;
        const bool live = interior && !(cls == CLS_SOLID || cls == CLS_OUTSIDE || (s == 1 && cls == CLS_MEMBRANE));
        float f[Q];
        float j[3] = {0.f, 0.f, 0.f};
        if (live) {
            const float* st = st_of(z);
#pragma unroll
            for (int k = 0; k < Q; ++k) f[k] = st[k * NT + tid];
            momentum(f, j);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) xch[(s * 3 + c) * NT + tid] = j[c];
        // the two warps of this row (one per component) meet here
        asm volatile("bar.sync %0, %1;\n" ::"r"(1 + row), "r"(64) : "memory");
        if (live) {
            float jo[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) jo[c] = xch[((s ^ 1) * 3 + c) * NT + tid];
            int zz;
            bool ok;
            const int cell = plane_cell(g, col, z, zz, ok);
            float* __restrict__ o = fout + (size_t)s * Q * g.plane + cell;
            const int pl = g.plane;
            const uint32_t a = adhw[(slot(z) * 2 + s) * NT + tid];
            collide_component<32, NT>(f, cls, (w0 & BIT_ADH) ? a : 0u, s, j, jo, ring, z, tid, P,
                                             [&](int k, float v) { o[(size_t)k * pl] = v; });
        }
    }
    cp_async_wait<0>();
}

template <int BY, int LEAD>
cudaError_t configure2() {
    static unsigned long long configured = 0;  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(sc_step2_kernel<BY, LEAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float) * step2_smem_floats<BY, LEAD>()));
        if (e != cudaSuccess) return e;
        configured |= bit;
    }
    return cudaSuccess;
}

template <int BY, int LEAD>
cudaError_t launch2(const float* fin, float* fout, const uint32_t* nbr, const uint32_t* nbr_nw, const uint32_t* adh,
                    const Geom& g, const Phys& p, int lz, cudaStream_t s) {
    constexpr int TY = BY - 2;
    dim3 grid((g.nx + 29) / 30, (g.ny + TY - 1) / TY, (g.nz + lz - 1) / lz);
    dim3 block(32, BY, 2);
    sc_step2_kernel<BY, LEAD>
        <<<grid, block, sizeof(float) * step2_smem_floats<BY, LEAD>(), s>>>(fin, fout, nbr, nbr_nw, adh, g, p, lz);
    return cudaGetLastError();
}

}  // namespace

bool tile2_supported(int by, int lead) { return lead == 2 && (by == 6 || by == 8); }

cudaError_t prepare_step2(const StepTile& t) {
    if (t.lz < 1 || !tile2_supported(t.by, t.lead)) return cudaErrorInvalidValue;
    return t.by == 6 ? configure2<6, 2>() : configure2<8, 2>();
}

cudaError_t launch_step2(const float* fin, float* fout, const uint32_t* nbr, const uint32_t* nbr_nw,
                         const uint32_t* adh, const Geom& g, const Phys& p, const StepTile& t, cudaStream_t s) {
    if (t.lz < 1 || !tile2_supported(t.by, t.lead)) return cudaErrorInvalidValue;
    return t.by == 6 ? launch2<6, 2>(fin, fout, nbr, nbr_nw, adh, g, p, t.lz, s)
                     : launch2<8, 2>(fin, fout, nbr, nbr_nw, adh, g, p, t.lz, s);
}

}  // namespace lbmk
