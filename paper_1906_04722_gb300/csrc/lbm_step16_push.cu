// lbm_step16_push.cu -- host side of the 16-bit push step (tensor maps, shape
// table queries, default segment length) and the FP16 instantiations of the
// kernel in lbm_step16_push.cuh.
#include "lbm_step16_push.cuh"

namespace lbmk {

namespace {

using Encode16Fn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

Encode16Fn encode16_fn() {
    static Encode16Fn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Encode16Fn>(p);
    }
    return fn;
}

}  // namespace

int push16_shape_count() { return N_PUSH16_SHAPES; }

int push16_shape_rows(int shape) {
    return (shape >= 0 && shape < N_PUSH16_SHAPES) ? kPush16Shapes[shape].by : 0;
}

int push16_shape_stages(int shape) {
    return (shape >= 0 && shape < N_PUSH16_SHAPES) ? kPush16Shapes[shape].ns : 0;
}

bool push16_step_applicable(const Geom& g) { return !g.px && !g.py && g.nx % 4 == 0; }

cudaError_t encode_push16_maps(const Geom& g, uint32_t* w0, uint32_t* w1, float2* r0, float2* r1, int by,
                               CUtensorMap (&mw)[2], CUtensorMap (&mr)[2]) {
    if (!push16_step_applicable(g) || by < 1) return cudaErrorInvalidValue;
    Encode16Fn enc = encode16_fn();
    if (!enc) return cudaErrorNotSupported;
    // words: (x, y, z, direction); R pairs: (component-interleaved x as floats, y, z)
    const cuuint64_t wd[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)Q};
    const cuuint64_t ws[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nxy * 4, (cuuint64_t)g.plane * 4};
    const cuuint32_t wbox[4] = {(cuuint32_t)P16BX, (cuuint32_t)by, 1, (cuuint32_t)Q};
    const cuuint64_t rd[3] = {(cuuint64_t)2 * g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t rs[2] = {(cuuint64_t)g.nx * 8, (cuuint64_t)g.nxy * 8};
    const cuuint32_t rbox[3] = {(cuuint32_t)(2 * P16BX), (cuuint32_t)by, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    uint32_t* wb[2] = {w0, w1};
    float2* rb[2] = {r0, r1};
    for (int i = 0; i < 2; ++i) {
        if (enc(&mw[i], CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, wb[i], wd, ws, wbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        if (enc(&mr[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, rb[i], rd, rs, rbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

int push16_default_lz(const Geom& g, int shape) {
    const int ty = push16_shape_rows(shape) - 2;
    if (ty <= 0) return 1;
    const long long tiles = (long long)((g.nx + P16XI - 1) / P16XI) * ((g.ny + ty - 1) / ty);
    long long segs = device_sm_count() / tiles;
    if (segs < 1) segs = 1;
    int lz = (int)((g.nz + segs - 1) / segs);
    if (lz > 32) lz = 32;
    if (lz < 4) lz = 4;
    if (lz > g.nz) lz = g.nz;
    return lz;
}

cudaError_t prepare_step16_push(int precision, int shape) {
    if (precision == 1) return prepare16_any<__half2>(shape);
    if (precision == 2) return prepare_step16_push_bf16(shape);
    return cudaErrorInvalidValue;
}

cudaError_t launch_step16_push(int precision, int shape, const CUtensorMap& tw, const CUtensorMap& tr,
                               uint32_t* wout, float2* Rout, const uint32_t* nbr, const uint32_t* nbr_nw,
                               const uint32_t* adh, const Geom& g, const Phys& p, int lz, int* err, cudaStream_t s) {
    if (precision == 1) return launch16_any<__half2>(shape, tw, tr, wout, Rout, nbr, nbr_nw, adh, g, p, lz, err, s);
    if (precision == 2) return launch_step16_push_bf16(shape, tw, tr, wout, Rout, nbr, nbr_nw, adh, g, p, lz, err, s);
    return cudaErrorInvalidValue;
}

}  // namespace lbmk
