// lbm_step16_push_bf16.cu -- the BF16 instantiations of the 16-bit push step
// (lbm_step16_push.cuh), compiled apart from the FP16 ones so that the two
// translation units build in parallel.
#include "lbm_step16_push.cuh"

namespace lbmk {

cudaError_t prepare_step16_push_bf16(int shape) { return prepare16_any<__nv_bfloat162>(shape); }

cudaError_t launch_step16_push_bf16(int shape, const CUtensorMap& tw, const CUtensorMap& tr, uint32_t* wout,
                                    float2* Rout, const uint32_t* nbr, const uint32_t* nbr_nw, const uint32_t* adh,
                                    const Geom& g, const Phys& p, int lz, int* err, cudaStream_t s) {
    return launch16_any<__nv_bfloat162>(shape, tw, tr, wout, Rout, nbr, nbr_nw, adh, g, p, lz, err, s);
}

}  // namespace lbmk
