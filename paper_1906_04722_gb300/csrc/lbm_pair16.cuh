// lbm_pair16.cuh -- a direction's two 16-bit deviations (wetting, non-wetting)
// packed in one 32-bit word, FP16 or BF16, converted with round-to-nearest.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <cstring>

namespace lbmk {

template <class H2>
struct Pair;

template <>
struct Pair<__half2> {
    static __device__ __forceinline__ float2 unpack(uint32_t u) {
        __half2 h;
        memcpy(&h, &u, 4);
        return __half22float2(h);
    }
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        uint32_t u;
        memcpy(&u, &h, 4);
        return u;
    }
    static __device__ __forceinline__ float round1(float v) { return __half2float(__float2half_rn(v)); }
};

template <>
struct Pair<__nv_bfloat162> {
    static __device__ __forceinline__ float2 unpack(uint32_t u) {
        __nv_bfloat162 h;
        memcpy(&h, &u, 4);
        return __bfloat1622float2(h);
    }
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        uint32_t u;
        memcpy(&u, &h, 4);
        return u;
    }
    static __device__ __forceinline__ float round1(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};

}  // namespace lbmk
