// Regrouping key of secondary rays for wavefront tracing: a 6-bit octahedral
// direction bin above the 24-bit Morton code of the ray origin, so that
// after a radix sort the rays of a warp leave neighbouring points in similar
// directions (shared by the shading and relighting wavefronts).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace irgs {

constexpr uint32_t kInvalidWaveKey = 0xffffffffu;   // sorts after every valid key

// Inverse of the order-preserving float view the scene's bounds are kept in.
__device__ __forceinline__ float bound_value(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// 8-bit value -> every third bit of a 24-bit word.
__device__ __forceinline__ uint32_t spread8(uint32_t v) {
    v &= 0xffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Regrouping key of a ray: octahedral direction bin (8 x 8) above the
// Morton code of the origin quantised to 256 cells per axis of the scene's
// centre bounds (clamped).
__device__ __forceinline__ uint32_t wave_key(f3 x, f3 d, const uint32_t* __restrict__ bounds) {
    const float c[3] = {x.x, x.y, x.z};
    uint32_t q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = bound_value(bounds[k]), hi = bound_value(bounds[3 + k]);
        const float ext = hi - lo;
        float t = ext > 0.f ? (c[k] - lo) / ext : 0.5f;
        t = t == t ? fminf(fmaxf(t, 0.f), 1.f) : 0.f;
        q[k] = (uint32_t)fminf(t * 256.f, 255.f);
    }
    const uint32_t morton = (spread8(q[0]) << 2) | (spread8(q[1]) << 1) | spread8(q[2]);
    const float l1 = fabsf(d.x) + fabsf(d.y) + fabsf(d.z);
    float u = d.x / l1, v = d.y / l1;
    if (d.z < 0.f) {
        const float uu = (1.f - fabsf(v)) * (u >= 0.f ? 1.f : -1.f);
        const float vv = (1.f - fabsf(u)) * (v >= 0.f ? 1.f : -1.f);
        u = uu;
        v = vv;
    }
    const uint32_t bu = (uint32_t)fminf(fmaxf((u * 0.5f + 0.5f) * 8.f, 0.f), 7.f);
    const uint32_t bv = (uint32_t)fminf(fmaxf((v * 0.5f + 0.5f) * 8.f, 0.f), 7.f);
    return ((bu << 3 | bv) << 24) | morton;
}

}  // namespace irgs
