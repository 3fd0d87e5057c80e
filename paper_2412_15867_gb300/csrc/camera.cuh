// Pinhole camera rays (irgs_camera), shared by the serving kernel, the
// camera-ray generator and the rasteriser. Written with explicit
// round-to-nearest operations so every kernel that inlines it produces
// bit-identical directions.
#pragma once

#include <cuda_runtime.h>

#include "../../include/irgs.h"
#include "common.cuh"

namespace irgs {

// Unit direction through the centre of pixel (px, py):
// normalize(forward + x right + y up), x = ((px + 0.5)/W 2 - 1) tan W/H,
// y = (1 - (py + 0.5)/H 2) tan.
__device__ __forceinline__ f3 camera_dir(const irgs_camera& c, float px, float py) {
    const float W = (float)c.width, H = (float)c.height;
    const float aspect = __fdiv_rn(W, H);
    const float sx = __fsub_rn(__fmul_rn(__fdiv_rn(__fadd_rn(px, 0.5f), W), 2.f), 1.f);
    const float sy = __fsub_rn(1.f, __fmul_rn(__fdiv_rn(__fadd_rn(py, 0.5f), H), 2.f));
    const float xn = __fmul_rn(__fmul_rn(sx, c.tan_half_fov), aspect);
    const float yn = __fmul_rn(sy, c.tan_half_fov);
    float v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = __fmaf_rn(c.up[k], yn, __fmaf_rn(c.right[k], xn, c.forward[k]));
    const float len2 = __fmaf_rn(v[0], v[0], __fmaf_rn(v[1], v[1], __fmul_rn(v[2], v[2])));
    const float inv = __frsqrt_rn(len2);
    return mk3(__fmul_rn(v[0], inv), __fmul_rn(v[1], inv), __fmul_rn(v[2], inv));
}

}  // namespace irgs
