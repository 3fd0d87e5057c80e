// Monte Carlo rendering equation at G-buffer points (IRGS Eq. 3 and 15) with
// the dielectric BRDF of Eq. 4 and the light split of Eq. 13-14: every
// incident ray is traced for its indirect radiance L_ind and visibility V,
// and L_i = V L_dir + L_ind with L_dir looked up in an equirectangular
// environment map. Incident directions are importance sampled per lobe
// (cosine-weighted for the diffuse term, GGX for the specular term), as in
// the paper's supplementary rendering of its composited scene.
//
// One warp shades one point: lanes take samples s = lane, lane + 32, ... and
// the per-point sums are reduced with a fixed butterfly, so a point's result
// depends only on (seed, point index, inputs), not on batching. The traced
// rays of a point share their origin; by default each lane walks its own
// stack (the directions spread over the hemisphere), IRGS_FLAG_WARP walks
// one stack for the warp. Both give identical results.
#include <cuda_runtime.h>

#include "scene.h"
#include "shade.cuh"
#include "trace.cuh"

namespace irgs {
namespace {

constexpr int kShadeThreads = 128;
__device__ __forceinline__ f3 ld3(const float* p, int64_t i) { return mk3(p[3 * i], p[3 * i + 1], p[3 * i + 2]); }

template <int K, bool WARP>
__global__ void __launch_bounds__(kShadeThreads) k_shade(SceneView S, const float* __restrict__ xg,
                                                         const float* __restrict__ ng, const float* __restrict__ ag,
                                                         const float* __restrict__ rg, const float* __restrict__ wog,
                                                         int64_t Pn, const float* __restrict__ env, int H, int W,
                                                         int nd, int ns, uint64_t seed, TraceParams TP,
                                                         float* __restrict__ rgb, float* __restrict__ vis,
                                                         float* __restrict__ ind) {
    static_assert(kShadeThreads == trace_threads<K>(), "k-buffer slots are laid out per block thread");
    const int lane = threadIdx.x & 31;
    const int64_t p = blockIdx.x * (int64_t)(kShadeThreads / 32) + (threadIdx.x >> 5);
    if (p >= Pn) return;
    ShadeSums o;
    shade_point_warp<K, WARP>(S, ld3(xg, p), ld3(ng, p), ld3(wog, p), ld3(ag, p), rg[p], (uint64_t)p, nd, ns, seed,
                              env, H, W, TP, o);
    if (lane == 0) {
        for (int c = 0; c < 3; ++c) rgb[3 * p + c] = o.rgb[c];
        if (vis != nullptr) vis[p] = o.vis;
        if (ind != nullptr)
            for (int c = 0; c < 3; ++c) ind[3 * p + c] = o.ind[c];
    }
}

}  // namespace

irgs_status launch_shade_mc(const SceneView& S, const float* x, const float* n, const float* albedo,
                            const float* rough, const float* wo, int64_t P, const float* env, int32_t H, int32_t W,
                            int32_t n_diffuse, int32_t n_spec, uint64_t seed, const irgs_trace_params& p,
                            float* rgb, float* vis, float* ind, cudaStream_t st) {
    if (P == 0) return IRGS_OK;
    const TraceParams TP = to_params(p);
    const int64_t blocks = (P + (kShadeThreads / 32) - 1) / (kShadeThreads / 32);
    const bool warp = (p.flags & IRGS_FLAG_WARP) != 0u;
#define IRGS_SHADE_LAUNCH(KK, WW)                                                                        \
    k_shade<KK, WW><<<(unsigned)blocks, kShadeThreads, 0, st>>>(S, x, n, albedo, rough, wo, P, env, H, W, \
                                                               n_diffuse, n_spec, seed, TP, rgb, vis, ind)
    switch (p.k) {
        case 8:
            if (warp) IRGS_SHADE_LAUNCH(8, true); else IRGS_SHADE_LAUNCH(8, false);
            break;
        case 16:
            if (warp) IRGS_SHADE_LAUNCH(16, true); else IRGS_SHADE_LAUNCH(16, false);
            break;
        default: return IRGS_ERR_UNSUPPORTED;
    }
#undef IRGS_SHADE_LAUNCH
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

}  // namespace irgs
