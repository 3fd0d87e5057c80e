// Monte Carlo rendering equation at G-buffer points (IRGS Eq. 3 and 15) with
// the dielectric BRDF of Eq. 4 and the light split of Eq. 13-14: every
// incident ray is traced for its indirect radiance L_ind and visibility V,
// and L_i = V L_dir + L_ind with L_dir looked up in an equirectangular
// environment map. Two estimators: split-lobe importance sampling (cosine-
// weighted diffuse, GGX specular, as in the paper's supplementary rendering
// of its composited scene) and stratified uniform hemisphere sampling (the
// form Eq. 15 writes out), selected by IRGS_FLAG_UNIFORM.
//
// One warp shades one point: lanes take samples s = lane, lane + 32, ... and
// the per-point sums are reduced with a fixed butterfly, so a point's result
// depends only on (seed, point index, inputs), not on batching. The traced
// rays of a point share their origin; by default each lane walks its own
// stack (the directions spread over the hemisphere), IRGS_FLAG_WARP walks
// one stack for the warp. Both give the same traces.
//
// The gradient (k_shade_backward) holds the sample directions fixed: with
// L = sum_p g_p . rgb_p and a sample's estimate term (w_a a_c + w_s) L_i,c,
//   dL/da_c  += g_c w_a L_i,c,
//   dL/dr    += sum_c g_c w_s (d ln f_s / dr) L_i,c,
//   dL/dL_ind = g_c (w_a a_c + w_s) =: gL_c,  dL/dO = -gL . L_dir,
//   dL/dL_dir texel += bilinear weight * gL_c V,
// and each traced ray is replayed backwards with (gL, g_O) as the upstream
// gradient of its colour and opacity (trace_bwd.cuh).
#include <cuda_runtime.h>

#include "scene.h"
#include "shade.cuh"
#include "trace.cuh"
#include "trace_bwd.cuh"

namespace irgs {
namespace {

constexpr int kShadeThreads = 128;
__device__ __forceinline__ f3 ld3(const float* p, int64_t i) { return mk3(p[3 * i], p[3 * i + 1], p[3 * i + 2]); }

template <int K, bool WARP>
__global__ void __launch_bounds__(kShadeThreads) k_shade(SceneView S, const float* __restrict__ xg,
                                                         const float* __restrict__ ng, const float* __restrict__ ag,
                                                         const float* __restrict__ rg, const float* __restrict__ wog,
                                                         int64_t Pn, const float* __restrict__ env, int H, int W,
                                                         int nd, int ns, int mode, uint64_t seed, TraceParams TP,
                                                         float* __restrict__ rgb, float* __restrict__ vis,
                                                         float* __restrict__ ind) {
    static_assert(kShadeThreads == trace_threads<K>(), "k-buffer slots are laid out per block thread");
    const int lane = threadIdx.x & 31;
    const int64_t p = blockIdx.x * (int64_t)(kShadeThreads / 32) + (threadIdx.x >> 5);
    if (p >= Pn) return;
    ShadeSums o;
    shade_point_warp<K, WARP>(S, ld3(xg, p), ld3(ng, p), ld3(wog, p), ld3(ag, p), rg[p], (uint64_t)p, nd, ns, mode,
                              seed, env, H, W, TP, o);
    if (lane == 0) {
        for (int c = 0; c < 3; ++c) rgb[3 * p + c] = o.rgb[c];
        if (vis != nullptr) vis[p] = o.vis;
        if (ind != nullptr)
            for (int c = 0; c < 3; ++c) ind[3 * p + c] = o.ind[c];
    }
}

template <int K, bool WARP>
__global__ void __launch_bounds__(kShadeThreads) k_shade_backward(
    SceneView S, const float* __restrict__ xg, const float* __restrict__ ng, const float* __restrict__ ag,
    const float* __restrict__ rg, const float* __restrict__ wog, int64_t Pn, const float* __restrict__ env, int H,
    int W, int nd, int ns, int mode, uint64_t seed, TraceParams TP, const float* __restrict__ g_rgb,
    float* __restrict__ g_albedo, float* __restrict__ g_rough, float* __restrict__ g_env,
    float* __restrict__ acc_rows) {
    static_assert(kShadeThreads == trace_threads<K>(), "k-buffer slots are laid out per block thread");
    __shared__ float4 rows_all[kShadeThreads * GradRow<3>::kStride / 4];
    float* rows = reinterpret_cast<float*>(rows_all) + (threadIdx.x & ~31) * GradRow<3>::kStride;
    const int lane = threadIdx.x & 31;
    const int64_t p = blockIdx.x * (int64_t)(kShadeThreads / 32) + (threadIdx.x >> 5);
    if (p >= Pn) return;
    const f3 x = ld3(xg, p), a = ld3(ag, p);
    const float av[3] = {a.x, a.y, a.z};
    const float g[3] = {g_rgb[3 * p], g_rgb[3 * p + 1], g_rgb[3 * p + 2]};
    if (g[0] == 0.f && g[1] == 0.f && g[2] == 0.f) return;   // uniform across the warp
    const ShadeFrame F = shade_frame(ld3(ng, p), ld3(wog, p), rg[p]);
    const int St = nd + ns;
    float ga[3] = {0.f, 0.f, 0.f}, gr = 0.f;
    bool ok = true;
    for (int base = 0; base < St; base += 32) {
        const ShadeSample d = draw_sample(F, mode, (uint64_t)p, base + lane, St, nd, seed);
        if (!WARP && !d.valid) continue;
        const Ray ray = make_ray(x, d.wi);
        MarchState<K, 3> st;
        ok &= march_forward<K, 3, WARP>(S, ray, TP, st, nullptr, 0, d.valid);
        float gL[3] = {0.f, 0.f, 0.f}, gO = 0.f;
        if (d.valid) sample_grad(F, d, mode, nd, ns, St, av, g, st.C, st.T, env, H, W, g_env, ga, gr, gL, gO);
        const bool live = d.valid && st.nh > 0;
        if (!WARP && !live) continue;
        ok &= march_backward<K, 3, WARP>(S, ray, TP, live, st.nh, st.C, st.D, st.T, gL, 0.f, gO, acc_rows, rows);
    }
    if (!ok) atomicOr(S.status, kErrStackOverflow);
#pragma unroll
    for (int k = 0; k < 3; ++k)
        for (int off = 16; off > 0; off >>= 1) ga[k] += __shfl_xor_sync(0xffffffffu, ga[k], off);
    for (int off = 16; off > 0; off >>= 1) gr += __shfl_xor_sync(0xffffffffu, gr, off);
    if (lane == 0) {
        for (int c = 0; c < 3; ++c) g_albedo[3 * p + c] += ga[c];
        g_rough[p] += gr;
    }
}

int shade_mode(const irgs_trace_params& p) { return (p.flags & IRGS_FLAG_UNIFORM) ? kModeUniform : kModeSplit; }

}  // namespace

// Directions of the secondary rays the estimator traces (the sampler of
// shade_point_warp without the traces): ray i = p * (nd + ns) + s.
__global__ void k_sample_rays(const float* __restrict__ ng, const float* __restrict__ rg,
                              const float* __restrict__ wog, int64_t Pn, int nd, int ns, int mode, uint64_t seed,
                              float* __restrict__ dir, int32_t* __restrict__ valid) {
    const int St = nd + ns;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= Pn * St) return;
    const int64_t p = i / St;
    const int s = (int)(i - p * St);
    const ShadeFrame F = shade_frame(mk3(ng[3 * p], ng[3 * p + 1], ng[3 * p + 2]),
                                     mk3(wog[3 * p], wog[3 * p + 1], wog[3 * p + 2]), rg[p]);
    const ShadeSample d = draw_sample(F, mode, (uint64_t)p, s, St, nd, seed);
    dir[3 * i] = d.wi.x;
    dir[3 * i + 1] = d.wi.y;
    dir[3 * i + 2] = d.wi.z;
    if (valid != nullptr) valid[i] = d.valid ? 1 : 0;
}

irgs_status launch_sample_rays(const float* n, const float* rough, const float* wo, int64_t P, int32_t nd,
                               int32_t ns, uint64_t seed, int mode, float* dir, int32_t* valid, cudaStream_t st) {
    const int64_t rays = P * (int64_t)(nd + ns);
    if (rays == 0) return IRGS_OK;
    const int T = 256;
    k_sample_rays<<<(unsigned)((rays + T - 1) / T), T, 0, st>>>(n, rough, wo, P, nd, ns, mode, seed, dir, valid);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

irgs_status launch_shade_mc(const SceneView& S, const float* x, const float* n, const float* albedo,
                            const float* rough, const float* wo, int64_t P, const float* env, int32_t H, int32_t W,
                            int32_t n_diffuse, int32_t n_spec, uint64_t seed, const irgs_trace_params& p,
                            float* rgb, float* vis, float* ind, cudaStream_t st) {
    if (P == 0) return IRGS_OK;
    const TraceParams TP = to_params(p);
    const int mode = shade_mode(p);
    const int64_t blocks = (P + (kShadeThreads / 32) - 1) / (kShadeThreads / 32);
    const bool warp = (p.flags & IRGS_FLAG_WARP) != 0u;
#define IRGS_SHADE_LAUNCH(KK, WW)                                                                        \
    k_shade<KK, WW><<<(unsigned)blocks, kShadeThreads, 0, st>>>(S, x, n, albedo, rough, wo, P, env, H, W, \
                                                               n_diffuse, n_spec, mode, seed, TP, rgb, vis, ind)
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

irgs_status launch_shade_mc_backward(const SceneView& S, const int32_t* perm, const float* x, const float* n,
                                     const float* albedo, const float* rough, const float* wo, int64_t P,
                                     const float* env, int32_t H, int32_t W, int32_t n_diffuse, int32_t n_spec,
                                     uint64_t seed, const irgs_trace_params& p, const float* g_rgb,
                                     float* g_albedo, float* g_rough, float* g_env, float* g_means, float* g_quats,
                                     float* g_scales, float* g_opacity, float* g_features, cudaStream_t st) {
    if (P == 0) return IRGS_OK;
    const TraceParams TP = to_params(p);
    const int mode = shade_mode(p);
    const bool warp = (p.flags & IRGS_FLAG_WARP) != 0u;
    constexpr int N = GradRow<3>::N;
    const size_t bytes = sizeof(float) * N * (size_t)(S.n > 0 ? S.n : 1);
    float* acc_rows = nullptr;
    cudaError_t e = scratch_alloc(reinterpret_cast<void**>(&acc_rows), bytes, st);
    if (e == cudaErrorMemoryAllocation) return IRGS_ERR_OOM;
    if (e != cudaSuccess) return IRGS_ERR_CUDA;
    e = cudaMemsetAsync(acc_rows, 0, bytes, st);
    if (e == cudaSuccess) {
        const int64_t blocks = (P + (kShadeThreads / 32) - 1) / (kShadeThreads / 32);
#define IRGS_SHADE_BWD(KK, WW)                                                                                     \
    k_shade_backward<KK, WW><<<(unsigned)blocks, kShadeThreads, 0, st>>>(S, x, n, albedo, rough, wo, P, env, H, W, \
                                                                        n_diffuse, n_spec, mode, seed, TP, g_rgb,  \
                                                                        g_albedo, g_rough, g_env, acc_rows)
        switch (p.k) {
            case 8:
                if (warp) IRGS_SHADE_BWD(8, true); else IRGS_SHADE_BWD(8, false);
                break;
            case 16:
                if (warp) IRGS_SHADE_BWD(16, true); else IRGS_SHADE_BWD(16, false);
                break;
            default: e = cudaErrorInvalidValue;
        }
#undef IRGS_SHADE_BWD
        if (e == cudaSuccess) {
            if (S.n > 0)
                k_grad_scatter<3><<<(unsigned)((S.n + 255) / 256), 256, 0, st>>>(perm, S.n, acc_rows, TP.fc, S.F,
                                                                                TP.off, g_means, g_quats, g_scales,
                                                                                g_opacity, g_features);
            count_launches(S.n > 0 ? 2 : 1);
            e = cudaGetLastError();
        }
    }
    const cudaError_t ef = cudaFreeAsync(acc_rows, st);
    if (e == cudaErrorInvalidValue) return IRGS_ERR_UNSUPPORTED;
    return (e == cudaSuccess && ef == cudaSuccess) ? IRGS_OK : IRGS_ERR_CUDA;
}

}  // namespace irgs
