// C ABI of libirgs.so (declared in include/irgs.h): argument validation,
// device selection and dispatch to the kernels' launchers.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "../../include/irgs.h"
#include "scene.h"

namespace irgs {
static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// One scratch pool per device, created on first use.
static std::mutex g_pool_mutex;
static cudaMemPool_t g_pools[256] = {};

cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st) {
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(g_pool_mutex);
        if (g_pools[device] == nullptr) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = device;
            cudaMemPool_t created;
            e = cudaMemPoolCreate(&created, &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = kScratchKeepBytes;
            e = cudaMemPoolSetAttribute(created, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) {
                cudaMemPoolDestroy(created);
                return e;
            }
            g_pools[device] = created;
        }
        pool = g_pools[device];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}
}  // namespace irgs

namespace {

bool finite(float x) { return isfinite(x) != 0; }

// Validate trace parameters against a scene. t_max may be +inf.
irgs_status check_params(const irgs_scene sc, const irgs_trace_params* p, bool shading = false) {
    if (p == nullptr) return IRGS_ERR_INVALID_ARG;
    if (!irgs::k_supported(p->k)) return IRGS_ERR_UNSUPPORTED;
    if (!finite(p->alpha_min) || !(p->alpha_min >= sc->alpha_min) || !(p->alpha_min > 0.f))
        return IRGS_ERR_INVALID_ARG;
    if (!finite(p->alpha_max) || !(p->alpha_max > p->alpha_min) || !(p->alpha_max <= 1.f))
        return IRGS_ERR_INVALID_ARG;
    if (!finite(p->T_min) || !(p->T_min >= 0.f) || !(p->T_min < 1.f)) return IRGS_ERR_INVALID_ARG;
    if (!finite(p->t_min) || !(p->t_min >= 0.f)) return IRGS_ERR_INVALID_ARG;
    if (isnan(p->t_max) || !(p->t_max > p->t_min)) return IRGS_ERR_INVALID_ARG;
    if (p->feat_count < 0 || p->feat_count > IRGS_MAX_FEATURES) return IRGS_ERR_INVALID_ARG;
    if (p->feat_count > 0 && (p->feat_offset < 0 || p->feat_offset + p->feat_count > sc->F))
        return IRGS_ERR_INVALID_ARG;
    const uint32_t allowed = IRGS_FLAG_PER_THREAD | IRGS_FLAG_WARP | (shading ? IRGS_FLAG_UNIFORM : 0u);
    if ((p->flags & ~allowed) != 0u) return IRGS_ERR_INVALID_ARG;
    if ((p->flags & IRGS_FLAG_PER_THREAD) && (p->flags & IRGS_FLAG_WARP)) return IRGS_ERR_INVALID_ARG;
    return IRGS_OK;
}

irgs_status use_device(irgs::DeviceGuard& g, const irgs_scene sc) {
    return g.set(sc->device) ? IRGS_OK : IRGS_ERR_CUDA;
}

// Shading runs as one fused kernel (a warp per point tracing its own
// samples) when a traversal flag is given, else as the regrouped wavefront.
bool fused_shading(const irgs_trace_params* p) {
    return (p->flags & (IRGS_FLAG_PER_THREAD | IRGS_FLAG_WARP)) != 0u;
}

int shade_mode(const irgs_trace_params* p) { return (p->flags & IRGS_FLAG_UNIFORM) ? 1 : 0; }

irgs_status check_shade(const irgs_scene sc, const irgs_trace_params* params, int64_t n_points, const float* env,
                        int32_t env_h, int32_t env_w, int32_t n_diffuse, int32_t n_spec) {
    if (sc == nullptr || n_points < 0) return IRGS_ERR_INVALID_ARG;
    irgs_status s = check_params(sc, params, true);
    if (s != IRGS_OK) return s;
    if (params->k != 8 && params->k != 16) return IRGS_ERR_UNSUPPORTED;
    if (params->feat_count != 3 || !(params->t_min > 0.f)) return IRGS_ERR_INVALID_ARG;
    if (n_diffuse < 0 || n_spec < 0 || n_diffuse + n_spec <= 0 || n_diffuse + n_spec > (1 << 24))
        return IRGS_ERR_INVALID_ARG;
    if ((params->flags & IRGS_FLAG_UNIFORM) && n_spec != 0) return IRGS_ERR_INVALID_ARG;
    if (env_h <= 0 || env_w <= 0 || !env) return IRGS_ERR_INVALID_ARG;
    if (n_points >= (int64_t)UINT32_MAX * 4) return IRGS_ERR_INVALID_ARG;
    return IRGS_OK;
}

// FP32 pipe probe: eight independent FMA chains per thread, 16 steps per
// loop pass (256 flops per thread per pass). The final sum is stored only if
// it equals a value it never reaches, which keeps the chains live.
__device__ float g_fma_sink;

__global__ void __launch_bounds__(256) k_fma_probe(float b, float c, int64_t iters) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1.0f + 1e-3f * k + 1e-7f * threadIdx.x;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == -12345.0f) g_fma_sink = s;
}

}  // namespace

extern "C" {

irgs_status irgs_probe_fma(int64_t iters, void* stream, double* flops) {
    if (iters <= 0 || iters > ((int64_t)1 << 40)) return IRGS_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return IRGS_ERR_CUDA;
    }
    const int blocks = sms * 8, threads = 256;
    k_fma_probe<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(0.9999999f, 1e-7f, iters);
    irgs::count_launches(1);
    if (cudaGetLastError() != cudaSuccess) return IRGS_ERR_CUDA;
    if (flops) *flops = (double)blocks * threads * (double)iters * 256.0;
    return IRGS_OK;
}

const char* irgs_status_string(irgs_status s) {
    switch (s) {
        case IRGS_OK: return "ok";
        case IRGS_ERR_INVALID_ARG: return "invalid argument";
        case IRGS_ERR_OOM: return "out of device memory";
        case IRGS_ERR_CUDA: return "CUDA error";
        case IRGS_ERR_NONFINITE: return "non-finite input";
        case IRGS_ERR_TIMEOUT: return "device wait timed out";
        case IRGS_ERR_UNSUPPORTED: return "unsupported configuration";
        case IRGS_ERR_DEVICE: return "device-side error recorded";
    }
    return "unknown status";
}

int32_t irgs_abi_version(void) { return IRGS_ABI_VERSION; }

uint64_t irgs_kernel_launches(void) { return irgs::g_launches.load(std::memory_order_relaxed); }

irgs_status irgs_build_scene(const irgs_surfels* s, float alpha_min, void* stream, irgs_scene* out) {
    return irgs_build_scene_ex(s, alpha_min, 0u, stream, out);
}

irgs_status irgs_build_scene_ex(const irgs_surfels* s, float alpha_min, uint32_t build_flags, void* stream,
                                irgs_scene* out) {
    if (s == nullptr || out == nullptr) return IRGS_ERR_INVALID_ARG;
    if ((build_flags & ~IRGS_BUILD_RADIX_TREE) != 0u) return IRGS_ERR_INVALID_ARG;
    if (s->n < 0 || s->n >= INT32_MAX) return IRGS_ERR_INVALID_ARG;
    if (s->num_features < 0 || s->num_features > 64) return IRGS_ERR_INVALID_ARG;
    if (!finite(alpha_min) || !(alpha_min > 0.f) || !(alpha_min < 1.f)) return IRGS_ERR_INVALID_ARG;
    if (s->n > 0 && (!s->means || !s->quats || !s->scales || !s->opacity)) return IRGS_ERR_INVALID_ARG;
    if (s->n > 0 && s->num_features > 0 && !s->features) return IRGS_ERR_INVALID_ARG;
    if (s->num_features == 0 && s->features) return IRGS_ERR_INVALID_ARG;
    cudaPointerAttributes at;
    if (s->n > 0) {
        if (cudaPointerGetAttributes(&at, s->means) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return IRGS_ERR_INVALID_ARG;
        }
    }
    irgs::DeviceGuard dg;
    if (s->n > 0 && !dg.set(at.device)) return IRGS_ERR_CUDA;
    return irgs::build_scene_impl(s, alpha_min, build_flags, static_cast<cudaStream_t>(stream), out);
}

irgs_status irgs_update_scene(irgs_scene sc, const irgs_surfels* s, void* stream) {
    if (sc == nullptr || s == nullptr) return IRGS_ERR_INVALID_ARG;
    if (s->n != sc->n || s->num_features != sc->F) return IRGS_ERR_INVALID_ARG;
    if (s->n > 0 && (!s->means || !s->quats || !s->scales || !s->opacity)) return IRGS_ERR_INVALID_ARG;
    if (s->n > 0 && s->num_features > 0 && !s->features) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    irgs_status st = use_device(dg, sc);
    if (st != IRGS_OK) return st;
    return irgs::update_scene_impl(sc, s, static_cast<cudaStream_t>(stream));
}

irgs_status irgs_refit_scene(irgs_scene sc, const irgs_surfels* s, void* stream) {
    if (sc == nullptr || s == nullptr) return IRGS_ERR_INVALID_ARG;
    if (s->n != sc->n || s->num_features != sc->F) return IRGS_ERR_INVALID_ARG;
    if (s->n > 0 && (!s->means || !s->quats || !s->scales || !s->opacity)) return IRGS_ERR_INVALID_ARG;
    if (s->n > 0 && s->num_features > 0 && !s->features) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    irgs_status st = use_device(dg, sc);
    if (st != IRGS_OK) return st;
    return irgs::refit_scene_impl(sc, s, static_cast<cudaStream_t>(stream));
}

irgs_status irgs_destroy_scene(irgs_scene sc) {
    if (sc == nullptr) return IRGS_OK;
    irgs::DeviceGuard dg;
    dg.set(sc->device);
    cudaDeviceSynchronize();
    irgs::free_scene(sc);
    return IRGS_OK;
}

irgs_status irgs_scene_info(irgs_scene sc, int64_t* n, int32_t* F, float* alpha_min, int64_t* bytes) {
    if (sc == nullptr) return IRGS_ERR_INVALID_ARG;
    if (n) *n = sc->n;
    if (F) *F = sc->F;
    if (alpha_min) *alpha_min = sc->alpha_min;
    if (bytes) *bytes = sc->bytes;
    return IRGS_OK;
}

irgs_status irgs_scene_status(irgs_scene sc, void* stream, uint32_t* bits) {
    if (sc == nullptr) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if (use_device(dg, sc) != IRGS_OK) return IRGS_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t h = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess) return IRGS_ERR_CUDA;
    if (cudaMemcpy(&h, sc->status, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return IRGS_ERR_CUDA;
    if (cudaMemset(sc->status, 0, sizeof(uint32_t)) != cudaSuccess) return IRGS_ERR_CUDA;
    if (bits) *bits = h;
    return h == 0u ? IRGS_OK : IRGS_ERR_DEVICE;
}

irgs_status irgs_scene_export(irgs_scene sc, int32_t* perm, uint32_t* keys, float* nodes, float* leaf_boxes) {
    if (sc == nullptr) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if (use_device(dg, sc) != IRGS_OK) return IRGS_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return IRGS_ERR_CUDA;
    const int64_t n = sc->n, nn = n > 1 ? n - 1 : 1;
    cudaError_t e = cudaSuccess;
    if (perm && n > 0) e = cudaMemcpy(perm, sc->perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && keys && n > 0) e = cudaMemcpy(keys, sc->keys, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && nodes) e = cudaMemcpy(nodes, sc->nodes, sizeof(irgs::Node) * nn, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && leaf_boxes && n > 0)
        e = cudaMemcpy(leaf_boxes, sc->leaf_box, sizeof(float) * 6 * n, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

irgs_status irgs_scene_export_wide(irgs_scene sc, float* nodes, int64_t cap, int64_t* n_wide) {
    if (sc == nullptr || cap < 0) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if (use_device(dg, sc) != IRGS_OK) return IRGS_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return IRGS_ERR_CUDA;
    int64_t nw = 1;
    if (sc->n > 1) {
        uint32_t allocated = 0;   // wide nodes the collapse allocated
        if (cudaMemcpy(&allocated, sc->wide_counters + 3, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return IRGS_ERR_CUDA;
        nw = (int64_t)allocated < sc->max_wide ? (int64_t)allocated : sc->max_wide;
    }
    if (n_wide) *n_wide = nw;
    const int64_t m = nw < cap ? nw : cap;
    if (nodes && m > 0 &&
        cudaMemcpy(nodes, sc->wide, sizeof(irgs::WideNode) * m, cudaMemcpyDeviceToHost) != cudaSuccess)
        return IRGS_ERR_CUDA;
    return IRGS_OK;
}

irgs_status irgs_trace_forward(irgs_scene sc, const float* ray_o, const float* ray_d, int64_t n_rays,
                               const irgs_trace_params* params, float* out_feat, float* out_depth,
                               float* out_opacity, int32_t* out_nhits, int32_t* out_hit_ids, int32_t max_hit_ids,
                               void* stream) {
    if (sc == nullptr || n_rays < 0) return IRGS_ERR_INVALID_ARG;
    irgs_status s = check_params(sc, params);
    if (s != IRGS_OK) return s;
    if (n_rays > 0 && (!ray_o || !ray_d || !out_depth || !out_opacity)) return IRGS_ERR_INVALID_ARG;
    if (n_rays > 0 && params->feat_count > 0 && !out_feat) return IRGS_ERR_INVALID_ARG;
    if (out_hit_ids && max_hit_ids <= 0) return IRGS_ERR_INVALID_ARG;
    if (n_rays >= (int64_t)UINT32_MAX * 128) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if ((s = use_device(dg, sc)) != IRGS_OK) return s;
    return irgs::launch_trace_forward(sc->view(), ray_o, ray_d, n_rays, *params, out_feat, out_depth, out_opacity,
                                      out_nhits, out_hit_ids, out_hit_ids ? max_hit_ids : 0,
                                      static_cast<cudaStream_t>(stream));
}

irgs_status irgs_trace_stats(irgs_scene sc, const float* ray_o, const float* ray_d, int64_t n_rays,
                             const irgs_trace_params* params, int32_t* out_stats, void* stream) {
    if (sc == nullptr || n_rays < 0) return IRGS_ERR_INVALID_ARG;
    irgs_status s = check_params(sc, params);
    if (s != IRGS_OK) return s;
    if (params->k != 16 || params->feat_count > 10) return IRGS_ERR_UNSUPPORTED;
    if (n_rays > 0 && (!ray_o || !ray_d || !out_stats)) return IRGS_ERR_INVALID_ARG;
    if (n_rays >= (int64_t)UINT32_MAX * 128) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if ((s = use_device(dg, sc)) != IRGS_OK) return s;
    return irgs::launch_trace_stats(sc->view(), ray_o, ray_d, n_rays, *params, out_stats,
                                    static_cast<cudaStream_t>(stream));
}

irgs_status irgs_trace_backward(irgs_scene sc, const float* ray_o, const float* ray_d, int64_t n_rays,
                                const irgs_trace_params* params, const float* out_feat, const float* out_depth,
                                const float* out_opacity, const int32_t* out_nhits, const int32_t* hit_ids,
                                int32_t max_hit_ids, const float* g_feat, const float* g_depth,
                                const float* g_opacity, float* g_means, float* g_quats, float* g_scales,
                                float* g_opacity_param, float* g_features, void* stream) {
    if (sc == nullptr || n_rays < 0) return IRGS_ERR_INVALID_ARG;
    irgs_status s = check_params(sc, params);
    if (s != IRGS_OK) return s;
    if (params->k != 8 && params->k != 16) return IRGS_ERR_UNSUPPORTED;
    if (n_rays > 0 && (!ray_o || !ray_d || !out_depth || !out_opacity || !out_nhits)) return IRGS_ERR_INVALID_ARG;
    if (n_rays > 0 && params->feat_count > 0 && (!out_feat || !g_feat)) return IRGS_ERR_INVALID_ARG;
    if (sc->n > 0 && (!g_means || !g_quats || !g_scales || !g_opacity_param)) return IRGS_ERR_INVALID_ARG;
    if (sc->n > 0 && sc->F > 0 && params->feat_count > 0 && !g_features) return IRGS_ERR_INVALID_ARG;
    if (hit_ids != nullptr && max_hit_ids <= 0) return IRGS_ERR_INVALID_ARG;
    if (n_rays >= (int64_t)UINT32_MAX * 128) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if ((s = use_device(dg, sc)) != IRGS_OK) return s;
    return irgs::launch_trace_backward(sc->view(), sc->perm, ray_o, ray_d, n_rays, *params, out_feat, out_depth,
                                       out_opacity, out_nhits, hit_ids, max_hit_ids, g_feat, g_depth, g_opacity,
                                       g_means, g_quats, g_scales, g_opacity_param, g_features,
                                       static_cast<cudaStream_t>(stream));
}

irgs_status irgs_shade_mc(irgs_scene sc, const float* x, const float* n, const float* albedo, const float* rough,
                          const float* wo, int64_t n_points, const float* env, int32_t env_h, int32_t env_w,
                          int32_t n_diffuse, int32_t n_spec, uint64_t seed, const irgs_trace_params* params,
                          float* out_rgb, float* out_vis, float* out_ind, void* stream) {
    irgs_status s = check_shade(sc, params, n_points, env, env_h, env_w, n_diffuse, n_spec);
    if (s != IRGS_OK) return s;
    if (n_points > 0 && (!x || !n || !albedo || !rough || !wo || !out_rgb)) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if ((s = use_device(dg, sc)) != IRGS_OK) return s;
    if (fused_shading(params))
        return irgs::launch_shade_mc(sc->view(), x, n, albedo, rough, wo, n_points, env, env_h, env_w, n_diffuse,
                                     n_spec, seed, *params, out_rgb, out_vis, out_ind,
                                     static_cast<cudaStream_t>(stream));
    return irgs::launch_shade_wave(sc->view(), sc->bounds, x, n, albedo, rough, wo, n_points, env, env_h, env_w,
                                   n_diffuse, n_spec, seed, shade_mode(params), *params, out_rgb, out_vis, out_ind,
                                   static_cast<cudaStream_t>(stream));
}

irgs_status irgs_shade_mc_backward(irgs_scene sc, const float* x, const float* n, const float* albedo,
                                   const float* rough, const float* wo, int64_t n_points, const float* env,
                                   int32_t env_h, int32_t env_w, int32_t n_diffuse, int32_t n_spec, uint64_t seed,
                                   const irgs_trace_params* params, const float* g_rgb, float* g_albedo,
                                   float* g_rough, float* g_env, float* g_means, float* g_quats, float* g_scales,
                                   float* g_opacity, float* g_features, void* stream) {
    irgs_status s = check_shade(sc, params, n_points, env, env_h, env_w, n_diffuse, n_spec);
    if (s != IRGS_OK) return s;
    if (n_points > 0 && (!x || !n || !albedo || !rough || !wo || !g_rgb || !g_albedo || !g_rough))
        return IRGS_ERR_INVALID_ARG;
    if (sc->n > 0 && (!g_means || !g_quats || !g_scales || !g_opacity || !g_features)) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if ((s = use_device(dg, sc)) != IRGS_OK) return s;
    if (fused_shading(params))
        return irgs::launch_shade_mc_backward(sc->view(), sc->perm, x, n, albedo, rough, wo, n_points, env, env_h,
                                              env_w, n_diffuse, n_spec, seed, *params, g_rgb, g_albedo, g_rough,
                                              g_env, g_means, g_quats, g_scales, g_opacity, g_features,
                                              static_cast<cudaStream_t>(stream));
    return irgs::launch_shade_wave_backward(sc->view(), sc->perm, sc->bounds, x, n, albedo, rough, wo, n_points, env,
                                            env_h, env_w, n_diffuse, n_spec, seed, shade_mode(params), *params,
                                            g_rgb, g_albedo, g_rough, g_env, g_means, g_quats, g_scales, g_opacity,
                                            g_features, static_cast<cudaStream_t>(stream));
}

irgs_status irgs_shade_sample_rays(const float* n, const float* rough, const float* wo, int64_t n_points,
                                  int32_t n_diffuse, int32_t n_spec, uint64_t seed, uint32_t flags, float* out_dir,
                                  int32_t* out_valid, void* stream) {
    if (n_points < 0 || n_diffuse < 0 || n_spec < 0 || n_diffuse + n_spec <= 0 || n_diffuse + n_spec > (1 << 24))
        return IRGS_ERR_INVALID_ARG;
    if ((flags & ~IRGS_FLAG_UNIFORM) != 0u || ((flags & IRGS_FLAG_UNIFORM) && n_spec != 0))
        return IRGS_ERR_INVALID_ARG;
    if (n_points > 0 && (!n || !rough || !wo || !out_dir)) return IRGS_ERR_INVALID_ARG;
    if (n_points >= (int64_t)UINT32_MAX * 4) return IRGS_ERR_INVALID_ARG;
    return irgs::launch_sample_rays(n, rough, wo, n_points, n_diffuse, n_spec, seed, (flags & IRGS_FLAG_UNIFORM) ? 1 : 0,
                                    out_dir, out_valid, static_cast<cudaStream_t>(stream));
}

irgs_status irgs_rasterize(irgs_scene sc, const irgs_camera* cam, const irgs_trace_params* params, float* out_feat,
                           float* out_depth, float* out_opacity, int32_t* out_nhits, void* stream) {
    if (sc == nullptr || cam == nullptr) return IRGS_ERR_INVALID_ARG;
    irgs_status s = check_params(sc, params);
    if (s != IRGS_OK) return s;
    if (params->flags != 0u || params->feat_count > 16) return IRGS_ERR_UNSUPPORTED;
    if (cam->width <= 0 || cam->height <= 0 || !(cam->tan_half_fov > 0.f)) return IRGS_ERR_INVALID_ARG;
    if ((int64_t)cam->width * cam->height > ((int64_t)1 << 31) - 1) return IRGS_ERR_INVALID_ARG;
    if (!out_depth || !out_opacity || (params->feat_count > 0 && !out_feat)) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if ((s = use_device(dg, sc)) != IRGS_OK) return s;
    return irgs::launch_rasterize(sc->view(), sc->leaf_box, *cam, *params, out_feat, out_depth, out_opacity,
                                  out_nhits, static_cast<cudaStream_t>(stream));
}

irgs_status irgs_envmap_create(const float* env, int32_t H, int32_t W, void* stream, irgs_envmap* out) {
    if (env == nullptr || out == nullptr || H <= 0 || W <= 0) return IRGS_ERR_INVALID_ARG;
    if ((int64_t)H * W > (int64_t)1 << 26) return IRGS_ERR_INVALID_ARG;
    return irgs::build_envmap_impl(env, H, W, static_cast<cudaStream_t>(stream), out);
}

irgs_status irgs_envmap_destroy(irgs_envmap m) {
    if (m == nullptr) return IRGS_OK;
    irgs::DeviceGuard dg;
    dg.set(m->device);
    cudaDeviceSynchronize();
    irgs::free_envmap(m);
    return IRGS_OK;
}

irgs_status irgs_envmap_export(irgs_envmap m, float* irr, float* pref, float* lut, double* row_cdf,
                               double* col_cdf, void* stream) {
    if (m == nullptr) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if (!dg.set(m->device)) return IRGS_ERR_CUDA;
    return irgs::export_envmap_impl(m, irr, pref, lut, row_cdf, col_cdf, static_cast<cudaStream_t>(stream));
}

irgs_status irgs_relight(irgs_scene sc, irgs_envmap m, const float* x, const float* n, const float* albedo,
                         const float* rough, const float* wo, int64_t n_points, int32_t n_samples, uint64_t seed,
                         const irgs_trace_params* params, float* out_rgb, float* out_vis, float* out_ind,
                         void* stream) {
    if (sc == nullptr || m == nullptr || n_points < 0) return IRGS_ERR_INVALID_ARG;
    irgs_status s = check_params(sc, params);
    if (s != IRGS_OK) return s;
    if (params->k != 8 && params->k != 16) return IRGS_ERR_UNSUPPORTED;
    if (params->feat_count != 7 || !(params->t_min > 0.f)) return IRGS_ERR_INVALID_ARG;
    if (n_samples <= 0 || n_samples > (1 << 24)) return IRGS_ERR_INVALID_ARG;
    if (m->device != sc->device) return IRGS_ERR_INVALID_ARG;
    if (n_points > 0 && (!x || !n || !albedo || !rough || !wo || !out_rgb)) return IRGS_ERR_INVALID_ARG;
    if (n_points >= (int64_t)UINT32_MAX * 4) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if ((s = use_device(dg, sc)) != IRGS_OK) return s;
    return irgs::launch_relight(sc->view(), sc->bounds, m, x, n, albedo, rough, wo, n_points, n_samples, seed,
                                *params, out_rgb, out_vis, out_ind, static_cast<cudaStream_t>(stream));
}

irgs_status irgs_relight_sample_rays(irgs_envmap m, int64_t n_points, int32_t n_samples, uint64_t seed,
                                    float* out_dir, float* out_pdf, int32_t* out_valid, void* stream) {
    if (m == nullptr || n_points < 0 || n_samples <= 0 || n_samples > (1 << 24)) return IRGS_ERR_INVALID_ARG;
    if (n_points > 0 && !out_dir) return IRGS_ERR_INVALID_ARG;
    if (n_points >= (int64_t)UINT32_MAX * 4) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if (!dg.set(m->device)) return IRGS_ERR_CUDA;
    return irgs::launch_relight_rays(m, n_points, n_samples, seed, out_dir, out_pdf, out_valid,
                                     static_cast<cudaStream_t>(stream));
}

irgs_status irgs_build_lbvh_noalloc(const irgs_surfels* s, float alpha_min, int32_t* perm, uint32_t* keys,
                                    float* nodes, float* leaf_boxes, void* stream) {
    if (s == nullptr) return IRGS_ERR_INVALID_ARG;
    if (s->n < 0 || s->n > IRGS_NOALLOC_MAX_SURFELS) return IRGS_ERR_INVALID_ARG;
    if (!finite(alpha_min) || !(alpha_min > 0.f) || !(alpha_min < 1.f)) return IRGS_ERR_INVALID_ARG;
    if (!nodes) return IRGS_ERR_INVALID_ARG;
    if (s->n > 0 && (!s->means || !s->quats || !s->scales || !s->opacity || !perm || !keys || !leaf_boxes))
        return IRGS_ERR_INVALID_ARG;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, nodes) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return IRGS_ERR_INVALID_ARG;
    }
    irgs::DeviceGuard dg;
    if (!dg.set(at.device)) return IRGS_ERR_CUDA;
    return irgs::build_lbvh_noalloc_impl(s, alpha_min, perm, keys, nodes, leaf_boxes,
                                         static_cast<cudaStream_t>(stream));
}

irgs_status irgs_build_lbvh_noalloc_status(int32_t device, void* stream, uint32_t* bits) {
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return IRGS_ERR_CUDA;
    }
    if (device < 0 || device >= count) return IRGS_ERR_INVALID_ARG;
    irgs::DeviceGuard dg;
    if (!dg.set(device)) return IRGS_ERR_CUDA;
    return irgs::lbvh_noalloc_status_impl(static_cast<cudaStream_t>(stream), bits);
}

}  // extern "C"
