// Host-side scene object and the internal launchers each translation unit
// provides. Not part of the public ABI (see include/irgs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

struct irgs_scene_s {
    int device = 0;
    int64_t n = 0;
    int32_t F = 0;
    float alpha_min = 0.f;
    uint32_t build_flags = 0;         // IRGS_BUILD_* of the hierarchy
    int64_t bytes = 0;

    // persistent scene data (Morton order)
    irgs::Node* nodes = nullptr;      // [max(n-1,1)]
    float4* rec = nullptr;            // [n*4]
    float* feat = nullptr;            // [n*F]
    float4* q_raw = nullptr;          // [n]
    float2* scale = nullptr;          // [n]
    float* leaf_box = nullptr;        // [n*6]
    uint32_t* keys = nullptr;         // [n] sorted Morton codes
    int32_t* perm = nullptr;          // [n] user index of Morton slot
    int32_t* inv_perm = nullptr;      // [n] Morton slot of user index
    uint32_t* status = nullptr;       // device error word
    irgs::WideNode* wide = nullptr;   // [max_wide] 4-wide hierarchy
    int64_t max_wide = 0;
    int2* wide_frontier = nullptr;    // [2n] (binary node, wide index) frontiers of the collapse
    uint32_t* wide_counters = nullptr;// [4] rotating frontier sizes, wide nodes allocated

    // build scratch (kept for rebuilds); after the gather, rec_user, box_user,
    // keys_tmp, vals_tmp and hist serve as the clustering build's working memory
    float4* rec_user = nullptr;       // [n*4]
    float* box_user = nullptr;        // [n*6]
    uint32_t* keys_tmp = nullptr;     // [n]
    int32_t* vals_tmp = nullptr;      // [n]
    uint32_t* hist = nullptr;         // [256 * tiles]
    uint32_t* bounds = nullptr;       // [6] ordered-bit centroid bounds
    int32_t* leaf_parent = nullptr;   // [n]
    int32_t* node_parent = nullptr;   // [max(n-1,1)]
    uint32_t* refit_flag = nullptr;   // [max(n-1,1)]

    irgs::SceneView view() const {
        irgs::SceneView v;
        v.nodes = nodes;
        v.wide = wide;
        v.rec = rec;
        v.feat = feat;
        v.q_raw = q_raw;
        v.scale = scale;
        v.inv_perm = inv_perm;
        v.status = status;
        v.n = n;
        v.F = F;
        v.alpha_min = alpha_min;
        return v;
    }
};

// Pre-integrated maps of one environment for the relighting query.
struct irgs_envmap_s {
    int device = 0;
    int32_t H = 0, W = 0;
    int64_t bytes = 0;
    float* env = nullptr;       // [H, W, 3] copy
    float* irr = nullptr;       // [IRGS_RELIGHT_IRR_H, IRGS_RELIGHT_IRR_W, 3]
    float* pref = nullptr;      // [IRGS_RELIGHT_LEVELS - 1, IRGS_RELIGHT_PREF_H, IRGS_RELIGHT_PREF_W, 3]
    float* lut = nullptr;       // [IRGS_RELIGHT_LUT_N, IRGS_RELIGHT_LUT_N, 2]
    double* row_cdf = nullptr;  // [H + 1]
    double* col_cdf = nullptr;  // [H, W + 1]
};

namespace irgs {

// Restores the calling thread's current device when an entry point that
// switched to its scene's device returns (a C library call must not change
// which device the caller's later CUDA calls go to).
class DeviceGuard {
  public:
    DeviceGuard() {
        if (cudaGetDevice(&prev_) != cudaSuccess) {
            cudaGetLastError();
            prev_ = -1;
        }
    }
    ~DeviceGuard() {
        if (switched_ && prev_ >= 0) cudaSetDevice(prev_);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
    bool set(int device) {
        if (device == prev_) return true;
        switched_ = true;
        return cudaSetDevice(device) == cudaSuccess;
    }

  private:
    int prev_ = -1;
    bool switched_ = false;
};

// raster.cu
irgs_status launch_rasterize(const SceneView& sv, const float* leaf_box, const irgs_camera& cam,
                             const irgs_trace_params& p, float* feat, float* depth, float* opac, int32_t* nhits,
                             cudaStream_t st);

// relight.cu
irgs_status build_envmap_impl(const float* env, int32_t H, int32_t W, cudaStream_t st, irgs_envmap* out);
void free_envmap(irgs_envmap m);
irgs_status export_envmap_impl(irgs_envmap m, float* irr, float* pref, float* lut, double* row_cdf,
                               double* col_cdf, cudaStream_t st);
irgs_status launch_sample_rays(const float* n, const float* rough, const float* wo, int64_t P, int32_t nd,
                               int32_t ns, uint64_t seed, int mode, float* dir, int32_t* valid, cudaStream_t st);
irgs_status launch_relight_rays(irgs_envmap m, int64_t P, int32_t n_samples, uint64_t seed, float* dir, float* pdf,
                                int32_t* valid, cudaStream_t st);
irgs_status launch_relight(const SceneView& sv, const uint32_t* bounds, irgs_envmap m, const float* x,
                           const float* n, const float* albedo, const float* rough, const float* wo, int64_t P,
                           int32_t n_samples, uint64_t seed, const irgs_trace_params& p, float* rgb, float* vis,
                           float* ind, cudaStream_t st);

// scene.cu
irgs_status build_scene_impl(const irgs_surfels* s, float alpha_min, uint32_t build_flags, cudaStream_t st,
                             irgs_scene* out);
irgs_status update_scene_impl(irgs_scene sc, const irgs_surfels* s, cudaStream_t st);
irgs_status refit_scene_impl(irgs_scene sc, const irgs_surfels* s, cudaStream_t st);
irgs_status build_lbvh_noalloc_impl(const irgs_surfels* s, float alpha_min, int32_t* perm, uint32_t* keys,
                                    float* nodes, float* leaf_boxes, cudaStream_t st);
irgs_status lbvh_noalloc_status_impl(cudaStream_t st, uint32_t* bits);
void free_scene(irgs_scene sc);
// Stable LSD radix sort of (keys, vals) pairs by the low key_bits bits of
// the keys (8-bit passes, rounded up to an even count; the result ends in
// keys/vals). keys_tmp/vals_tmp hold n entries, hist sort_hist_words(n) words.
int64_t sort_hist_words(int64_t n);
cudaError_t sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys_tmp, int32_t* vals_tmp, uint32_t* hist,
                       int64_t n, cudaStream_t st, int key_bits = 32);
// In-place exclusive prefix sum of m words (one block; for up to a few million).
cudaError_t scan_exclusive(uint32_t* a, int64_t m, cudaStream_t st);
// In-place exclusive prefix sum of m words by tiles (any m); sums holds
// scan_long_words(m) words of scratch.
int64_t scan_long_words(int64_t m);
cudaError_t scan_exclusive_long(uint32_t* a, int64_t m, uint32_t* sums, cudaStream_t st);
// The flagged indices of flags[0..m) (0/1 words; flags[m] must be 0) in
// order: list[0..count) and *count (device). flags is overwritten by its
// prefix sums; sums holds scan_long_words(m + 1) words.
cudaError_t flags_to_list(uint32_t* flags, int64_t m, uint32_t* sums, int32_t* list, uint32_t* count,
                          cudaStream_t st);

// trace_fwd.cu
irgs_status launch_trace_forward(const SceneView& sv, const float* ro, const float* rd, int64_t R,
                                 const irgs_trace_params& p, float* feat, float* depth, float* opac,
                                 int32_t* nhits, int32_t* ids, int32_t max_ids, cudaStream_t st);
irgs_status launch_trace_stats(const SceneView& S, const float* ro, const float* rd, int64_t R,
                               const irgs_trace_params& p, int32_t* stats, cudaStream_t st);
// trace_bwd.cu
irgs_status launch_trace_backward(const SceneView& sv, const int32_t* perm, const float* ro, const float* rd, int64_t R,
                                  const irgs_trace_params& p, const float* feat, const float* depth,
                                  const float* opac, const int32_t* nhits, const int32_t* hit_ids,
                                  int32_t max_hit_ids, const float* g_feat,
                                  const float* g_depth, const float* g_opac, float* g_means,
                                  float* g_quats, float* g_scales, float* g_opacity, float* g_features,
                                  cudaStream_t st);
// shade.cu
irgs_status launch_shade_mc(const SceneView& sv, const float* x, const float* n, const float* albedo,
                            const float* rough, const float* wo, int64_t P, const float* env, int32_t H,
                            int32_t W, int32_t n_diffuse, int32_t n_spec, uint64_t seed,
                            const irgs_trace_params& p, float* rgb, float* vis, float* ind,
                            cudaStream_t st);
// shade_wave.cu: the same estimates and gradients with the secondary rays
// regrouped by direction and origin (bounds: the scene's ordered-bit centre
// bounds)
irgs_status launch_shade_wave(const SceneView& sv, const uint32_t* bounds, const float* x, const float* n,
                              const float* albedo, const float* rough, const float* wo, int64_t P, const float* env,
                              int32_t H, int32_t W, int32_t n_diffuse, int32_t n_spec, uint64_t seed, int mode,
                              const irgs_trace_params& p, float* rgb, float* vis, float* ind, cudaStream_t st,
                              uint64_t key_base = 0, const float* valid = nullptr);
irgs_status launch_shade_wave_backward(const SceneView& sv, const int32_t* perm, const uint32_t* bounds,
                                       const float* x, const float* n, const float* albedo, const float* rough,
                                       const float* wo, int64_t P, const float* env, int32_t H, int32_t W,
                                       int32_t n_diffuse, int32_t n_spec, uint64_t seed, int mode,
                                       const irgs_trace_params& p, const float* g_rgb, float* g_albedo,
                                       float* g_rough, float* g_env, float* g_means, float* g_quats, float* g_scales,
                                       float* g_opacity, float* g_features, cudaStream_t st);
irgs_status launch_shade_mc_backward(const SceneView& sv, const int32_t* perm, const float* x, const float* n,
                                     const float* albedo, const float* rough, const float* wo, int64_t P,
                                     const float* env, int32_t H, int32_t W, int32_t n_diffuse, int32_t n_spec,
                                     uint64_t seed, const irgs_trace_params& p, const float* g_rgb,
                                     float* g_albedo, float* g_rough, float* g_env, float* g_means, float* g_quats,
                                     float* g_scales, float* g_opacity, float* g_features, cudaStream_t st);

// k-buffer sizes that are compiled in
inline bool k_supported(int k) { return k == 1 || k == 4 || k == 8 || k == 16 || k == 32; }

}  // namespace irgs
