/*
 * irgs.h -- C ABI of the GB300 2D Gaussian ray tracer (libirgs.so).
 *
 * Differentiable ray tracing of 2D Gaussian surfels as defined by IRGS
 * (Gu et al., "IRGS: Inter-Reflective Gaussian Splatting with 2D Gaussian Ray
 * Tracing", CVPR 2025, arXiv 2412.15867): the ray-splat intersection of
 * Eq. 6, the surfel response of Eq. 7, front-to-back alpha blending (Eq. 2)
 * into Trace(r_o, r_d) of Eq. 8, its gradient (the tracer is differentiable,
 * Sec. 3.3, so indirect radiance can be optimised), and the Monte Carlo rendering
 * equation of Eq. 15 with the light split of Eq. 13-14.
 *
 * Conventions shared by every entry point
 *  - Array arguments are DEVICE pointers to C-contiguous float32 / int32 data
 *    owned by the caller. The library never frees them and never keeps them
 *    after the call returns (the scene keeps its own copies).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). All work is
 *    enqueued asynchronously on it; a call returns once the work is queued.
 *  - The return status covers argument validation and launch errors. Errors
 *    that kernels detect (traversal stack overflow) are recorded in the
 *    scene's status word and reported by irgs_scene_status().
 *  - Per-call scratch is stream-ordered: taken from the library's own
 *    memory pool on the current device and freed on the call's stream. The
 *    pool keeps up to 32 GiB of freed scratch for later calls instead of
 *    returning it to the driver; it is released when the process ends.
 *  - No entry point exits or aborts the process. Build/destroy of one scene
 *    must not race with other calls on that scene; concurrent traces of one
 *    scene are safe (they only read it).
 *  - Quaternions are (w, x, y, z) and need not be normalised; the rotation
 *    columns are the tangents t_u, t_v and the normal n = t_u x t_v (Sec. 3.2).
 *    Scales (s_u, s_v) > 0 and opacities in [0, 1] are activated values.
 */
#ifndef IRGS_H
#define IRGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IRGS_ABI_VERSION 3
#define IRGS_MAX_FEATURES 16   /* blended channels per trace call */

typedef enum {
    IRGS_OK = 0,
    IRGS_ERR_INVALID_ARG = 1,   /* a pointer, size or parameter is invalid       */
    IRGS_ERR_OOM = 2,           /* device memory allocation failed               */
    IRGS_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed          */
    IRGS_ERR_NONFINITE = 4,     /* reserved: non-finite input detected           */
    IRGS_ERR_TIMEOUT = 5,       /* reserved: a bounded device wait gave up       */
    IRGS_ERR_UNSUPPORTED = 6,   /* e.g. a k-buffer size that is not compiled in  */
    IRGS_ERR_DEVICE = 7         /* a kernel recorded an error (stack overflow)   */
} irgs_status;

/* Opaque scene: owns a Morton-ordered packed copy of the surfels, their
 * features, and a linear BVH over the surfels' support-disk bounding boxes. */
typedef struct irgs_scene_s* irgs_scene;

/* Surfel cloud in user order (device pointers, float32, C-contiguous). */
typedef struct {
    const float* means;       /* [n, 3] centres mu                                */
    const float* quats;       /* [n, 4] rotation quaternions (w, x, y, z)          */
    const float* scales;      /* [n, 2] (s_u, s_v) > 0                             */
    const float* opacity;     /* [n] opacity o in [0, 1]                          */
    const float* features;    /* [n, num_features], NULL iff num_features == 0     */
    int64_t n;                /* number of surfels, 0 <= n < 2^31 - 1              */
    int32_t num_features;     /* channels per surfel, 0 .. 64                      */
} irgs_surfels;

/* Parameters of one trace (Eq. 2, 6-8 and the termination rule of Sec. 4). */
typedef struct {
    int32_t k;            /* k-buffer size: 1, 4, 8, 16 or 32 (8 and 16 everywhere) */
    float alpha_min;      /* hits need alpha >= alpha_min; >= the scene's value     */
    float alpha_max;      /* alpha = min(alpha_max, o exp(-rho^2/2)), <= 1          */
    float T_min;          /* stop after the hit that makes T < T_min, in [0, 1)     */
    float t_min;          /* hits need tau > t_min (>= 0)                           */
    float t_max;          /* hits need tau < t_max (may be +inf)                    */
    int32_t feat_offset;  /* first blended feature channel                          */
    int32_t feat_count;   /* blended channels, 0 .. IRGS_MAX_FEATURES               */
    uint32_t flags;       /* IRGS_FLAG_* bits, 0 for the defaults                   */
} irgs_trace_params;

/* Traversal policy (results are identical either way, only speed differs).
 * Default for irgs_trace_forward / irgs_trace_backward: warp-coherent -- the
 * 32 rays of a warp walk one shared stack, best for coherent batches such as
 * camera rays in image order. Default for irgs_shade_mc / _backward: the
 * secondary rays of all points are regrouped by direction and origin and
 * traced with one stack per ray. IRGS_FLAG_PER_THREAD forces an independent
 * stack per ray (for shading: the fused kernel, a warp per point tracing its
 * own samples); IRGS_FLAG_WARP forces the warp-coherent walk (for shading:
 * the fused kernel with a warp-shared stack). Setting both is invalid. */
#define IRGS_FLAG_PER_THREAD 1u
#define IRGS_FLAG_WARP 2u
/* Shading only (irgs_shade_mc / irgs_shade_mc_backward): the stratified
 * uniform hemisphere estimator of Eq. 15 instead of split-lobe importance
 * sampling; n_spec must be 0. Rejected by the trace entry points. */
#define IRGS_FLAG_UNIFORM 4u

/* Human-readable name of a status code (static storage). */
const char* irgs_status_string(irgs_status status);

/* Measurement probe (the paper has no counterpart): one launch of a kernel
 * that keeps the FP32 FMA pipes of every SM of the current device busy
 * (8 blocks of 256 threads per SM, eight independent FMA chains per thread,
 * `iters` passes of 16 dependent steps each). *flops receives the launch's
 * FP32 flop count (2 per FMA); the caller times the launch on `stream` and
 * divides, which gives the measured FP32 peak that bounds the intersection
 * arithmetic of Eq. 6-7. Enqueued on `stream`; allocates nothing. */
irgs_status irgs_probe_fma(int64_t iters, void* stream, double* flops);

/* IRGS_ABI_VERSION of the loaded library. */
int32_t irgs_abi_version(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (all devices and threads; a diagnostic for benchmarks). */
uint64_t irgs_kernel_launches(void);

/*
 * Build a scene from a surfel cloud (Sec. 3.2, bounding proxies and BVH;
 * Eq. 5 gives the support radius). Each surfel is bounded by the box of its
 * support disk rho <= rho_c, rho_c = min(3, sqrt(2 ln(o / alpha_min))),
 * where rho^2 = u^2 + v^2 of Eq. 7; surfels with o < alpha_min never hit.
 * The library copies the surfels into Morton order and builds the BVH on the
 * device, enqueued on `stream`: Morton codes, radix sort, a binary hierarchy
 * by locally-ordered clustering of the sorted leaf boxes (the Karras radix
 * tree instead when clustering would give a tree more than 60 levels high),
 * and its collapse into a 4-wide hierarchy for traversal.
 *   surfels   : device arrays, read during the call's stream work only.
 *   alpha_min : the smallest alpha cutoff later traces may use (> 0).
 *   out       : receives the new scene handle (caller owns it; free it with
 *               irgs_destroy_scene). Unchanged on error.
 * The scene allocates device memory (about 200 B per surfel plus features)
 * with cudaMalloc; IRGS_ERR_OOM if that fails.
 */
irgs_status irgs_build_scene(const irgs_surfels* surfels, float alpha_min, void* stream,
                             irgs_scene* out);

/*
 * irgs_build_scene with a choice of binary hierarchy (Sec. 3.2, the BVH over
 * the bounding proxies). build_flags = 0 is irgs_build_scene: locally-ordered
 * clustering of the sorted leaves, the radix tree only as its fallback.
 * IRGS_BUILD_RADIX_TREE builds the Karras (2012) radix tree over the sorted
 * Morton codes (equal codes split by index) and refits its boxes bottom-up:
 * faster to build, slower to trace. Traces give identical results on
 * either tree. The choice is kept for irgs_update_scene. Other bits of
 * build_flags: IRGS_ERR_INVALID_ARG; the rest as for irgs_build_scene.
 */
#define IRGS_BUILD_RADIX_TREE 1u
irgs_status irgs_build_scene_ex(const irgs_surfels* surfels, float alpha_min, uint32_t build_flags, void* stream,
                                irgs_scene* out);

/*
 * Rebuild an existing scene in place from new surfel values (same n and
 * num_features): the BVH update that a training loop runs every iteration
 * because the geometry changes (Sec. 4).
 * Reuses the scene's device buffers, allocates nothing, and is enqueued on
 * `stream`; traces already enqueued on other streams must finish first.
 * IRGS_ERR_INVALID_ARG if n or num_features differ from the scene's.
 */
irgs_status irgs_update_scene(irgs_scene scene, const irgs_surfels* surfels, void* stream);

/*
 * Refit an existing scene to new surfel values (same n and num_features)
 * without rebuilding it: records, boxes and features are recomputed in the
 * Morton order of the last build, and the boxes of its hierarchy are
 * refitted bottom-up (the per-iteration BVH update of Sec. 4 done as a
 * refit). Traces stay exact (every box bounds its subtree); only traversal
 * speed can degrade as surfels drift from the order the tree was built for,
 * so callers rebuild with irgs_update_scene now and then. Allocates nothing;
 * enqueued on `stream`. IRGS_ERR_INVALID_ARG if n or num_features differ.
 */
irgs_status irgs_refit_scene(irgs_scene scene, const irgs_surfels* surfels, void* stream);

/* Free a scene and all its device memory (synchronises the device first).
 * NULL is accepted and ignored. */
irgs_status irgs_destroy_scene(irgs_scene scene);

/* Scene facts: surfel count, feature channels, alpha_min and device bytes.
 * Any output pointer may be NULL. */
irgs_status irgs_scene_info(irgs_scene scene, int64_t* n, int32_t* num_features,
                            float* alpha_min, int64_t* device_bytes);

/* Synchronise `stream`, then read and clear the scene's device error word.
 * Returns IRGS_OK or IRGS_ERR_DEVICE; *bits (may be NULL) receives the raw
 * word (bit 0: a traversal stack overflowed and that ray's result is
 * incomplete; bit 1: the hierarchy failed a consistency bound; bit 2: a hit
 * list given to irgs_trace_backward held an index outside the scene, and
 * that ray's gradient is incomplete). */
irgs_status irgs_scene_status(irgs_scene scene, void* stream, uint32_t* bits);

/*
 * Copy the scene's structure to HOST buffers for inspection and tests
 * (synchronous). Any pointer may be NULL.
 *   perm      : [n] int32, user index of each Morton-ordered surfel.
 *   keys      : [n] uint32, sorted 30-bit Morton codes.
 *   nodes     : [max(n-1,1), 16] float32, internal nodes: child 0 box
 *               (lo xyz, hi xyz), child 1 box, then the two child ids as
 *               int32 bits (>= 0 internal node, < 0 leaf ~m, INT32_MIN none),
 *               then two unused words.
 *   leaf_boxes: [n, 6] float32, (lo xyz, hi xyz) of each Morton-ordered leaf.
 */
irgs_status irgs_scene_export(irgs_scene scene, int32_t* perm, uint32_t* keys, float* nodes,
                              float* leaf_boxes);

/*
 * Copy the 4-wide hierarchy the tracing kernels walk (root = node 0) to a
 * HOST buffer (synchronous). *n_wide receives the node count; nodes [cap,
 * 32] float32 receives min(cap, n_wide) nodes laid out as six float4 rows
 * lo.x lo.y lo.z hi.x hi.y hi.z (component k = child k), one int4 row of
 * child ids (>= 0 wide node, < 0 leaf ~m, INT32_MIN none) and one row whose
 * first int is the child count. Either pointer may be NULL.
 */
irgs_status irgs_scene_export_wide(irgs_scene scene, float* nodes, int64_t cap, int64_t* n_wide);

/*
 * Forward trace, Trace(r_o, r_d) of Eq. 8 for n_rays rays. For each ray
 * every surfel hit with t_min < tau < t_max is found (Eq. 6-7: tau =
 * n.(mu - o)/(n.d), u = (p - mu).t_u / s_u, v = (p - mu).t_v / s_v, alpha =
 * min(alpha_max, o exp(-(u^2+v^2)/2)), kept if rho <= rho_c and alpha >=
 * alpha_min, no hit if |n.d| < 1e-8 |d|), and hits are blended front to back
 * in (tau, index) order with a k-buffer (Eq. 2): w = T alpha, T *= 1 - alpha,
 * stopping after the hit that makes T < T_min.
 *   ray_o, ray_d  : [n_rays, 3] origins and directions (any non-zero length;
 *                   tau is in units of |d|).
 *   out_feat      : [n_rays, feat_count] sum of w f (Eq. 8/9, unnormalised).
 *   out_depth     : [n_rays] sum of w tau (Eq. 9, unnormalised).
 *   out_opacity   : [n_rays] 1 - T_final (o_rt of Eq. 8).
 *   out_nhits     : [n_rays] int32 blended hits, or NULL.
 *   out_hit_ids   : [n_rays, max_hit_ids] int32 user indices of the first
 *                   min(n_hits, max_hit_ids) blended hits in blend order,
 *                   followed by -1 if n_hits < max_hit_ids; later entries
 *                   are not written. NULL to skip. irgs_trace_backward can
 *                   take this list instead of replaying the traversal.
 * Outputs are overwritten. n_rays may be 0. With the warp-coherent walk,
 * k = 16 and at least 2^20 rays, rays still marching after each of the
 * first three k-buffer rounds are regrouped into full warps; that takes
 * 56 to 104 bytes per ray of scratch (72 at 4..10 channels), allocated and
 * freed stream-ordered (the library's scratch pool) on `stream`; if that allocation
 * fails the rays are marched without regrouping. Results are the same
 * either way.
 */
irgs_status irgs_trace_forward(irgs_scene scene, const float* ray_o, const float* ray_d,
                               int64_t n_rays, const irgs_trace_params* params,
                               float* out_feat, float* out_depth, float* out_opacity,
                               int32_t* out_nhits, int32_t* out_hit_ids, int32_t max_hit_ids,
                               void* stream);

/*
 * Diagnostic: the forward march of irgs_trace_forward (k = 16, feat_count
 * <= 10, same traversal policy flags) with per-ray counters instead of
 * outputs. out_stats [n_rays, 4] int32: k-buffer rounds, BVH nodes fetched
 * (in the warp-coherent walk: fetched by the warp while this ray was still
 * marching), surfel tests, k-buffer insertions.
 */
irgs_status irgs_trace_stats(irgs_scene scene, const float* ray_o, const float* ray_d, int64_t n_rays,
                             const irgs_trace_params* params, int32_t* out_stats, void* stream);

/*
 * Backward of irgs_trace_forward for the loss
 *   L = sum_r g_feat[r].feat[r] + g_depth[r] depth[r] + g_opacity[r] opacity[r].
 * Each ray's blended hits are taken from the forward's hit list when one is
 * given and holds them all (n_hits <= max_hit_ids), else found again by
 * replaying the k-buffer march; each hit is recomputed with the forward's
 * arithmetic. dL/d(parameter) is ADDED into the user-order gradient arrays
 * (the caller zeroes them first).
 *   out_feat, out_depth, out_opacity, out_nhits: the forward's outputs for
 *                   the same scene, rays and params (required).
 *   hit_ids, max_hit_ids: the out_hit_ids list of that forward call, or
 *                   NULL (then max_hit_ids is ignored); max_hit_ids > 0.
 *   g_feat [n_rays, feat_count], g_depth [n_rays], g_opacity [n_rays]:
 *                   upstream gradients; g_depth / g_opacity may be NULL (0).
 *   g_means [n,3], g_quats [n,4] (w.r.t. the raw, unnormalised quaternion),
 *   g_scales [n,2], g_opacity_param [n], g_features [n, num_features]
 *                   (only the traced channel range receives gradient).
 * The surfel gradient pointers must all be non-NULL.
 */
irgs_status irgs_trace_backward(irgs_scene scene, const float* ray_o, const float* ray_d,
                                int64_t n_rays, const irgs_trace_params* params,
                                const float* out_feat, const float* out_depth,
                                const float* out_opacity, const int32_t* out_nhits,
                                const int32_t* hit_ids, int32_t max_hit_ids,
                                const float* g_feat, const float* g_depth, const float* g_opacity,
                                float* g_means, float* g_quats, float* g_scales,
                                float* g_opacity_param, float* g_features, void* stream);

/*
 * Monte Carlo rendering equation at G-buffer points (Eq. 3, 15), with the
 * dielectric BRDF of Eq. 4 and incident light L_i = V L_dir + L_ind whose
 * (L_ind, 1 - V) come from tracing (x, w_i) (Eq. 13-14). D is GGX
 * (alpha_g = roughness^2), F is Schlick with F0 = 0.04 on (w_o.h), G is
 * separable Schlick-GGX with k = alpha_g / 2; the normal is flipped when
 * n.w_o <= 0. Two estimators:
 *  - default, split-lobe importance sampling (supplementary "Composited
 *    scene details"): n_diffuse cosine-weighted samples estimate the diffuse
 *    term (a L_i each) and n_spec GGX samples estimate the specular term
 *    (F G (w_o.h) L_i / ((n.w_o)(n.h)) each; a sample below the horizon adds
 *    0 but counts);
 *  - IRGS_FLAG_UNIFORM (n_spec = 0): S = n_diffuse directions uniform over
 *    the hemisphere, stratified in cos(theta) (sample s has cos(theta) =
 *    (s + u1) / S), estimate 2 pi / S sum (f_d + f_s) L_i (w_i.n) (Eq. 15).
 * Random numbers: SplitMix64 stream of `seed`, output index
 * (p * (n_diffuse + n_spec) + s) * 2 + dim, top 24 bits.
 *   x, n, albedo, wo : [n_points, 3]; rough : [n_points].
 *   env   : [env_h, env_w, 3] equirectangular radiance, z up, row = polar
 *           angle acos(z), column = azimuth atan2(y, x) from -pi; bilinear,
 *           wrapping in azimuth and clamping in polar angle.
 *   params: the secondary-ray trace; feat_count must be 3 (radiance c of the
 *           surfels, Sec. 3.3) and t_min > 0 is the self-hit offset.
 *   out_rgb [n_points, 3]; out_vis [n_points] and out_ind [n_points, 3]
 *           (means of V and L_ind over the cosine samples, or over all
 *           samples in the uniform mode) may be NULL.
 * Results do not depend on how points are batched into calls.
 */
irgs_status irgs_shade_mc(irgs_scene scene, const float* x, const float* n, const float* albedo,
                          const float* rough, const float* wo, int64_t n_points, const float* env,
                          int32_t env_h, int32_t env_w, int32_t n_diffuse, int32_t n_spec,
                          uint64_t seed, const irgs_trace_params* params, float* out_rgb,
                          float* out_vis, float* out_ind, void* stream);

/*
 * Gradient of irgs_shade_mc (same scene, points, sample counts, seed and
 * params) for the loss L = sum_p g_rgb[p].rgb[p], with the sample directions
 * held fixed (their dependence on roughness and on the normal is not
 * differentiated: the estimate of the gradient stays unbiased for the
 * roughness). Each sample's secondary ray is traced again and replayed
 * backwards (as irgs_trace_backward, with upstream gradients dL/dL_ind and
 * dL/dO = -dL/dL_ind . L_dir). All outputs are ADDED to:
 *   g_albedo [n_points, 3], g_rough [n_points] (required);
 *   g_env [env_h, env_w, 3] (bilinear taps, atomics; NULL to skip);
 *   g_means [n,3], g_quats [n,4] (raw quaternion), g_scales [n,2],
 *   g_opacity [n], g_features [n, num_features] (channels feat_offset ..
 *   feat_offset + 2 only) (all required).
 * Points whose g_rgb row is zero are skipped. Needs scratch of 64 bytes per
 * surfel from the stream-ordered allocator (IRGS_ERR_OOM if it fails).
 */
irgs_status irgs_shade_mc_backward(irgs_scene scene, const float* x, const float* n, const float* albedo,
                                   const float* rough, const float* wo, int64_t n_points, const float* env,
                                   int32_t env_h, int32_t env_w, int32_t n_diffuse, int32_t n_spec,
                                   uint64_t seed, const irgs_trace_params* params, const float* g_rgb,
                                   float* g_albedo, float* g_rough, float* g_env, float* g_means,
                                   float* g_quats, float* g_scales, float* g_opacity, float* g_features,
                                   void* stream);

/*
 * The incident directions irgs_shade_mc draws (Eq. 15's samples; cosine /
 * GGX half-vector sampling of the supplementary "Composited scene details",
 * or the stratified uniform directions with IRGS_FLAG_UNIFORM in `flags`),
 * without tracing them: sample s of point p is ray i = p (n_diffuse +
 * n_spec) + s, starting at x[p] (not written). n, wo : [n_points, 3], rough
 * : [n_points] device arrays as for irgs_shade_mc. out_dir [n_points S, 3]
 * receives the unit direction w_i, out_valid [n_points S] (may be NULL) 1
 * where the sample is traced and 0 where it lies below the horizon (adds 0
 * but counts). Same random numbers, frame and arithmetic as the estimator.
 */
irgs_status irgs_shade_sample_rays(const float* n, const float* rough, const float* wo, int64_t n_points,
                                  int32_t n_diffuse, int32_t n_spec, uint64_t seed, uint32_t flags,
                                  float* out_dir, int32_t* out_valid, void* stream);

/* ---------------------------------------------------------------------- */
/* Relighting (supplementary "Relighting details", Eq. 18).               */
/* ---------------------------------------------------------------------- */

/* Sizes of the pre-integrated maps. */
#define IRGS_RELIGHT_IRR_H 32
#define IRGS_RELIGHT_IRR_W 64
#define IRGS_RELIGHT_LEVELS 6
#define IRGS_RELIGHT_PREF_H 64
#define IRGS_RELIGHT_PREF_W 128
#define IRGS_RELIGHT_LUT_N 32

typedef struct irgs_envmap_s* irgs_envmap;

/*
 * Pre-integrate an environment for relighting (all maps equirect, z up,
 * texel centres as in irgs_shade_mc, over all H x W texels t of the
 * environment, each of constant radiance E_t over its exact band solid
 * angle dOmega_t seen from its centre direction w_t):
 *   irradiance  Irr(N) = 1/pi sum_t E_t max(0, w_t.N) dOmega_t, at the centres
 *               of a 32 x 64 map;
 *   prefilter   for roughness rho_l = l/5, l = 1..5, at the centres R of
 *               64 x 128 maps: sum_t E_t D(R.h_t) max(0, w_t.R) dOmega_t /
 *               sum_t D(R.h_t) max(0, w_t.R) dOmega_t, h_t = normalise(w_t + R),
 *               D GGX with alpha_g = rho^2 (split sum with n = v = R; level 0
 *               is the environment itself);
 *   BRDF table  over cell centres (n.v, rho) = ((i+0.5)/32, (j+0.5)/32): the
 *               split-sum factors A, B of int f_s (w.n) dw = F0 A + B (Schlick
 *               F split into F0 (1 - c^5) + c^5, c = 1 - v.h), from 1024
 *               Hammersley GGX half vectors ((k+0.5)/1024, radical inverse);
 *   sampling    FP64 cdfs of the texel weights lum(E_t) sin(theta of the row
 *               centre), lum = 0.2126 r + 0.7152 g + 0.0722 b, per row over
 *               columns and over rows.
 *   env : device [H, W, 3] radiance, copied (the caller keeps ownership).
 *   out : receives the handle; free it with irgs_envmap_destroy.
 * Enqueued on `stream`; allocates about 1.2 MB + 28 H W bytes of device memory.
 */
irgs_status irgs_envmap_create(const float* env, int32_t H, int32_t W, void* stream, irgs_envmap* out);

/* Synchronises the device, then frees the maps. NULL is ignored. */
irgs_status irgs_envmap_destroy(irgs_envmap envmap);

/* Copy the maps out (any pointer may be NULL; device or host memory, copied
 * with cudaMemcpyAsync on `stream`): irr [32,64,3], pref [5,64,128,3]
 * (levels 1..5), lut [32,32,2] (A, B), row_cdf [H+1], col_cdf [H, W+1]. */
irgs_status irgs_envmap_export(irgs_envmap envmap, float* irr, float* pref, float* lut, double* row_cdf,
                               double* col_cdf, void* stream);

/*
 * Relighting estimate at G-buffer points under the environment of `envmap`:
 *   rgb = 1/S sum_s f(w_s, w_o) L_i(w_s) max(0, w_s.n) / pdf(w_s)
 * with f the point's BRDF as in irgs_shade_mc (n flipped towards w_o), w_s
 * drawn by importance sampling the environment (row from the row cdf at
 * u1 x total, column from that row's cdf at u2 x row weight, the leftover
 * fractions placing w_s uniformly in (phi, theta) inside the texel; pdf =
 * (weight / total) W H / (2 pi^2 sin theta)), uniforms as in irgs_shade_mc
 * with S = n_samples. Each w_s is traced (params.feat_offset selects 7
 * channels [albedo (3), roughness, normal (3)], feat_count = 7, t_min > 0):
 * with O = 1 - V the traced opacity, the blend gives A_r = sum(w a)/O,
 * R_r = sum(w r)/O, N_r = normalise(sum(w n)) flipped to face v = -w_s, and
 *   L_i = V E(w_s) + O (A_r Irr(N_r) + Pref(reflect(v, N_r), R_r)
 *                        (0.04 A + B)(N_r.v, R_r)),
 * Pref linear between its two nearest roughness levels, all maps bilinear.
 * out_rgb [P,3]; out_vis [P] and out_ind [P,3] (means of V and of the
 * indirect term over all samples) may be NULL. By default the samples of
 * all points are regrouped by direction and origin and traced with one
 * stack per ray (scratch from the stream-ordered allocator, ~64 bytes per
 * sample in chunks of at most 2^26); IRGS_FLAG_PER_THREAD selects the fused
 * kernel (a warp per point tracing its own samples). Both give the same
 * traces.
 */
irgs_status irgs_relight(irgs_scene scene, irgs_envmap envmap, const float* x, const float* n,
                         const float* albedo, const float* rough, const float* wo, int64_t n_points,
                         int32_t n_samples, uint64_t seed, const irgs_trace_params* params,
                         float* out_rgb, float* out_vis, float* out_ind, void* stream);

/*
 * The environment-importance directions irgs_relight draws (Eq. 18's
 * samples), without tracing them: sample s of point p is ray i = p
 * n_samples + s. out_dir [n_points n_samples, 3] unit directions, out_pdf
 * (may be NULL) their solid-angle density, out_valid (may be NULL) 1 where
 * the sample is used. Device arrays; the directions depend only on the
 * environment, the seed and the keys (p, s).
 */
irgs_status irgs_relight_sample_rays(irgs_envmap envmap, int64_t n_points, int32_t n_samples, uint64_t seed,
                                    float* out_dir, float* out_pdf, int32_t* out_valid, void* stream);

/* ---------------------------------------------------------------------- */
/* Serving: several resident scenes, many requests per persistent launch. */
/* ---------------------------------------------------------------------- */

/* Pinhole camera. Pixel p of a request is numbered tile by tile: tiles of
 * tile_w x tile_h pixels in row-major tile order, row-major inside a tile
 * (tile_w = tile_h = 1 gives plain row-major order); width and height must
 * be multiples of the tile. The ray of pixel (px, py) starts at `origin`
 * and points along normalize(forward + x right + y up) with
 * x = ((px + 0.5)/width * 2 - 1) tan_half_fov width/height and
 * y = (1 - (py + 0.5)/height * 2) tan_half_fov. */
typedef struct {
    float origin[3];
    float forward[3];       /* unit view direction          */
    float right[3];         /* unit image x axis            */
    float up[3];            /* unit image y axis (up)       */
    float tan_half_fov;     /* tan(vertical field of view/2) */
    int32_t width, height;
    int32_t tile_w, tile_h;
} irgs_camera;

typedef enum { IRGS_JOB_RENDER = 0, IRGS_JOB_RELIGHT = 1 } irgs_job_kind;

/* One request of a serving step. Device pointers; the caller owns them.
 *   render : feat [P, render.feat_count], depth [P], opacity [P] (Eq. 8).
 *   relight: gbuffer, 16 P floats written by G-buffer tiles and read by
 *            shade tiles, planar: x [P, 3], then n [P, 3], albedo [P, 3],
 *            roughness [P], w_o [P, 3], valid [P] (1 where the opacity
 *            exceeds 0.5), opacity [P] and [P] unused, one after the other;
 *            rgb [P, 3] (Eq. 15 with n_diffuse cosine + n_spec GGX samples
 *            per pixel against env [env_h, env_w, 3], random stream `seed`,
 *            stream point = pixel index p, exactly as irgs_shade_mc keys
 *            point p; pixels whose valid entry is 0 get 0).
 * P = width x height of the camera. Render and G-buffer tiles trace the
 * camera's ray of pixel p, or, when ray_o and ray_d are both non-NULL, the
 * caller's ray p of ray_o / ray_d [P, 3] (the camera then only sets P). */
typedef struct {
    int32_t kind;           /* irgs_job_kind (informational)          */
    int32_t scene;          /* index into the server's scenes         */
    irgs_camera cam;
    int32_t n_diffuse, n_spec;
    uint64_t seed;
    const float* env;
    int32_t env_h, env_w;
    float* feat;
    float* depth;
    float* opacity;
    float* gbuffer;
    float* rgb;
    const float* ray_o;     /* optional explicit rays [P, 3] (both or neither) */
    const float* ray_d;
} irgs_job;

typedef enum { IRGS_TILE_RENDER = 0, IRGS_TILE_GBUFFER = 1, IRGS_TILE_SHADE = 2 } irgs_tile_kind;

/* A unit of work: pixels (render / G-buffer) or G-buffer points (shade)
 * [first, first + count) of job `job`. A shade tile must run in a later
 * step than the G-buffer tiles of the same pixels. */
typedef struct {
    int32_t kind;
    int32_t job;
    int32_t first;
    int32_t count;
} irgs_tile;

typedef struct irgs_server_s* irgs_server;

/*
 * Create a server over resident scenes (the scenes must outlive it and must
 * not be rebuilt while a step runs). `render` traces camera rays (k = 16,
 * feat_count <= 10); G-buffer tiles trace the 7 material channels starting
 * at `material_offset` (albedo 3, roughness 1, normal 3) with the render
 * parameters otherwise; `shade` traces the secondary rays (k = 16,
 * feat_count = 3 radiance channels, t_min > 0, flags 0: served shading is
 * the split-lobe estimator through the wavefront path). Allocates pinned staging
 * for max_jobs jobs and max_tiles tiles and its device copy.
 */
irgs_status irgs_server_create(const irgs_scene* scenes, int32_t n_scenes, int32_t max_jobs, int32_t max_tiles,
                               int32_t material_offset, const irgs_trace_params* render,
                               const irgs_trace_params* shade, irgs_server* out);

/* Host (pinned) tables the caller fills before each step: jobs[max_jobs],
 * tiles[max_tiles]. They may be rewritten only after the previous step's
 * work has completed on its stream. */
irgs_status irgs_server_staging(irgs_server server, irgs_job** jobs, irgs_tile** tiles);

/*
 * Run one step: validate the first n_jobs / n_tiles table entries, copy the
 * tables to the device and launch one persistent kernel whose blocks pull
 * the render and G-buffer tiles until none is left. With use_graph != 0 the
 * copy, counter reset and launch are captured into a CUDA graph on the first
 * such call and replayed afterwards. The shade tiles follow: each run of
 * consecutive tiles of one job over consecutive points is shaded by the
 * wavefront path of irgs_shade_mc (scratch from the stream-ordered
 * allocator, as there). Ordered after prior work on `stream`; later work on
 * `stream` waits for the step. Returns once the work is enqueued.
 */
irgs_status irgs_server_step(irgs_server server, int32_t n_jobs, int32_t n_tiles, int32_t use_graph,
                             void* stream);

/* Free a server (synchronises its stream first). NULL is ignored. */
irgs_status irgs_server_destroy(irgs_server server);

/* Rays of pixels [first, first + count) of a camera, written to device
 * arrays ray_o / ray_d [count, 3] (the same rays a server step traces). */
irgs_status irgs_camera_rays(const irgs_camera* cam, int64_t first, int64_t count, float* ray_o, float* ray_d,
                             void* stream);

/*
 * 2D Gaussian rasterisation of a G-buffer (Sec. 3.3: the stage-I/II maps of
 * Eq. 9-10 are rasterised, not traced). Row-major width x height image of
 * `cam` (its tile fields are ignored). For each pixel and its camera ray d,
 * the surfels whose centre has view depth z_c = (mu - origin).forward >
 * params->t_min are blended with Eq. 2 (w = T alpha, stop after the hit that
 * makes T < T_min) in ascending (z_c, user index) order. Per surfel:
 *   rho3^2 = u^2 + v^2 of the ray's intersection with its plane (Eq. 6-7),
 *            +inf if |n.d| < 1e-8 or tau <= 0;
 *   rho2^2 = |pixel centre - projected centre|^2 / (1/2)   (pixels; the
 *            2DGS screen-space low-pass filter);
 *   rho^2 = min(rho3^2, rho2^2); kept if rho^2 <= rho_c^2 and
 *   alpha = min(alpha_max, o exp(-rho^2/2)) >= alpha_min; its depth is tau
 *   if rho3^2 <= rho2^2, else (mu - origin).d.
 * Outputs as irgs_trace_forward: out_feat [P, feat_count], out_depth [P],
 * out_opacity [P], out_nhits [P] (or NULL), P = width x height. Uses scratch
 * from the stream-ordered allocator and synchronises `stream` once (to size
 * the per-tile lists). params->flags must be 0.
 */
irgs_status irgs_rasterize(irgs_scene scene, const irgs_camera* cam, const irgs_trace_params* params,
                           float* out_feat, float* out_depth, float* out_opacity, int32_t* out_nhits,
                           void* stream);

/*
 * Allocation-free LBVH build (the paper has no counterpart; this is a
 * deployment variant of irgs_build_scene).
 *
 * Some callers cannot let a library allocate device memory: applications
 * that own every byte of GPU memory through their own arena or budget, and
 * loops that cannot afford the device-wide synchronisation a cudaMalloc or
 * cudaFree implies. For them this call builds the same hierarchy as
 * irgs_build_scene -- Morton order, sorted keys, internal nodes and leaf
 * boxes, identical to what irgs_scene_export returns for the same surfels
 * -- into buffers the caller passes, and allocates nothing: its working
 * memory is one fixed array of about 6.5 MB inside the library (a
 * file-scope __device__ array that every GPU which loads the library holds
 * until the process exits).
 *   surfels   : device arrays as for irgs_build_scene; features are ignored.
 *               n must not exceed IRGS_NOALLOC_MAX_SURFELS, otherwise the
 *               call returns IRGS_ERR_INVALID_ARG and does nothing.
 *   alpha_min : as for irgs_build_scene (> 0).
 *   perm      : [n] int32 device buffer, user index of each Morton slot.
 *   keys      : [n] uint32 device buffer, sorted Morton codes.
 *   nodes     : [max(n-1,1), 16] float32 device buffer (layout as in
 *               irgs_scene_export).
 *   leaf_boxes: [n, 6] float32 device buffer.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture. All calls share the one array and it keeps the last call's
 * contents; calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it, so serialise them. Work is enqueued on `stream`.
 * Errors the kernels detect (a hierarchy that fails a consistency bound)
 * land in a status word inside the array: read it with
 * irgs_build_lbvh_noalloc_status before the next build.
 */
#define IRGS_NOALLOC_MAX_SURFELS 32768
irgs_status irgs_build_lbvh_noalloc(const irgs_surfels* surfels, float alpha_min, int32_t* perm,
                                    uint32_t* keys, float* nodes, float* leaf_boxes, void* stream);

/* Device-side outcome of the last irgs_build_lbvh_noalloc on `device`: waits
 * for `stream` (the build's stream), then copies the build's status word out
 * of the shared array into *bits (NULL to skip) without clearing it. Returns
 * IRGS_OK if it is 0, else IRGS_ERR_DEVICE with the bits of
 * irgs_scene_status (2: the hierarchy failed a consistency bound, so the
 * nodes must not be used). The next build on that device overwrites the
 * word, so read it before starting another. Allocates nothing. */
irgs_status irgs_build_lbvh_noalloc_status(int32_t device, void* stream, uint32_t* bits);

#ifdef __cplusplus
}
#endif

#endif /* IRGS_H */
