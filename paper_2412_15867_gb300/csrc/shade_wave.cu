// Wavefront Monte Carlo shading (IRGS Eq. 13-15) and its gradient.
//
// The fused shading kernel traces the samples of one point from one warp:
// its 32 rays share an origin but spread over the hemisphere, so a warp
// walks 32 unrelated paths through the hierarchy. Here the secondary rays of
// a batch of points are made first (one thread per sample), regrouped by a
// 30-bit key -- a 6-bit octahedral bin of the direction above the 24-bit
// Morton code of the origin -- with a stable radix sort, and traced in that
// order, so the rays of a warp leave neighbouring points in similar
// directions and walk similar paths. Each lane keeps its own stack: these
// rays are still too spread for one warp-wide walk (a shared stack visited
// 8x the nodes), but their independent walks now diverge little (1.8x the
// throughput of unsorted rays on the 1M-surfel scene). The per-point estimate then reads the stored
// traces (L_ind, V) and applies the same per-sample arithmetic as the fused
// kernel (shade_point_warp), with the same fixed reduction order.
//
// The gradient reuses the regrouping: the forward pass of the backward also
// saves each ray's hit list; a per-point kernel turns the upstream gradient
// into albedo / roughness / environment gradients and into each ray's
// upstream (dL/dL_ind, dL/dO); the rays are then run backwards in sorted
// order from their hit lists (rays with longer lists replay the march).
//
// Rays are processed in chunks of whole points, at most kWaveChunkRays rays
// each, so the scratch (~390 bytes per ray with the gradient) stays bounded;
// a chunk is sorted as a whole, and the denser its points the more a warp's
// regrouped rays share their paths (one chunk of 41M rays traces 6-7%
// faster than three of at most 2^24).
#include <cuda_runtime.h>

#include "scene.h"
#include "shade.cuh"
#include "trace.cuh"
#include "trace_bwd.cuh"
#include "wave.cuh"

namespace irgs {
namespace {

constexpr int kWaveThreads = 128;
constexpr int64_t kWaveChunkRays = int64_t(1) << 26;
constexpr int kWaveSavedHits = 64;   // 12% of secondary rays blend more than 32 hits, 0.02% more than 64
constexpr int kWaveReplayBlocks = 1024;   // grid-stride blocks for the few rays whose hit list did not fit

__device__ __forceinline__ f3 ld3w(const float* p, int64_t i) { return mk3(p[3 * i], p[3 * i + 1], p[3 * i + 2]); }

// One thread per sample of points [p0, p0 + rays / St): direction (w = 1 if
// the sample is valid) and its regrouping key (invalid samples sort last).
// Point p draws the random numbers of point number key_base + p; a point
// whose `valid` entry (if given) is not above 0.5 traces nothing.
__global__ void k_wave_gen(const float* __restrict__ xg, const float* __restrict__ ng, const float* __restrict__ rg,
                           const float* __restrict__ wog, int64_t p0, int64_t rays, int St, int nd, int mode,
                           uint64_t seed, const uint32_t* __restrict__ bounds, float4* __restrict__ dir,
                           uint32_t* __restrict__ key, int32_t* __restrict__ val, uint64_t key_base,
                           const float* __restrict__ valid) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rays) return;
    const int64_t p = p0 + i / St;
    const int s = (int)(i % St);
    if (valid != nullptr && !(valid[p] > 0.5f)) {
        dir[i] = make_float4(0.f, 0.f, 1.f, 0.f);
        key[i] = kInvalidWaveKey;
        val[i] = (int32_t)i;
        return;
    }
    const ShadeFrame F = shade_frame(ld3w(ng, p), ld3w(wog, p), rg[p]);
    const ShadeSample d = draw_sample(F, mode, key_base + (uint64_t)p, s, St, nd, seed);
    dir[i] = make_float4(d.wi.x, d.wi.y, d.wi.z, d.valid ? 1.f : 0.f);
    key[i] = d.valid ? wave_key(ld3w(xg, p), d.wi, bounds) : kInvalidWaveKey;
    val[i] = (int32_t)i;
}

// Trace the rays in regrouped order; res[i] = (L_ind, V).
// With SAVE the blended hit ids (user order, -1 terminated) and the hit
// counts are kept for the backward.
template <int K, bool SAVE>
__global__ void __launch_bounds__(kWaveThreads, 6) k_wave_trace(SceneView S, TraceParams P,
                                                                const float* __restrict__ xg, int64_t p0, int St,
                                                                const float4* __restrict__ dir,
                                                                const int32_t* __restrict__ order, int64_t rays,
                                                                float4* __restrict__ res, int32_t* __restrict__ nh,
                                                                int32_t* __restrict__ ids, int max_ids) {
    static_assert(kWaveThreads == trace_threads<K>(), "k-buffer slots are laid out per block thread");
    const int64_t j = blockIdx.x * (int64_t)kWaveThreads + threadIdx.x;
    const int64_t i = j < rays ? order[j] : 0;
    const float4 d4 = dir[i];
    const bool live = j < rays && d4.w != 0.f;
    const int64_t p = p0 + i / St;
    const Ray ray = make_ray(ld3w(xg, p), mk3(d4.x, d4.y, d4.z));
    MarchState<K, 3> st;
    int32_t* my_ids = (SAVE && live) ? ids + i * (int64_t)max_ids : nullptr;
    const bool ok = march_forward<K, 3, false>(S, ray, P, st, my_ids, max_ids, live);
    if (j >= rays) return;
    if (!live) {   // every sample gets an entry, so no reader sees unwritten scratch
        res[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (SAVE) nh[i] = 0;
        return;
    }
    if (!ok) atomicOr(S.status, kErrStackOverflow);
    res[i] = make_float4(st.C[0], st.C[1], st.C[2], st.T);
    if (SAVE) {
        nh[i] = st.nh;
        if (st.nh < max_ids) my_ids[st.nh] = -1;
    }
}

// The same traces in compacted rounds: round 1 on every ray of the order;
// rays still marching store their state (C, D, T, hit count, next key) at
// their sorted position and are regrouped, keeping the sorted order, for
// rounds 2 and 3; the rest run to completion. Per ray the rounds and their
// arithmetic are march_forward's (per lane), so the results are the same.
enum WaveRound { kWaveFirst = 0, kWaveNext = 1, kWaveLast = 2 };
constexpr int kWaveStateF4 = 3;   // C[3], D, T, hit count, next key (2 words), next user index

template <int K, bool SAVE, int MODE>
__global__ void __launch_bounds__(kWaveThreads, 6) k_wave_round(
    SceneView S, TraceParams P, const float* __restrict__ xg, int64_t p0, int St, const float4* __restrict__ dir,
    const int32_t* __restrict__ order, int64_t rays, float4* __restrict__ res, int32_t* __restrict__ nh,
    int32_t* __restrict__ ids, int max_ids, const int32_t* __restrict__ list, const uint32_t* __restrict__ count,
    float4* __restrict__ state, uint32_t* __restrict__ flags) {
    static_assert(kWaveThreads == trace_threads<K>(), "k-buffer slots are laid out per block thread");
    const int64_t t = blockIdx.x * (int64_t)kWaveThreads + threadIdx.x;
    const int64_t n = MODE == kWaveFirst ? rays : (int64_t)*count;
    if (t >= n) return;
    const int64_t j = MODE == kWaveFirst ? t : (int64_t)list[t];
    const int64_t i = order[j];
    const float4 d4 = dir[i];
    if (MODE == kWaveFirst && d4.w == 0.f) {   // every sample gets an entry, so no reader sees unwritten scratch
        res[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (SAVE) nh[i] = 0;
        return;
    }
    const Ray ray = make_ray(ld3w(xg, p0 + i / St), mk3(d4.x, d4.y, d4.z));
    MarchState<K, 3> st;
    uint64_t last_key = depth_key(P.t_min, 0.f);
    int32_t last_u = INT32_MAX;
    if (MODE == kWaveFirst) {
        st.C[0] = st.C[1] = st.C[2] = 0.f;
        st.D = 0.f;
        st.T = 1.f;
        st.nh = 0;
    } else {
        const float4 a = state[j * kWaveStateF4], b = state[j * kWaveStateF4 + 1], c = state[j * kWaveStateF4 + 2];
        st.C[0] = a.x; st.C[1] = a.y; st.C[2] = a.z;
        st.D = a.w;
        st.T = b.x;
        st.nh = __float_as_int(b.y);
        last_key = ((uint64_t)__float_as_uint(b.w) << 32) | (uint64_t)__float_as_uint(b.z);
        last_u = __float_as_int(c.x);
    }
    int32_t* my_ids = SAVE ? ids + i * (int64_t)max_ids : nullptr;
    KBuffer<K, trace_threads<K>()> kb;
    kb.bind();
    bool ok = true, done = false;
    do {
        ok &= collect_round(S, ray, P, last_key, last_u, kb);
        done = blend_round<K, 3>(S, P, kb, st, my_ids, max_ids, last_key, last_u);
    } while (MODE == kWaveLast && !done);
    if (!ok) atomicOr(S.status, kErrStackOverflow);
    if (done) {
        res[i] = make_float4(st.C[0], st.C[1], st.C[2], st.T);
        if (SAVE) {
            nh[i] = st.nh;
            if (st.nh < max_ids) my_ids[st.nh] = -1;
        }
    } else {
        state[j * kWaveStateF4] = make_float4(st.C[0], st.C[1], st.C[2], st.D);
        state[j * kWaveStateF4 + 1] = make_float4(st.T, __int_as_float(st.nh), __uint_as_float((uint32_t)last_key),
                                                  __uint_as_float((uint32_t)(last_key >> 32)));
        state[j * kWaveStateF4 + 2] = make_float4(__int_as_float(last_u), 0.f, 0.f, 0.f);
        flags[j] = 1u;
    }
}

// Per-point estimate from the stored traces (warp per point).
template <int K>
__global__ void __launch_bounds__(kWaveThreads) k_wave_shade(SceneView S, const float* __restrict__ xg,
                                                             const float* __restrict__ ng,
                                                             const float* __restrict__ ag,
                                                             const float* __restrict__ rg,
                                                             const float* __restrict__ wog, int64_t p0, int64_t np,
                                                             const float* __restrict__ env, int H, int W, int nd,
                                                             int ns, int mode, uint64_t seed, TraceParams TP,
                                                             const float4* __restrict__ res, float* __restrict__ rgb,
                                                             float* __restrict__ vis, float* __restrict__ ind,
                                                             uint64_t key_base, const float* __restrict__ valid) {
    const int lane = threadIdx.x & 31;
    const int64_t k = blockIdx.x * (int64_t)(kWaveThreads / 32) + (threadIdx.x >> 5);
    if (k >= np) return;
    const int64_t p = p0 + k;
    const int St = nd + ns;
    ShadeSums o;
    if (valid != nullptr && !(valid[p] > 0.5f)) {   // background: no estimate (warp-uniform)
        o.rgb[0] = o.rgb[1] = o.rgb[2] = 0.f;
        o.ind[0] = o.ind[1] = o.ind[2] = 0.f;
        o.vis = 0.f;
    } else {
        shade_point_warp<K, false, true>(S, ld3w(xg, p), ld3w(ng, p), ld3w(wog, p), ld3w(ag, p), rg[p],
                                         key_base + (uint64_t)p, nd, ns, mode, seed, env, H, W, TP, o, res + k * St);
    }
    if (lane == 0) {
        for (int c = 0; c < 3; ++c) rgb[3 * p + c] = o.rgb[c];
        if (vis != nullptr) vis[p] = o.vis;
        if (ind != nullptr)
            for (int c = 0; c < 3; ++c) ind[3 * p + c] = o.ind[c];
    }
}

// Per-point gradient (warp per point): albedo, roughness and environment
// gradients, and up[i] = (dL/dL_ind, dL/dO) of each of its rays.
__global__ void __launch_bounds__(kWaveThreads) k_wave_grad_point(
    const float* __restrict__ ng, const float* __restrict__ ag, const float* __restrict__ rg,
    const float* __restrict__ wog, int64_t p0, int64_t np, const float* __restrict__ env, int H, int W, int nd,
    int ns, int mode, uint64_t seed, const float4* __restrict__ res, const float* __restrict__ g_rgb,
    float* __restrict__ g_albedo, float* __restrict__ g_rough, float* __restrict__ g_env, float4* __restrict__ up) {
    const int lane = threadIdx.x & 31;
    const int64_t k = blockIdx.x * (int64_t)(kWaveThreads / 32) + (threadIdx.x >> 5);
    if (k >= np) return;
    const int64_t p = p0 + k;
    const int St = nd + ns;
    const float g[3] = {g_rgb[3 * p], g_rgb[3 * p + 1], g_rgb[3 * p + 2]};
    const f3 a = ld3w(ag, p);
    const float av[3] = {a.x, a.y, a.z};
    const ShadeFrame F = shade_frame(ld3w(ng, p), ld3w(wog, p), rg[p]);
    float ga[3] = {0.f, 0.f, 0.f}, gr = 0.f;
    for (int s = lane; s < St; s += 32) {
        const ShadeSample d = draw_sample(F, mode, (uint64_t)p, s, St, nd, seed);
        float gL[3] = {0.f, 0.f, 0.f}, gO = 0.f;
        if (d.valid) {
            const float4 t = __ldg(res + k * St + s);
            const float C[3] = {t.x, t.y, t.z};
            sample_grad(F, d, mode, nd, ns, St, av, g, C, t.w, env, H, W, g_env, ga, gr, gL, gO);
        }
        up[k * St + s] = make_float4(gL[0], gL[1], gL[2], gO);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        for (int off = 16; off > 0; off >>= 1) ga[c] += __shfl_xor_sync(0xffffffffu, ga[c], off);
    for (int off = 16; off > 0; off >>= 1) gr += __shfl_xor_sync(0xffffffffu, gr, off);
    if (lane == 0) {
        for (int c = 0; c < 3; ++c) g_albedo[3 * p + c] += ga[c];
        g_rough[p] += gr;
    }
}

// Backward of one ray in regrouped order (sorted position j): from its saved
// hit list (LISTED) or by replaying its march.
template <int K, bool LISTED>
__device__ __forceinline__ void wave_backward_ray(const SceneView& S, const TraceParams& P,
                                                  const float* __restrict__ xg, int64_t p0, int St,
                                                  const float4* __restrict__ dir, int64_t i,
                                                  const float4* __restrict__ res, int n_hits,
                                                  const int32_t* __restrict__ ids, int max_ids, float4 u4,
                                                  float* __restrict__ acc_rows, float* rows) {
    const float4 d4 = dir[i];
    const int64_t p = p0 + i / St;
    const Ray ray = make_ray(ld3w(xg, p), mk3(d4.x, d4.y, d4.z));
    const float4 t = res[i];
    const float Cf[3] = {t.x, t.y, t.z};
    const float gC[3] = {u4.x, u4.y, u4.z};
    if (LISTED) {
        listed_backward<3>(S, ray, P, ids + i * (int64_t)max_ids, n_hits, Cf, 0.f, t.w, gC, 0.f, u4.w, acc_rows,
                           rows);
    } else {
        const bool ok = march_backward<K, 3, false>(S, ray, P, true, n_hits, Cf, 0.f, t.w, gC, 0.f, u4.w, acc_rows,
                                                    rows);
        if (!ok) atomicOr(S.status, kErrStackOverflow);
    }
}

// Backward from the saved hit lists, one thread per sorted ray; rays whose
// list did not fit (more than max_ids hits) are appended to replay_list for
// k_wave_replay.
template <int K>
__global__ void __launch_bounds__(kWaveThreads) k_wave_backward(SceneView S, TraceParams P,
                                                                const float* __restrict__ xg, int64_t p0, int St,
                                                                const float4* __restrict__ dir,
                                                                const int32_t* __restrict__ order, int64_t rays,
                                                                const float4* __restrict__ res,
                                                                const int32_t* __restrict__ nh,
                                                                const int32_t* __restrict__ ids, int max_ids,
                                                                const float4* __restrict__ up,
                                                                float* __restrict__ acc_rows,
                                                                int32_t* __restrict__ replay_list,
                                                                uint32_t* __restrict__ replay_count) {
    static_assert(kWaveThreads == trace_threads<K>(), "k-buffer slots are laid out per block thread");
    __shared__ float4 rows_all[kWaveThreads * GradRow<3>::kStride / 4];
    float* rows = reinterpret_cast<float*>(rows_all) + (threadIdx.x & ~31) * GradRow<3>::kStride;
    const int64_t j = blockIdx.x * (int64_t)kWaveThreads + threadIdx.x;
    if (j >= rays) return;
    const int64_t i = order[j];
    const int n_hits = nh[i];   // 0 for samples that drew no ray
    if (n_hits <= 0) return;
    const float4 u4 = up[i];
    if (u4.x == 0.f && u4.y == 0.f && u4.z == 0.f && u4.w == 0.f) return;
    if (n_hits > max_ids) {
        replay_list[atomicAdd(replay_count, 1u)] = (int32_t)j;
        return;
    }
    wave_backward_ray<K, true>(S, P, xg, p0, St, dir, i, res, n_hits, ids, max_ids, u4, acc_rows, rows);
}

// The rays of replay_list replay their march backwards (the list's length is
// what the listing launch left in replay_count). Consecutive entries go to
// different blocks, so the few long replays spread over every SM.
template <int K>
__global__ void __launch_bounds__(kWaveThreads) k_wave_replay(SceneView S, TraceParams P,
                                                              const float* __restrict__ xg, int64_t p0, int St,
                                                              const float4* __restrict__ dir,
                                                              const int32_t* __restrict__ order,
                                                              const float4* __restrict__ res,
                                                              const int32_t* __restrict__ nh,
                                                              const float4* __restrict__ up,
                                                              float* __restrict__ acc_rows,
                                                              const int32_t* __restrict__ replay_list,
                                                              const uint32_t* __restrict__ replay_count) {
    static_assert(kWaveThreads == trace_threads<K>(), "k-buffer slots are laid out per block thread");
    __shared__ float4 rows_all[kWaveThreads * GradRow<3>::kStride / 4];
    float* rows = reinterpret_cast<float*>(rows_all) + (threadIdx.x & ~31) * GradRow<3>::kStride;
    const int64_t n = *replay_count;
    for (int64_t t = threadIdx.x * (int64_t)gridDim.x + blockIdx.x; t < n; t += (int64_t)gridDim.x * kWaveThreads) {
        const int64_t i = order[replay_list[t]];
        wave_backward_ray<K, false>(S, P, xg, p0, St, dir, i, res, nh[i], nullptr, 0, up[i], acc_rows, rows);
    }
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

// Scratch of one chunk (stream-ordered allocation).
struct WaveScratch {
    float4* dir = nullptr;
    uint32_t* key = nullptr;
    int32_t* val = nullptr;
    uint32_t* key_tmp = nullptr;
    int32_t* val_tmp = nullptr;
    uint32_t* hist = nullptr;
    float4* res = nullptr;
    int32_t* nh = nullptr;
    int32_t* ids = nullptr;
    float4* up = nullptr;
    uint32_t* flags = nullptr;   // [rays + 1] continue flags, then their prefix sums
    int32_t* list = nullptr;     // [rays] continuing rays (sorted positions)
    uint32_t* count = nullptr;   // [1] and the scan's tile sums after it
    float4* state = nullptr;     // [rays * kWaveStateF4] march state between rounds
    unsigned char* base = nullptr;

    cudaError_t alloc(int64_t rays, bool backward, cudaStream_t st) {
        const int64_t hw = sort_hist_words(rays);
        size_t off = 0;
        auto take = [&](size_t bytes) {
            const size_t o = off;
            off += (bytes + 255) & ~size_t(255);
            return o;
        };
        const size_t o_dir = take(sizeof(float4) * rays), o_key = take(4 * rays), o_val = take(4 * rays);
        const size_t o_kt = take(4 * rays), o_vt = take(4 * rays), o_hist = take(4 * hw);
        const size_t o_res = take(sizeof(float4) * rays);
        const size_t o_flags = take(4 * (rays + 1)), o_list = take(4 * rays);
        const size_t o_count = take(4 * (1 + scan_long_words(rays + 1)));
        const size_t o_state = take(sizeof(float4) * kWaveStateF4 * rays);
        size_t o_nh = 0, o_ids = 0, o_up = 0;
        if (backward) {
            o_nh = take(4 * rays);
            o_ids = take(sizeof(int32_t) * kWaveSavedHits * rays);
            o_up = take(sizeof(float4) * rays);
        }
        cudaError_t e = scratch_alloc(reinterpret_cast<void**>(&base), off, st);
        if (e != cudaSuccess) return e;
        dir = reinterpret_cast<float4*>(base + o_dir);
        key = reinterpret_cast<uint32_t*>(base + o_key);
        val = reinterpret_cast<int32_t*>(base + o_val);
        key_tmp = reinterpret_cast<uint32_t*>(base + o_kt);
        val_tmp = reinterpret_cast<int32_t*>(base + o_vt);
        hist = reinterpret_cast<uint32_t*>(base + o_hist);
        res = reinterpret_cast<float4*>(base + o_res);
        flags = reinterpret_cast<uint32_t*>(base + o_flags);
        list = reinterpret_cast<int32_t*>(base + o_list);
        count = reinterpret_cast<uint32_t*>(base + o_count);
        state = reinterpret_cast<float4*>(base + o_state);
        if (backward) {
            nh = reinterpret_cast<int32_t*>(base + o_nh);
            ids = reinterpret_cast<int32_t*>(base + o_ids);
            up = reinterpret_cast<float4*>(base + o_up);
        }
        return cudaSuccess;
    }
    cudaError_t release(cudaStream_t st) { return base ? cudaFreeAsync(base, st) : cudaSuccess; }
};

int64_t chunk_points(int St) {
    const int64_t pc = kWaveChunkRays / St;
    return pc > 0 ? pc : 1;
}

// Trace the sorted rays of one chunk into w.res (and, with SAVE, the hit
// counts and lists): compacted rounds when the scene has surfels.
template <int K, bool SAVE>
cudaError_t wave_trace(const SceneView& S, const TraceParams& TP, const float* x, int64_t p0, int St, int64_t rays,
                       WaveScratch& w, cudaStream_t st) {
    int32_t* ids = SAVE ? w.ids : nullptr;
    int32_t* nh = SAVE ? w.nh : nullptr;
    const int max_ids = SAVE ? kWaveSavedHits : 0;
    if (S.n == 0) {
        k_wave_trace<K, SAVE><<<grid_for(rays, kWaveThreads), kWaveThreads, 0, st>>>(S, TP, x, p0, St, w.dir, w.val,
                                                                                    rays, w.res, nh, ids, max_ids);
        count_launches(1);
        return cudaGetLastError();
    }
    const unsigned g = grid_for(rays, kWaveThreads);
    cudaError_t e = cudaMemsetAsync(w.flags, 0, sizeof(uint32_t) * (rays + 1), st);
    if (e != cudaSuccess) return e;
    k_wave_round<K, SAVE, kWaveFirst><<<g, kWaveThreads, 0, st>>>(S, TP, x, p0, St, w.dir, w.val, rays, w.res, nh, ids,
                                                                  max_ids, w.list, w.count, w.state, w.flags);
    count_launches(1);
    for (int round = 2; round <= 4 && e == cudaSuccess; ++round) {
        e = flags_to_list(w.flags, rays, w.count + 1, w.list, w.count, st);
        if (e != cudaSuccess) break;
        if (round < 4) {
            e = cudaMemsetAsync(w.flags, 0, sizeof(uint32_t) * (rays + 1), st);
            if (e != cudaSuccess) break;
            k_wave_round<K, SAVE, kWaveNext><<<g, kWaveThreads, 0, st>>>(S, TP, x, p0, St, w.dir, w.val, rays, w.res,
                                                                         nh, ids, max_ids, w.list, w.count, w.state,
                                                                         w.flags);
        } else {
            k_wave_round<K, SAVE, kWaveLast><<<g, kWaveThreads, 0, st>>>(S, TP, x, p0, St, w.dir, w.val, rays, w.res,
                                                                         nh, ids, max_ids, w.list, w.count, w.state,
                                                                         w.flags);
        }
        count_launches(1);
        e = cudaGetLastError();
    }
    return e;
}

template <int K>
cudaError_t wave_forward(const SceneView& S, const uint32_t* bounds, const float* x, const float* n, const float* a,
                         const float* r, const float* wo, int64_t P, const float* env, int H, int W, int nd, int ns,
                         int mode, uint64_t seed, const TraceParams& TP, float* rgb, float* vis, float* ind,
                         cudaStream_t st, uint64_t key_base, const float* valid) {
    const int St = nd + ns;
    const int64_t pc = chunk_points(St);
    WaveScratch w;
    cudaError_t e = w.alloc((P < pc ? P : pc) * St, false, st);
    if (e != cudaSuccess) return e;
    for (int64_t p0 = 0; p0 < P && e == cudaSuccess; p0 += pc) {
        const int64_t np = P - p0 < pc ? P - p0 : pc;
        const int64_t rays = np * St;
        k_wave_gen<<<grid_for(rays, 256), 256, 0, st>>>(x, n, r, wo, p0, rays, St, nd, mode, seed, bounds, w.dir,
                                                        w.key, w.val, key_base, valid);
        e = sort_pairs(w.key, w.val, w.key_tmp, w.val_tmp, w.hist, rays, st);
        if (e != cudaSuccess) break;
        e = wave_trace<K, false>(S, TP, x, p0, St, rays, w, st);
        if (e != cudaSuccess) break;
        k_wave_shade<K><<<grid_for(np, kWaveThreads / 32), kWaveThreads, 0, st>>>(
            S, x, n, a, r, wo, p0, np, env, H, W, nd, ns, mode, seed, TP, w.res, rgb, vis, ind, key_base, valid);
        count_launches(2);
        e = cudaGetLastError();
    }
    const cudaError_t ef = w.release(st);
    return e != cudaSuccess ? e : ef;
}

template <int K>
cudaError_t wave_backward(const SceneView& S, const int32_t* perm, const uint32_t* bounds, const float* x,
                          const float* n, const float* a, const float* r, const float* wo, int64_t P,
                          const float* env, int H, int W, int nd, int ns, int mode, uint64_t seed,
                          const TraceParams& TP, const float* g_rgb, float* g_albedo, float* g_rough, float* g_env,
                          float* g_means, float* g_quats, float* g_scales, float* g_opacity, float* g_features,
                          cudaStream_t st) {
    constexpr int N = GradRow<3>::N;
    const int St = nd + ns;
    const int64_t pc = chunk_points(St);
    const size_t row_bytes = sizeof(float) * N * (size_t)(S.n > 0 ? S.n : 1);
    float* acc_rows = nullptr;
    cudaError_t e = scratch_alloc(reinterpret_cast<void**>(&acc_rows), row_bytes, st);
    if (e != cudaSuccess) return e;
    WaveScratch w;
    e = cudaMemsetAsync(acc_rows, 0, row_bytes, st);
    if (e == cudaSuccess) e = w.alloc((P < pc ? P : pc) * St, true, st);
    for (int64_t p0 = 0; p0 < P && e == cudaSuccess; p0 += pc) {
        const int64_t np = P - p0 < pc ? P - p0 : pc;
        const int64_t rays = np * St;
        k_wave_gen<<<grid_for(rays, 256), 256, 0, st>>>(x, n, r, wo, p0, rays, St, nd, mode, seed, bounds, w.dir,
                                                        w.key, w.val, 0ull, nullptr);
        e = sort_pairs(w.key, w.val, w.key_tmp, w.val_tmp, w.hist, rays, st);
        if (e != cudaSuccess) break;
        const unsigned g = grid_for(rays, kWaveThreads);
        e = wave_trace<K, true>(S, TP, x, p0, St, rays, w, st);
        if (e != cudaSuccess) break;
        k_wave_grad_point<<<grid_for(np, kWaveThreads / 32), kWaveThreads, 0, st>>>(
            n, a, r, wo, p0, np, env, H, W, nd, ns, mode, seed, w.res, g_rgb, g_albedo, g_rough, g_env, w.up);
        e = cudaMemsetAsync(w.count, 0, sizeof(uint32_t), st);
        if (e != cudaSuccess) break;
        k_wave_backward<K><<<g, kWaveThreads, 0, st>>>(S, TP, x, p0, St, w.dir, w.val, rays, w.res, w.nh, w.ids,
                                                       kWaveSavedHits, w.up, acc_rows, w.list, w.count);
        k_wave_replay<K><<<kWaveReplayBlocks, kWaveThreads, 0, st>>>(S, TP, x, p0, St, w.dir, w.val, w.res, w.nh,
                                                                     w.up, acc_rows, w.list, w.count);
        count_launches(4);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && S.n > 0) {
        k_grad_scatter<3><<<grid_for(S.n, 256), 256, 0, st>>>(perm, S.n, acc_rows, TP.fc, S.F, TP.off, g_means,
                                                             g_quats, g_scales, g_opacity, g_features);
        count_launches(1);
        e = cudaGetLastError();
    }
    const cudaError_t ef = w.release(st);
    const cudaError_t ea = cudaFreeAsync(acc_rows, st);
    if (e != cudaSuccess) return e;
    return ef != cudaSuccess ? ef : ea;
}

irgs_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return IRGS_OK;
    return e == cudaErrorMemoryAllocation ? IRGS_ERR_OOM : IRGS_ERR_CUDA;
}

}  // namespace

irgs_status launch_shade_wave(const SceneView& S, const uint32_t* bounds, const float* x, const float* n,
                              const float* albedo, const float* rough, const float* wo, int64_t P, const float* env,
                              int32_t H, int32_t W, int32_t n_diffuse, int32_t n_spec, uint64_t seed, int mode,
                              const irgs_trace_params& p, float* rgb, float* vis, float* ind, cudaStream_t st,
                              uint64_t key_base, const float* valid) {
    if (P == 0) return IRGS_OK;
    const TraceParams TP = to_params(p);
    switch (p.k) {
        case 8:
            return to_status(wave_forward<8>(S, bounds, x, n, albedo, rough, wo, P, env, H, W, n_diffuse, n_spec,
                                             mode, seed, TP, rgb, vis, ind, st, key_base, valid));
        case 16:
            return to_status(wave_forward<16>(S, bounds, x, n, albedo, rough, wo, P, env, H, W, n_diffuse, n_spec,
                                              mode, seed, TP, rgb, vis, ind, st, key_base, valid));
        default: return IRGS_ERR_UNSUPPORTED;
    }
}

irgs_status launch_shade_wave_backward(const SceneView& S, const int32_t* perm, const uint32_t* bounds,
                                       const float* x, const float* n, const float* albedo, const float* rough,
                                       const float* wo, int64_t P, const float* env, int32_t H, int32_t W,
                                       int32_t n_diffuse, int32_t n_spec, uint64_t seed, int mode,
                                       const irgs_trace_params& p, const float* g_rgb, float* g_albedo,
                                       float* g_rough, float* g_env, float* g_means, float* g_quats, float* g_scales,
                                       float* g_opacity, float* g_features, cudaStream_t st) {
    if (P == 0) return IRGS_OK;
    const TraceParams TP = to_params(p);
    switch (p.k) {
        case 8:
            return to_status(wave_backward<8>(S, perm, bounds, x, n, albedo, rough, wo, P, env, H, W, n_diffuse,
                                              n_spec, mode, seed, TP, g_rgb, g_albedo, g_rough, g_env, g_means,
                                              g_quats, g_scales, g_opacity, g_features, st));
        case 16:
            return to_status(wave_backward<16>(S, perm, bounds, x, n, albedo, rough, wo, P, env, H, W, n_diffuse,
                                               n_spec, mode, seed, TP, g_rgb, g_albedo, g_rough, g_env, g_means,
                                               g_quats, g_scales, g_opacity, g_features, st));
        default: return IRGS_ERR_UNSUPPORTED;
    }
}

}  // namespace irgs
