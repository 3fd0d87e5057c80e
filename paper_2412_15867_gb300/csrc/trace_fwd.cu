// Forward trace kernel: one thread per ray, Trace(r_o, r_d) of IRGS Eq. 8.
#include <cuda_runtime.h>

#include "scene.h"
#include "trace.cuh"

namespace irgs {
namespace {


// 6 resident blocks per SM (24 warps) keep the latency-bound walk fed; the
// k-buffers of 6 blocks take 192 KB of shared memory.
template <int K, int FB, bool WARP>
__global__ void __launch_bounds__(trace_threads<K>(), K <= 16 ? 6 : 4) k_trace_forward(SceneView S, const float* __restrict__ ro,
                                                               const float* __restrict__ rd, int64_t R,
                                                               TraceParams P, float* __restrict__ feat,
                                                               float* __restrict__ depth, float* __restrict__ opac,
                                                               int32_t* __restrict__ nhits, int32_t* __restrict__ ids,
                                                               int max_ids) {
    const int64_t r = blockIdx.x * (int64_t)trace_threads<K>() + threadIdx.x;
    const bool live = r < R;
    if (!WARP && !live) return;
    const int64_t q = live ? r : 0;   // lanes without a ray follow the warp with a dummy ray
    const Ray ray = make_ray(mk3(ro[3 * q], ro[3 * q + 1], ro[3 * q + 2]),
                             mk3(rd[3 * q], rd[3 * q + 1], rd[3 * q + 2]));
    int32_t* my_ids = (ids != nullptr && live) ? ids + r * (int64_t)max_ids : nullptr;
    MarchState<K, FB> st;
    const bool ok = march_forward<K, FB, WARP>(S, ray, P, st, my_ids, max_ids, live);
    if (!live) return;
    if (my_ids != nullptr && st.nh < max_ids) my_ids[st.nh] = -1;   // terminator
    if (!ok) atomicOr(S.status, kErrStackOverflow);
#pragma unroll
    for (int c = 0; c < FB; ++c)
        if (c < P.fc) feat[r * P.fc + c] = st.C[c];
    depth[r] = st.D;
    opac[r] = 1.0f - st.T;
    if (nhits != nullptr) nhits[r] = st.nh;
}

// ---------------------------------------------------------------------------
// Compacted rounds (large warp-coherent batches). Rays need 1 to ~6 k-buffer
// rounds (2 on average at k = 16 in camera views), and a warp walks as many
// rounds as its slowest ray, mostly with few lanes still active. Here round
// 1 runs on every ray; rays not done after it store their march state and
// are regrouped, in ray order, into full warps for round 2, again for round
// 3, and the remaining few run to completion. Per ray the rounds and their
// arithmetic are those of march_forward, so the results are bitwise the
// same; only which rays share a warp changes.
enum RoundMode { kRoundFirst = 0, kRoundNext = 1, kRoundLast = 2 };

// Between rounds: C[FB], D, T, hit count, next key (2 words), next user index.
template <int FB>
struct RoundState {
    static constexpr int kF4 = (FB + 6 + 3) / 4;
};

template <int K, int FB, int MODE>
__global__ void __launch_bounds__(trace_threads<K>(), K <= 16 ? 6 : 4) k_trace_round(
    SceneView S, const float* __restrict__ ro, const float* __restrict__ rd, int64_t R, TraceParams P,
    float* __restrict__ feat, float* __restrict__ depth, float* __restrict__ opac, int32_t* __restrict__ nhits,
    int32_t* __restrict__ ids, int max_ids, const int32_t* __restrict__ list, const uint32_t* __restrict__ count,
    float4* __restrict__ state, uint32_t* __restrict__ flags) {
    constexpr int SW = RoundState<FB>::kF4;
    const int64_t t = blockIdx.x * (int64_t)trace_threads<K>() + threadIdx.x;
    const int64_t n = MODE == kRoundFirst ? R : (int64_t)*count;
    if (__all_sync(kFullWarp, t >= n)) return;   // nothing for this warp
    const bool live = t < n;
    const int64_t r = live ? (MODE == kRoundFirst ? t : (int64_t)list[t]) : 0;
    const Ray ray = make_ray(mk3(ro[3 * r], ro[3 * r + 1], ro[3 * r + 2]),
                             mk3(rd[3 * r], rd[3 * r + 1], rd[3 * r + 2]));
    MarchState<K, FB> st;
    uint64_t last_key = depth_key(P.t_min, 0.f);
    int32_t last_u = INT32_MAX;
    if (MODE == kRoundFirst || !live) {
#pragma unroll
        for (int c = 0; c < FB; ++c) st.C[c] = 0.f;
        st.D = 0.f;
        st.T = 1.f;
        st.nh = 0;
    } else {
        float w[4 * SW];
#pragma unroll
        for (int q = 0; q < SW; ++q) {
            const float4 v = state[r * SW + q];
            w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int c = 0; c < FB; ++c) st.C[c] = w[c];
        st.D = w[FB];
        st.T = w[FB + 1];
        st.nh = __float_as_int(w[FB + 2]);
        last_key = ((uint64_t)__float_as_uint(w[FB + 4]) << 32) | (uint64_t)__float_as_uint(w[FB + 3]);
        last_u = __float_as_int(w[FB + 5]);
    }
    int32_t* my_ids = (ids != nullptr && live) ? ids + r * (int64_t)max_ids : nullptr;
    KBuffer<K, trace_threads<K>()> kb;
    kb.bind();
    bool ok = true, done = !live;
    do {
        ok &= collect_round_warp(S, ray, P, last_key, last_u, kb, !done);
        if (!done) done = blend_round<K, FB>(S, P, kb, st, my_ids, max_ids, last_key, last_u);
    } while (MODE == kRoundLast && __any_sync(kFullWarp, !done));
    if (!live) return;
    if (!ok) atomicOr(S.status, kErrStackOverflow);
    if (done) {
        if (my_ids != nullptr && st.nh < max_ids) my_ids[st.nh] = -1;   // terminator
#pragma unroll
        for (int c = 0; c < FB; ++c)
            if (c < P.fc) feat[r * P.fc + c] = st.C[c];
        depth[r] = st.D;
        opac[r] = 1.0f - st.T;
        if (nhits != nullptr) nhits[r] = st.nh;
    } else {
        float w[4 * SW];
#pragma unroll
        for (int c = 0; c < FB; ++c) w[c] = st.C[c];
        w[FB] = st.D;
        w[FB + 1] = st.T;
        w[FB + 2] = __int_as_float(st.nh);
        w[FB + 3] = __uint_as_float((uint32_t)last_key);
        w[FB + 4] = __uint_as_float((uint32_t)(last_key >> 32));
        w[FB + 5] = __int_as_float(last_u);
#pragma unroll
        for (int c = FB + 6; c < 4 * SW; ++c) w[c] = 0.f;
#pragma unroll
        for (int q = 0; q < SW; ++q) state[r * SW + q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        flags[r] = 1u;
    }
}

// Batches at least this large take the compacted rounds.
constexpr int64_t kRoundMinRays = int64_t(1) << 20;
constexpr int kCompactedRounds = 3;   // regroup after rounds 1, 2 and 3; rounds 4+ run to completion

template <int K, int FB>
cudaError_t launch_rounds(const SceneView& S, const float* ro, const float* rd, int64_t R, const TraceParams& P,
                          float* feat, float* depth, float* opac, int32_t* nhits, int32_t* ids, int max_ids,
                          cudaStream_t st) {
    constexpr int threads = trace_threads<K>();
    constexpr int SW = RoundState<FB>::kF4;
    const int64_t sums = scan_long_words(R + 1);
    // scratch: flags / positions [R + 1], list [R], count, scan sums, then the states (16-byte aligned)
    const int64_t words = (R + 1) + R + 1 + sums;
    const size_t state_off = (size_t)((words * 4 + 255) / 256 * 256);
    const size_t bytes = state_off + sizeof(float4) * SW * (size_t)R;
    unsigned char* base = nullptr;
    cudaError_t e = scratch_alloc(reinterpret_cast<void**>(&base), bytes, st);
    if (e != cudaSuccess) return e;
    uint32_t* flags = reinterpret_cast<uint32_t*>(base);
    int32_t* list = reinterpret_cast<int32_t*>(flags + R + 1);
    uint32_t* count = reinterpret_cast<uint32_t*>(list + R);
    uint32_t* scan_sums = count + 1;
    float4* state = reinterpret_cast<float4*>(base + state_off);
    const unsigned grid = (unsigned)((R + threads - 1) / threads);
    e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * (R + 1), st);
    if (e == cudaSuccess) {
        k_trace_round<K, FB, kRoundFirst><<<grid, threads, 0, st>>>(S, ro, rd, R, P, feat, depth, opac, nhits, ids,
                                                                     max_ids, list, count, state, flags);
        count_launches(1);
        for (int round = 2; round <= kCompactedRounds + 1 && e == cudaSuccess; ++round) {
            e = flags_to_list(flags, R, scan_sums, list, count, st);
            if (e != cudaSuccess) break;
            if (round <= kCompactedRounds) {
                e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * (R + 1), st);
                if (e != cudaSuccess) break;
                k_trace_round<K, FB, kRoundNext><<<grid, threads, 0, st>>>(S, ro, rd, R, P, feat, depth, opac, nhits,
                                                                           ids, max_ids, list, count, state, flags);
            } else {
                k_trace_round<K, FB, kRoundLast><<<grid, threads, 0, st>>>(S, ro, rd, R, P, feat, depth, opac, nhits,
                                                                           ids, max_ids, list, count, state, flags);
            }
            count_launches(1);
            e = cudaGetLastError();
        }
    }
    const cudaError_t ef = cudaFreeAsync(base, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e != cudaSuccess ? e : ef;
}

template <int K, int FB, bool WARP>
cudaError_t launch(const SceneView& S, const float* ro, const float* rd, int64_t R, const TraceParams& P,
                   float* feat, float* depth, float* opac, int32_t* nhits, int32_t* ids, int max_ids,
                   cudaStream_t st) {
    if constexpr (WARP && K == 16) {
        // the ray list holds int32 indices; without room for the scratch the
        // single-kernel march below does the same work
        if (R >= kRoundMinRays && R < INT32_MAX && S.n > 0) {
            const cudaError_t e = launch_rounds<K, FB>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st);
            if (e != cudaErrorMemoryAllocation) return e;
            cudaGetLastError();   // clear the failed allocation
        }
    }
    constexpr int threads = trace_threads<K>();
    const int64_t blocks = (R + threads - 1) / threads;
    k_trace_forward<K, FB, WARP><<<(unsigned)blocks, threads, 0, st>>>(S, ro, rd, R, P, feat, depth, opac,
                                                                           nhits, ids, max_ids);
    count_launches(1);
    return cudaGetLastError();
}

template <int K, bool WARP>
cudaError_t launch_f(const SceneView& S, const float* ro, const float* rd, int64_t R, const TraceParams& P,
                     float* feat, float* depth, float* opac, int32_t* nhits, int32_t* ids, int max_ids,
                     cudaStream_t st) {
    if (P.fc <= 3) return launch<K, 3, WARP>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st);
    if (P.fc <= 10) return launch<K, 10, WARP>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st);
    return launch<K, 16, WARP>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st);
}

template <int K>
cudaError_t launch_k(bool warp, const SceneView& S, const float* ro, const float* rd, int64_t R,
                     const TraceParams& P, float* feat, float* depth, float* opac, int32_t* nhits, int32_t* ids,
                     int max_ids, cudaStream_t st) {
    return warp ? launch_f<K, true>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st)
                : launch_f<K, false>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st);
}

// Diagnostic: the forward march with per-ray counters (K = 16, <= 10 channels).
template <bool WARP>
__global__ void __launch_bounds__(128) k_trace_stats(SceneView S, const float* __restrict__ ro,
                                                     const float* __restrict__ rd, int64_t R, TraceParams P,
                                                     int32_t* __restrict__ stats) {
    const int64_t r = blockIdx.x * (int64_t)128 + threadIdx.x;
    const bool live = r < R;
    if (!WARP && !live) return;
    const int64_t q = live ? r : 0;
    const Ray ray = make_ray(mk3(ro[3 * q], ro[3 * q + 1], ro[3 * q + 2]),
                             mk3(rd[3 * q], rd[3 * q + 1], rd[3 * q + 2]));
    MarchState<16, 10> st;
    TraceStats ts = {0, 0, 0, 0};
    march_forward<16, 10, WARP, true>(S, ray, P, st, nullptr, 0, live, &ts);
    if (!live) return;
    stats[4 * r] = ts.rounds;
    stats[4 * r + 1] = ts.nodes;
    stats[4 * r + 2] = ts.leaves;
    stats[4 * r + 3] = ts.inserts;
}

}  // namespace

irgs_status launch_trace_stats(const SceneView& S, const float* ro, const float* rd, int64_t R,
                               const irgs_trace_params& p, int32_t* stats, cudaStream_t st) {
    if (R == 0) return IRGS_OK;
    const TraceParams P = to_params(p);
    const unsigned blocks = (unsigned)((R + 127) / 128);
    if ((p.flags & IRGS_FLAG_PER_THREAD) == 0u)
        k_trace_stats<true><<<blocks, 128, 0, st>>>(S, ro, rd, R, P, stats);
    else
        k_trace_stats<false><<<blocks, 128, 0, st>>>(S, ro, rd, R, P, stats);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

irgs_status launch_trace_forward(const SceneView& S, const float* ro, const float* rd, int64_t R,
                                 const irgs_trace_params& p, float* feat, float* depth, float* opac,
                                 int32_t* nhits, int32_t* ids, int32_t max_ids, cudaStream_t st) {
    if (R == 0) return IRGS_OK;
    const TraceParams P = to_params(p);
    cudaError_t e;
    const bool warp = (p.flags & IRGS_FLAG_PER_THREAD) == 0u;
    switch (p.k) {
        case 1: e = launch_k<1>(warp, S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st); break;
        case 4: e = launch_k<4>(warp, S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st); break;
        case 8: e = launch_k<8>(warp, S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st); break;
        case 16: e = launch_k<16>(warp, S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st); break;
        case 32: e = launch_k<32>(warp, S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st); break;
        default: return IRGS_ERR_UNSUPPORTED;
    }
    if (e == cudaErrorMemoryAllocation) return IRGS_ERR_OOM;
    return e == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

}  // namespace irgs
