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

template <int K, int FB, bool WARP>
cudaError_t launch(const SceneView& S, const float* ro, const float* rd, int64_t R, const TraceParams& P,
                   float* feat, float* depth, float* opac, int32_t* nhits, int32_t* ids, int max_ids,
                   cudaStream_t st) {
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
    return e == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

}  // namespace irgs
