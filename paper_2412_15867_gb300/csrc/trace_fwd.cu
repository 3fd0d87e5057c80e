// Forward trace kernel: one thread per ray, Trace(r_o, r_d) of IRGS Eq. 8.
#include <cuda_runtime.h>

#include "scene.h"
#include "trace.cuh"

namespace irgs {
namespace {

constexpr int kFwdThreads = 128;

template <int K, int FB>
__global__ void __launch_bounds__(kFwdThreads) k_trace_forward(SceneView S, const float* __restrict__ ro,
                                                               const float* __restrict__ rd, int64_t R,
                                                               TraceParams P, float* __restrict__ feat,
                                                               float* __restrict__ depth, float* __restrict__ opac,
                                                               int32_t* __restrict__ nhits, int32_t* __restrict__ ids,
                                                               int max_ids) {
    const int64_t r = blockIdx.x * (int64_t)kFwdThreads + threadIdx.x;
    if (r >= R) return;
    const Ray ray = make_ray(mk3(ro[3 * r], ro[3 * r + 1], ro[3 * r + 2]),
                             mk3(rd[3 * r], rd[3 * r + 1], rd[3 * r + 2]));
    int32_t* my_ids = nullptr;
    if (ids != nullptr) {
        my_ids = ids + r * (int64_t)max_ids;
        for (int j = 0; j < max_ids; ++j) my_ids[j] = -1;
    }
    MarchState<K, FB> st;
    const bool ok = march_forward<K, FB>(S, ray, P, st, my_ids, max_ids);
    if (!ok) atomicOr(S.status, kErrStackOverflow);
#pragma unroll
    for (int c = 0; c < FB; ++c)
        if (c < P.fc) feat[r * P.fc + c] = st.C[c];
    depth[r] = st.D;
    opac[r] = 1.0f - st.T;
    if (nhits != nullptr) nhits[r] = st.nh;
}

template <int K, int FB>
cudaError_t launch(const SceneView& S, const float* ro, const float* rd, int64_t R, const TraceParams& P,
                   float* feat, float* depth, float* opac, int32_t* nhits, int32_t* ids, int max_ids,
                   cudaStream_t st) {
    const int64_t blocks = (R + kFwdThreads - 1) / kFwdThreads;
    k_trace_forward<K, FB><<<(unsigned)blocks, kFwdThreads, 0, st>>>(S, ro, rd, R, P, feat, depth, opac, nhits,
                                                                     ids, max_ids);
    count_launches(1);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_f(const SceneView& S, const float* ro, const float* rd, int64_t R, const TraceParams& P,
                     float* feat, float* depth, float* opac, int32_t* nhits, int32_t* ids, int max_ids,
                     cudaStream_t st) {
    if (P.fc <= 3) return launch<K, 3>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st);
    if (P.fc <= 10) return launch<K, 10>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st);
    return launch<K, 16>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st);
}

}  // namespace

irgs_status launch_trace_forward(const SceneView& S, const float* ro, const float* rd, int64_t R,
                                 const irgs_trace_params& p, float* feat, float* depth, float* opac,
                                 int32_t* nhits, int32_t* ids, int32_t max_ids, cudaStream_t st) {
    if (R == 0) return IRGS_OK;
    const TraceParams P = to_params(p);
    cudaError_t e;
    switch (p.k) {
        case 1: e = launch_f<1>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st); break;
        case 4: e = launch_f<4>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st); break;
        case 8: e = launch_f<8>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st); break;
        case 16: e = launch_f<16>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st); break;
        case 32: e = launch_f<32>(S, ro, rd, R, P, feat, depth, opac, nhits, ids, max_ids, st); break;
        default: return IRGS_ERR_UNSUPPORTED;
    }
    return e == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

}  // namespace irgs
