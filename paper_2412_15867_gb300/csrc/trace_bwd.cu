// Backward trace kernels: each ray's hits come from the forward's saved hit
// list or from a replay of its march (trace_bwd.cuh); the surfel gradients
// are accumulated in Morton order and then added into the caller's
// user-order arrays.
#include <cuda_runtime.h>

#include "scene.h"
#include "trace.cuh"
#include "trace_bwd.cuh"

namespace irgs {
namespace {

constexpr int kBwdThreads = 128;

// Which rays a launch handles.
enum BwdMode {
    kReplayAll = 0,    // every ray replays the march (no hit lists)
    kListed = 1,       // rays whose whole hit list was saved; no traversal code
    kReplayLong = 2,   // rays whose hit list did not fit replay the march
};

// Per-ray inputs of the backward (forward outputs and upstream gradients).
template <int FB>
struct RayGrad {
    float gC[FB], Cf[FB];
    float gD, gO, Df, Tfin;
};

template <int FB>
__device__ __forceinline__ void load_ray_grad(RayGrad<FB>& g, int64_t q, const TraceParams& P,
                                              const float* __restrict__ out_feat, const float* __restrict__ out_depth,
                                              const float* __restrict__ out_opac, const float* __restrict__ g_featv,
                                              const float* __restrict__ g_depthv,
                                              const float* __restrict__ g_opacv) {
#pragma unroll
    for (int c = 0; c < FB; ++c) {
        g.gC[c] = c < P.fc ? g_featv[q * P.fc + c] : 0.f;
        g.Cf[c] = c < P.fc ? out_feat[q * P.fc + c] : 0.f;
    }
    g.gD = g_depthv != nullptr ? g_depthv[q] : 0.f;
    g.gO = g_opacv != nullptr ? g_opacv[q] : 0.f;
    g.Df = out_depth[q];
    g.Tfin = 1.0f - out_opac[q];
}

template <int K, int FB, bool WARP, int MODE>
__global__ void __launch_bounds__(kBwdThreads) k_trace_backward(
    SceneView S, const float* __restrict__ ro, const float* __restrict__ rd, int64_t R, TraceParams P,
    const float* __restrict__ out_feat, const float* __restrict__ out_depth, const float* __restrict__ out_opac,
    const int32_t* __restrict__ out_nhits, const int32_t* __restrict__ hit_ids, int max_ids,
    const float* __restrict__ g_featv, const float* __restrict__ g_depthv, const float* __restrict__ g_opacv,
    float* __restrict__ acc_rows) {
    static_assert(kBwdThreads == trace_threads<K>(), "k-buffer slots are laid out per block thread");
    __shared__ float4 rows_all[kBwdThreads * GradRow<FB>::kStride / 4];
    float* rows = reinterpret_cast<float*>(rows_all) + (threadIdx.x & ~31) * GradRow<FB>::kStride;
    const int64_t r = blockIdx.x * (int64_t)kBwdThreads + threadIdx.x;
    if (S.n == 0) return;
    const int nh_total = r < R ? out_nhits[r] : 0;
    const bool mine = nh_total > 0 && (MODE == kReplayAll || (MODE == kListed) == (nh_total <= max_ids));
    if (MODE == kListed || !WARP) {
        if (!mine) return;
    } else if (!__any_sync(kFullWarp, mine)) {
        return;   // the whole warp has nothing to replay
    }
    const int64_t q = mine ? r : 0;   // lanes without work follow the warp with a dummy ray
    const Ray ray = make_ray(mk3(ro[3 * q], ro[3 * q + 1], ro[3 * q + 2]),
                             mk3(rd[3 * q], rd[3 * q + 1], rd[3 * q + 2]));
    RayGrad<FB> g;
    load_ray_grad<FB>(g, q, P, out_feat, out_depth, out_opac, g_featv, g_depthv, g_opacv);
    if (MODE == kListed) {
        listed_backward<FB>(S, ray, P, hit_ids + q * (int64_t)max_ids, nh_total, g.Cf, g.Df, g.Tfin, g.gC, g.gD,
                            g.gO, acc_rows, rows);
    } else {
        const bool ok = march_backward<K, FB, WARP>(S, ray, P, mine, nh_total, g.Cf, g.Df, g.Tfin, g.gC, g.gD, g.gO,
                                                    acc_rows, rows);
        if (mine && !ok) atomicOr(S.status, kErrStackOverflow);
    }
}

// Pointers of one backward call (see irgs_trace_backward).
struct BwdArgs {
    const int32_t* perm;
    const float *ro, *rd;
    int64_t R;
    const float *feat, *depth, *opac;
    const int32_t *nhits, *ids;
    int max_ids;
    const float *gf, *gd, *go;
    float *gm, *gq, *gs, *gop, *gfe;
};

template <int K, int FB, bool WARP>
cudaError_t launch(const SceneView& S, const TraceParams& P, const BwdArgs& a, cudaStream_t st) {
    constexpr int N = GradRow<FB>::N;
    const size_t bytes = sizeof(float) * N * (size_t)(S.n > 0 ? S.n : 1);
    float* acc_rows = nullptr;
    cudaError_t e = scratch_alloc(reinterpret_cast<void**>(&acc_rows), bytes, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(acc_rows, 0, bytes, st);
    if (e == cudaSuccess) {
        const int64_t blocks = (a.R + kBwdThreads - 1) / kBwdThreads;
        const unsigned grid = (unsigned)blocks;
#define IRGS_BWD(MODE)                                                                                  \
    k_trace_backward<K, FB, WARP, MODE><<<grid, kBwdThreads, 0, st>>>(S, a.ro, a.rd, a.R, P, a.feat, a.depth, \
                                                                      a.opac, a.nhits, a.ids, a.max_ids, a.gf, \
                                                                      a.gd, a.go, acc_rows)
        if (a.ids != nullptr) {
            IRGS_BWD(kListed);
            IRGS_BWD(kReplayLong);
            count_launches(1);
        } else {
            IRGS_BWD(kReplayAll);
        }
#undef IRGS_BWD
        if (S.n > 0)
            k_grad_scatter<FB><<<(unsigned)((S.n + 255) / 256), 256, 0, st>>>(a.perm, S.n, acc_rows, P.fc, S.F, P.off,
                                                                             a.gm, a.gq, a.gs, a.gop, a.gfe);
        count_launches(S.n > 0 ? 2 : 1);
        e = cudaGetLastError();
    }
    cudaError_t ef = cudaFreeAsync(acc_rows, st);
    return e != cudaSuccess ? e : ef;
}

template <int K, bool WARP>
cudaError_t launch_f(const SceneView& S, const TraceParams& P, const BwdArgs& a, cudaStream_t st) {
    if (P.fc <= 3) return launch<K, 3, WARP>(S, P, a, st);
    if (P.fc <= 10) return launch<K, 10, WARP>(S, P, a, st);
    return launch<K, 16, WARP>(S, P, a, st);
}

template <int K>
cudaError_t launch_k(bool warp, const SceneView& S, const TraceParams& P, const BwdArgs& a, cudaStream_t st) {
    return warp ? launch_f<K, true>(S, P, a, st) : launch_f<K, false>(S, P, a, st);
}

}  // namespace

irgs_status launch_trace_backward(const SceneView& S, const int32_t* perm, const float* ro, const float* rd, int64_t R,
                                  const irgs_trace_params& p, const float* feat, const float* depth,
                                  const float* opac, const int32_t* nhits, const int32_t* hit_ids,
                                  int32_t max_hit_ids, const float* g_feat, const float* g_depth, const float* g_opac,
                                  float* g_means, float* g_quats, float* g_scales, float* g_opacity,
                                  float* g_features, cudaStream_t st) {
    if (R == 0) return IRGS_OK;
    const TraceParams P = to_params(p);
    const BwdArgs a{perm,  ro,     rd,      R,       feat,     depth,     opac,      nhits,     hit_ids,
                    hit_ids != nullptr ? max_hit_ids : 0, g_feat, g_depth, g_opac, g_means, g_quats, g_scales,
                    g_opacity, g_features};
    const bool warp = (p.flags & IRGS_FLAG_PER_THREAD) == 0u;
    cudaError_t e;
    switch (p.k) {
        case 8: e = launch_k<8>(warp, S, P, a, st); break;
        case 16: e = launch_k<16>(warp, S, P, a, st); break;
        default: return IRGS_ERR_UNSUPPORTED;
    }
    if (e == cudaErrorMemoryAllocation) return IRGS_ERR_OOM;
    return e == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

}  // namespace irgs
