// Backward of one ray's blend (the gradient of Trace, IRGS Eq. 8; the
// tracer is differentiable, Sec. 3.3), shared by the trace backward and the
// shading backward kernels.
//
// For the loss L = g_C.C + g_D D + g_O O and hits j = 0..J-1 in depth order,
// with w_j = T_j alpha_j and v_j = g_C.f_j + g_D tau_j:
//   dL/dalpha_j = T_j v_j - (S_j - g_O T_J) / (1 - alpha_j),
//   S_j = sum_{m>j} w_m v_m = g_C.(C - C_<=j) + g_D (D - D_<=j),
// where C_<=j, D_<=j are the running sums up to and including hit j (the
// suffix comes from the forward's totals minus the replayed prefix). The
// chain then runs alpha -> (o, rho^2) -> (u, v) -> (p - mu, tau) -> (mu, t_u,
// t_v, n, s_u, s_v) -> raw quaternion (Eq. 6-7 and the rotation of the unit
// quaternion). The hits come either from replaying the march (same traversal
// and arithmetic as the forward) or from the hit list the forward saved.
// Per-hit gradients are summed across the lanes of a warp that hold the same
// surfel and added with vector atomics into a Morton-ordered scratch
// accumulator, which k_grad_scatter finally adds into the caller's
// user-order arrays.
#pragma once

#include <cuda_runtime.h>

#include "trace.cuh"

namespace irgs {

// Per-surfel gradient row in the Morton-ordered scratch accumulator (16-byte
// aligned, added with vector atomics), packed without gaps:
//   g_mu.x g_mu.y g_mu.z g_o | g_q.w g_q.x g_q.y g_q.z | g_su g_sv g_f0 g_f1 | g_f2 ...
// (the traced channels follow the scales; the row is padded to a multiple of
// 4 floats: 20 floats = 5 vector atomics at 10 channels)
template <int FB>
struct GradRow {
    static constexpr int N = (10 + FB + 3) / 4 * 4;   // floats per row
    // row stride of the per-warp shared exchange: rows are written and read
    // as float4; an odd number of float4 per row keeps the 8 lanes of each
    // 128-bit shared-memory phase on distinct banks
    static constexpr int kStride = (N / 4) % 2 ? N : N + 4;
    float v[N];
};

// Add row g for Morton slot m: lanes of the warp holding the same slot are
// summed first (match mask + per-lane rows in shared memory; each lane of
// the group sums a share of the row's float4 columns over the group and
// adds them with one float4 atomic each); a lane alone adds its row directly.
template <int FB>
__device__ __forceinline__ void accumulate_row(const GradRow<FB>& g, int32_t m, float* __restrict__ acc_rows,
                                               float* rows /* [32][kStride] this warp, 16-byte aligned */) {
    constexpr int N = GradRow<FB>::N;
    constexpr int S = GradRow<FB>::kStride;
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, m);
    const int lane = threadIdx.x & 31;
    float4* dst = reinterpret_cast<float4*>(acc_rows + (int64_t)m * N);
    if (peers == (1u << lane)) {
#pragma unroll
        for (int q = 0; q < N / 4; ++q)
            atomicAdd(dst + q, make_float4(g.v[4 * q], g.v[4 * q + 1], g.v[4 * q + 2], g.v[4 * q + 3]));
        return;
    }
    float4* mine = reinterpret_cast<float4*>(rows + lane * S);
#pragma unroll
    for (int q = 0; q < N / 4; ++q) mine[q] = make_float4(g.v[4 * q], g.v[4 * q + 1], g.v[4 * q + 2], g.v[4 * q + 3]);
    __syncwarp(peers);
    // the peers split the row's float4 columns: the lane of rank r sums
    // columns r, r + p, ... over the group and adds each with one atomic
    const int p = __popc(peers);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    for (int q = rank; q < N / 4; q += p) {
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
        unsigned rest = peers;
        while (rest) {
            const int l = __ffs(rest) - 1;
            rest &= rest - 1;
            const float4 o = reinterpret_cast<const float4*>(rows + l * S)[q];
            sum.x += o.x;
            sum.y += o.y;
            sum.z += o.z;
            sum.w += o.w;
        }
        atomicAdd(dst + q, sum);
    }
    __syncwarp(peers);
}

// Add the Morton-ordered rows into the caller's user-order gradients
// (each user index is touched by exactly one thread: no atomics).
template <int FB>
__global__ void k_grad_scatter(const int32_t* __restrict__ perm, int64_t n, const float* __restrict__ acc_rows,
                               int fc, int F, int off, float* __restrict__ g_means, float* __restrict__ g_quats,
                               float* __restrict__ g_scales, float* __restrict__ g_opac, float* __restrict__ g_feat) {
    constexpr int N = GradRow<FB>::N;
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= n) return;
    const int64_t u = perm[m];
    const float4* r = reinterpret_cast<const float4*>(acc_rows + m * N);
    const float4 a = r[0], q = r[1];
    const float2 sc = *reinterpret_cast<const float2*>(r + 2);
    g_means[3 * u] += a.x;
    g_means[3 * u + 1] += a.y;
    g_means[3 * u + 2] += a.z;
    g_opac[u] += a.w;
    g_quats[4 * u] += q.x;
    g_quats[4 * u + 1] += q.y;
    g_quats[4 * u + 2] += q.z;
    g_quats[4 * u + 3] += q.w;
    g_scales[2 * u] += sc.x;
    g_scales[2 * u + 1] += sc.y;
    const float* f = acc_rows + m * N + 10;
    for (int c = 0; c < fc; ++c) g_feat[u * F + off + c] += f[c];
}

// Running state of one ray's backward: the blended prefix sums C_<=j, D_<=j
// and the transmittance T_j in front of the next hit.
template <int FB>
struct BwdAcc {
    float C[FB];
    float D, T;
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int c = 0; c < FB; ++c) C[c] = 0.f;
        D = 0.f;
        T = 1.f;
    }
};

// Gradient of the next blended hit, surfel m (Morton slot), given the
// forward's outputs (Cf, Df, Tfin) and the upstream gradients: recomputes
// the hit with the forward's arithmetic (bitwise the same alpha and depth),
// adds its row to the accumulator and advances the running state.
template <int FB>
__device__ __forceinline__ void backward_hit(const SceneView& S, const Ray& ray, const TraceParams& P, int32_t m,
                                             BwdAcc<FB>& st, const float (&Cf)[FB], float Df, float Tfin,
                                             const float (&gC)[FB], float gD, float gO,
                                             float* __restrict__ acc_rows, float* rows) {
    const float4* Rp = S.rec + (int64_t)m * kRecF4;
    const float4 r0 = ldg4(Rp), r1 = ldg4(Rp + 1), r2 = ldg4(Rp + 2), r3 = ldg4(Rp + 3);
    float kh, kl, a;
    HitGeom hg;
    surfel_hit<true>(r0, r1, r2, r3, ray, P.alpha_min, P.alpha_max, kh, kl, a, &hg);
    const float tau = kh + 0.0f;
    const float w = __fmul_rn(st.T, a);
    float fv[FB];
    load_channels<FB>(S.feat + (int64_t)m * S.F + P.off, P.fc, ((S.F | P.off) & 1) == 0, fv);
    float v = __fmul_rn(gD, tau), Sj = 0.f;
#pragma unroll
    for (int c = 0; c < FB; ++c) {
        st.C[c] = c < P.fc ? __fmaf_rn(w, fv[c], st.C[c]) : 0.f;
        v = fmaf(gC[c], fv[c], v);
        Sj = fmaf(gC[c], Cf[c] - st.C[c], Sj);
    }
    st.D = __fmaf_rn(w, tau, st.D);
    Sj = fmaf(gD, Df - st.D, Sj);
    // gradients need no correctly rounded quotients: one 2-ulp reciprocal
    // (__fdividef) per divisor; every divisor here is a normal number
    const float dA = st.T * v - (Sj - gO * Tfin) * __fdividef(1.0f, 1.0f - a);

    const float2 sc = __ldg(&S.scale[m]);
    const float4 q = __ldg(&S.q_raw[m]);
    const float isx = __fdividef(1.0f, sc.x), isy = __fdividef(1.0f, sc.y);
    GradRow<FB> gv;
    const bool clamped = hg.a_raw >= P.alpha_max;
    const float g_o = clamped ? 0.f : dA * hg.G;
    const float g_rho2 = clamped ? 0.f : -0.5f * dA * a;
    const float gu = 2.f * g_rho2 * hg.u, gvv = 2.f * g_rho2 * hg.v;
    const f3 tus = mk3(r1.x, r1.y, r1.z), tvs = mk3(r2.x, r2.y, r2.z), nn = mk3(r3.x, r3.y, r3.z);
    const f3 ge = add3(mul3(tus, gu), mul3(tvs, gvv));
    const float gtau = w * gD + dot3(ge, ray.d);
    const float s_t = gtau * __fdividef(1.0f, hg.den);
    const f3 gmu = sub3(mul3(nn, s_t), ge);
    const f3 gn = mul3(hg.e, -s_t);
    const f3 gtu = mul3(hg.e, gu * isx);
    const f3 gtv = mul3(hg.e, gvv * isy);
    // raw quaternion: derivative of the rotation columns, then of q / |q|
    const float iqn = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float qw = q.x * iqn, qx = q.y * iqn, qy = q.z * iqn, qz = q.w * iqn;
    const float hw = 2.f * (qz * gtu.y - qy * gtu.z - qz * gtv.x + qx * gtv.z + qy * gn.x - qx * gn.y);
    const float hx = 2.f * (qy * gtu.y + qz * gtu.z + qy * gtv.x - 2.f * qx * gtv.y + qw * gtv.z + qz * gn.x -
                            qw * gn.y - 2.f * qx * gn.z);
    const float hy = 2.f * (-2.f * qy * gtu.x + qx * gtu.y - qw * gtu.z + qx * gtv.x + qz * gtv.z + qw * gn.x +
                            qz * gn.y - 2.f * qy * gn.z);
    const float hz = 2.f * (-2.f * qz * gtu.x + qw * gtu.y + qx * gtu.z - qw * gtv.x - 2.f * qz * gtv.y +
                            qy * gtv.z + qx * gn.x + qy * gn.y);
    const float proj = qw * hw + qx * hx + qy * hy + qz * hz;
    gv.v[0] = gmu.x; gv.v[1] = gmu.y; gv.v[2] = gmu.z;
    gv.v[3] = g_o;
    gv.v[4] = (hw - qw * proj) * iqn;
    gv.v[5] = (hx - qx * proj) * iqn;
    gv.v[6] = (hy - qy * proj) * iqn;
    gv.v[7] = (hz - qz * proj) * iqn;
    gv.v[8] = -gu * hg.u * isx;
    gv.v[9] = -gvv * hg.v * isy;
#pragma unroll
    for (int c = 0; c < GradRow<FB>::N - 10; ++c) gv.v[10 + c] = c < FB ? w * gC[c] : 0.f;
    accumulate_row<FB>(gv, m, acc_rows, rows);
    st.T = __fmul_rn(st.T, __fsub_rn(1.0f, a));
}

// Replay of one ray (all 32 lanes together when WARP): the march is repeated
// with the same traversal and arithmetic as the forward, capped at nh_total
// composited hits; Cf, Df, Tfin are the forward's outputs and gC, gD, gO the
// upstream gradients. rows is this warp's [32][N+1] shared scratch. Returns
// false if a traversal stack overflowed.
template <int K, int FB, bool WARP>
__device__ __forceinline__ bool march_backward(const SceneView& S, const Ray& ray, const TraceParams& P, bool live,
                                               int nh_total, const float (&Cf)[FB], float Df, float Tfin,
                                               const float (&gC)[FB], float gD, float gO,
                                               float* __restrict__ acc_rows, float* rows) {
    BwdAcc<FB> st;
    st.init();
    int nh = 0;
    uint64_t last_key = depth_key(P.t_min, 0.f);
    int32_t last_u = INT32_MAX;
    KBuffer<K, trace_threads<K>()> kb;
    kb.bind();
    bool ok = true, done = !live;
    while (WARP ? __any_sync(kFullWarp, !done) : !done) {
        if (WARP)
            ok &= collect_round_warp(S, ray, P, last_key, last_u, kb, !done);
        else
            ok &= collect_round(S, ray, P, last_key, last_u, kb);
        if (done) continue;
        for (int j = 0; j < kb.cnt && nh < nh_total; ++j, ++nh)
            backward_hit<FB>(S, ray, P, kb.m_at(j), st, Cf, Df, Tfin, gC, gD, gO, acc_rows, rows);
        if (nh >= nh_total || kb.cnt < K) {
            done = true;
        } else {
            last_key = kb.tail_key;
            last_u = uid_of(S.rec, kb.tail_m);
        }
    }
    return ok;
}

// Backward from the forward's saved hit list (user indices in blend order,
// as irgs_trace_forward writes them): no traversal.
template <int FB>
__device__ __forceinline__ void listed_backward(const SceneView& S, const Ray& ray, const TraceParams& P,
                                                const int32_t* __restrict__ ids, int nh_total, const float (&Cf)[FB],
                                                float Df, float Tfin, const float (&gC)[FB], float gD, float gO,
                                                float* __restrict__ acc_rows, float* rows) {
    BwdAcc<FB> st;
    st.init();
    if (nh_total <= 0) return;
    // The lookups run ahead of the hit being processed: the id of hit j + 2
    // and the Morton slot of hit j + 1 are in flight while hit j is. An id
    // outside [0, n) is not a list the forward wrote for this scene: the hits
    // before it are processed, then the ray stops with an error bit.
    int32_t u = __ldg(ids);
    if (u < 0 || u >= S.n) {
        atomicOr(S.status, kErrBadHitList);
        return;
    }
    int32_t m_next = __ldg(&S.inv_perm[u]);
    u = nh_total > 1 ? __ldg(ids + 1) : 0;
    for (int j = 0; j < nh_total; ++j) {
        const int32_t m = m_next;
        bool bad = false;
        if (j + 1 < nh_total) {
            if (u < 0 || u >= S.n) bad = true;
            else m_next = __ldg(&S.inv_perm[u]);
        }
        u = j + 2 < nh_total ? __ldg(ids + j + 2) : 0;
        backward_hit<FB>(S, ray, P, m, st, Cf, Df, Tfin, gC, gD, gO, acc_rows, rows);
        if (bad) {
            atomicOr(S.status, kErrBadHitList);
            return;
        }
    }
}

}  // namespace irgs
