// Per-point Monte Carlo estimate of the rendering equation (IRGS Eq. 3, 15)
// with the BRDF of Eq. 4 and the light split of Eq. 13-14, shared by the
// shading kernel and the serving kernel. One warp shades one point: lanes
// take samples s = lane, lane + 32, ...; the sums are reduced with a fixed
// butterfly, so a point's result depends only on (seed, point key, inputs).
#pragma once

#include <cuda_runtime.h>

#include "trace.cuh"

namespace irgs {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kF0 = 0.04f;

// Orthonormal basis (b1, b2, n) around a unit n (Duff et al. 2017).
__device__ __forceinline__ void onb(f3 n, f3& b1, f3& b2) {
    const float sgn = n.z >= 0.f ? 1.f : -1.f;
    const float a = -1.f / (sgn + n.z);
    const float b = n.x * n.y * a;
    b1 = mk3(1.f + sgn * n.x * n.x * a, sgn * b, -sgn * n.x);
    b2 = mk3(b, sgn + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ f3 from_local(f3 l, f3 b1, f3 b2, f3 n) {
    return add3(add3(mul3(b1, l.x), mul3(b2, l.y)), mul3(n, l.z));
}

// Bilinear equirectangular lookup: azimuth atan2(y,x) wraps, polar angle
// from +z clamps; texel centres at ((phi+pi)/2pi W - 0.5, theta/pi H - 0.5).
__device__ __forceinline__ f3 env_lookup(const float* __restrict__ env, int H, int W, f3 w) {
    const float phi = atan2f(w.y, w.x);
    const float theta = atan2f(sqrtf(w.x * w.x + w.y * w.y), w.z);
    const float x = (phi + kPi) * (0.5f / kPi) * (float)W - 0.5f;
    const float y = theta * (1.0f / kPi) * (float)H - 0.5f;
    const float x0f = floorf(x), y0f = floorf(y);
    const float fx = x - x0f, fy = y - y0f;
    int x0 = (int)x0f, y0 = (int)y0f;
    int x1 = x0 + 1, y1 = y0 + 1;
    x0 = ((x0 % W) + W) % W;
    x1 = ((x1 % W) + W) % W;
    y0 = y0 < 0 ? 0 : (y0 > H - 1 ? H - 1 : y0);
    y1 = y1 < 0 ? 0 : (y1 > H - 1 ? H - 1 : y1);
    const float* p00 = env + ((int64_t)y0 * W + x0) * 3;
    const float* p01 = env + ((int64_t)y0 * W + x1) * 3;
    const float* p10 = env + ((int64_t)y1 * W + x0) * 3;
    const float* p11 = env + ((int64_t)y1 * W + x1) * 3;
    float o[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float top = (1.f - fx) * __ldg(p00 + c) + fx * __ldg(p01 + c);
        const float bot = (1.f - fx) * __ldg(p10 + c) + fx * __ldg(p11 + c);
        o[c] = (1.f - fy) * top + fy * bot;
    }
    return mk3(o[0], o[1], o[2]);
}


struct ShadeSums {
    float rgb[3];   // diffuse mean + specular mean
    float vis;      // mean V over the cosine samples
    float ind[3];   // mean L_ind over the cosine samples
};

// All 32 lanes of a warp call this with the same point; every lane returns
// the point's sums. WARP selects the warp-coherent traversal.
template <int K, bool WARP>
__device__ __forceinline__ void shade_point_warp(const SceneView& S, f3 x, f3 n_in, f3 wo_in, f3 a, float rough,
                                                 uint64_t p, int nd, int ns, uint64_t seed,
                                                 const float* __restrict__ env, int H, int W, const TraceParams& TP,
                                                 ShadeSums& out) {
    const int lane = threadIdx.x & 31;
    f3 n = normalize3(n_in);
    const f3 wo = normalize3(wo_in);
    float no = dot3(n, wo);
    if (no <= 0.f) {
        n = mul3(n, -1.f);
        no = -no;
    }
    const float alpha_g = rough * rough;
    const float a2 = alpha_g * alpha_g;
    const float kk = 0.5f * alpha_g;
    const float G1o = no / (no * (1.f - kk) + kk);
    f3 b1, b2;
    onb(n, b1, b2);
    const int St = nd + ns;
    float sd[3] = {0.f, 0.f, 0.f}, ss[3] = {0.f, 0.f, 0.f}, si[3] = {0.f, 0.f, 0.f}, sv = 0.f;
    // lane l takes samples l, l + 32, ...; the trip count is the same for the
    // whole warp so the warp-coherent walk keeps every lane in the loop
    for (int base = 0; base < St; base += 32) {
        const int s = base + lane;
        const bool diffuse = s < nd;
        bool valid = s < St;
        f3 wi = mk3(0.f, 0.f, 1.f), h = mk3(0.f, 0.f, 1.f);
        float oh = 0.f, nh = 0.f;
        if (valid) {
            const uint64_t i0 = ((uint64_t)p * (uint64_t)St + (uint64_t)s) * 2ull;
            const float u1 = u01_from_bits(splitmix64_at(seed, i0));
            const float u2 = u01_from_bits(splitmix64_at(seed, i0 + 1));
            float sp, cp;
            sincospif(2.f * u2, &sp, &cp);
            if (diffuse) {
                const float r = sqrtf(u1);
                wi = normalize3(from_local(mk3(r * cp, r * sp, sqrtf(fmaxf(0.f, 1.f - u1))), b1, b2, n));
            } else {
                const float c2 = (1.f - u1) / (1.f + (a2 - 1.f) * u1);
                const float ct = sqrtf(c2), st = sqrtf(fmaxf(0.f, 1.f - c2));
                h = normalize3(from_local(mk3(st * cp, st * sp, ct), b1, b2, n));
                oh = dot3(wo, h);
                wi = normalize3(sub3(mul3(h, 2.f * oh), wo));
                nh = dot3(n, h);
                valid = oh > 0.f && dot3(wi, n) > 0.f;   // below the horizon: adds 0
            }
        }
        if (!WARP && !valid) continue;
        const Ray ray = make_ray(x, wi);
        MarchState<K, 3> st;
        const bool ok = march_forward<K, 3, WARP>(S, ray, TP, st, nullptr, 0, valid);
        if (!valid) continue;
        if (!ok) atomicOr(S.status, kErrStackOverflow);
        const float V = st.T;
        const f3 Ld = env_lookup(env, H, W, wi);
        const float Li[3] = {V * Ld.x + st.C[0], V * Ld.y + st.C[1], V * Ld.z + st.C[2]};
        if (diffuse) {
            sd[0] += a.x * Li[0];
            sd[1] += a.y * Li[1];
            sd[2] += a.z * Li[2];
            si[0] += st.C[0];
            si[1] += st.C[1];
            si[2] += st.C[2];
            sv += V;
        } else {
            const float ni = dot3(n, wi);
            const float om = 1.f - oh, om2 = om * om;
            const float Fr = kF0 + (1.f - kF0) * (om2 * om2 * om);
            const float G1i = ni / (ni * (1.f - kk) + kk);
            const float wgt = Fr * G1i * G1o * oh / (no * nh);
            ss[0] += wgt * Li[0];
            ss[1] += wgt * Li[1];
            ss[2] += wgt * Li[2];
        }
    }
    float acc[10] = {sd[0], sd[1], sd[2], ss[0], ss[1], ss[2], si[0], si[1], si[2], sv};
#pragma unroll
    for (int k = 0; k < 10; ++k)
        for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
    const float inv_d = nd > 0 ? 1.f / (float)nd : 0.f;
    const float inv_s = ns > 0 ? 1.f / (float)ns : 0.f;
    for (int c = 0; c < 3; ++c) out.rgb[c] = acc[c] * inv_d + acc[3 + c] * inv_s;
    out.vis = acc[9] * inv_d;
    for (int c = 0; c < 3; ++c) out.ind[c] = acc[6 + c] * inv_d;
}

}  // namespace irgs
