// Per-point Monte Carlo estimate of the rendering equation (IRGS Eq. 3, 15)
// with the BRDF of Eq. 4 and the light split of Eq. 13-14, shared by the
// shading kernels (forward and gradient) and the serving kernel. One warp
// shades one point: lanes take samples s = lane, lane + 32, ...; the sums are
// reduced with a fixed butterfly, so a point's result depends only on
// (seed, point key, inputs).
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

// Bilinear equirectangular taps: azimuth atan2(y,x) wraps, polar angle from
// +z clamps; texel centres at ((phi+pi)/2pi W - 0.5, theta/pi H - 0.5).
struct EnvTaps {
    int64_t i00, i01, i10, i11;   // texel indices (row-major [H][W])
    float fx, fy;                 // bilinear fractions
};

__device__ __forceinline__ EnvTaps env_taps(int H, int W, f3 w) {
    const float phi = atan2f(w.y, w.x);
    const float theta = atan2f(sqrtf(w.x * w.x + w.y * w.y), w.z);
    const float x = (phi + kPi) * (0.5f / kPi) * (float)W - 0.5f;
    const float y = theta * (1.0f / kPi) * (float)H - 0.5f;
    const float x0f = floorf(x), y0f = floorf(y);
    EnvTaps t;
    t.fx = x - x0f;
    t.fy = y - y0f;
    int x0 = (int)x0f, y0 = (int)y0f;
    int x1 = x0 + 1, y1 = y0 + 1;
    x0 = ((x0 % W) + W) % W;
    x1 = ((x1 % W) + W) % W;
    y0 = y0 < 0 ? 0 : (y0 > H - 1 ? H - 1 : y0);
    y1 = y1 < 0 ? 0 : (y1 > H - 1 ? H - 1 : y1);
    t.i00 = (int64_t)y0 * W + x0;
    t.i01 = (int64_t)y0 * W + x1;
    t.i10 = (int64_t)y1 * W + x0;
    t.i11 = (int64_t)y1 * W + x1;
    return t;
}

__device__ __forceinline__ f3 env_lookup(const float* __restrict__ env, int H, int W, f3 w) {
    const EnvTaps t = env_taps(H, W, w);
    const float* p00 = env + t.i00 * 3;
    const float* p01 = env + t.i01 * 3;
    const float* p10 = env + t.i10 * 3;
    const float* p11 = env + t.i11 * 3;
    float o[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float top = (1.f - t.fx) * __ldg(p00 + c) + t.fx * __ldg(p01 + c);
        const float bot = (1.f - t.fx) * __ldg(p10 + c) + t.fx * __ldg(p11 + c);
        o[c] = (1.f - t.fy) * top + t.fy * bot;
    }
    return mk3(o[0], o[1], o[2]);
}

// Adds g_c * (bilinear weight) to the four taps of direction w (the
// gradient of env_lookup with respect to the texels).
__device__ __forceinline__ void env_lookup_grad(float* __restrict__ g_env, int H, int W, f3 w, const float (&g)[3]) {
    const EnvTaps t = env_taps(H, W, w);
    const float w00 = (1.f - t.fy) * (1.f - t.fx), w01 = (1.f - t.fy) * t.fx;
    const float w10 = t.fy * (1.f - t.fx), w11 = t.fy * t.fx;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        atomicAdd(g_env + t.i00 * 3 + c, w00 * g[c]);
        atomicAdd(g_env + t.i01 * 3 + c, w01 * g[c]);
        atomicAdd(g_env + t.i10 * 3 + c, w10 * g[c]);
        atomicAdd(g_env + t.i11 * 3 + c, w11 * g[c]);
    }
}

// Estimators of the rendering equation (Eq. 15):
//   split:   cosine-weighted samples for the diffuse lobe and GGX samples of
//            the half vector for the specular lobe, each lobe averaged over
//            its own samples;
//   uniform: stratified uniform hemisphere directions, stratum s of S in
//            cos(theta), 2 pi / S sum (f_d + f_s) L_i (w_i.n).
constexpr int kModeSplit = 0;
constexpr int kModeUniform = 1;

// Shading frame of a point: unit normal flipped towards w_o, the ONB
// around it and the BRDF constants of its roughness.
struct ShadeFrame {
    f3 n, wo, b1, b2;
    float no, rough, alpha_g, a2, kk, G1o;
};

__device__ __forceinline__ ShadeFrame shade_frame(f3 n_in, f3 wo_in, float rough) {
    ShadeFrame F;
    F.n = normalize3(n_in);
    F.wo = normalize3(wo_in);
    F.no = dot3(F.n, F.wo);
    if (F.no <= 0.f) {
        F.n = mul3(F.n, -1.f);
        F.no = -F.no;
    }
    F.rough = rough;
    F.alpha_g = rough * rough;
    F.a2 = F.alpha_g * F.alpha_g;
    F.kk = 0.5f * F.alpha_g;
    F.G1o = F.no / (F.no * (1.f - F.kk) + F.kk);
    onb(F.n, F.b1, F.b2);
    return F;
}

// Incident direction of sample s (of St) of point key p. Split mode:
// s < nd cosine-weighted (diffuse = true), else reflected about a GGX half
// vector (valid = false below the horizon: it adds 0 but still counts).
// Uniform mode: stratified in cos(theta); valid = false on the horizon.
struct ShadeSample {
    f3 wi, h;
    float oh, nh;
    bool valid, diffuse;
};

__device__ __forceinline__ ShadeSample draw_sample(const ShadeFrame& F, int mode, uint64_t p, int s, int St, int nd,
                                                   uint64_t seed) {
    ShadeSample d;
    d.wi = mk3(0.f, 0.f, 1.f);
    d.h = mk3(0.f, 0.f, 1.f);
    d.oh = 0.f;
    d.nh = 0.f;
    d.diffuse = mode == kModeSplit && s < nd;
    d.valid = s < St;
    if (!d.valid) return d;
    const uint64_t i0 = ((uint64_t)p * (uint64_t)St + (uint64_t)s) * 2ull;
    const float u1 = u01_from_bits(splitmix64_at(seed, i0));
    const float u2 = u01_from_bits(splitmix64_at(seed, i0 + 1));
    float sp, cp;
    sincospif(2.f * u2, &sp, &cp);
    if (mode == kModeUniform) {
        const float z = ((float)s + u1) / (float)St;
        const float rr = sqrtf(fmaxf(0.f, (1.f - z) * (1.f + z)));
        d.wi = normalize3(from_local(mk3(rr * cp, rr * sp, z), F.b1, F.b2, F.n));
        d.h = normalize3(add3(d.wi, F.wo));
        d.oh = dot3(F.wo, d.h);
        d.nh = dot3(F.n, d.h);
        d.valid = z > 0.f;
    } else if (d.diffuse) {
        const float r = sqrtf(u1);
        d.wi = normalize3(from_local(mk3(r * cp, r * sp, sqrtf(fmaxf(0.f, 1.f - u1))), F.b1, F.b2, F.n));
    } else {
        // cos^2 = (1 - u1) / den and sin^2 = a2 u1 / den with den = (1 - u1) + a2 u1
        // (1 - u1 is exact): both keep their relative accuracy for a narrow lobe,
        // where 1 - cos^2 would cancel
        const float om = 1.f - u1;
        const float inv_den = 1.f / fmaf(F.a2, u1, om);
        const float ct = sqrtf(om * inv_den), st = sqrtf(F.a2 * u1 * inv_den);
        d.h = normalize3(from_local(mk3(st * cp, st * sp, ct), F.b1, F.b2, F.n));
        d.oh = dot3(F.wo, d.h);
        d.wi = normalize3(sub3(mul3(d.h, 2.f * d.oh), F.wo));
        d.nh = dot3(F.n, d.h);
        d.valid = d.oh > 0.f && dot3(d.wi, F.n) > 0.f;
    }
    return d;
}

// Schlick Fresnel on w_o.h with F0 = 0.04.
__device__ __forceinline__ float fresnel(float oh) {
    const float om = 1.f - oh, om2 = om * om;
    return kF0 + (1.f - kF0) * (om2 * om2 * om);
}

// q = (n.h)^2 (alpha^2 - 1) + 1 of the GGX distribution, written as
// |n x h|^2 + (n.h)^2 alpha^2 so that it keeps its relative accuracy near
// the peak of a narrow lobe.
__device__ __forceinline__ float ggx_q(const ShadeFrame& F, f3 h, float nh) {
    const f3 c = cross3(F.n, h);
    return fmaf(nh * nh, F.a2, dot3(c, c));
}

// d ln(D G1(w_i) G1(w_o)) / d roughness (directions held fixed):
//   d ln D / dr = 4/r - 8 r^3 (n.h)^2 / q,
//   d ln G1(c) / dr = -r (1 - c) / (c (1 - k) + k),  k = r^2 / 2.
__device__ __forceinline__ float dln_spec_dr(const ShadeFrame& F, float q, float nh, float ni) {
    const float r = F.rough;
    const float dD = 4.f / r - 8.f * r * F.alpha_g * nh * nh / q;
    const float dGi = -r * (1.f - ni) / (ni * (1.f - F.kk) + F.kk);
    const float dGo = -r * (1.f - F.no) / (F.no * (1.f - F.kk) + F.kk);
    return dD + dGi + dGo;
}

// Per-sample factor on L_i (channel-independent parts): the estimate adds
// (wa * a_c + ws) * L_i,c for channel c, with d/da_c = wa and d/dr = ws * dln.
struct SampleWeight {
    float wa, ws, dln;
};

__device__ __forceinline__ SampleWeight sample_weight(const ShadeFrame& F, const ShadeSample& d, int mode, int nd,
                                                      int ns, int St, bool want_dln) {
    SampleWeight w;
    w.dln = 0.f;
    const float ni = dot3(F.n, d.wi);
    if (mode == kModeUniform) {
        const float q = ggx_q(F, d.h, d.nh);
        const float D = F.a2 / (kPi * q * q);
        const float G1i = ni / (ni * (1.f - F.kk) + F.kk);
        const float fs_cos = D * fresnel(d.oh) * G1i * F.G1o / (4.f * F.no);   // f_s (w_i.n)
        const float inv = 1.f / (float)St;
        w.wa = 2.f * ni * inv;
        w.ws = 2.f * kPi * fs_cos * inv;
        if (want_dln) w.dln = dln_spec_dr(F, q, d.nh, ni);
    } else if (d.diffuse) {
        w.wa = 1.f / (float)nd;
        w.ws = 0.f;
    } else {
        const float G1i = ni / (ni * (1.f - F.kk) + F.kk);
        w.wa = 0.f;
        w.ws = fresnel(d.oh) * G1i * F.G1o * d.oh / (F.no * d.nh) / (float)ns;
        if (want_dln) w.dln = dln_spec_dr(F, ggx_q(F, d.h, d.nh), d.nh, ni);
    }
    return w;
}

// Gradient of one valid sample's estimate term (directions held fixed),
// given its trace (L_ind = C, visibility V) and the point's upstream g:
// adds g_c w_a L_i,c to ga, sum_c g_c w_s (d ln f_s/dr) L_i,c to gr, the
// bilinear taps of gL_c V to g_env (if not NULL), and returns the upstream
// gradient of the trace: gL_c = g_c (w_a a_c + w_s), gO = -gL.L_dir.
__device__ __forceinline__ void sample_grad(const ShadeFrame& F, const ShadeSample& d, int mode, int nd, int ns,
                                            int St, const float (&av)[3], const float (&g)[3], const float (&C)[3],
                                            float V, const float* __restrict__ env, int H, int W,
                                            float* __restrict__ g_env, float (&ga)[3], float& gr, float (&gL)[3],
                                            float& gO) {
    const f3 Ld = env_lookup(env, H, W, d.wi);
    const float Ldv[3] = {Ld.x, Ld.y, Ld.z};
    const SampleWeight w = sample_weight(F, d, mode, nd, ns, St, true);
    gO = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float Li = V * Ldv[c] + C[c];
        gL[c] = g[c] * (w.wa * av[c] + w.ws);
        ga[c] += g[c] * w.wa * Li;
        gr += g[c] * w.ws * w.dln * Li;
        gO -= gL[c] * Ldv[c];
    }
    if (g_env != nullptr) {
        const float ge[3] = {gL[0] * V, gL[1] * V, gL[2] * V};
        env_lookup_grad(g_env, H, W, d.wi, ge);
    }
}

struct ShadeSums {
    float rgb[3];   // the estimate of Eq. 15
    float vis;      // mean V over the cosine samples (split) or all samples (uniform)
    float ind[3];   // mean L_ind over the same samples
};

// All 32 lanes of a warp call this with the same point; every lane returns
// the point's sums. WARP selects the warp-coherent traversal. With TRACED the
// samples' traces were made beforehand: traced[s] = (L_ind, V) of sample s
// of this point (the same values the march gives), and nothing is traced.
template <int K, bool WARP, bool TRACED = false>
__device__ __forceinline__ void shade_point_warp(const SceneView& S, f3 x, f3 n_in, f3 wo_in, f3 a, float rough,
                                                 uint64_t p, int nd, int ns, int mode, uint64_t seed,
                                                 const float* __restrict__ env, int H, int W, const TraceParams& TP,
                                                 ShadeSums& out, const float4* __restrict__ traced = nullptr) {
    const int lane = threadIdx.x & 31;
    const ShadeFrame F = shade_frame(n_in, wo_in, rough);
    const int St = nd + ns;
    float sd[3] = {0.f, 0.f, 0.f}, ss[3] = {0.f, 0.f, 0.f}, si[3] = {0.f, 0.f, 0.f}, sv = 0.f, cnt = 0.f;
    // lane l takes samples l, l + 32, ...; the trip count is the same for the
    // whole warp so the warp-coherent walk keeps every lane in the loop
    for (int base = 0; base < St; base += 32) {
        const ShadeSample d = draw_sample(F, mode, p, base + lane, St, nd, seed);
        if ((TRACED || !WARP) && !d.valid) continue;
        MarchState<K, 3> st;
        if (TRACED) {
            const float4 t = __ldg(traced + base + lane);
            st.C[0] = t.x;
            st.C[1] = t.y;
            st.C[2] = t.z;
            st.T = t.w;
        } else {
            const Ray ray = make_ray(x, d.wi);
            const bool ok = march_forward<K, 3, WARP>(S, ray, TP, st, nullptr, 0, d.valid);
            if (!d.valid) continue;
            if (!ok) atomicOr(S.status, kErrStackOverflow);
        }
        const float V = st.T;
        const f3 Ld = env_lookup(env, H, W, d.wi);
        const float Li[3] = {V * Ld.x + st.C[0], V * Ld.y + st.C[1], V * Ld.z + st.C[2]};
        const SampleWeight w = sample_weight(F, d, mode, nd, ns, St, false);
        if (mode == kModeUniform) {
            sd[0] += (w.wa * a.x + w.ws) * Li[0];
            sd[1] += (w.wa * a.y + w.ws) * Li[1];
            sd[2] += (w.wa * a.z + w.ws) * Li[2];
        } else if (d.diffuse) {
            sd[0] += a.x * Li[0];
            sd[1] += a.y * Li[1];
            sd[2] += a.z * Li[2];
        } else {
            ss[0] += w.ws * Li[0];
            ss[1] += w.ws * Li[1];
            ss[2] += w.ws * Li[2];
        }
        if (mode == kModeUniform || d.diffuse) {
            si[0] += st.C[0];
            si[1] += st.C[1];
            si[2] += st.C[2];
            sv += V;
            cnt += 1.f;
        }
    }
    float acc[11] = {sd[0], sd[1], sd[2], ss[0], ss[1], ss[2], si[0], si[1], si[2], sv, cnt};
#pragma unroll
    for (int k = 0; k < 11; ++k)
        for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
    const float inv_c = acc[10] > 0.f ? 1.f / acc[10] : 0.f;
    if (mode == kModeUniform) {
        for (int c = 0; c < 3; ++c) out.rgb[c] = acc[c];
    } else {
        const float inv_d = nd > 0 ? 1.f / (float)nd : 0.f;
        for (int c = 0; c < 3; ++c) out.rgb[c] = acc[c] * inv_d + acc[3 + c];
    }
    out.vis = acc[9] * inv_c;
    for (int c = 0; c < 3; ++c) out.ind[c] = acc[6 + c] * inv_c;
}

}  // namespace irgs
