// Relighting query (IRGS supplementary "Relighting details", Eq. 18; Sec. 4,
// relighting paragraph).
//
// Under a new environment the surfels' optimised radiance no longer holds,
// so each incident ray instead blends the albedo, roughness and normal of
// the surfels it crosses (normalised blend weights) and that aggregate
// surface is shaded with pre-integrated maps of the environment:
//   L_ind = O (A_r Irr(N_r) + Pref(reflect(v, N_r), R_r) (F0 A + B)(N_r.v, R_r)),
// O = 1 - V the ray's opacity, v = -w_i, Irr the diffuse irradiance map,
// Pref the split-sum prefiltered radiance and (A, B) the split-sum BRDF
// table. Incident directions are drawn by importance sampling the
// environment's intensity. Pre-integration (once per environment):
//   irradiance  Irr(N) = 1/pi sum_t E_t max(0, w_t.N) dOmega_t      [32 x 64]
//   prefilter   Pref_l(R) = sum_t E_t D_l(R.h_t) (w_t.R)+ dOmega_t / sum_t D_l (w_t.R)+ dOmega_t,
//               roughness l/5, l = 1..5                               [64 x 128 each]
//   BRDF table  A, B over (n.v, roughness) cell centres, 1024 Hammersley
//               GGX half vectors per cell                             [32 x 32]
//   sampling    row and per-row column cdfs of lum(E) sin(theta_row), FP64
// over all environment texels t (centre direction w_t, exact band solid
// angle dOmega_t). One block per output texel sums the environment with a
// fixed order, so the maps are deterministic.
#include <cuda_runtime.h>

#include <new>

#include "scene.h"
#include "shade.cuh"
#include "trace.cuh"
#include "wave.cuh"

namespace irgs {
namespace {

constexpr int kIrrH = IRGS_RELIGHT_IRR_H, kIrrW = IRGS_RELIGHT_IRR_W;
constexpr int kLevels = IRGS_RELIGHT_LEVELS;
constexpr int kPrefH = IRGS_RELIGHT_PREF_H, kPrefW = IRGS_RELIGHT_PREF_W;
constexpr int kLutN = IRGS_RELIGHT_LUT_N;
constexpr int kLutSamples = 1024;
constexpr int kReduceThreads = 256;
constexpr int kRelightThreads = 128;

// Centre direction of texel (row, col) of an h x w equirect map.
__device__ __forceinline__ f3 texel_dir(int h, int w, int row, int col) {
    float st, ct, sp, cp;
    sincospif(((float)row + 0.5f) / (float)h, &st, &ct);
    sincospif(((float)col + 0.5f) * 2.f / (float)w - 1.f, &sp, &cp);
    return mk3(st * cp, st * sp, ct);
}

// Solid angle of a texel of `row`: (cos t0 - cos t1) 2 pi / W written as
// 2 sin((t0 + t1)/2) sin((t1 - t0)/2) 2 pi / W (no cancellation at the poles).
__device__ __forceinline__ float texel_solid_angle(int H, int W, int row) {
    const float m = sinpif(((float)row + 0.5f) / (float)H);
    const float h = sinpif(0.5f / (float)H);
    return 2.f * m * h * 2.f * kPi / (float)W;
}

template <int N>
__device__ __forceinline__ void block_sum(float (&v)[N]) {
    __shared__ float part[N][kReduceThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k)
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if (lane == 0)
        for (int k = 0; k < N; ++k) part[k][warp] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < N; ++k) {
            float s = 0.f;
            for (int w = 0; w < kReduceThreads / 32; ++w) s += part[k][w];
            v[k] = s;
        }
}

// One block per irradiance texel.
__global__ void __launch_bounds__(kReduceThreads) k_irradiance(const float* __restrict__ env, int H, int W,
                                                               float* __restrict__ irr) {
    const int i = blockIdx.x;
    const f3 N = texel_dir(kIrrH, kIrrW, i / kIrrW, i % kIrrW);
    float acc[3] = {0.f, 0.f, 0.f};
    for (int t = threadIdx.x; t < H * W; t += kReduceThreads) {
        const int r = t / W, c = t - r * W;
        const float cs = dot3(texel_dir(H, W, r, c), N);
        if (cs <= 0.f) continue;
        const float wgt = cs * texel_solid_angle(H, W, r);
        const float* e = env + (int64_t)t * 3;
        acc[0] = fmaf(e[0], wgt, acc[0]);
        acc[1] = fmaf(e[1], wgt, acc[1]);
        acc[2] = fmaf(e[2], wgt, acc[2]);
    }
    block_sum<3>(acc);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) irr[(int64_t)i * 3 + k] = acc[k] * (1.f / kPi);
}

// One block per texel of prefilter levels 1 .. kLevels - 1.
__global__ void __launch_bounds__(kReduceThreads) k_prefilter(const float* __restrict__ env, int H, int W,
                                                              float* __restrict__ pref) {
    const int per_level = kPrefH * kPrefW;
    const int level = 1 + blockIdx.x / per_level;
    const int i = blockIdx.x % per_level;
    const float rho = (float)level / (float)(kLevels - 1);
    const float a2 = rho * rho * rho * rho;
    const f3 R = texel_dir(kPrefH, kPrefW, i / kPrefW, i % kPrefW);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t = threadIdx.x; t < H * W; t += kReduceThreads) {
        const int r = t / W, c = t - r * W;
        const f3 w = texel_dir(H, W, r, c);
        const float cs = dot3(w, R);
        if (cs <= 0.f) continue;
        const f3 h = normalize3(add3(w, R));
        const float nh = dot3(R, h);
        const f3 x = cross3(R, h);
        const float q = fmaf(nh * nh, a2, dot3(x, x));   // (n.h)^2 (a2 - 1) + 1 without cancellation
        const float wgt = a2 / (kPi * q * q) * cs * texel_solid_angle(H, W, r);
        const float* e = env + (int64_t)t * 3;
        acc[0] = fmaf(e[0], wgt, acc[0]);
        acc[1] = fmaf(e[1], wgt, acc[1]);
        acc[2] = fmaf(e[2], wgt, acc[2]);
        acc[3] += wgt;
    }
    block_sum<4>(acc);
    if (threadIdx.x == 0) {
        float* o = pref + ((int64_t)(level - 1) * per_level + i) * 3;
        for (int k = 0; k < 3; ++k) o[k] = acc[3] > 0.f ? acc[k] / acc[3] : 0.f;
    }
}

// One thread per table cell.
__global__ void k_brdf_table(float* __restrict__ lut) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= kLutN * kLutN) return;
    const int i = cell / kLutN, j = cell % kLutN;
    const float mu = ((float)i + 0.5f) / (float)kLutN, rho = ((float)j + 0.5f) / (float)kLutN;
    const float ag = rho * rho, a2 = ag * ag, kk = 0.5f * ag;
    const f3 v = mk3(sqrtf(1.f - mu * mu), 0.f, mu);
    float A = 0.f, B = 0.f;
    for (int s = 0; s < kLutSamples; ++s) {
        const float u1 = ((float)s + 0.5f) / (float)kLutSamples;
        const float u2 = (float)__brev((unsigned)s) * 2.3283064365386963e-10f;   // radical inverse, base 2
        const float om = 1.f - u1;
        const float inv = 1.f / fmaf(a2, u1, om);
        const float ct = sqrtf(om * inv), st = sqrtf(a2 * u1 * inv);
        float sp, cp;
        sincospif(2.f * u2, &sp, &cp);
        const f3 h = mk3(st * cp, st * sp, ct);
        const float vh = dot3(v, h);
        const float lz = 2.f * vh * h.z - v.z;
        if (lz <= 0.f || vh <= 0.f) continue;
        const float G = (lz / (lz * (1.f - kk) + kk)) * (mu / (mu * (1.f - kk) + kk));
        const float gv = G * vh / (h.z * mu);
        const float om5 = 1.f - vh, om52 = om5 * om5;
        const float fc = om52 * om52 * om5;
        A += (1.f - fc) * gv;
        B += fc * gv;
    }
    lut[cell * 2] = A / (float)kLutSamples;
    lut[cell * 2 + 1] = B / (float)kLutSamples;
}

// Importance-sampling tables, FP64, sequential in row-major order (the sums
// are deterministic): one thread per row for the column cdfs, then one
// thread for the row cdf.
__global__ void k_env_col_cdf(const float* __restrict__ env, int H, int W, double* __restrict__ col_cdf) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    const double s = sin(((double)r + 0.5) * 3.14159265358979323846 / (double)H);
    double* cc = col_cdf + (int64_t)r * (W + 1);
    double run = 0.0;
    cc[0] = 0.0;
    for (int c = 0; c < W; ++c) {
        const float* e = env + ((int64_t)r * W + c) * 3;
        const double lum = __dadd_rn(__dadd_rn(__dmul_rn(0.2126, (double)e[0]), __dmul_rn(0.7152, (double)e[1])),
                                     __dmul_rn(0.0722, (double)e[2]));
        run = __dadd_rn(run, __dmul_rn(lum, s));
        cc[c + 1] = run;
    }
}

__global__ void k_env_row_cdf(const double* __restrict__ col_cdf, int H, int W, double* __restrict__ row_cdf) {
    double run = 0.0;
    row_cdf[0] = 0.0;
    for (int r = 0; r < H; ++r) {
        run = __dadd_rn(run, col_cdf[(int64_t)r * (W + 1) + W]);
        row_cdf[r + 1] = run;
    }
}

// Largest k in [0, n) with cdf[k] <= t (cdf[0] <= t < cdf[n]).
__device__ __forceinline__ int cdf_find(const double* __restrict__ cdf, int n, double t) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cdf[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// Environment sample from (u1, u2) (row, then column within the row; the
// leftover fractions place the direction inside the texel). Returns false
// if the environment has no weight.
__device__ __forceinline__ bool env_sample(const double* __restrict__ row_cdf, const double* __restrict__ col_cdf,
                                           int H, int W, double u1, double u2, f3& w, float& pdf) {
    const double total = row_cdf[H];
    if (!(total > 0.0)) return false;
    const double t1 = u1 * total;
    const int r = cdf_find(row_cdf, H, t1);
    const double* cc = col_cdf + (int64_t)r * (W + 1);
    const double rw = cc[W];
    const double fv = (t1 - row_cdf[r]) / rw;
    const double t2 = u2 * rw;
    const int c = cdf_find(cc, W, t2);
    const double wt = cc[c + 1] - cc[c];
    const double fu = (t2 - cc[c]) / wt;
    double st, ct, sp, cp;
    sincospi(((double)r + fv) / (double)H, &st, &ct);
    sincospi(((double)c + fu) * 2.0 / (double)W - 1.0, &sp, &cp);
    w = mk3((float)(st * cp), (float)(st * sp), (float)ct);
    pdf = st > 0.0 ? (float)((wt / total) * (double)W * (double)H / (2.0 * 3.14159265358979323846 *
                                                                       3.14159265358979323846 * st))
                   : 0.f;
    return pdf > 0.f;
}

struct EnvMaps {
    const float *env, *irr, *pref, *lut;
    const double *row_cdf, *col_cdf;
    int H, W;
};

// Split-sum prefiltered radiance at roughness rho: linear between the two
// nearest levels (level 0 is the environment).
__device__ __forceinline__ f3 pref_lookup(const EnvMaps& M, f3 d, float rho) {
    rho = fminf(fmaxf(rho, 0.f), 1.f);
    const float t = rho * (float)(kLevels - 1);
    int l0 = (int)floorf(t);
    l0 = l0 > kLevels - 2 ? kLevels - 2 : l0;
    const float f = t - (float)l0;
    const f3 a = l0 == 0 ? env_lookup(M.env, M.H, M.W, d)
                         : env_lookup(M.pref + (int64_t)(l0 - 1) * kPrefH * kPrefW * 3, kPrefH, kPrefW, d);
    const f3 b = env_lookup(M.pref + (int64_t)l0 * kPrefH * kPrefW * 3, kPrefH, kPrefW, d);
    return add3(mul3(a, 1.f - f), mul3(b, f));
}

// Bilinear lookup of the BRDF table at (mu, rho), coordinates clamped to the
// cell centres.
__device__ __forceinline__ float2 lut_lookup(const float* __restrict__ lut, float mu, float rho) {
    const float x = fminf(fmaxf(mu * kLutN - 0.5f, 0.f), (float)(kLutN - 1));
    const float y = fminf(fmaxf(rho * kLutN - 0.5f, 0.f), (float)(kLutN - 1));
    int i0 = (int)floorf(x), j0 = (int)floorf(y);
    i0 = i0 > kLutN - 2 ? kLutN - 2 : i0;
    j0 = j0 > kLutN - 2 ? kLutN - 2 : j0;
    const float fx = x - (float)i0, fy = y - (float)j0;
    const float2* L = reinterpret_cast<const float2*>(lut);
    const float2 a = __ldg(L + i0 * kLutN + j0), b = __ldg(L + i0 * kLutN + j0 + 1);
    const float2 c = __ldg(L + (i0 + 1) * kLutN + j0), d = __ldg(L + (i0 + 1) * kLutN + j0 + 1);
    return make_float2((1.f - fx) * ((1.f - fy) * a.x + fy * b.x) + fx * ((1.f - fy) * c.x + fy * d.x),
                       (1.f - fx) * ((1.f - fy) * a.y + fy * b.y) + fx * ((1.f - fy) * c.y + fy * d.y));
}

__device__ __forceinline__ f3 ld3r(const float* p, int64_t i) { return mk3(p[3 * i], p[3 * i + 1], p[3 * i + 2]); }

// One environment sample w (density pdf) of a point, given its trace (the
// blended [albedo, roughness, normal] C and transmittance T): adds the
// estimate term f L_i (w.n) / pdf to acc[0..2], V to acc[3] and L_ind to
// acc[4..6].
__device__ __forceinline__ void relight_sample(const EnvMaps& M, const ShadeFrame& F, f3 a, f3 w, float pdf,
                                               const float (&C)[7], float T, float (&acc)[7]) {
    const float V = T, O = 1.f - T;
    f3 Lind = mk3(0.f, 0.f, 0.f);
    if (O > 0.f) {
        const f3 Ar = mul3(mk3(C[0], C[1], C[2]), 1.f / O);
        const float Rr = C[3] / O;
        const f3 v = mul3(w, -1.f);
        f3 Nr = mk3(C[4], C[5], C[6]);
        const float len2 = dot3(Nr, Nr);
        Nr = len2 > 1e-24f ? mul3(Nr, rsqrtf(len2)) : v;
        if (dot3(Nr, v) < 0.f) Nr = mul3(Nr, -1.f);
        const float mu = fminf(dot3(Nr, v), 1.f);
        const f3 refl = sub3(mul3(Nr, 2.f * mu), v);
        const f3 irr = env_lookup(M.irr, kIrrH, kIrrW, Nr);
        const f3 pf = pref_lookup(M, refl, Rr);
        const float2 AB = lut_lookup(M.lut, mu, Rr);
        const float spec = kF0 * AB.x + AB.y;
        Lind = mul3(add3(mk3(Ar.x * irr.x, Ar.y * irr.y, Ar.z * irr.z), mul3(pf, spec)), O);
    }
    acc[3] += V;
    acc[4] += Lind.x;
    acc[5] += Lind.y;
    acc[6] += Lind.z;
    const float ni = dot3(F.n, w);
    if (ni <= 0.f) return;
    const f3 h = normalize3(add3(w, F.wo));
    const float nh = dot3(F.n, h), oh = dot3(F.wo, h);
    const float q = ggx_q(F, h, nh);
    const float D = F.a2 / (kPi * q * q);
    const float G1i = ni / (ni * (1.f - F.kk) + F.kk);
    const float fs_cos = D * fresnel(oh) * G1i * F.G1o / (4.f * F.no);   // f_s (w.n)
    const f3 E = env_lookup(M.env, M.H, M.W, w);
    const float Li[3] = {V * E.x + Lind.x, V * E.y + Lind.y, V * E.z + Lind.z};
    const float av[3] = {a.x, a.y, a.z};
    const float inv_pdf = 1.f / pdf;
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] += (av[c] * (1.f / kPi) * ni + fs_cos) * Li[c] * inv_pdf;
}

// Final per-point sums of a warp (fixed butterfly order).
__device__ __forceinline__ void relight_write(float (&acc)[7], int lane, int64_t p, int Sn, float* __restrict__ rgb,
                                              float* __restrict__ vis, float* __restrict__ ind) {
#pragma unroll
    for (int k = 0; k < 7; ++k)
        for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
    if (lane == 0) {
        const float inv = 1.f / (float)Sn;
        for (int c = 0; c < 3; ++c) rgb[3 * p + c] = acc[c] * inv;
        if (vis != nullptr) vis[p] = acc[3] * inv;
        if (ind != nullptr)
            for (int c = 0; c < 3; ++c) ind[3 * p + c] = acc[4 + c] * inv;
    }
}

// Environment sample s of point p (uniforms as in the shading estimate).
__device__ __forceinline__ bool relight_dir(const EnvMaps& M, int64_t p, int s, int Sn, uint64_t seed, f3& w,
                                            float& pdf) {
    const uint64_t i0 = ((uint64_t)p * (uint64_t)Sn + (uint64_t)s) * 2ull;
    const double u1 = (double)u01_from_bits(splitmix64_at(seed, i0));
    const double u2 = (double)u01_from_bits(splitmix64_at(seed, i0 + 1));
    return env_sample(M.row_cdf, M.col_cdf, M.H, M.W, u1, u2, w, pdf);
}

// One warp per point; lanes take samples s = lane, lane + 32, ...; the traced
// channels are [albedo (3), roughness, normal (3)].
template <int K>
__global__ void __launch_bounds__(kRelightThreads) k_relight(SceneView S, EnvMaps M, const float* __restrict__ xg,
                                                             const float* __restrict__ ng,
                                                             const float* __restrict__ ag,
                                                             const float* __restrict__ rg,
                                                             const float* __restrict__ wog, int64_t Pn, int Sn,
                                                             uint64_t seed, TraceParams TP, float* __restrict__ rgb,
                                                             float* __restrict__ vis, float* __restrict__ ind) {
    static_assert(kRelightThreads == trace_threads<K>(), "k-buffer slots are laid out per block thread");
    const int lane = threadIdx.x & 31;
    const int64_t p = blockIdx.x * (int64_t)(kRelightThreads / 32) + (threadIdx.x >> 5);
    if (p >= Pn) return;
    const f3 x = ld3r(xg, p), a = ld3r(ag, p);
    const ShadeFrame F = shade_frame(ld3r(ng, p), ld3r(wog, p), rg[p]);
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // rgb, V, L_ind
    for (int s = lane; s < Sn; s += 32) {
        f3 w;
        float pdf;
        if (!relight_dir(M, p, s, Sn, seed, w, pdf)) continue;
        MarchState<K, 7> st;
        const bool ok = march_forward<K, 7, false>(S, make_ray(x, w), TP, st, nullptr, 0, true);
        if (!ok) atomicOr(S.status, kErrStackOverflow);
        relight_sample(M, F, a, w, pdf, st.C, st.T, acc);
    }
    relight_write(acc, lane, p, Sn, rgb, vis, ind);
}

// Wavefront form: samples generated one thread each, regrouped by direction
// bin and origin, traced in that order with one stack per ray, then
// estimated per point from the stored traces with the same per-sample
// arithmetic and reduction order as k_relight.
__global__ void k_relight_gen(EnvMaps M, const float* __restrict__ xg, int64_t p0, int64_t rays, int Sn,
                              uint64_t seed, const uint32_t* __restrict__ bounds, float4* __restrict__ dir,
                              uint32_t* __restrict__ key, int32_t* __restrict__ val) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rays) return;
    const int64_t p = p0 + i / Sn;
    f3 w = mk3(0.f, 0.f, 1.f);
    float pdf = 0.f;
    const bool ok = relight_dir(M, p, (int)(i % Sn), Sn, seed, w, pdf);
    dir[i] = make_float4(w.x, w.y, w.z, ok ? pdf : 0.f);
    key[i] = ok ? wave_key(ld3r(xg, p), w, bounds) : kInvalidWaveKey;
    val[i] = (int32_t)i;
}

template <int K>
__global__ void __launch_bounds__(kRelightThreads, 6) k_relight_trace(SceneView S, TraceParams P,
                                                                      const float* __restrict__ xg, int64_t p0,
                                                                      int Sn, const float4* __restrict__ dir,
                                                                      const int32_t* __restrict__ order,
                                                                      int64_t rays, float4* __restrict__ res) {
    static_assert(kRelightThreads == trace_threads<K>(), "k-buffer slots are laid out per block thread");
    const int64_t j = blockIdx.x * (int64_t)kRelightThreads + threadIdx.x;
    if (j >= rays) return;
    const int64_t i = order[j];
    const float4 d4 = dir[i];
    MarchState<K, 7> st;
    if (d4.w > 0.f) {
        const bool ok = march_forward<K, 7, false>(S, make_ray(ld3r(xg, p0 + i / Sn), mk3(d4.x, d4.y, d4.z)), P,
                                                   st, nullptr, 0, true);
        if (!ok) atomicOr(S.status, kErrStackOverflow);
    } else {
#pragma unroll
        for (int c = 0; c < 7; ++c) st.C[c] = 0.f;
        st.T = 1.f;
    }
    res[2 * i] = make_float4(st.C[0], st.C[1], st.C[2], st.C[3]);
    res[2 * i + 1] = make_float4(st.C[4], st.C[5], st.C[6], st.T);
}

// The same traces in compacted rounds: round 1 on every sorted ray; rays
// still marching store their state (C[7], D, T, hit count, next key) at
// their sorted position and are regrouped, in sorted order, for rounds 2
// and 3; the rest run to completion. Per ray the rounds and their
// arithmetic are march_forward's (per lane), so the results are the same.
enum RelightRound { kRelFirst = 0, kRelNext = 1, kRelLast = 2 };
constexpr int kRelightStateF4 = 4;

template <int K, int MODE>
__global__ void __launch_bounds__(kRelightThreads, 6) k_relight_round(
    SceneView S, TraceParams P, const float* __restrict__ xg, int64_t p0, int Sn, const float4* __restrict__ dir,
    const int32_t* __restrict__ order, int64_t rays, float4* __restrict__ res, const int32_t* __restrict__ list,
    const uint32_t* __restrict__ count, float4* __restrict__ state, uint32_t* __restrict__ flags) {
    static_assert(kRelightThreads == trace_threads<K>(), "k-buffer slots are laid out per block thread");
    const int64_t t = blockIdx.x * (int64_t)kRelightThreads + threadIdx.x;
    const int64_t n = MODE == kRelFirst ? rays : (int64_t)*count;
    if (t >= n) return;
    const int64_t j = MODE == kRelFirst ? t : (int64_t)list[t];
    const int64_t i = order[j];
    const float4 d4 = dir[i];
    MarchState<K, 7> st;
    uint64_t last_key = depth_key(P.t_min, 0.f);
    int32_t last_u = INT32_MAX;
    if (MODE == kRelFirst) {
#pragma unroll
        for (int c = 0; c < 7; ++c) st.C[c] = 0.f;
        st.D = 0.f;
        st.T = 1.f;
        st.nh = 0;
        if (!(d4.w > 0.f)) {
            res[2 * i] = make_float4(0.f, 0.f, 0.f, 0.f);
            res[2 * i + 1] = make_float4(0.f, 0.f, 0.f, 1.f);
            return;
        }
    } else {
        float w[16];
#pragma unroll
        for (int q = 0; q < kRelightStateF4; ++q) {
            const float4 v = state[j * kRelightStateF4 + q];
            w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int c = 0; c < 7; ++c) st.C[c] = w[c];
        st.D = w[7];
        st.T = w[8];
        st.nh = __float_as_int(w[9]);
        last_key = ((uint64_t)__float_as_uint(w[11]) << 32) | (uint64_t)__float_as_uint(w[10]);
        last_u = __float_as_int(w[12]);
    }
    const Ray ray = make_ray(ld3r(xg, p0 + i / Sn), mk3(d4.x, d4.y, d4.z));
    KBuffer<K, trace_threads<K>()> kb;
    kb.bind();
    bool ok = true, done = false;
    do {
        ok &= collect_round(S, ray, P, last_key, last_u, kb);
        done = blend_round<K, 7>(S, P, kb, st, nullptr, 0, last_key, last_u);
    } while (MODE == kRelLast && !done);
    if (!ok) atomicOr(S.status, kErrStackOverflow);
    if (done) {
        res[2 * i] = make_float4(st.C[0], st.C[1], st.C[2], st.C[3]);
        res[2 * i + 1] = make_float4(st.C[4], st.C[5], st.C[6], st.T);
    } else {
        float w[16];
#pragma unroll
        for (int c = 0; c < 7; ++c) w[c] = st.C[c];
        w[7] = st.D;
        w[8] = st.T;
        w[9] = __int_as_float(st.nh);
        w[10] = __uint_as_float((uint32_t)last_key);
        w[11] = __uint_as_float((uint32_t)(last_key >> 32));
        w[12] = __int_as_float(last_u);
        w[13] = w[14] = w[15] = 0.f;
#pragma unroll
        for (int q = 0; q < kRelightStateF4; ++q)
            state[j * kRelightStateF4 + q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        flags[j] = 1u;
    }
}

__global__ void __launch_bounds__(kRelightThreads) k_relight_shade(EnvMaps M, const float* __restrict__ ng,
                                                                   const float* __restrict__ ag,
                                                                   const float* __restrict__ rg,
                                                                   const float* __restrict__ wog, int64_t p0,
                                                                   int64_t np, int Sn, const float4* __restrict__ dir,
                                                                   const float4* __restrict__ res,
                                                                   float* __restrict__ rgb, float* __restrict__ vis,
                                                                   float* __restrict__ ind) {
    const int lane = threadIdx.x & 31;
    const int64_t k = blockIdx.x * (int64_t)(kRelightThreads / 32) + (threadIdx.x >> 5);
    if (k >= np) return;
    const int64_t p = p0 + k;
    const f3 a = ld3r(ag, p);
    const ShadeFrame F = shade_frame(ld3r(ng, p), ld3r(wog, p), rg[p]);
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int s = lane; s < Sn; s += 32) {
        const int64_t i = k * Sn + s;
        const float4 d4 = __ldg(dir + i);
        if (!(d4.w > 0.f)) continue;
        const float4 r0 = __ldg(res + 2 * i), r1 = __ldg(res + 2 * i + 1);
        const float C[7] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z};
        relight_sample(M, F, a, mk3(d4.x, d4.y, d4.z), d4.w, C, r1.w, acc);
    }
    relight_write(acc, lane, p, Sn, rgb, vis, ind);
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

constexpr int64_t kRelightChunkRays = int64_t(1) << 26;

template <int K>
cudaError_t relight_wave(const SceneView& S, const uint32_t* bounds, const EnvMaps& M, const float* x,
                         const float* n, const float* a, const float* r, const float* wo, int64_t P, int Sn,
                         uint64_t seed, const TraceParams& TP, float* rgb, float* vis, float* ind, cudaStream_t st) {
    const int64_t pc = kRelightChunkRays / Sn > 0 ? kRelightChunkRays / Sn : 1;
    const int64_t cap = (P < pc ? P : pc) * Sn;
    const int64_t hw = sort_hist_words(cap);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const int64_t sums = scan_long_words(cap + 1);
    const size_t bytes = al(16 * cap) + 4 * al(4 * cap) + al(4 * hw) + al(32 * cap) + al(4 * (cap + 1)) +
                         al(4 * cap) + al(4 * (1 + sums)) + al(16 * kRelightStateF4 * cap);
    unsigned char* base = nullptr;
    cudaError_t e = scratch_alloc(reinterpret_cast<void**>(&base), bytes, st);
    if (e != cudaSuccess) return e;
    size_t off = 0;
    auto take = [&](size_t b) { unsigned char* q = base + off; off += al(b); return q; };
    float4* dir = reinterpret_cast<float4*>(take(16 * cap));
    uint32_t* key = reinterpret_cast<uint32_t*>(take(4 * cap));
    int32_t* val = reinterpret_cast<int32_t*>(take(4 * cap));
    uint32_t* ktmp = reinterpret_cast<uint32_t*>(take(4 * cap));
    int32_t* vtmp = reinterpret_cast<int32_t*>(take(4 * cap));
    uint32_t* hist = reinterpret_cast<uint32_t*>(take(4 * hw));
    float4* res = reinterpret_cast<float4*>(take(32 * cap));
    uint32_t* flags = reinterpret_cast<uint32_t*>(take(4 * (cap + 1)));
    int32_t* list = reinterpret_cast<int32_t*>(take(4 * cap));
    uint32_t* count = reinterpret_cast<uint32_t*>(take(4 * (1 + sums)));
    float4* state = reinterpret_cast<float4*>(take(16 * kRelightStateF4 * cap));
    for (int64_t p0 = 0; p0 < P && e == cudaSuccess; p0 += pc) {
        const int64_t np = P - p0 < pc ? P - p0 : pc;
        const int64_t rays = np * Sn;
        k_relight_gen<<<grid_for(rays, 256), 256, 0, st>>>(M, x, p0, rays, Sn, seed, bounds, dir, key, val);
        e = sort_pairs(key, val, ktmp, vtmp, hist, rays, st);
        if (e != cudaSuccess) break;
        if (S.n == 0) {
            k_relight_trace<K><<<grid_for(rays, kRelightThreads), kRelightThreads, 0, st>>>(S, TP, x, p0, Sn, dir,
                                                                                          val, rays, res);
            count_launches(1);
        } else {
            const unsigned g = grid_for(rays, kRelightThreads);
            e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * (rays + 1), st);
            if (e != cudaSuccess) break;
            k_relight_round<K, kRelFirst><<<g, kRelightThreads, 0, st>>>(S, TP, x, p0, Sn, dir, val, rays, res, list,
                                                                          count, state, flags);
            count_launches(1);
            for (int round = 2; round <= 4 && e == cudaSuccess; ++round) {
                e = flags_to_list(flags, rays, count + 1, list, count, st);
                if (e != cudaSuccess) break;
                if (round < 4) {
                    e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * (rays + 1), st);
                    if (e != cudaSuccess) break;
                    k_relight_round<K, kRelNext><<<g, kRelightThreads, 0, st>>>(S, TP, x, p0, Sn, dir, val, rays, res,
                                                                                 list, count, state, flags);
                } else {
                    k_relight_round<K, kRelLast><<<g, kRelightThreads, 0, st>>>(S, TP, x, p0, Sn, dir, val, rays, res,
                                                                                 list, count, state, flags);
                }
                count_launches(1);
            }
            if (e != cudaSuccess) break;
        }
        k_relight_shade<<<grid_for(np, kRelightThreads / 32), kRelightThreads, 0, st>>>(M, n, a, r, wo, p0, np, Sn,
                                                                                       dir, res, rgb, vis, ind);
        count_launches(2);
        e = cudaGetLastError();
    }
    const cudaError_t ef = cudaFreeAsync(base, st);
    return e != cudaSuccess ? e : ef;
}

template <class T>
cudaError_t dalloc(T** p, size_t count, int64_t& bytes) {
    const size_t b = sizeof(T) * (count > 0 ? count : 1);
    bytes += (int64_t)b;
    return cudaMalloc(reinterpret_cast<void**>(p), b);
}

}  // namespace

void free_envmap(irgs_envmap m) {
    if (m == nullptr) return;
    void* ptrs[] = {m->env, m->irr, m->pref, m->lut, m->row_cdf, m->col_cdf};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete m;
}

irgs_status build_envmap_impl(const float* env, int32_t H, int32_t W, cudaStream_t st, irgs_envmap* out) {
    irgs_envmap m = new (std::nothrow) irgs_envmap_s();
    if (m == nullptr) return IRGS_ERR_OOM;
    cudaGetDevice(&m->device);
    m->H = H;
    m->W = W;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(dalloc(&m->env, (size_t)H * W * 3, m->bytes));
    A(dalloc(&m->irr, (size_t)kIrrH * kIrrW * 3, m->bytes));
    A(dalloc(&m->pref, (size_t)(kLevels - 1) * kPrefH * kPrefW * 3, m->bytes));
    A(dalloc(&m->lut, (size_t)kLutN * kLutN * 2, m->bytes));
    A(dalloc(&m->row_cdf, (size_t)H + 1, m->bytes));
    A(dalloc(&m->col_cdf, (size_t)H * (W + 1), m->bytes));
    if (e != cudaSuccess) {
        free_envmap(m);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? IRGS_ERR_OOM : IRGS_ERR_CUDA;
    }
    A(cudaMemcpyAsync(m->env, env, sizeof(float) * (size_t)H * W * 3, cudaMemcpyDeviceToDevice, st));
    k_irradiance<<<kIrrH * kIrrW, kReduceThreads, 0, st>>>(m->env, H, W, m->irr);
    k_prefilter<<<(kLevels - 1) * kPrefH * kPrefW, kReduceThreads, 0, st>>>(m->env, H, W, m->pref);
    k_brdf_table<<<(kLutN * kLutN + 127) / 128, 128, 0, st>>>(m->lut);
    k_env_col_cdf<<<(H + 127) / 128, 128, 0, st>>>(m->env, H, W, m->col_cdf);
    k_env_row_cdf<<<1, 1, 0, st>>>(m->col_cdf, H, W, m->row_cdf);
    count_launches(5);
    A(cudaGetLastError());
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        free_envmap(m);
        return IRGS_ERR_CUDA;
    }
    *out = m;
    return IRGS_OK;
}

irgs_status export_envmap_impl(irgs_envmap m, float* irr, float* pref, float* lut, double* row_cdf,
                               double* col_cdf, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    const cudaMemcpyKind k = cudaMemcpyDefault;
    if (irr) A(cudaMemcpyAsync(irr, m->irr, sizeof(float) * kIrrH * kIrrW * 3, k, st));
    if (pref) A(cudaMemcpyAsync(pref, m->pref, sizeof(float) * (kLevels - 1) * kPrefH * kPrefW * 3, k, st));
    if (lut) A(cudaMemcpyAsync(lut, m->lut, sizeof(float) * kLutN * kLutN * 2, k, st));
    if (row_cdf) A(cudaMemcpyAsync(row_cdf, m->row_cdf, sizeof(double) * (m->H + 1), k, st));
    if (col_cdf) A(cudaMemcpyAsync(col_cdf, m->col_cdf, sizeof(double) * (size_t)m->H * (m->W + 1), k, st));
    return e == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

// Directions of the environment-importance samples the relighting traces:
// ray i = p * n_samples + s (they depend on the keys only, not on the point).
__global__ void k_relight_rays(EnvMaps M, int64_t rays, int Sn, uint64_t seed, float* __restrict__ dir,
                               float* __restrict__ pdf_out, int32_t* __restrict__ valid) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rays) return;
    f3 w = mk3(0.f, 0.f, 1.f);
    float pdf = 0.f;
    const bool ok = relight_dir(M, i / Sn, (int)(i % Sn), Sn, seed, w, pdf);
    dir[3 * i] = w.x;
    dir[3 * i + 1] = w.y;
    dir[3 * i + 2] = w.z;
    if (pdf_out != nullptr) pdf_out[i] = ok ? pdf : 0.f;
    if (valid != nullptr) valid[i] = ok ? 1 : 0;
}

irgs_status launch_relight_rays(irgs_envmap m, int64_t P, int32_t n_samples, uint64_t seed, float* dir, float* pdf,
                                int32_t* valid, cudaStream_t st) {
    const int64_t rays = P * (int64_t)n_samples;
    if (rays == 0) return IRGS_OK;
    const EnvMaps M{m->env, m->irr, m->pref, m->lut, m->row_cdf, m->col_cdf, m->H, m->W};
    const int T = 256;
    k_relight_rays<<<(unsigned)((rays + T - 1) / T), T, 0, st>>>(M, rays, n_samples, seed, dir, pdf, valid);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

irgs_status launch_relight(const SceneView& S, const uint32_t* bounds, irgs_envmap m, const float* x,
                           const float* n, const float* albedo, const float* rough, const float* wo, int64_t P,
                           int32_t n_samples, uint64_t seed, const irgs_trace_params& p, float* rgb, float* vis,
                           float* ind, cudaStream_t st) {
    if (P == 0) return IRGS_OK;
    const TraceParams TP = to_params(p);
    const EnvMaps M{m->env, m->irr, m->pref, m->lut, m->row_cdf, m->col_cdf, m->H, m->W};
    cudaError_t e = cudaSuccess;
    if ((p.flags & IRGS_FLAG_PER_THREAD) != 0u) {
        // fused: a warp per point tracing its own samples
        const int64_t blocks = (P + kRelightThreads / 32 - 1) / (kRelightThreads / 32);
        switch (p.k) {
            case 8:
                k_relight<8><<<(unsigned)blocks, kRelightThreads, 0, st>>>(S, M, x, n, albedo, rough, wo, P,
                                                                          n_samples, seed, TP, rgb, vis, ind);
                break;
            case 16:
                k_relight<16><<<(unsigned)blocks, kRelightThreads, 0, st>>>(S, M, x, n, albedo, rough, wo, P,
                                                                           n_samples, seed, TP, rgb, vis, ind);
                break;
            default: return IRGS_ERR_UNSUPPORTED;
        }
        count_launches(1);
        e = cudaGetLastError();
    } else {
        switch (p.k) {
            case 8:
                e = relight_wave<8>(S, bounds, M, x, n, albedo, rough, wo, P, n_samples, seed, TP, rgb, vis, ind, st);
                break;
            case 16:
                e = relight_wave<16>(S, bounds, M, x, n, albedo, rough, wo, P, n_samples, seed, TP, rgb, vis, ind,
                                     st);
                break;
            default: return IRGS_ERR_UNSUPPORTED;
        }
    }
    if (e == cudaErrorMemoryAllocation) return IRGS_ERR_OOM;
    return e == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

}  // namespace irgs
