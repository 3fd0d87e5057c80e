// Per-ray traversal of the LBVH with a register k-buffer and front-to-back
// compositing -- Trace(r_o, r_d) of IRGS Eq. 8 with the intersection of Eq. 6,
// the response of Eq. 7 and the blending of Eq. 2. Shared by the forward,
// backward and shading kernels, which must reproduce each other's hit order
// and arithmetic bit for bit; every operation whose rounding matters is
// therefore written with explicit round-to-nearest intrinsics.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace irgs {

struct TraceParams {
    float alpha_min, alpha_max, T_min, t_min, t_max;
    int32_t off, fc;
};

struct Ray {
    f3 o, d;           // origin and direction as given
    f3 inv;            // 1/d with zero components replaced (slab test only)
    f3 oinv;           // o * inv
    float inv_dd;      // 1 / |d|^2
    float graze;       // 1e-8 |d|
    int nrx, nry, nrz; // row of a wide node holding each axis' entry plane (lo if inv >= 0, else hi)
};

__device__ __forceinline__ Ray make_ray(f3 o, f3 d) {
    Ray r;
    r.o = o;
    r.d = d;
    auto safe = [](float x) { return fabsf(x) < 1e-20f ? copysignf(1e-20f, x) : x; };
    r.inv = mk3(1.0f / safe(d.x), 1.0f / safe(d.y), 1.0f / safe(d.z));
    r.oinv = mk3(o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z);
    float dd = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
    r.inv_dd = 1.0f / dd;
    r.graze = 1e-8f * sqrtf(dd);
    r.nrx = r.inv.x >= 0.f ? 0 : 3;
    r.nry = r.inv.y >= 0.f ? 1 : 4;
    r.nrz = r.inv.z >= 0.f ? 2 : 5;
    return r;
}

// Geometry of an accepted hit that the backward pass needs.
struct HitGeom {
    f3 e;          // p - mu
    float u, v;    // Eq. 7 local coordinates
    float G;       // exp(-rho^2/2)
    float a_raw;   // o G before the clamp
    float den;     // n . d
};

// Ray/surfel test (Eq. 6-7) evaluated around a rebased origin
// o' = o + t_r d, t_r = (mu - o).d / |d|^2 (closest approach to mu), so the
// cancellation that plain FP32 suffers when |o - mu| >> scale disappears:
//   a   = mu - o exactly as a float pair (two_sum),
//   dl  = mu - o' = fma(-t_r, d, a_hi) + a_lo          (small, nearly exact)
//   tau = t_r + n.dl / n.d,  p - mu = (tau - t_r) d - dl.
// The depth is returned as the exact pair (kh, kl) = two_sum(t_r, tau - t_r).
// A candidate whose rounded depth kh lies outside [kh_lo, kh_hi] is rejected
// before the support and opacity tests (callers pass bounds that only cut
// candidates their own key tests would reject).
template <bool GEOM>
__device__ __forceinline__ bool surfel_hit(const float4& r0, const float4& r1, const float4& r2, const float4& r3,
                                           const Ray& ray, float amin, float amax, float& kh, float& kl,
                                           float& alpha, HitGeom* g, float kh_lo = -INFINITY,
                                           float kh_hi = INFINITY) {
    float ahx, alx, ahy, aly, ahz, alz;
    two_sum(r0.x, -ray.o.x, ahx, alx);
    two_sum(r0.y, -ray.o.y, ahy, aly);
    two_sum(r0.z, -ray.o.z, ahz, alz);
    const f3 d = ray.d;
    float tr = __fmul_rn(__fmaf_rn(ahx, d.x, __fmaf_rn(ahy, d.y, __fmul_rn(ahz, d.z))), ray.inv_dd);
    float dlx = __fadd_rn(__fmaf_rn(-tr, d.x, ahx), alx);
    float dly = __fadd_rn(__fmaf_rn(-tr, d.y, ahy), aly);
    float dlz = __fadd_rn(__fmaf_rn(-tr, d.z, ahz), alz);
    float den = __fmaf_rn(r3.x, d.x, __fmaf_rn(r3.y, d.y, __fmul_rn(r3.z, d.z)));
    if (!(fabsf(den) >= ray.graze)) return false;
    float num = __fmaf_rn(r3.x, dlx, __fmaf_rn(r3.y, dly, __fmul_rn(r3.z, dlz)));
    float tp = __fdiv_rn(num, den);
    two_sum(tr, tp, kh, kl);
    if (kh < kh_lo || kh > kh_hi) return false;
    float ex = __fmaf_rn(tp, d.x, -dlx);
    float ey = __fmaf_rn(tp, d.y, -dly);
    float ez = __fmaf_rn(tp, d.z, -dlz);
    float u = __fmaf_rn(ex, r1.x, __fmaf_rn(ey, r1.y, __fmul_rn(ez, r1.z)));
    float v = __fmaf_rn(ex, r2.x, __fmaf_rn(ey, r2.y, __fmul_rn(ez, r2.z)));
    float rho2 = __fmaf_rn(u, u, __fmul_rn(v, v));
    if (!(rho2 <= r1.w)) return false;
    float G = __expf(__fmul_rn(-0.5f, rho2));
    float a_raw = __fmul_rn(r0.w, G);
    alpha = fminf(a_raw, amax);
    if (!(alpha >= amin)) return false;
    if (GEOM) {
        g->e = mk3(ex, ey, ez);
        g->u = u;
        g->v = v;
        g->G = G;
        g->a_raw = a_raw;
        g->den = den;
    }
    return true;
}

__device__ __forceinline__ void slab2(const Node& nd, const Ray& r, float& tn0, float& tf0, float& tn1,
                                      float& tf1) {
    // child 0: lo = (a.x,a.y,a.z) hi = (a.w,b.x,b.y); child 1: lo = (b.z,b.w,c.x) hi = (c.y,c.z,c.w)
    float x0 = fmaf(nd.a.x, r.inv.x, -r.oinv.x), x1 = fmaf(nd.a.w, r.inv.x, -r.oinv.x);
    float y0 = fmaf(nd.a.y, r.inv.y, -r.oinv.y), y1 = fmaf(nd.b.x, r.inv.y, -r.oinv.y);
    float z0 = fmaf(nd.a.z, r.inv.z, -r.oinv.z), z1 = fmaf(nd.b.y, r.inv.z, -r.oinv.z);
    tn0 = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fminf(z0, z1));
    tf0 = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fmaxf(z0, z1));
    x0 = fmaf(nd.b.z, r.inv.x, -r.oinv.x); x1 = fmaf(nd.c.y, r.inv.x, -r.oinv.x);
    y0 = fmaf(nd.b.w, r.inv.y, -r.oinv.y); y1 = fmaf(nd.c.z, r.inv.y, -r.oinv.y);
    z0 = fmaf(nd.c.x, r.inv.z, -r.oinv.z); z1 = fmaf(nd.c.w, r.inv.z, -r.oinv.z);
    tn1 = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fminf(z0, z1));
    tf1 = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fmaxf(z0, z1));
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ WideNode load_wide(const WideNode* w, int i) {
    const float4* p = reinterpret_cast<const float4*>(w + i);
    WideNode n;
    n.lox = ldg4(p);
    n.loy = ldg4(p + 1);
    n.loz = ldg4(p + 2);
    n.hix = ldg4(p + 3);
    n.hiy = ldg4(p + 4);
    n.hiz = ldg4(p + 5);
    n.child = ldg4i(reinterpret_cast<const int4*>(p + 6));
    return n;
}

// Slab intervals of the four children of a wide node.
__device__ __forceinline__ void slab4(const WideNode& w, const Ray& r, float tn[4], float tf[4]) {
    const float lx[4] = {w.lox.x, w.lox.y, w.lox.z, w.lox.w}, hx[4] = {w.hix.x, w.hix.y, w.hix.z, w.hix.w};
    const float ly[4] = {w.loy.x, w.loy.y, w.loy.z, w.loy.w}, hy[4] = {w.hiy.x, w.hiy.y, w.hiy.z, w.hiy.w};
    const float lz[4] = {w.loz.x, w.loz.y, w.loz.z, w.loz.w}, hz[4] = {w.hiz.x, w.hiz.y, w.hiz.z, w.hiz.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float x0 = fmaf(lx[k], r.inv.x, -r.oinv.x), x1 = fmaf(hx[k], r.inv.x, -r.oinv.x);
        const float y0 = fmaf(ly[k], r.inv.y, -r.oinv.y), y1 = fmaf(hy[k], r.inv.y, -r.oinv.y);
        const float z0 = fmaf(lz[k], r.inv.z, -r.oinv.z), z1 = fmaf(hz[k], r.inv.z, -r.oinv.z);
        tn[k] = max3f(fminf(x0, x1), fminf(y0, y1), fminf(z0, z1));
        tf[k] = min3f(fmaxf(x0, x1), fmaxf(y0, y1), fmaxf(z0, z1));
    }
}

// A wide node's child boxes as the ray meets them: for each axis the plane
// it enters through (lo where 1/d >= 0, else hi) and the one it leaves
// through, selected by which rows are loaded.
struct WideNodeRay {
    float4 nx, ny, nz, fx, fy, fz;
    int4 child;
};

__device__ __forceinline__ WideNodeRay load_wide_ray(const WideNode* w, int i, const Ray& r) {
    const float4* p = reinterpret_cast<const float4*>(w + i);
    WideNodeRay n;
    n.nx = ldg4(p + r.nrx);
    n.ny = ldg4(p + r.nry);
    n.nz = ldg4(p + r.nrz);
    n.fx = ldg4(p + (r.nrx ^ 3));   // rows 0 <-> 3, 1 <-> 4, 2 <-> 5
    n.fy = ldg4(p + (r.nry ^ 5));
    n.fz = ldg4(p + (r.nrz ^ 7));
    n.child = ldg4i(reinterpret_cast<const int4*>(p + 6));
    return n;
}

// Slab intervals of the four children from the entry / exit planes: the same
// values slab4 gives (fma(v, inv, -oinv) is monotone in v for a fixed sign
// of inv, so the entry plane's distance is the minimum of the pair), with
// no per-axis min/max.
__device__ __forceinline__ void slab4_ray(const WideNodeRay& w, const Ray& r, float tn[4], float tf[4]) {
    const float nx[4] = {w.nx.x, w.nx.y, w.nx.z, w.nx.w}, fx[4] = {w.fx.x, w.fx.y, w.fx.z, w.fx.w};
    const float ny[4] = {w.ny.x, w.ny.y, w.ny.z, w.ny.w}, fy[4] = {w.fy.x, w.fy.y, w.fy.z, w.fy.w};
    const float nz[4] = {w.nz.x, w.nz.y, w.nz.z, w.nz.w}, fz[4] = {w.fz.x, w.fz.y, w.fz.z, w.fz.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        tn[k] = max3f(fmaf(nx[k], r.inv.x, -r.oinv.x), fmaf(ny[k], r.inv.y, -r.oinv.y),
                      fmaf(nz[k], r.inv.z, -r.oinv.z));
        tf[k] = min3f(fmaf(fx[k], r.inv.x, -r.oinv.x), fmaf(fy[k], r.inv.y, -r.oinv.y),
                      fmaf(fz[k], r.inv.z, -r.oinv.z));
    }
}

// Conservative slack on depths compared against box intervals.
__device__ __forceinline__ float tslack(float t) { return 1e-5f * (1.0f + fabsf(t)); }

__device__ __forceinline__ Node load_node(const Node* nodes, int i) {
    const float4* p = reinterpret_cast<const float4*>(nodes + i);
    Node nd;
    nd.a = ldg4(p);
    nd.b = ldg4(p + 1);
    nd.c = ldg4(p + 2);
    nd.d = ldg4i(reinterpret_cast<const int4*>(p + 3));
    return nd;
}

// User index of the surfel in Morton slot m (carried in its record's r2.w).
__device__ __forceinline__ int32_t uid_of(const float4* rec, int32_t m) {
    return __float_as_int(__ldg(&rec[(int64_t)m * kRecF4 + 2].w));
}

// k-buffer of the K nearest hits after `last`, sorted by (key, user index),
// kept in shared memory as 16-byte entries {key (8 B), Morton index, alpha}:
// slot j of thread t lives at [j * THREADS + t], so a warp touching the same
// slot reads consecutive 16-byte words, and one shift step of the insertion
// is one 128-bit load and one 128-bit store. Insertion shifts only the
// entries behind the new one (hits mostly arrive front to back, so the shift
// is usually short); the last entry is cached in registers for the cheap
// "does it fit" test and the traversal's far bound. Two hits with the same
// exact depth key are ordered by user index, which is read from the
// record only on that (rare) tie.
template <int K, int THREADS>
struct KBuffer {
    static constexpr int kThreads = THREADS;
    uint4* e;   // x, y: key (low, high); z: Morton index; w: alpha bits
    int cnt;
    uint64_t tail_key;
    int32_t tail_m;

    __device__ __forceinline__ void bind() {
        __shared__ uint4 s_e[K * THREADS];
        e = s_e + threadIdx.x;
        cnt = 0;
    }
    __device__ __forceinline__ static uint64_t key_of(const uint4& v) {
        return ((uint64_t)v.y << 32) | (uint64_t)v.x;
    }
    __device__ __forceinline__ void clear() { cnt = 0; }
    __device__ __forceinline__ bool full() const { return cnt == K; }
    __device__ __forceinline__ uint64_t key_at(int j) const { return key_of(e[j * THREADS]); }
    __device__ __forceinline__ int32_t m_at(int j) const { return (int32_t)e[j * THREADS].z; }
    __device__ __forceinline__ float a_at(int j) const { return __uint_as_float(e[j * THREADS].w); }
    // does the hit (k, user index u) belong before the full buffer's last entry?
    __device__ __forceinline__ bool fits(uint64_t k, int32_t u, const float4* rec) const {
        return cnt < K || k < tail_key || (k == tail_key && u < uid_of(rec, tail_m));
    }
    // insert (k, Morton index mm, user index u, alpha aa); the caller checked fits()
    __device__ __forceinline__ void insert(uint64_t k, int32_t mm, int32_t u, float aa, const float4* rec) {
        int j = (cnt < K ? cnt : K - 1) - 1;
        while (j >= 0) {
            const uint4 v = e[j * THREADS];
            const uint64_t kj = key_of(v);
            if (!(k < kj || (k == kj && u < uid_of(rec, (int32_t)v.z)))) break;
            e[(j + 1) * THREADS] = v;
            --j;
        }
        e[(j + 1) * THREADS] = make_uint4((uint32_t)k, (uint32_t)(k >> 32), (uint32_t)mm, __float_as_uint(aa));
        if (cnt < K) ++cnt;
        if (cnt == K) {
            const uint4 t = e[(K - 1) * THREADS];
            tail_key = key_of(t);
            tail_m = (int32_t)t.z;
        }
    }
};

// Threads per block of the tracing kernels for a k-buffer of K entries
// (the shared-memory k-buffer takes K * THREADS * 16 bytes).
template <int K>
__host__ __device__ constexpr int trace_threads() { return K > 16 ? 64 : 128; }

__device__ __forceinline__ float key_depth(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }

// Per-ray traversal counters of the diagnostic build (STATS = true).
struct TraceStats {
    int rounds, nodes, leaves, inserts;
};

// Test surfel m against the ray and insert it into the k-buffer if its
// (key, user index) lies strictly after (last_key, last_u) and before the
// buffer's last entry.
template <class KB, bool STATS = false>
__device__ __forceinline__ void leaf_insert(const SceneView& S, const Ray& ray, const TraceParams& P, int32_t m,
                                            uint64_t last_key, int32_t last_u, KB& kb, float& t_hi,
                                            TraceStats* ts = nullptr) {
    if (STATS) ts->leaves++;
    const float4* R = S.rec + (int64_t)m * kRecF4;
    const float4 r0 = ldg4(R), r1 = ldg4(R + 1), r2 = ldg4(R + 2), r3 = ldg4(R + 3);
    float kh, kl, a;
    // a rounded depth below the last blended key's, or above the full
    // buffer's last entry (t_hi, else t_max), cannot pass the key tests
    // below; kh >= key_depth(last_key) >= t_min >= 0 also makes the key
    // order that of the depths, and the first round's last_key = (t_min, 0)
    // with last_u = INT32_MAX admits exactly the depths beyond t_min
    if (!surfel_hit<false>(r0, r1, r2, r3, ray, P.alpha_min, P.alpha_max, kh, kl, a, nullptr, key_depth(last_key),
                           t_hi))
        return;
    const uint64_t key = depth_key(kh, kl);
    const int32_t u = __float_as_int(r2.w);
    const bool after = key > last_key || (key == last_key && u > last_u);
    const bool before = kh < P.t_max || (kh == P.t_max && kl < 0.f);
    if (after && before && kb.fits(key, u, S.rec)) {
        if (STATS) ts->inserts++;
        kb.insert(key, m, u, a, S.rec);
        if (kb.full()) t_hi = key_depth(kb.tail_key);
    }
}

// One round: gather the K nearest hits strictly after (last_key, last_u).
// Returns false if the traversal stack overflowed.
template <class KB, bool STATS = false>
__device__ __forceinline__ bool collect_round(const SceneView& S, const Ray& ray, const TraceParams& P,
                                              uint64_t last_key, int32_t last_u, KB& kb,
                                              TraceStats* ts = nullptr) {
    int2 stack[kStackSize];   // (node, entry depth bits): one 8-byte word per entry
    int sp = 0;
    int2 top = make_int2(0, 0);
    bool has_top = false;
    bool ok = true;
    kb.clear();
    const float t_lo = key_depth(last_key);
    const float lo_c = t_lo - tslack(t_lo);
    float t_hi = P.t_max;
    int ni = 0;
    // each wide node is fetched at most once per round in a valid tree
    const int max_visits = S.n + 64 < (int64_t)INT32_MAX ? (int)(S.n + 64) : INT32_MAX;
    for (int visits = 0;; ++visits) {
        if (visits > max_visits) {
            ok = false;
            break;
        }
        const WideNodeRay nd = load_wide_ray(S.wide, ni, ray);
        if (STATS) ts->nodes++;
        float tn[4], tf[4];
        slab4_ray(nd, ray, tn, tf);
        const int c[4] = {nd.child.x, nd.child.y, nd.child.z, nd.child.w};
        float hi_c = t_hi + tslack(t_hi);
        bool h[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) h[k] = tn[k] <= tf[k] && tf[k] >= lo_c && tn[k] <= hi_c;   // empty slots: empty box
        {
            // lanes of a warp walk different nodes here: each tests its own
            // needed leaves in one loop, so lanes run their i-th leaf test
            // together whatever slot it sits in (slot order kept per lane)
            unsigned mask = 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) mask |= (h[k] && c[k] < 0) ? (1u << k) : 0u;
            while (mask != 0u) {
                const int k = __ffs(mask) - 1;
                mask &= mask - 1u;
                const int ck = k == 0 ? c[0] : k == 1 ? c[1] : k == 2 ? c[2] : c[3];
                leaf_insert<KB, STATS>(S, ray, P, ~ck, last_key, last_u, kb, t_hi, ts);
            }
        }
        hi_c = t_hi + tslack(t_hi);
        // internal children still in reach: descend into the nearest, push the rest far first
        float t[4];
        int nv = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool v = h[k] && c[k] >= 0 && tn[k] <= hi_c;
            t[k] = v ? tn[k] : INFINITY;
            nv += v;
        }
        if (nv == 0) {
            bool found = false;
            if (has_top) {   // the most recent entry, kept in registers
                has_top = false;
                if (__int_as_float(top.y) <= hi_c) {
                    ni = top.x;
                    found = true;
                }
            }
            while (!found && sp > 0) {
                --sp;
                const int2 e = stack[sp];
                if (__int_as_float(e.y) <= hi_c) {
                    ni = e.x;
                    found = true;
                }
            }
            if (!found) break;
            continue;
        }
        // repeatedly take the farthest remaining child onto the stack
        for (int r = 0; r < nv - 1; ++r) {
            int far = -1;
            float tfar = -INFINITY;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (t[k] != INFINITY && t[k] >= tfar) {
                    tfar = t[k];
                    far = k;
                }
            int2 ent = make_int2(0, 0);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k == far) {
                    ent = make_int2(c[k], __float_as_int(t[k]));
                    t[k] = INFINITY;
                }
            if (has_top) {
                if (sp < kStackSize) stack[sp++] = top;
                else ok = false;
            }
            top = ent;
            has_top = true;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (t[k] != INFINITY) ni = c[k];
    }
    return ok;
}

constexpr unsigned kFullWarp = 0xffffffffu;

// Warp-coherent round: the 32 lanes of a warp walk one shared traversal
// stack (entry e lives in register e/32 of lane e%32). A child is visited when
// any lane's ray overlaps its box inside that lane's (t_lo, t_hi) window;
// each lane tests leaves with its own ray and keeps its own k-buffer, so the
// result per ray equals the per-thread round. All 32 lanes must call this
// together (inactive lanes pass active = false).
template <class KB, bool STATS = false>
__device__ __forceinline__ bool collect_round_warp(const SceneView& S, const Ray& ray, const TraceParams& P,
                                                   uint64_t last_key, int32_t last_u, KB& kb, bool active,
                                                   TraceStats* ts = nullptr) {
    kb.clear();
    const int lane = threadIdx.x & 31;
    const float t_lo = key_depth(last_key);
    const float lo_c = t_lo - tslack(t_lo);
    float t_hi = P.t_max;
    int st0 = 0, st1 = 0;
    int sp = 0;
    bool ok = true;
    int ni = 0;
    const int max_visits = S.n + 64 < (int64_t)INT32_MAX ? (int)(S.n + 64) : INT32_MAX;
    for (int visits = 0;; ++visits) {
        if (visits > max_visits) {
            ok = false;
            break;
        }
        const WideNodeRay nd = load_wide_ray(S.wide, ni, ray);
        if (STATS && active) ts->nodes++;
        float tn[4], tf[4];
        slab4_ray(nd, ray, tn, tf);
        const int c[4] = {nd.child.x, nd.child.y, nd.child.z, nd.child.w};
        float hi_c = t_hi + tslack(t_hi);
        bool h[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            h[k] = active && tn[k] <= tf[k] && tf[k] >= lo_c && tn[k] <= hi_c;   // empty slots: empty box
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (h[k] && c[k] < 0) leaf_insert<KB, STATS>(S, ray, P, ~c[k], last_key, last_u, kb, t_hi, ts);
        hi_c = t_hi + tslack(t_hi);
        // internal children some lane still needs; order them by the entry
        // depth seen by the first lane that needs each
        float t[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
        int nv = 0;
        if (max(max(c[0], c[1]), max(c[2], c[3])) >= 0) {   // the node (same for the warp) has internal children
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned b = __ballot_sync(kFullWarp, h[k] && c[k] >= 0 && tn[k] <= hi_c);
                const int src = b ? __ffs(b) - 1 : 0;
                const float tk = __shfl_sync(kFullWarp, tn[k], src);
                t[k] = b ? tk : INFINITY;
                nv += b ? 1 : 0;
            }
        }
        if (nv == 0) {
            if (sp == 0) break;
            --sp;
            ni = __shfl_sync(kFullWarp, (sp >> 5) ? st1 : st0, sp & 31);
            continue;
        }
        for (int r = 0; r < nv - 1; ++r) {
            int far = -1;
            float tfar = -INFINITY;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (t[k] != INFINITY && t[k] >= tfar) {
                    tfar = t[k];
                    far = k;
                }
            int farc = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k == far) {
                    farc = c[k];
                    t[k] = INFINITY;
                }
            if (sp < kStackSize) {
                if (lane == (sp & 31)) {
                    if (sp >> 5) st1 = farc; else st0 = farc;
                }
                ++sp;
            } else {
                ok = false;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (t[k] != INFINITY) ni = c[k];
    }
    return ok;
}

// Full forward march of one ray: rounds of collect + blend until the
// transmittance drops below T_min or no further hit exists.
template <int K, int FB>
struct MarchState {
    float C[FB];
    float D, T;
    int nh;
};

// The traced channels f[0..fc) of one surfel, zero beyond fc; as 8-byte
// pairs when f is 8-byte aligned for every surfel (even row length and
// offset).
template <int FB>
__device__ __forceinline__ void load_channels(const float* __restrict__ f, int fc, bool pairs, float (&fv)[FB]) {
    if (pairs) {
#pragma unroll
        for (int c = 0; c < FB; c += 2) {
            const float2 t = c + 1 < fc ? __ldg(reinterpret_cast<const float2*>(f + c))
                                        : make_float2(c < fc ? __ldg(f + c) : 0.f, 0.f);
            fv[c] = t.x;
            if (c + 1 < FB) fv[c + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int c = 0; c < FB; ++c) fv[c] = c < fc ? __ldg(f + c) : 0.f;
    }
}

// Blend the round's buffered hits in order (Eq. 2, Eq. 8) until the
// transmittance drops below T_min (the crossing hit included). Returns true
// when the ray is done: terminated, or fewer than K hits were left; else
// (last_key, last_u) move to the buffer's last entry (its key and user
// index) for the next round.
template <int K, int FB, class KB>
__device__ __forceinline__ bool blend_round(const SceneView& S, const TraceParams& P, const KB& kb,
                                            MarchState<K, FB>& st, int32_t* ids, int max_ids, uint64_t& last_key,
                                            int32_t& last_u) {
    bool done = false;
    for (int j = 0; j < kb.cnt && !done; ++j) {
        const float a = kb.a_at(j);
        const int32_t m = kb.m_at(j);
        const float w = __fmul_rn(st.T, a);
        float fv[FB];
        load_channels<FB>(S.feat + (int64_t)m * S.F + P.off, P.fc, ((S.F | P.off) & 1) == 0, fv);
#pragma unroll
        for (int c = 0; c < FB; ++c)
            if (c < P.fc) st.C[c] = __fmaf_rn(w, fv[c], st.C[c]);
        st.D = __fmaf_rn(w, key_depth(kb.key_at(j)), st.D);
        st.T = __fmul_rn(st.T, __fsub_rn(1.0f, a));
        if (ids != nullptr && st.nh < max_ids) ids[st.nh] = __float_as_int(__ldg(&S.rec[(int64_t)m * kRecF4 + 2].w));
        st.nh++;
        if (st.T < P.T_min) done = true;
    }
    if (!done) {
        if (kb.cnt < K) {
            done = true;
        } else {
            last_key = kb.tail_key;
            last_u = uid_of(S.rec, kb.tail_m);
        }
    }
    return done;
}

// WARP = true: all 32 lanes of the warp call this together (lanes without a
// ray pass live = false) and traverse warp-coherently.
template <int K, int FB, bool WARP, bool STATS = false>
__device__ __forceinline__ bool march_forward(const SceneView& S, const Ray& ray, const TraceParams& P,
                                              MarchState<K, FB>& st, int32_t* ids, int max_ids,
                                              bool live = true, TraceStats* ts = nullptr) {
#pragma unroll
    for (int c = 0; c < FB; ++c) st.C[c] = 0.f;
    st.D = 0.f;
    st.T = 1.f;
    st.nh = 0;
    bool ok = true;
    if (S.n == 0) return ok;
    uint64_t last_key = depth_key(P.t_min, 0.f);
    int32_t last_u = INT32_MAX;
    KBuffer<K, trace_threads<K>()> kb;
    kb.bind();
    bool done = !live;
    while (WARP ? __any_sync(kFullWarp, !done) : !done) {
        if (STATS && !done) ts->rounds++;
        if (WARP)
            ok &= collect_round_warp<decltype(kb), STATS>(S, ray, P, last_key, last_u, kb, !done, ts);
        else
            ok &= collect_round<decltype(kb), STATS>(S, ray, P, last_key, last_u, kb, ts);
        if (done) continue;
        done = blend_round<K, FB>(S, P, kb, st, ids, max_ids, last_key, last_u);
    }
    return ok;
}

__host__ __device__ inline TraceParams to_params(const irgs_trace_params& p) {
    TraceParams t;
    t.alpha_min = p.alpha_min;
    t.alpha_max = p.alpha_max;
    t.T_min = p.T_min;
    t.t_min = p.t_min;
    t.t_max = p.t_max;
    t.off = p.feat_offset;
    t.fc = p.feat_count;
    return t;
}

}  // namespace irgs
