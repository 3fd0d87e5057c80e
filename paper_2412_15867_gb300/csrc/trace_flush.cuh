// Single-pass ordered march of a warp of rays: Trace(r_o, r_d) of IRGS Eq. 8
// with the k-buffer of Sec. 3.2 used as a window of pending hits instead of
// a batch that is blended only after a whole traversal round.
//
// The 32 rays of a warp walk one shared stack as in collect_round_warp. Each
// stack entry also carries a lower bound of the depth at which any ray of
// the warp can meet its subtree (the smallest entry depth over the lanes that
// need it; a lane that does not need a subtree has no hit in it), and the
// stack keeps the prefix minimum of these bounds. Before each node visit the
// bound B of everything not yet visited is min(the node's own bound, the
// prefix minimum of the stack). Every undiscovered hit of a lane then lies at
// depth >= B - slack, so the lane's pending hits with depth below B - slack
// are final: they are blended in (key, user index) order at once, and a ray
// whose transmittance drops below T_min stops walking right there.
//
// The pending hits sit in a ring of K slots. When it is full the farthest one
// bounds the walk (the cut: nodes beyond it are culled and later hits are
// dropped, exactly as the far bound of a full k-buffer); a ray whose ring was
// ever full this pass and is not done after it starts another pass after its
// last blended hit. Per ray the hits are blended in the same order with the
// same arithmetic as march_forward, so the results are bitwise the same; the
// traversal only visits fewer nodes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "trace.cuh"

namespace irgs {

// Pending hits of one ray: a ring of K 16-byte entries {key (8 B), Morton
// index, alpha} in shared memory (slot j of thread t at [j * THREADS + t]),
// sorted by (key, user index) from `head`, `cnt` of them. cut_key / cut_m:
// the farthest hit admitted since the ring was last full (UINT64_MAX: it has
// not been full this pass).
template <int K, int THREADS>
struct KRing {
    static_assert((K & (K - 1)) == 0, "ring size must be a power of two");
    uint4* e;
    int head, cnt;
    uint64_t cut_key;
    int32_t cut_m;

    __device__ __forceinline__ void bind() {
        __shared__ uint4 s_e[K * THREADS];
        e = s_e + threadIdx.x;
        clear();
    }
    __device__ __forceinline__ void clear() {
        head = 0;
        cnt = 0;
        cut_key = UINT64_MAX;
        cut_m = 0;
    }
    __device__ __forceinline__ static uint64_t key_of(const uint4& v) {
        return ((uint64_t)v.y << 32) | (uint64_t)v.x;
    }
    __device__ __forceinline__ uint4& at(int i) const { return e[((head + i) & (K - 1)) * THREADS]; }
    __device__ __forceinline__ bool was_full() const { return cut_key != UINT64_MAX; }
    // does the hit (k, user index u) come before the cut?
    __device__ __forceinline__ bool fits(uint64_t k, int32_t u, const float4* rec) const {
        return k < cut_key || (k == cut_key && u < uid_of(rec, cut_m));
    }
    // insert (k, Morton index mm, user index u, alpha aa); the caller checked fits()
    __device__ __forceinline__ void insert(uint64_t k, int32_t mm, int32_t u, float aa, const float4* rec) {
        int j = (cnt < K ? cnt : K - 1) - 1;
        while (j >= 0) {
            const uint4 v = at(j);
            const uint64_t kj = key_of(v);
            if (!(k < kj || (k == kj && u < uid_of(rec, (int32_t)v.z)))) break;
            at(j + 1) = v;
            --j;
        }
        at(j + 1) = make_uint4((uint32_t)k, (uint32_t)(k >> 32), (uint32_t)mm, __float_as_uint(aa));
        if (cnt < K) ++cnt;
        if (cnt == K) {
            const uint4 t = at(K - 1);
            cut_key = key_of(t);
            cut_m = (int32_t)t.z;
        }
    }
    __device__ __forceinline__ void pop() {
        head = (head + 1) & (K - 1);
        --cnt;
    }
};

// Signed-integer image of a float with the same order (for warp reductions).
__device__ __forceinline__ int ordered_int(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : (i ^ 0x7fffffff);
}
__device__ __forceinline__ float from_ordered_int(int i) { return __int_as_float(i >= 0 ? i : (i ^ 0x7fffffff)); }

// Test surfel m and insert it into the ring if its (key, user index) lies
// strictly after the last blended hit (last_key, Morton slot last_m; none if
// last_m < 0) and before the cut.
template <class KR, bool STATS>
__device__ __forceinline__ void leaf_insert_ring(const SceneView& S, const Ray& ray, const TraceParams& P, int32_t m,
                                                 uint64_t last_key, int32_t last_m, KR& kb, float& t_hi,
                                                 TraceStats* ts) {
    if (STATS) ts->leaves++;
    const float4* R = S.rec + (int64_t)m * kRecF4;
    const float4 r0 = ldg4(R), r1 = ldg4(R + 1), r2 = ldg4(R + 2), r3 = ldg4(R + 3);
    float kh, kl, a;
    if (!surfel_hit<false>(r0, r1, r2, r3, ray, P.alpha_min, P.alpha_max, kh, kl, a, nullptr, key_depth(last_key),
                           t_hi))
        return;
    const uint64_t key = depth_key(kh, kl);
    const int32_t u = __float_as_int(r2.w);
    const bool past_min = kh > P.t_min || (kh == P.t_min && kl > 0.f);
    const bool after =
        past_min && (key > last_key || (key == last_key && last_m >= 0 && u > uid_of(S.rec, last_m)));
    const bool before = kh < P.t_max || (kh == P.t_max && kl < 0.f);
    if (after && before && kb.fits(key, u, S.rec)) {
        if (STATS) ts->inserts++;
        kb.insert(key, m, u, a, S.rec);
        if (kb.was_full()) t_hi = key_depth(kb.cut_key);
    }
}

// Blend the ring's front hits with depth below `bound` (all of them for
// bound = +inf) until T < T_min. Returns true when the ray is done.
template <int K, int FB, class KR>
__device__ __forceinline__ bool flush_front(const SceneView& S, const TraceParams& P, KR& kb, float bound,
                                            MarchState<K, FB>& st, int32_t* ids, int max_ids, uint64_t& last_key,
                                            int32_t& last_m) {
    while (kb.cnt > 0) {
        const uint4 v = kb.at(0);
        const uint64_t key = KR::key_of(v);
        const float kh = key_depth(key);
        if (!(kh < bound)) break;
        const float a = __uint_as_float(v.w);
        const int32_t m = (int32_t)v.z;
        const float w = __fmul_rn(st.T, a);
        const float* f = S.feat + (int64_t)m * S.F + P.off;
#pragma unroll
        for (int c = 0; c < FB; ++c)
            if (c < P.fc) st.C[c] = __fmaf_rn(w, __ldg(f + c), st.C[c]);
        st.D = __fmaf_rn(w, kh, st.D);
        st.T = __fmul_rn(st.T, __fsub_rn(1.0f, a));
        if (ids != nullptr && st.nh < max_ids) ids[st.nh] = __float_as_int(__ldg(&S.rec[(int64_t)m * kRecF4 + 2].w));
        st.nh++;
        kb.pop();
        last_key = key;
        last_m = m;
        if (st.T < P.T_min) return true;
    }
    return false;
}

// The forward march of a warp (all 32 lanes call it; lanes without a ray pass
// live = false). Returns false if the traversal stack overflowed.
template <int K, int FB, bool STATS = false>
__device__ __forceinline__ bool march_forward_flush(const SceneView& S, const Ray& ray, const TraceParams& P,
                                                    MarchState<K, FB>& st, int32_t* ids, int max_ids, bool live,
                                                    TraceStats* ts = nullptr) {
#pragma unroll
    for (int c = 0; c < FB; ++c) st.C[c] = 0.f;
    st.D = 0.f;
    st.T = 1.f;
    st.nh = 0;
    bool ok = true;
    if (S.n == 0) return ok;
    KRing<K, trace_threads<K>()> kb;
    kb.bind();
    const int lane = threadIdx.x & 31;
    uint64_t last_key = depth_key(P.t_min, 0.f);
    int32_t last_m = -1;
    bool done = !live;
    const int64_t max_visits = S.n + 64;
    while (__any_sync(kFullWarp, !done)) {
        if (STATS && !done) ts->rounds++;
        kb.clear();
        float t_hi = P.t_max;
        int st0 = 0, st1 = 0;         // stack: node of entry e in lane e % 32, register e / 32
        float pm0 = INFINITY, pm1 = INFINITY;   // and the prefix minimum of the entry bounds
        float pm_top = INFINITY;      // prefix minimum of the whole stack (warp-uniform)
        float bnd = -INFINITY;        // bound of the node about to be visited (none for the root)
        int sp = 0;
        int ni = 0;
        for (int64_t visits = 0;; ++visits) {
            if (!done) {
                const float B = fminf(bnd, pm_top);
                if (B > -INFINITY && kb.cnt > 0)
                    done = flush_front<K, FB>(S, P, kb, B - tslack(B), st, ids, max_ids, last_key, last_m);
            }
            if (__all_sync(kFullWarp, done)) break;
            if (visits > max_visits) {
                ok = false;
                break;
            }
            const bool active = !done;
            const WideNodeRay nd = load_wide_ray(S.wide, ni, ray);
            if (STATS && active) ts->nodes++;
            float tn[4], tf[4];
            slab4_ray(nd, ray, tn, tf);
            const int c[4] = {nd.child.x, nd.child.y, nd.child.z, nd.child.w};
            const float t_lo = key_depth(last_key);
            const float lo_c = t_lo - tslack(t_lo);
            float hi_c = t_hi + tslack(t_hi);
            bool h[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                h[k] = active && c[k] != kNoChild && tn[k] <= tf[k] && tf[k] >= lo_c && tn[k] <= hi_c;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (h[k] && c[k] < 0) leaf_insert_ring<decltype(kb), STATS>(S, ray, P, ~c[k], last_key, last_m, kb,
                                                                            t_hi, ts);
            hi_c = t_hi + tslack(t_hi);
            // internal children some lane still needs, each with the smallest
            // entry depth over those lanes (its bound and its visiting order)
            float t[4];
            int nv = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool need = h[k] && c[k] >= 0 && tn[k] <= hi_c;
                const int r = __reduce_min_sync(kFullWarp, need ? ordered_int(tn[k]) : INT32_MAX);
                t[k] = r != INT32_MAX ? from_ordered_int(r) : INFINITY;
                nv += r != INT32_MAX ? 1 : 0;
            }
            if (nv == 0) {
                if (sp == 0) break;
                --sp;
                const bool hiw = (sp >> 5) != 0;
                ni = __shfl_sync(kFullWarp, hiw ? st1 : st0, sp & 31);
                bnd = __shfl_sync(kFullWarp, hiw ? pm1 : pm0, sp & 31);   // prefix minimum through this entry
                pm_top = sp > 0 ? __shfl_sync(kFullWarp, ((sp - 1) >> 5) ? pm1 : pm0, (sp - 1) & 31) : INFINITY;
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
                    pm_top = fminf(pm_top, tfar);
                    if (lane == (sp & 31)) {
                        if (sp >> 5) {
                            st1 = farc;
                            pm1 = pm_top;
                        } else {
                            st0 = farc;
                            pm0 = pm_top;
                        }
                    }
                    ++sp;
                } else {
                    ok = false;
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (t[k] != INFINITY) {
                    ni = c[k];
                    bnd = t[k];
                }
        }
        // end of the pass: what is still pending is final
        if (!done) done = flush_front<K, FB>(S, P, kb, INFINITY, st, ids, max_ids, last_key, last_m);
        // a ray whose ring never filled has seen every hit after its last key
        if (!done && !kb.was_full()) done = true;
    }
    return ok;
}

}  // namespace irgs
