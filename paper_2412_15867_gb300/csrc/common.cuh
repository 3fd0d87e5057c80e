// Device-side building blocks shared by the scene builder, the tracer and the
// shading kernel: small vector math, error-free float transforms, the packed
// node / surfel layouts in HBM, and the counter-based random generator.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/irgs.h"

namespace irgs {

// ---------------------------------------------------------------------------
// Error bits of the per-scene device status word.
constexpr uint32_t kErrStackOverflow = 1u;   // a ray's traversal stack overflowed
constexpr uint32_t kErrBadTree = 2u;         // the hierarchy failed a consistency bound
constexpr uint32_t kErrBadHitList = 4u;      // a saved hit list held an index outside the scene

// Traversal stack depth. Karras trees over 30-bit keys with index tie-breaks
// are at most 30 + 31 levels deep; the stack holds deferred siblings only.
constexpr int kStackSize = 64;

// Child id encoding in a node: >= 0 internal node, < 0 leaf (~m, m = Morton
// index of the surfel), kNoChild = absent.
constexpr int32_t kNoChild = INT32_MIN;

// ---------------------------------------------------------------------------
// HBM layouts.
//
// Internal node (64 B, one 128-byte line holds two): both children's boxes
// are stored in the parent so one fetch decides which children to visit.
//   a = {b0.lo.x, b0.lo.y, b0.lo.z, b0.hi.x}
//   b = {b0.hi.y, b0.hi.z, b1.lo.x, b1.lo.y}
//   c = {b1.lo.z, b1.hi.x, b1.hi.y, b1.hi.z}
//   d = {child0, child1, -, -}
struct __align__(16) Node {
    float4 a, b, c;
    int4 d;
};

// 4-wide node (128 B, one cache line): the boxes of up to four children in
// structure-of-arrays form (component k of each float4 belongs to child k)
// and the child ids (same encoding as Node; kNoChild for empty slots).
struct __align__(16) WideNode {
    float4 lox, loy, loz, hix, hiy, hiz;
    int4 child;
    int4 pad;
};

// Packed surfel record, Morton order (64 B = 4 x float4):
//   r0 = {mu.x, mu.y, mu.z, opacity}
//   r1 = {t_u/s_u (xyz), rho_c^2}        rho_c^2 < 0: never hit
//   r2 = {t_v/s_v (xyz), user index as int bits}
//   r3 = {n (xyz), 0}
constexpr int kRecF4 = 4;

// ---------------------------------------------------------------------------
struct f3 {
    float x, y, z;
};
__device__ __forceinline__ f3 mk3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ float dot3(f3 a, f3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ f3 add3(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 sub3(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 mul3(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ f3 cross3(f3 a, f3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ f3 normalize3(f3 a) {
    float r = rsqrtf(dot3(a, a));
    return mul3(a, r);
}

// Error-free sum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Order-preserving unsigned view of a float (total order on finite values,
// -0 and +0 must be normalised by the caller).
__device__ __forceinline__ uint32_t ordered_bits(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Sort key of a hit at depth tau = kh + kl (kh >= 0 is the rounded depth,
// kl the exact remainder): lexicographic (kh, kl) as one 64-bit integer.
// Only valid for kh >= 0 (callers reject tau <= t_min with t_min >= 0 first).
__device__ __forceinline__ uint64_t depth_key(float kh, float kl) {
    return (static_cast<uint64_t>(__float_as_uint(kh + 0.0f)) << 32) | ordered_bits(kl + 0.0f);
}

// ---------------------------------------------------------------------------
// Read-only vector loads through the non-coherent path.
__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }
__device__ __forceinline__ int4 ldg4i(const int4* p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): output i of the stream seeded with
// `seed` is the variant-13 mixer applied to seed + (i + 1) * golden gamma.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// Top 24 bits as a float in [0, 1) (exact).
__device__ __forceinline__ float u01_from_bits(uint64_t z) {
    return static_cast<float>(static_cast<uint32_t>(z >> 40)) * (1.0f / 16777216.0f);
}

// ---------------------------------------------------------------------------
// Process-wide count of kernel launches (capi.cu owns the counter).
void count_launches(uint64_t k);

// Stream-ordered scratch of the current device from the library's own pool
// (capi.cu): freed blocks stay in the pool up to kScratchKeepBytes, so the
// large per-call scratch is not mapped again on every call. Free with
// cudaFreeAsync.
constexpr uint64_t kScratchKeepBytes = uint64_t(32) << 30;
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st);

// ---------------------------------------------------------------------------
// Device view of a scene (plain pointers, passed by value to kernels).
struct SceneView {
    const Node* nodes;     // [max(n-1,1)] binary hierarchy
    const WideNode* wide;  // 4-wide hierarchy traversed by the kernels, root 0
    const float4* rec;     // [n * 4]
    const float* feat;     // [n, F] Morton order
    const float4* q_raw;   // [n] raw quaternion (w,x,y,z), Morton order
    const float2* scale;   // [n] (s_u, s_v), Morton order
    const int32_t* inv_perm;  // [n] Morton slot of user index u
    uint32_t* status;      // device error word
    int64_t n;
    int32_t F;
    float alpha_min;
};

}  // namespace irgs
