// Scene construction: surfel packing and support boxes (K1), Morton codes (K2),
// stable LSD radix sort (K3), the binary hierarchy by locally-ordered
// clustering over the sorted leaves (K4; the Karras hierarchy as fallback),
// bottom-up box refit (K5) and the 4-wide collapse (K6). IRGS bounds each 2D Gaussian by a proxy enclosing the region
// where its response reaches alpha_min (Sec. 3.2, Eq. 5) and builds a BVH over
// the proxies; here the proxy is the axis-aligned box of the support disk and
// the BVH is a linear BVH built entirely on the device.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <new>

#include "common.cuh"
#include "scene.h"

namespace irgs {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortChunks = 16;                             // 32-key chunks per warp
constexpr int kTile = kSortThreads * kSortChunks;           // 4096 keys per tile

__device__ __forceinline__ uint32_t f2ord(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// ---------------------------------------------------------------------------
// K1: per-surfel frame (FP64, then rounded once), support radius, packed
// record (user order) and padded support-disk box; centroid bounds.
__global__ void k_surfel_boxes(const float* __restrict__ means, const float* __restrict__ quats,
                               const float* __restrict__ scales, const float* __restrict__ opac,
                               int64_t n, double alpha_min, float4* __restrict__ rec_user,
                               float* __restrict__ box_user, uint32_t* __restrict__ bounds) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (i < n) {
        double mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
        double w = quats[4 * i], x = quats[4 * i + 1], y = quats[4 * i + 2], z = quats[4 * i + 3];
        double su = scales[2 * i], sv = scales[2 * i + 1];
        double o = opac[i];
        double qn = sqrt(w * w + x * x + y * y + z * z);
        bool ok = qn > 0.0 && isfinite(qn) && su > 0.0 && sv > 0.0 && isfinite(su) && isfinite(sv) &&
                  isfinite(mu[0]) && isfinite(mu[1]) && isfinite(mu[2]) && isfinite(o);
        double tu[3] = {1, 0, 0}, tv[3] = {0, 1, 0}, nn[3] = {0, 0, 1};
        if (ok) {
            w /= qn; x /= qn; y /= qn; z /= qn;
            // rotation columns of the unit quaternion (w,x,y,z)
            tu[0] = 1.0 - 2.0 * (y * y + z * z); tu[1] = 2.0 * (x * y + w * z); tu[2] = 2.0 * (x * z - w * y);
            tv[0] = 2.0 * (x * y - w * z); tv[1] = 1.0 - 2.0 * (x * x + z * z); tv[2] = 2.0 * (y * z + w * x);
            nn[0] = 2.0 * (x * z + w * y); nn[1] = 2.0 * (y * z - w * x); nn[2] = 1.0 - 2.0 * (x * x + y * y);
        }
        // support radius: alpha reaches alpha_min at rho^2 = 2 ln(o/alpha_min), capped at 3 sigma
        double rc2 = -1.0;
        if (ok && o > 0.0) {
            double r2 = 2.0 * log(o / alpha_min);
            rc2 = r2 < 9.0 ? r2 : 9.0;
        }
        if (!(rc2 >= 0.0)) rc2 = -1.0;
        if (!ok) su = sv = 1.0;
        float4* R = rec_user + 4 * i;
        int32_t uid = (int32_t)i;
        R[0] = make_float4((float)mu[0], (float)mu[1], (float)mu[2], (float)o);
        R[1] = make_float4((float)(tu[0] / su), (float)(tu[1] / su), (float)(tu[2] / su), (float)rc2);
        R[2] = make_float4((float)(tv[0] / sv), (float)(tv[1] / sv), (float)(tv[2] / sv), __int_as_float(uid));
        R[3] = make_float4((float)nn[0], (float)nn[1], (float)nn[2], 0.f);
        double rc = rc2 >= 0.0 ? sqrt(rc2) : 0.0;
        float* B = box_user + 6 * i;
        for (int k = 0; k < 3; ++k) {
            double m = ok ? mu[k] : 0.0;
            double a = su * tu[k], b = sv * tv[k];
            double e = rc * sqrt(a * a + b * b);
            e = e * (1.0 + 1e-5) + 1e-6 * (1.0 + fabs(m));
            if (rc2 < 0.0) e = 0.0;   // never hit: a point box at the centre
            B[k] = __double2float_rd(m - e);
            B[3 + k] = __double2float_ru(m + e);
            cmin[k] = cmax[k] = (float)m;
        }
    }
    // block reduction of the centroid bounds
    for (int k = 0; k < 3; ++k) {
        for (int off = 16; off > 0; off >>= 1) {
            cmin[k] = fminf(cmin[k], __shfl_xor_sync(0xffffffffu, cmin[k], off));
            cmax[k] = fmaxf(cmax[k], __shfl_xor_sync(0xffffffffu, cmax[k], off));
        }
    }
    if ((threadIdx.x & 31) == 0 && cmin[0] <= cmax[0]) {
        for (int k = 0; k < 3; ++k) {
            atomicMin(&bounds[k], f2ord(cmin[k]));
            atomicMax(&bounds[3 + k], f2ord(cmax[k]));
        }
    }
}

// K2: 30-bit Morton code of each centre inside the centroid bounds.
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_morton(const float4* __restrict__ rec_user, int64_t n, const uint32_t* __restrict__ bounds,
                         uint32_t* __restrict__ keys, int32_t* __restrict__ vals) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 r0 = rec_user[4 * i];
    float c[3] = {r0.x, r0.y, r0.z};
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
        float lo = ord2f(bounds[k]), hi = ord2f(bounds[3 + k]);
        float ext = hi - lo;
        float t = ext > 0.f ? (c[k] - lo) / ext : 0.5f;
        int v = (int)(t * 1024.0f);
        v = v < 0 ? 0 : (v > 1023 ? 1023 : v);
        if (!(t == t)) v = 0;
        q[k] = (uint32_t)v;
    }
    keys[i] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    vals[i] = (int32_t)i;
}

// ---------------------------------------------------------------------------
// K3: stable LSD radix sort, 8 bits per pass. Per pass: tile histograms,
// one exclusive scan over (digit, tile), and a stable scatter that ranks keys
// inside a tile with warp match masks in (warp, chunk, lane) order.
__global__ void k_sort_hist(const uint32_t* __restrict__ keys, int64_t n, int shift, int tiles,
                            uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    for (int d = threadIdx.x; d < 256; d += blockDim.x) h[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kTile;
    for (int j = threadIdx.x; j < kTile; j += blockDim.x) {
        int64_t i = base + j;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * tiles + blockIdx.x] = h[d];
}

// Exclusive scan of `m` counters with one block of 1024 threads.
__global__ void k_scan_exclusive(uint32_t* __restrict__ a, int64_t m) {
    __shared__ uint32_t part[1024];
    int t = threadIdx.x;
    int64_t per = (m + 1023) / 1024;
    int64_t b = t * per, e = b + per < m ? b + per : m;
    uint32_t s = 0;
    for (int64_t i = b; i < e; ++i) s += a[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = part[t] - s;   // exclusive prefix of this thread's chunk
    for (int64_t i = b; i < e; ++i) {
        uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

// Multi-block exclusive scan for long arrays: each block scans a tile of
// kScanTile words in place and records the tile total; the totals are scanned
// by k_scan_exclusive; a last pass adds each tile's offset.
constexpr int kScanThreads = 1024;
constexpr int kScanTile = 4 * kScanThreads;

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(uint32_t* __restrict__ a, int64_t m,
                                                              uint32_t* __restrict__ sums) {
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + 4 * threadIdx.x;
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = base + k < m ? a[base + k] : 0u;
    const uint32_t t = v[0] + v[1] + v[2] + v[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = t;   // inclusive scan of the thread totals within the warp
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;   // exclusive warp offsets
        if (lane == kScanThreads / 32 - 1) sums[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run = warp_tot[warp] + inc - t;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < m) a[base + k] = run;
        run += v[k];
    }
}

__global__ void k_scan_add(uint32_t* __restrict__ a, int64_t m, const uint32_t* __restrict__ sums) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) a[i] += sums[i / kScanTile];
}

// Exclusive scan of m words using `sums` (ceil(m / kScanTile) words) as scratch.
void scan_long(uint32_t* a, int64_t m, uint32_t* sums, cudaStream_t st) {
    const int64_t tiles = (m + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(a, m, sums);
    k_scan_exclusive<<<1, 1024, 0, st>>>(sums, tiles);
    k_scan_add<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(a, m, sums);
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(
    const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t n, int shift, int tiles,
    const uint32_t* __restrict__ offs, uint32_t* __restrict__ kout, int32_t* __restrict__ vout) {
    __shared__ uint32_t wcnt[kSortWarps][256];
    __shared__ uint32_t gofs[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        gofs[d] = offs[(int64_t)d * tiles + blockIdx.x];
        for (int w = 0; w < kSortWarps; ++w) wcnt[w][d] = 0;
    }
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * kTile + warp * (32 * kSortChunks);
    uint32_t key[kSortChunks];
    int32_t val[kSortChunks];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int c = 0; c < kSortChunks; ++c) {
        int64_t i = wbase + c * 32 + lane;
        key[c] = i < n ? kin[i] : 0u;
        val[c] = i < n ? vin[i] : 0;
    }
    // phase 1: per-warp digit counts
#pragma unroll
    for (int c = 0; c < kSortChunks; ++c) {
        int64_t i = wbase + c * 32 + lane;
        uint32_t dg = i < n ? ((key[c] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, dg);
        if (dg < 256u && (peers & lt) == 0u) wcnt[warp][dg] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // phase 2: exclusive scan over warps per digit
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            uint32_t v = wcnt[w][d];
            wcnt[w][d] = run;
            run += v;
        }
    }
    __syncthreads();
    // phase 3: stable scatter
#pragma unroll
    for (int c = 0; c < kSortChunks; ++c) {
        int64_t i = wbase + c * 32 + lane;
        uint32_t dg = i < n ? ((key[c] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, dg);
        if (dg < 256u) {
            uint32_t pos = gofs[dg] + wcnt[warp][dg] + __popc(peers & lt);
            kout[pos] = key[c];
            vout[pos] = val[c];
        }
        __syncwarp();
        if (dg < 256u && (peers & lt) == 0u) wcnt[warp][dg] += __popc(peers);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Gather into Morton order: packed records, leaf boxes, features, raw
// quaternions and scales.
__global__ void k_gather(const int32_t* __restrict__ perm, int64_t n, const float4* __restrict__ rec_user,
                         const float* __restrict__ box_user, const float* __restrict__ quats,
                         const float* __restrict__ scales, float4* __restrict__ rec, float* __restrict__ leaf_box,
                         float4* __restrict__ q_raw, float2* __restrict__ scale, int32_t* __restrict__ inv_perm) {
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= n) return;
    int64_t u = perm[m];
    if (inv_perm != nullptr) inv_perm[u] = (int32_t)m;
    for (int k = 0; k < 4; ++k) rec[4 * m + k] = rec_user[4 * u + k];
    for (int k = 0; k < 6; ++k) leaf_box[6 * m + k] = box_user[6 * u + k];
    q_raw[m] = make_float4(quats[4 * u], quats[4 * u + 1], quats[4 * u + 2], quats[4 * u + 3]);
    scale[m] = make_float2(scales[2 * u], scales[2 * u + 1]);
}

__global__ void k_gather_feat(const int32_t* __restrict__ perm, int64_t n, int F, const float* __restrict__ fin,
                              float* __restrict__ fout) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n * F) return;
    int64_t m = j / F, c = j - m * F;
    fout[j] = fin[(int64_t)perm[m] * F + c];
}

// ---------------------------------------------------------------------------
// K4: Karras (2012) hierarchy. delta(i,j) is the common prefix length of the
// sorted keys, extended by the index bits when keys are equal.
__device__ __forceinline__ int kdelta(const uint32_t* __restrict__ k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    uint32_t a = k[i], b = k[j];
    if (a == b) return 32 + __clz((uint32_t)i ^ (uint32_t)j);
    return __clz(a ^ b);
}

// With `gate` set it runs only if *gate != 0 (the clustering build's fallback).
__global__ void k_karras(const uint32_t* __restrict__ keys, int64_t n, Node* __restrict__ nodes,
                         int32_t* __restrict__ leaf_parent, int32_t* __restrict__ node_parent,
                         const uint32_t* __restrict__ gate) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n - 1 || (gate != nullptr && *gate == 0u)) return;
    int d = (kdelta(keys, n, i, i + 1) - kdelta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = kdelta(keys, n, i, i - d);
    int64_t lmax = 2;
    while (kdelta(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
    int64_t l = 0;
    for (int64_t t = lmax / 2; t >= 1; t /= 2)
        if (kdelta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int64_t j = i + l * d;
    int dnode = kdelta(keys, n, i, j);
    int64_t s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (kdelta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int64_t g = i + s * d + (d < 0 ? -1 : 0);
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    int32_t left = (lo == g) ? ~(int32_t)g : (int32_t)g;
    int32_t right = (hi == g + 1) ? ~(int32_t)(g + 1) : (int32_t)(g + 1);
    nodes[i].d = make_int4(left, right, 0, 0);
    if (left < 0) leaf_parent[~left] = (int32_t)i; else node_parent[left] = (int32_t)i;
    if (right < 0) leaf_parent[~right] = (int32_t)i; else node_parent[right] = (int32_t)i;
    if (i == 0) node_parent[0] = -1;
}

// K5: bottom-up refit. The second thread to reach a node writes both child
// boxes into it and moves up; the first one stops.
__device__ __forceinline__ void child_box(const Node* nodes, const float* leaf_box, int32_t c, float b[6]) {
    if (c < 0) {
        const float* L = leaf_box + 6 * (int64_t)(~c);
        for (int k = 0; k < 6; ++k) b[k] = __ldcg(L + k);
    } else {
        const float4* p = reinterpret_cast<const float4*>(nodes + c);
        float4 a = __ldcg(p), bb = __ldcg(p + 1), cc = __ldcg(p + 2);
        b[0] = fminf(a.x, bb.z); b[1] = fminf(a.y, bb.w); b[2] = fminf(a.z, cc.x);
        b[3] = fmaxf(a.w, cc.y); b[4] = fmaxf(bb.x, cc.z); b[5] = fmaxf(bb.y, cc.w);
    }
}

__global__ void k_refit(int64_t n, const float* __restrict__ leaf_box, const int32_t* __restrict__ leaf_parent,
                        const int32_t* __restrict__ node_parent, Node* nodes, uint32_t* flags, uint32_t* status,
                        const uint32_t* __restrict__ gate) {
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= n || (gate != nullptr && *gate == 0u)) return;
    int32_t p = leaf_parent[m];
    // a valid hierarchy is at most 62 levels deep (30 key bits + 32 index bits)
    for (int level = 0; p >= 0; ++level) {
        if (level > 128 || p >= n - 1) {
            atomicOr(status, kErrBadTree);
            return;
        }
        __threadfence();
        const uint32_t arrived = atomicAdd(&flags[p], 1u);
        if (arrived == 0u) return;
        if (arrived != 1u) {
            atomicOr(status, kErrBadTree);
            return;
        }
        int4 ch = __ldcg(&nodes[p].d);
        float b0[6], b1[6];
        child_box(nodes, leaf_box, ch.x, b0);
        child_box(nodes, leaf_box, ch.y, b1);
        nodes[p].a = make_float4(b0[0], b0[1], b0[2], b0[3]);
        nodes[p].b = make_float4(b0[4], b0[5], b1[0], b1[1]);
        nodes[p].c = make_float4(b1[2], b1[3], b1[4], b1[5]);
        p = node_parent[p];
    }
}

// Root of a one-surfel (or empty) scene: child 0 = leaf 0 (if any), child 1 absent.
__global__ void k_tiny_root(int64_t n, const float* __restrict__ leaf_box, Node* nodes) {
    float b[6] = {0, 0, 0, 0, 0, 0};
    if (n == 1)
        for (int k = 0; k < 6; ++k) b[k] = leaf_box[k];
    nodes[0].a = make_float4(b[0], b[1], b[2], b[3]);
    nodes[0].b = make_float4(b[4], b[5], 0.f, 0.f);
    nodes[0].c = make_float4(0.f, 0.f, 0.f, 0.f);
    nodes[0].d = make_int4(n == 1 ? ~0 : kNoChild, kNoChild, 0, 0);
}

// ---------------------------------------------------------------------------
// K4 (default): locally-ordered agglomerative clustering over the sorted
// leaves (PLOC, Meister and Bittner 2018). In each round every cluster looks
// at the kPlocRadius clusters on either side in Morton order and picks the
// one whose union box has the smallest surface area; mutually chosen pairs
// merge into a new internal node. Equal areas are ordered by (distance in
// the order, parity of the lower index, lower index): a strict order on
// pairs, so the best pair of a round is always mutual (every round merges)
// and runs of equal boxes pair up as (0,1), (2,3), ... Node ids follow
// (round, position), so the tree is the same on every run; the root is made
// last and gets id 0. A cluster is (id, lo, hi) with its subtree height in
// lo.w. The rounds run over all clusters until at most kPlocFinishCap are
// left; one block then merges the rest in shared memory. A tree higher than
// kPlocMaxHeight (possible only for contrived inputs) is replaced by the
// Karras hierarchy, whose depth the 4-wide collapse and the refit assume.
//
// Working memory: the build's user-order buffers, dead after the gather:
// cluster boxes in rec_user (4 x n float4: lo and hi, two copies), cluster ids
// in keys_tmp / vals_tmp, per-tile kept lists in box_user (n int2), and the
// round counters and tile counts in hist.
constexpr int kPlocRadius = 16;
constexpr int kPlocBlock = 1024;
constexpr int kPlocFinishCap = kPlocBlock;
constexpr int kPlocMaxRounds = 64;
constexpr int kPlocMaxHeight = 60;
// state words: cluster count before each round, then nodes made before each
// round, then the fallback flag
constexpr int kPlocMade = kPlocMaxRounds + 1;
constexpr int kPlocFallback = 2 * (kPlocMaxRounds + 1);
constexpr int kPlocStateWords = kPlocFallback + 1;
constexpr int kPlocTileWords = 136;   // tile counts start here in hist

__device__ __forceinline__ float union_area(const float4& alo, const float4& ahi, const float4& blo,
                                            const float4& bhi) {
    const float dx = fmaxf(ahi.x, bhi.x) - fminf(alo.x, blo.x);
    const float dy = fmaxf(ahi.y, bhi.y) - fminf(alo.y, blo.y);
    const float dz = fmaxf(ahi.z, bhi.z) - fminf(alo.z, blo.z);
    const float a = dx * dy + dy * dz + dz * dx;
    return isnan(a) ? INFINITY : a;
}

// Nearest neighbour of cluster i among [i - R, i + R] of [0, count); boxes
// of cluster g at s_lo / s_hi[g - base].
__device__ __forceinline__ int64_t ploc_nearest(int64_t i, int64_t count, const float4* s_lo, const float4* s_hi,
                                                int64_t base) {
    const float4 lo = s_lo[i - base], hi = s_hi[i - base];
    float bc = INFINITY;
    int bd = 0;
    int64_t bm = 0, bj = -1;
    for (int o = -kPlocRadius; o <= kPlocRadius; ++o) {
        const int64_t j = i + o;
        if (o == 0 || j < 0 || j >= count) continue;
        const float c = union_area(lo, hi, s_lo[j - base], s_hi[j - base]);
        const int d = o < 0 ? -o : o;
        const int64_t m = o < 0 ? j : i;
        bool better = bj < 0 || c < bc;
        if (bj >= 0 && c == bc) {
            if (d != bd) better = d < bd;
            else if ((m & 1) != (bm & 1)) better = (m & 1) < (bm & 1);
            else better = m < bm;
        }
        if (better) { bc = c; bd = d; bm = m; bj = j; }
    }
    return bj;
}

// Exclusive scan of one value per thread over the block (blockDim.x a
// multiple of 32); s_warp holds 33 words. Returns the prefix, *total the sum.
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < nw ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        if (lane < nw) s_warp[lane] = wi - w;
        if (lane == nw - 1) s_warp[32] = wi;
    }
    __syncthreads();
    const uint32_t r = s_warp[warp] + inc - v;
    *total = s_warp[32];
    __syncthreads();
    return r;
}

// Internal node k with children a, b (ids as in Node::d) and their boxes;
// returns the merged cluster's box (height in lo.w).
__device__ __forceinline__ void ploc_node(int32_t k, int32_t a, int32_t b, const float4& alo, const float4& ahi,
                                          const float4& blo, const float4& bhi, Node* nodes, int32_t* leaf_parent,
                                          int32_t* node_parent, float4& lo, float4& hi) {
    nodes[k].a = make_float4(alo.x, alo.y, alo.z, ahi.x);
    nodes[k].b = make_float4(ahi.y, ahi.z, blo.x, blo.y);
    nodes[k].c = make_float4(blo.z, bhi.x, bhi.y, bhi.z);
    nodes[k].d = make_int4(a, b, 0, 0);
    if (a < 0) leaf_parent[~a] = k; else node_parent[a] = k;
    if (b < 0) leaf_parent[~b] = k; else node_parent[b] = k;
    lo = make_float4(fminf(alo.x, blo.x), fminf(alo.y, blo.y), fminf(alo.z, blo.z), fmaxf(alo.w, blo.w) + 1.f);
    hi = make_float4(fmaxf(ahi.x, bhi.x), fmaxf(ahi.y, bhi.y), fmaxf(ahi.z, bhi.z), 0.f);
}

__global__ void k_ploc_init(int64_t n, const float* __restrict__ leaf_box, int32_t* __restrict__ cid,
                            float4* __restrict__ clo, float4* __restrict__ chi, uint32_t* __restrict__ state,
                            int32_t* __restrict__ node_parent) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < kPlocStateWords) state[i] = i == 0 ? (uint32_t)n : 0u;
    if (i == 0) node_parent[0] = -1;
    if (i >= n) return;
    const float* b = leaf_box + 6 * i;
    cid[i] = ~(int32_t)i;
    clo[i] = make_float4(b[0], b[1], b[2], 0.f);
    chi[i] = make_float4(b[3], b[4], b[5], 0.f);
}

// One round, block b: nearest neighbours of its clusters (and of R clusters
// on either side, whose choices decide mutuality), then the block's kept
// clusters in order as (source index, partner or -1) in kept[b * block ...],
// their number and the number of merges in tile_cnt[2b], [2b + 1].
__global__ void __launch_bounds__(kPlocBlock) k_ploc_round(int r, const uint32_t* __restrict__ state,
                                                           const float4* __restrict__ clo,
                                                           const float4* __restrict__ chi, int2* __restrict__ kept,
                                                           uint32_t* __restrict__ tile_cnt) {
    constexpr int H = 2 * kPlocRadius;
    __shared__ float4 s_lo[kPlocBlock + 2 * H], s_hi[kPlocBlock + 2 * H];
    __shared__ int32_t s_nn[kPlocBlock + 2 * kPlocRadius];
    __shared__ uint32_t s_warp[33];
    const int64_t count = state[r];
    const int64_t b0 = (int64_t)blockIdx.x * kPlocBlock;
    if (count <= kPlocFinishCap || b0 >= count) return;
    const int64_t base = b0 - H;
    for (int t = threadIdx.x; t < kPlocBlock + 2 * H; t += kPlocBlock) {
        const int64_t g = base + t;
        if (g >= 0 && g < count) {
            s_lo[t] = clo[g];
            s_hi[t] = chi[g];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kPlocBlock + 2 * kPlocRadius; t += kPlocBlock) {
        const int64_t g = b0 - kPlocRadius + t;
        s_nn[t] = (g >= 0 && g < count) ? (int32_t)ploc_nearest(g, count, s_lo, s_hi, base) : -1;
    }
    __syncthreads();
    const int64_t i = b0 + threadIdx.x;
    uint32_t keep = 0u, maker = 0u;
    int32_t j = -1;
    if (i < count) {
        const int32_t c = s_nn[threadIdx.x + kPlocRadius];
        const bool mutual = c >= 0 && s_nn[c - (b0 - kPlocRadius)] == (int32_t)i;
        keep = (mutual && c < i) ? 0u : 1u;
        maker = (mutual && c > i) ? 1u : 0u;
        j = maker ? c : -1;
    }
    uint32_t tot;
    const uint32_t pre = block_scan(keep | (maker << 16), s_warp, &tot);
    if (keep) kept[b0 + (pre & 0xffffu)] = make_int2((int32_t)i, j);
    if (threadIdx.x == 0) {
        tile_cnt[2 * blockIdx.x] = tot & 0xffffu;
        tile_cnt[2 * blockIdx.x + 1] = tot >> 16;
    }
}

// Compaction of round r into the other cluster buffer; merges become nodes
// numbered by (nodes made before the round + merges before them).
__global__ void __launch_bounds__(kPlocBlock) k_ploc_compact(
    int r, int64_t n, uint32_t* __restrict__ state, const uint32_t* __restrict__ tile_cnt,
    const int2* __restrict__ kept, const int32_t* __restrict__ cid, const float4* __restrict__ clo,
    const float4* __restrict__ chi, int32_t* __restrict__ cid2, float4* __restrict__ clo2, float4* __restrict__ chi2,
    Node* __restrict__ nodes, int32_t* __restrict__ leaf_parent, int32_t* __restrict__ node_parent,
    uint32_t* status) {
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_red[2][32];
    const int64_t count = state[r];
    const uint32_t made = state[kPlocMade + r];
    if (count <= kPlocFinishCap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            state[r + 1] = (uint32_t)count;
            state[kPlocMade + r + 1] = made;
        }
        return;
    }
    const int64_t b0 = (int64_t)blockIdx.x * kPlocBlock;
    if (b0 >= count) return;
    // kept clusters and merges of the tiles before this one
    uint32_t ko = 0u, mo = 0u;
    for (int64_t t = threadIdx.x; t < blockIdx.x; t += blockDim.x) {
        ko += tile_cnt[2 * t];
        mo += tile_cnt[2 * t + 1];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ko += __shfl_xor_sync(0xffffffffu, ko, off);
        mo += __shfl_xor_sync(0xffffffffu, mo, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_red[0][warp] = ko;
        s_red[1][warp] = mo;
    }
    __syncthreads();
    ko = 0u;
    mo = 0u;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        ko += s_red[0][w];
        mo += s_red[1][w];
    }
    const uint32_t nk = tile_cnt[2 * blockIdx.x];
    const int t = threadIdx.x;
    const int2 e = (uint32_t)t < nk ? kept[b0 + t] : make_int2(-1, -1);
    uint32_t tot;
    const uint32_t rank = block_scan((uint32_t)t < nk && e.y >= 0 ? 1u : 0u, s_warp, &tot);
    if ((uint32_t)t < nk) {
        const int64_t dst = (int64_t)ko + t;
        if (e.y >= 0) {
            const int64_t idx = (int64_t)made + mo + rank;
            if (idx > n - 2) {
                atomicOr(status, kErrBadTree);
            } else {
                const int32_t k = (int32_t)(n - 2 - idx);
                float4 lo, hi;
                ploc_node(k, cid[e.x], cid[e.y], clo[e.x], chi[e.x], clo[e.y], chi[e.y], nodes, leaf_parent,
                          node_parent, lo, hi);
                cid2[dst] = k;
                clo2[dst] = lo;
                chi2[dst] = hi;
            }
        } else {
            cid2[dst] = cid[e.x];
            clo2[dst] = clo[e.x];
            chi2[dst] = chi[e.x];
        }
    }
    if ((int64_t)(b0 + kPlocBlock) >= count && threadIdx.x == 0) {
        state[r + 1] = ko + nk;
        state[kPlocMade + r + 1] = made + mo + tot;
    }
}

// One block: the clusters left after the rounds (pairs of neighbours first
// while more than kPlocFinishCap remain, which only contrived inputs leave),
// then rounds in shared memory down to the root; a root higher than
// kPlocMaxHeight raises the fallback flag.
__global__ void __launch_bounds__(kPlocBlock) k_ploc_finish(int rounds, int64_t n, uint32_t* __restrict__ state,
                                                            int32_t* cid0, float4* clo0, float4* chi0, int32_t* cid1,
                                                            float4* clo1, float4* chi1, Node* __restrict__ nodes,
                                                            int32_t* __restrict__ leaf_parent,
                                                            int32_t* __restrict__ node_parent, uint32_t* status) {
    __shared__ float4 s_lo[kPlocFinishCap], s_hi[kPlocFinishCap];
    __shared__ int32_t s_id[kPlocFinishCap], s_nn[kPlocFinishCap];
    __shared__ uint32_t s_warp[33];
    // the rounds that ran are a prefix; after e of them the clusters are in buffer e & 1
    int e = 0;
    while (e < rounds && state[e] > (uint32_t)kPlocFinishCap) ++e;
    int64_t c = state[e];
    int64_t made = state[kPlocMade + e];
    int src = e & 1;
    for (int level = 0; c > kPlocFinishCap && level < 64; ++level) {
        const int32_t* sid = src ? cid1 : cid0;
        const float4* slo = src ? clo1 : clo0;
        const float4* shi = src ? chi1 : chi0;
        int32_t* did = src ? cid0 : cid1;
        float4* dlo = src ? clo0 : clo1;
        float4* dhi = src ? chi0 : chi1;
        const int64_t half = c / 2;
        for (int64_t t = threadIdx.x; t < (c + 1) / 2; t += blockDim.x) {
            if (t < half) {
                const int64_t idx = made + t;
                if (idx > n - 2) {
                    atomicOr(status, kErrBadTree);
                    continue;
                }
                const int32_t k = (int32_t)(n - 2 - idx);
                float4 lo, hi;
                ploc_node(k, sid[2 * t], sid[2 * t + 1], slo[2 * t], shi[2 * t], slo[2 * t + 1], shi[2 * t + 1],
                          nodes, leaf_parent, node_parent, lo, hi);
                did[t] = k;
                dlo[t] = lo;
                dhi[t] = hi;
            } else {
                did[t] = sid[c - 1];
                dlo[t] = slo[c - 1];
                dhi[t] = shi[c - 1];
            }
        }
        made += half;
        c = (c + 1) / 2;
        src ^= 1;
        __syncthreads();
    }
    if (c > kPlocFinishCap) {   // cannot happen: 64 halvings
        if (threadIdx.x == 0) atomicOr(status, kErrBadTree);
        return;
    }
    {
        const int32_t* sid = src ? cid1 : cid0;
        const float4* slo = src ? clo1 : clo0;
        const float4* shi = src ? chi1 : chi0;
        for (int t = threadIdx.x; t < c; t += blockDim.x) {
            s_id[t] = sid[t];
            s_lo[t] = slo[t];
            s_hi[t] = shi[t];
        }
    }
    __syncthreads();
    const int t = threadIdx.x;
    for (int round = 0; c > 1 && round < kPlocFinishCap; ++round) {
        const int32_t nn = t < c ? (int32_t)ploc_nearest(t, c, s_lo, s_hi, 0) : -1;
        s_nn[t] = nn;
        __syncthreads();
        bool keep = false, maker = false;
        int32_t id = 0;
        float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo, plo = lo, phi = lo;
        int32_t pid = 0;
        if (t < c) {
            const bool mutual = nn >= 0 && s_nn[nn] == t;
            keep = !(mutual && nn < t);
            maker = mutual && nn > t;
            id = s_id[t];
            lo = s_lo[t];
            hi = s_hi[t];
            if (maker) {
                pid = s_id[nn];
                plo = s_lo[nn];
                phi = s_hi[nn];
            }
        }
        uint32_t tot;
        const uint32_t pre = block_scan((keep ? 1u : 0u) | (maker ? 0x10000u : 0u), s_warp, &tot);
        if (maker) {
            const int64_t idx = made + (pre >> 16);
            if (idx > n - 2) {
                atomicOr(status, kErrBadTree);
            } else {
                const int32_t k = (int32_t)(n - 2 - idx);
                float4 mlo, mhi;
                ploc_node(k, id, pid, lo, hi, plo, phi, nodes, leaf_parent, node_parent, mlo, mhi);
                id = k;
                lo = mlo;
                hi = mhi;
            }
        }
        if (keep) {
            s_id[pre & 0xffffu] = id;
            s_lo[pre & 0xffffu] = lo;
            s_hi[pre & 0xffffu] = hi;
        }
        made += tot >> 16;
        c = tot & 0xffffu;
        __syncthreads();
    }
    if (t == 0) {
        if (c != 1 || made != n - 1 || s_id[0] != 0) {
            atomicOr(status, kErrBadTree);
            state[kPlocFallback] = 1u;
        } else if (s_lo[0].w > (float)kPlocMaxHeight) {
            state[kPlocFallback] = 1u;
        }
    }
}

__device__ __forceinline__ void node_child(const Node& nd, int s, int32_t& c, float b[6]) {
    if (s == 0) {
        c = nd.d.x;
        b[0] = nd.a.x; b[1] = nd.a.y; b[2] = nd.a.z; b[3] = nd.a.w; b[4] = nd.b.x; b[5] = nd.b.y;
    } else {
        c = nd.d.y;
        b[0] = nd.b.z; b[1] = nd.b.w; b[2] = nd.c.x; b[3] = nd.c.y; b[4] = nd.c.z; b[5] = nd.c.w;
    }
}

// K6, greedy form: wide nodes are made top-down, one frontier level per
// launch. A wide node starts from the two children of its binary node and
// repeatedly replaces the internal child of largest box surface area by that
// child's two children, until it has four (or only leaves). Its internal
// children get new wide indices and form the next frontier. Levels read and
// clear rotating counters, so the host never waits on them.
constexpr int kWideLevels = 64;   // >= the binary depth: each level consumes one binary level at least

__device__ __forceinline__ float box_area(const float b[6]) {
    const float dx = b[3] - b[0], dy = b[4] - b[1], dz = b[5] - b[2];
    return dx * dy + dy * dz + dz * dx;
}

__global__ void k_wide_root(int64_t n, int2* __restrict__ frontier, uint32_t* __restrict__ counters) {
    frontier[0] = make_int2(0, 0);   // binary root -> wide node 0
    counters[0] = n > 1 ? 1u : 0u;   // level 0 frontier size
    counters[1] = 0u;
    counters[2] = 0u;
    counters[3] = 1u;                // wide nodes allocated
}

__global__ void k_wide_level(int level, const Node* __restrict__ nodes, const int2* __restrict__ cur,
                             int2* __restrict__ next, uint32_t* __restrict__ counters, int64_t max_wide,
                             WideNode* __restrict__ wide, uint32_t* status) {
    const uint32_t cnt = counters[level % 3];
    uint32_t* next_count = counters + (level + 1) % 3;
    if (blockIdx.x == 0 && threadIdx.x == 0) counters[(level + 2) % 3] = 0u;   // the level after next
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int2 e = cur[i];
        int32_t cid[4] = {kNoChild, kNoChild, kNoChild, kNoChild};
        float box[4][6] = {};
        const Node nd = nodes[e.x];
        node_child(nd, 0, cid[0], box[0]);
        node_child(nd, 1, cid[1], box[1]);
        int m = 2;
        while (m < 4) {
            int best = -1;
            float ba = -1.f;
            for (int k = 0; k < m; ++k)
                if (cid[k] >= 0) {
                    const float a = box_area(box[k]);
                    if (a > ba) {
                        ba = a;
                        best = k;
                    }
                }
            if (best < 0) break;
            const Node cn = nodes[cid[best]];
            node_child(cn, 1, cid[m], box[m]);
            node_child(cn, 0, cid[best], box[best]);
            ++m;
        }
        int32_t out[4] = {kNoChild, kNoChild, kNoChild, kNoChild};
        // empty slots get an empty box (lo = +inf, hi = -inf): no ray's slab
        // interval meets it, so the walks need no test of the child id
        for (int k = m; k < 4; ++k)
            for (int j = 0; j < 3; ++j) {
                box[k][j] = INFINITY;
                box[k][3 + j] = -INFINITY;
            }
        for (int k = 0; k < m; ++k) {
            if (cid[k] < 0) {
                out[k] = cid[k];
                continue;
            }
            const uint32_t w = atomicAdd(counters + 3, 1u);
            if ((int64_t)w >= max_wide) {
                atomicOr(status, kErrBadTree);
                continue;
            }
            out[k] = (int32_t)w;
            next[atomicAdd(next_count, 1u)] = make_int2(cid[k], (int32_t)w);
        }
        WideNode o;
        o.lox = make_float4(box[0][0], box[1][0], box[2][0], box[3][0]);
        o.loy = make_float4(box[0][1], box[1][1], box[2][1], box[3][1]);
        o.loz = make_float4(box[0][2], box[1][2], box[2][2], box[3][2]);
        o.hix = make_float4(box[0][3], box[1][3], box[2][3], box[3][3]);
        o.hiy = make_float4(box[0][4], box[1][4], box[2][4], box[3][4]);
        o.hiz = make_float4(box[0][5], box[1][5], box[2][5], box[3][5]);
        o.child = make_int4(out[0], out[1], out[2], out[3]);
        o.pad = make_int4(m, 0, 0, 0);
        wide[e.y] = o;
    }
}

// After the last level the frontier must be empty.
__global__ void k_wide_check(const uint32_t* __restrict__ counters, uint32_t* status) {
    if (counters[kWideLevels % 3] != 0u) atomicOr(status, kErrBadTree);
}

// Wide root of a one-surfel (or empty) scene.
__global__ void k_wide_tiny(int64_t n, const float* __restrict__ leaf_box, WideNode* wide) {
    WideNode o;
    const float e = INFINITY;   // empty slots: lo = +inf, hi = -inf
    float b[6] = {e, e, e, -e, -e, -e};
    if (n == 1)
        for (int k = 0; k < 6; ++k) b[k] = leaf_box[k];
    o.lox = make_float4(b[0], e, e, e);
    o.loy = make_float4(b[1], e, e, e);
    o.loz = make_float4(b[2], e, e, e);
    o.hix = make_float4(b[3], -e, -e, -e);
    o.hiy = make_float4(b[4], -e, -e, -e);
    o.hiz = make_float4(b[5], -e, -e, -e);
    o.child = make_int4(n == 1 ? ~0 : kNoChild, kNoChild, kNoChild, kNoChild);
    o.pad = make_int4(n == 1 ? 1 : 0, 0, 0, 0);
    wide[0] = o;
}

template <class T>
cudaError_t dalloc(T** p, size_t count, int64_t& bytes) {
    size_t b = sizeof(T) * (count > 0 ? count : 1);
    bytes += (int64_t)b;
    return cudaMalloc(reinterpret_cast<void**>(p), b);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

}  // namespace

void free_scene(irgs_scene sc) {
    if (!sc) return;
    void* ptrs[] = {sc->nodes, sc->rec, sc->feat, sc->q_raw, sc->scale, sc->leaf_box, sc->keys,
                    sc->perm, sc->inv_perm, sc->status, sc->rec_user, sc->box_user, sc->keys_tmp, sc->vals_tmp,
                    sc->hist, sc->bounds, sc->leaf_parent, sc->node_parent, sc->refit_flag, sc->wide,
                    sc->wide_frontier, sc->wide_counters};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete sc;
}

// Rounds of the clustering build for n leaves: about four per halving of the
// cluster count down to kPlocFinishCap, plus margin (rounds past that point
// return at once).
static int ploc_rounds(int64_t n) {
    int r = 8;
    for (int64_t c = n; c > kPlocFinishCap; c = (c + 1) / 2) r += 4;
    return r < kPlocMaxRounds ? r : kPlocMaxRounds;
}

// Enqueue the clustering build of the binary hierarchy (n > 1) over the
// sorted leaf boxes; returns the device word that is nonzero when the
// Karras hierarchy has to replace it.
static const uint32_t* enqueue_ploc(irgs_scene sc, cudaStream_t st) {
    const int64_t n = sc->n;
    int32_t* cid[2] = {reinterpret_cast<int32_t*>(sc->keys_tmp), sc->vals_tmp};
    float4* lo[2] = {sc->rec_user, sc->rec_user + 2 * n};
    float4* hi[2] = {sc->rec_user + n, sc->rec_user + 3 * n};
    int2* kept = reinterpret_cast<int2*>(sc->box_user);
    uint32_t* state = sc->hist;
    uint32_t* tile_cnt = sc->hist + kPlocTileWords;
    const int rounds = ploc_rounds(n);
    const unsigned tiles = (unsigned)((n + kPlocBlock - 1) / kPlocBlock);
    const int64_t init = n > kPlocStateWords ? n : kPlocStateWords;
    k_ploc_init<<<blocks_for(init, 256), 256, 0, st>>>(n, sc->leaf_box, cid[0], lo[0], hi[0], state,
                                                        sc->node_parent);
    for (int r = 0; r < rounds; ++r) {
        const int s = r & 1, d = s ^ 1;
        k_ploc_round<<<tiles, kPlocBlock, 0, st>>>(r, state, lo[s], hi[s], kept, tile_cnt);
        k_ploc_compact<<<tiles, kPlocBlock, 0, st>>>(r, n, state, tile_cnt, kept, cid[s], lo[s], hi[s], cid[d],
                                                     lo[d], hi[d], sc->nodes, sc->leaf_parent, sc->node_parent,
                                                     sc->status);
    }
    k_ploc_finish<<<1, kPlocBlock, 0, st>>>(rounds, n, state, cid[0], lo[0], hi[0], cid[1], lo[1], hi[1], sc->nodes,
                                            sc->leaf_parent, sc->node_parent, sc->status);
    count_launches(2 + 2 * rounds);
    return state + kPlocFallback;
}

// Enqueue the greedy 4-wide collapse of the scene's binary hierarchy (n > 1).
static void enqueue_wide(irgs_scene sc, cudaStream_t st) {
    const int64_t n = sc->n;
    int2* a = sc->wide_frontier;
    int2* b = sc->wide_frontier + n;
    // a grid-stride loop over the frontier: four 256-thread blocks per SM
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sc->device) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 1;
    }
    k_wide_root<<<1, 1, 0, st>>>(n, a, sc->wide_counters);
    for (int level = 0; level < kWideLevels; ++level) {
        k_wide_level<<<sms * 4, 256, 0, st>>>(level, sc->nodes, a, b, sc->wide_counters, sc->max_wide, sc->wide,
                                             sc->status);
        int2* t = a; a = b; b = t;
    }
    k_wide_check<<<1, 1, 0, st>>>(sc->wide_counters, sc->status);
    count_launches(kWideLevels + 2);
}

// Enqueue the whole build (K1-K5) for surfels `s` into the scene's buffers.
static irgs_status enqueue_build(irgs_scene sc, const irgs_surfels* s, cudaStream_t st) {
    const int64_t n = sc->n;
    const int32_t F = sc->F;
    const int64_t nn = n > 1 ? n - 1 : 1;
    const int64_t tiles = (n + kTile - 1) / kTile;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(cudaMemsetAsync(sc->nodes, 0, sizeof(Node) * nn, st));
    A(cudaMemsetAsync(sc->refit_flag, 0, sizeof(uint32_t) * nn, st));
    // bounds: mins start at the largest ordered value, maxes at the smallest
    A(cudaMemsetAsync(sc->bounds, 0xff, 3 * sizeof(uint32_t), st));
    A(cudaMemsetAsync(sc->bounds + 3, 0x00, 3 * sizeof(uint32_t), st));
    if (n > 0) {
        const int T = 256;
        k_surfel_boxes<<<blocks_for(n, T), T, 0, st>>>(s->means, s->quats, s->scales, s->opacity, n,
                                                       (double)sc->alpha_min, sc->rec_user, sc->box_user, sc->bounds);
        k_morton<<<blocks_for(n, T), T, 0, st>>>(sc->rec_user, n, sc->bounds, sc->keys, sc->perm);
        // 4 passes ping-pong: keys/perm -> tmp -> keys/perm ...
        uint32_t* ka = sc->keys; int32_t* va = sc->perm;
        uint32_t* kb = sc->keys_tmp; int32_t* vb = sc->vals_tmp;
        for (int shift = 0; shift < 32; shift += 8) {
            k_sort_hist<<<(unsigned)tiles, 256, 0, st>>>(ka, n, shift, (int)tiles, sc->hist);
            k_scan_exclusive<<<1, 1024, 0, st>>>(sc->hist, 256 * tiles);
            k_sort_scatter<<<(unsigned)tiles, kSortThreads, 0, st>>>(ka, va, n, shift, (int)tiles, sc->hist, kb, vb);
            uint32_t* tk = ka; ka = kb; kb = tk;
            int32_t* tv = va; va = vb; vb = tv;
        }
        // after an even number of passes the sorted data is back in keys/perm
        k_gather<<<blocks_for(n, T), T, 0, st>>>(sc->perm, n, sc->rec_user, sc->box_user, s->quats, s->scales,
                                                 sc->rec, sc->leaf_box, sc->q_raw, sc->scale, sc->inv_perm);
        if (F > 0)
            k_gather_feat<<<blocks_for(n * F, T), T, 0, st>>>(sc->perm, n, F, s->features, sc->feat);
        if (n > 1) {
            // the radix tree runs when asked for, else only if the clustering raises its fallback flag
            const uint32_t* gate = (sc->build_flags & IRGS_BUILD_RADIX_TREE) ? nullptr : enqueue_ploc(sc, st);
            k_karras<<<blocks_for(n - 1, T), T, 0, st>>>(sc->keys, n, sc->nodes, sc->leaf_parent, sc->node_parent,
                                                         gate);
            k_refit<<<blocks_for(n, T), T, 0, st>>>(n, sc->leaf_box, sc->leaf_parent, sc->node_parent, sc->nodes,
                                                    sc->refit_flag, sc->status, gate);
        }
    }
    if (n <= 1) k_tiny_root<<<1, 1, 0, st>>>(n, sc->leaf_box, sc->nodes);
    // boxes, morton, 4 x (hist, scan, scatter), gather = 15; + features; + the fallback karras/refit (the
    // clustering counts its own) or the tiny root
    count_launches(n == 0 ? 1 : 15 + (F > 0) + (n == 1 ? 1 : 2));
    if (sc->wide != nullptr) {
        if (n > 1) {
            enqueue_wide(sc, st);
        } else {
            k_wide_tiny<<<1, 1, 0, st>>>(n, sc->leaf_box, sc->wide);
            count_launches(1);
        }
    }
    A(cudaGetLastError());
    return e == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

int64_t sort_hist_words(int64_t n) {
    const int64_t tiles = (n + kTile - 1) / kTile;
    const int64_t words = 256 * (tiles > 0 ? tiles : 1);
    return words + (words + kScanTile - 1) / kScanTile;   // digit counts, then the scan's tile sums
}

cudaError_t sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys_tmp, int32_t* vals_tmp, uint32_t* hist,
                       int64_t n, cudaStream_t st, int key_bits) {
    if (n <= 0) return cudaSuccess;
    const int64_t tiles = (n + kTile - 1) / kTile;
    // an even number of 8-bit passes, so that the result ends in keys / vals
    const int passes = ((key_bits + 15) / 16) * 2;
    uint32_t* ka = keys; int32_t* va = vals;
    uint32_t* kb = keys_tmp; int32_t* vb = vals_tmp;
    for (int shift = 0; shift < 8 * passes; shift += 8) {
        k_sort_hist<<<(unsigned)tiles, 256, 0, st>>>(ka, n, shift, (int)tiles, hist);
        scan_long(hist, 256 * tiles, hist + 256 * tiles, st);
        k_sort_scatter<<<(unsigned)tiles, kSortThreads, 0, st>>>(ka, va, n, shift, (int)tiles, hist, kb, vb);
        uint32_t* tk = ka; ka = kb; kb = tk;
        int32_t* tv = va; va = vb; vb = tv;
    }
    count_launches(5 * passes);
    return cudaGetLastError();
}

cudaError_t scan_exclusive(uint32_t* a, int64_t m, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_scan_exclusive<<<1, 1024, 0, st>>>(a, m);
    count_launches(1);
    return cudaGetLastError();
}

int64_t scan_long_words(int64_t m) { return (m + kScanTile - 1) / kScanTile + 1; }

namespace {
// pos[0..m] = exclusive prefix of 0/1 flags: list[pos[j]] = j for every
// flagged j, *count = pos[m].
__global__ void k_flag_list(const uint32_t* __restrict__ pos, int64_t m, int32_t* __restrict__ list,
                            uint32_t* __restrict__ count) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j == 0) *count = pos[m];
    if (j < m && pos[j + 1] != pos[j]) list[pos[j]] = (int32_t)j;
}
}  // namespace

cudaError_t flags_to_list(uint32_t* flags, int64_t m, uint32_t* sums, int32_t* list, uint32_t* count,
                          cudaStream_t st) {
    cudaError_t e = scan_exclusive_long(flags, m + 1, sums, st);
    if (e != cudaSuccess) return e;
    k_flag_list<<<(unsigned)((m + 255) / 256 > 0 ? (m + 255) / 256 : 1), 256, 0, st>>>(flags, m, list, count);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t scan_exclusive_long(uint32_t* a, int64_t m, uint32_t* sums, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    scan_long(a, m, sums, st);
    count_launches(3);
    return cudaGetLastError();
}

irgs_status build_scene_impl(const irgs_surfels* s, float alpha_min, uint32_t build_flags, cudaStream_t st,
                             irgs_scene* out) {
    const int64_t n = s->n;
    const int32_t F = s->num_features;
    irgs_scene sc = new (std::nothrow) irgs_scene_s();
    if (!sc) return IRGS_ERR_OOM;
    cudaGetDevice(&sc->device);
    sc->n = n;
    sc->F = F;
    sc->alpha_min = alpha_min;
    sc->build_flags = build_flags;
    const int64_t nn = n > 1 ? n - 1 : 1;
    const int64_t tiles = (n + kTile - 1) / kTile;
    int64_t& B = sc->bytes;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(dalloc(&sc->nodes, nn, B));
    A(dalloc(&sc->rec, 4 * n, B));
    A(dalloc(&sc->feat, (size_t)n * F, B));
    A(dalloc(&sc->q_raw, n, B));
    A(dalloc(&sc->scale, n, B));
    A(dalloc(&sc->leaf_box, 6 * n, B));
    A(dalloc(&sc->keys, n, B));
    A(dalloc(&sc->perm, n, B));
    A(dalloc(&sc->inv_perm, n, B));
    A(dalloc(&sc->status, 1, B));
    A(dalloc(&sc->rec_user, 4 * n, B));
    A(dalloc(&sc->box_user, 6 * n, B));
    A(dalloc(&sc->keys_tmp, n, B));
    A(dalloc(&sc->vals_tmp, n, B));
    A(dalloc(&sc->hist, 256 * (tiles > 0 ? tiles : 1), B));
    A(dalloc(&sc->bounds, 6, B));
    A(dalloc(&sc->leaf_parent, n, B));
    A(dalloc(&sc->node_parent, nn, B));
    A(dalloc(&sc->refit_flag, nn, B));
    // every wide node takes at least one binary internal node
    sc->max_wide = nn + 1;
    A(dalloc(&sc->wide, sc->max_wide, B));
    A(dalloc(&sc->wide_frontier, 2 * (n > 0 ? n : 1), B));
    A(dalloc(&sc->wide_counters, 4, B));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_scene(sc);
        return e == cudaErrorMemoryAllocation ? IRGS_ERR_OOM : IRGS_ERR_CUDA;
    }
    if (cudaMemsetAsync(sc->status, 0, sizeof(uint32_t), st) != cudaSuccess) {
        free_scene(sc);
        return IRGS_ERR_CUDA;
    }
    irgs_status r = enqueue_build(sc, s, st);
    if (r != IRGS_OK) {
        cudaStreamSynchronize(st);
        free_scene(sc);
        return r;
    }
    *out = sc;
    return IRGS_OK;
}

irgs_status update_scene_impl(irgs_scene sc, const irgs_surfels* s, cudaStream_t st) {
    return enqueue_build(sc, s, st);
}

// Refit: new surfel values in the Morton order and hierarchy of the last
// build. Records, leaf boxes and features are recomputed and gathered with
// the kept permutation, the binary boxes are refitted bottom-up and the
// 4-wide nodes re-emitted from them (their layout depends only on the
// topology). Every box still bounds its subtree, so traces stay exact; only
// the quality of the tree can degrade as surfels move.
irgs_status refit_scene_impl(irgs_scene sc, const irgs_surfels* s, cudaStream_t st) {
    const int64_t n = sc->n;
    const int32_t F = sc->F;
    const int64_t nn = n > 1 ? n - 1 : 1;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(cudaMemsetAsync(sc->refit_flag, 0, sizeof(uint32_t) * nn, st));
    A(cudaMemsetAsync(sc->bounds, 0xff, 3 * sizeof(uint32_t), st));
    A(cudaMemsetAsync(sc->bounds + 3, 0x00, 3 * sizeof(uint32_t), st));
    const int T = 256;
    if (n > 0) {
        k_surfel_boxes<<<blocks_for(n, T), T, 0, st>>>(s->means, s->quats, s->scales, s->opacity, n,
                                                       (double)sc->alpha_min, sc->rec_user, sc->box_user, sc->bounds);
        k_gather<<<blocks_for(n, T), T, 0, st>>>(sc->perm, n, sc->rec_user, sc->box_user, s->quats, s->scales,
                                                 sc->rec, sc->leaf_box, sc->q_raw, sc->scale, sc->inv_perm);
        if (F > 0)
            k_gather_feat<<<blocks_for(n * F, T), T, 0, st>>>(sc->perm, n, F, s->features, sc->feat);
        if (n > 1)
            k_refit<<<blocks_for(n, T), T, 0, st>>>(n, sc->leaf_box, sc->leaf_parent, sc->node_parent, sc->nodes,
                                                    sc->refit_flag, sc->status, nullptr);
    }
    if (n <= 1) k_tiny_root<<<1, 1, 0, st>>>(n, sc->leaf_box, sc->nodes);
    if (n > 1) {
        enqueue_wide(sc, st);
    } else {
        k_wide_tiny<<<1, 1, 0, st>>>(n, sc->leaf_box, sc->wide);
    }
    // boxes, gather, features, refit (or the tiny root and tiny wide node); the collapse counts its own
    count_launches(n == 0 ? 2 : (n == 1 ? 4 + (F > 0) : 3 + (F > 0)));
    A(cudaGetLastError());
    return e == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Allocation-free build: all working memory of the build comes from one
// file-scope device array; the caller provides the outputs.
namespace {

constexpr int64_t kNoallocMax = IRGS_NOALLOC_MAX_SURFELS;
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }
constexpr int64_t kNoallocTiles = (kNoallocMax + kTile - 1) / kTile;
constexpr size_t kNoallocBytes =
    align_up(sizeof(float4) * 4 * kNoallocMax) * 2 +      // records in user and Morton order
    align_up(sizeof(float) * 6 * kNoallocMax) +           // user-order boxes
    align_up(sizeof(float4) * kNoallocMax) +              // raw quaternions
    align_up(sizeof(float2) * kNoallocMax) +              // scales
    align_up(sizeof(uint32_t) * kNoallocMax) * 2 +        // sort ping-pong keys / values
    align_up(sizeof(int32_t) * kNoallocMax) * 3 +         // leaf parents, node parents, refit flags
    align_up(sizeof(uint32_t) * 256 * kNoallocTiles) +    // digit histograms
    align_up(sizeof(uint32_t) * 6) + align_up(sizeof(uint32_t));   // bounds, status word

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[256] = {};

// Device address of the scratch array on the current device (looked up once
// per device). Returns nullptr if the lookup fails.
void* noalloc_scratch(int device) {
    if (device < 0 || device >= 256) return nullptr;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_ptr[device] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_noalloc_ptr[device] = p;
    }
    return g_noalloc_ptr[device];
}

}  // namespace

// The scratch array's carve-out for one allocation-free build: the scene
// view's work buffers and its device status word. Returns the bytes used.
size_t noalloc_carve(unsigned char* base, irgs_scene_s& sc) {
    const int64_t M = kNoallocMax;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base + off;
        off += align_up(bytes);
        return p;
    };
    sc.rec_user = reinterpret_cast<float4*>(take(sizeof(float4) * 4 * M));
    sc.rec = reinterpret_cast<float4*>(take(sizeof(float4) * 4 * M));
    sc.box_user = reinterpret_cast<float*>(take(sizeof(float) * 6 * M));
    sc.q_raw = reinterpret_cast<float4*>(take(sizeof(float4) * M));
    sc.scale = reinterpret_cast<float2*>(take(sizeof(float2) * M));
    sc.keys_tmp = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * M));
    sc.vals_tmp = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * M));
    sc.leaf_parent = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * M));
    sc.node_parent = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * M));
    sc.refit_flag = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * M));
    sc.hist = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * 256 * kNoallocTiles));
    sc.bounds = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * 6));
    sc.status = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t)));
    return off;
}

irgs_status build_lbvh_noalloc_impl(const irgs_surfels* s, float alpha_min, int32_t* perm, uint32_t* keys,
                                    float* nodes, float* leaf_boxes, cudaStream_t st) {
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return IRGS_ERR_CUDA;
    unsigned char* base = static_cast<unsigned char*>(noalloc_scratch(device));
    if (base == nullptr) return IRGS_ERR_CUDA;
    irgs_scene_s sc;   // a view onto caller buffers and the scratch array
    sc.device = device;
    sc.n = s->n;
    sc.F = 0;
    sc.alpha_min = alpha_min;
    const size_t used = noalloc_carve(base, sc);
    sc.keys = keys;
    sc.perm = perm;
    sc.nodes = reinterpret_cast<Node*>(nodes);
    sc.leaf_box = leaf_boxes;
    if (used > kNoallocBytes) return IRGS_ERR_CUDA;   // carve-out mismatch (cannot happen)
    if (cudaMemsetAsync(sc.status, 0, sizeof(uint32_t), st) != cudaSuccess) return IRGS_ERR_CUDA;
    return enqueue_build(&sc, s, st);
}

irgs_status lbvh_noalloc_status_impl(cudaStream_t st, uint32_t* bits) {
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return IRGS_ERR_CUDA;
    unsigned char* base = static_cast<unsigned char*>(noalloc_scratch(device));
    if (base == nullptr) return IRGS_ERR_CUDA;
    irgs_scene_s sc;
    noalloc_carve(base, sc);
    uint32_t h = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess) return IRGS_ERR_CUDA;
    if (cudaMemcpy(&h, sc.status, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return IRGS_ERR_CUDA;
    if (bits) *bits = h;
    return h == 0u ? IRGS_OK : IRGS_ERR_DEVICE;
}

}  // namespace irgs
