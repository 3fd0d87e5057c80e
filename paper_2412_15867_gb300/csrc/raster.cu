// 2D Gaussian tile rasteriser for G-buffers (IRGS Sec. 3.3: the depth,
// normal, albedo and roughness maps of Eq. 9-10 come from 2DGS
// rasterisation; the shading then runs per pixel).
//
// Per pixel the surfels in front of the near plane are blended (Eq. 2) in
// ascending order of their centre's view depth (ties by user index), each
// with rho^2 = min(rho3^2, rho2^2): rho3 from the pixel ray's intersection
// with the surfel plane (Eq. 6-7; +inf when grazing or behind the camera),
// rho2 the distance of the pixel centre to the projected surfel centre over
// sigma = sqrt(1/2) pixel (the 2DGS screen-space low-pass filter). A surfel
// counts where rho^2 <= rho_c^2 and alpha = min(alpha_max, o exp(-rho^2/2))
// >= alpha_min; its depth is the intersection's tau when the ray term
// wins, else the centre's distance along the ray.
//
// Pipeline, GB300 style: per surfel a conservative 16x16-tile rectangle
// (the projected corners of its padded support box, united with the
// filter's disc around the projected centre); one (tile, depth) pair per
// covered tile, emitted in user order; a stable radix sort by depth, then
// by tile; per-tile ranges; then one block of 256 threads per tile walks its
// list in 256-surfel chunks staged in shared memory, each thread blending
// its pixel until T < T_min, the block stopping when every pixel is done.
#include <cuda_runtime.h>

#include "camera.cuh"
#include "scene.h"
#include "trace.cuh"

namespace irgs {
namespace {

constexpr int kTileSide = 16;
constexpr int kTilePix = kTileSide * kTileSide;
constexpr int kRasterFB = 16;          // blended channels handled per pixel
constexpr float kFilterSigma2 = 0.5f;  // screen-space filter variance (pixels^2)

struct RasterCam {
    f3 o, fw, rt, up;
    float tan_half, aspect;
    int W, H, tiles_x, tiles_y;
};

__device__ __forceinline__ void project(const RasterCam& c, f3 p, float& z, float& px, float& py) {
    const f3 q = sub3(p, c.o);
    z = dot3(q, c.fw);
    const float xs = dot3(q, c.rt) / z, ys = dot3(q, c.up) / z;
    px = (xs / (c.tan_half * c.aspect) + 1.f) * 0.5f * (float)c.W - 0.5f;
    py = (1.f - ys / c.tan_half) * 0.5f * (float)c.H - 0.5f;
}

// Per surfel (user order): centre depth key and covered tile rectangle.
__global__ void k_raster_prep(SceneView S, const float* __restrict__ leaf_box, RasterCam c, float near,
                              uint32_t* __restrict__ zkey, int4* __restrict__ rect, uint32_t* __restrict__ count) {
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= S.n) return;
    const int32_t m = S.inv_perm[u];
    const float4 r0 = __ldg(S.rec + (int64_t)m * kRecF4), r1 = __ldg(S.rec + (int64_t)m * kRecF4 + 1);
    const f3 mu = mk3(r0.x, r0.y, r0.z);
    float zc, pxc, pyc;
    project(c, mu, zc, pxc, pyc);
    count[u] = 0;
    if (!(zc > near) || r1.w < 0.f) return;
    // the filter's support: rho2^2 <= rho_c^2 within rho_c sigma pixels of the centre
    const float rf = sqrtf(fmaxf(r1.w, 0.f) * kFilterSigma2);
    float x0 = pxc - rf, x1 = pxc + rf, y0 = pyc - rf, y1 = pyc + rf;
    // the ray term: the support disc lies in the padded leaf box; project its corners
    const float* b = leaf_box + (int64_t)m * 6;
    bool full = false;
    for (int k = 0; k < 8; ++k) {
        const f3 p = mk3(b[(k & 1) ? 3 : 0], b[(k & 2) ? 4 : 1], b[(k & 4) ? 5 : 2]);
        float z, px, py;
        project(c, p, z, px, py);
        if (!(z > 1e-6f)) {
            full = true;   // the box reaches the camera plane: any pixel may see it
            break;
        }
        x0 = fminf(x0, px); x1 = fmaxf(x1, px);
        y0 = fminf(y0, py); y1 = fmaxf(y1, py);
    }
    int px0, px1, py0, py1;
    if (full) {
        px0 = 0; py0 = 0; px1 = c.W - 1; py1 = c.H - 1;
    } else {
        // one pixel of slack for rounding, then clamp to the image
        x0 = fmaxf(x0 - 1.f, -1.f); y0 = fmaxf(y0 - 1.f, -1.f);
        x1 = fminf(x1 + 1.f, (float)c.W); y1 = fminf(y1 + 1.f, (float)c.H);
        px0 = (int)ceilf(x0); px1 = (int)floorf(x1);
        py0 = (int)ceilf(y0); py1 = (int)floorf(y1);
        px0 = max(px0, 0); py0 = max(py0, 0);
        px1 = min(px1, c.W - 1); py1 = min(py1, c.H - 1);
        if (px1 < px0 || py1 < py0) return;
    }
    const int4 t = make_int4(px0 / kTileSide, py0 / kTileSide, px1 / kTileSide, py1 / kTileSide);
    rect[u] = t;
    count[u] = (uint32_t)((t.z - t.x + 1) * (t.w - t.y + 1));
    zkey[u] = __float_as_uint(zc);   // zc > 0: the float bits order like the values
}

// One (depth, tile, Morton slot) triple per covered tile, in user order.
__global__ void k_raster_emit(SceneView S, RasterCam c, const uint32_t* __restrict__ zkey,
                              const int4* __restrict__ rect, const uint32_t* __restrict__ count,
                              const uint32_t* __restrict__ offset, uint32_t* __restrict__ depth_key,
                              uint32_t* __restrict__ tile_key, int32_t* __restrict__ slot,
                              int32_t* __restrict__ pair) {
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= S.n || count[u] == 0) return;
    const int4 t = rect[u];
    const int32_t m = S.inv_perm[u];
    uint32_t j = offset[u];
    for (int ty = t.y; ty <= t.w; ++ty)
        for (int tx = t.x; tx <= t.z; ++tx, ++j) {
            depth_key[j] = zkey[u];
            tile_key[j] = (uint32_t)(ty * c.tiles_x + tx);
            slot[j] = m;
            pair[j] = (int32_t)j;
        }
}

__global__ void k_raster_total(const uint32_t* __restrict__ offset, const uint32_t* __restrict__ count, int64_t n,
                               uint64_t* __restrict__ total) {
    *total = n > 0 ? (uint64_t)offset[n - 1] + count[n - 1] : 0ull;
}

// Tile keys in depth order (the second sort's input).
__global__ void k_raster_gather_tiles(const uint32_t* __restrict__ tile_key, const int32_t* __restrict__ order,
                                      int64_t total, uint32_t* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < total) out[i] = tile_key[order[i]];
}

__global__ void k_raster_ranges(const uint32_t* __restrict__ tiles_sorted, int64_t total, int2* __restrict__ range) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const uint32_t t = tiles_sorted[i];
    if (i == 0 || tiles_sorted[i - 1] != t) range[t].x = (int)i;
    if (i == total - 1 || tiles_sorted[i + 1] != t) range[t].y = (int)(i + 1);
}

// rho3^2 and tau of the pixel ray against one surfel (the ray origin is
// rebased to the closest approach to the centre, as in the tracer, so that
// u and v keep their digits for small surfels far from the camera);
// returns false when grazing or behind the camera.
__device__ __forceinline__ bool ray_term(const float4& r0, const float4& r1, const float4& r2, const float4& r3,
                                         f3 o, f3 d, float& rho2, float& tau) {
    float ahx, alx, ahy, aly, ahz, alz;
    two_sum(r0.x, -o.x, ahx, alx);
    two_sum(r0.y, -o.y, ahy, aly);
    two_sum(r0.z, -o.z, ahz, alz);
    const float tr = __fmaf_rn(ahx, d.x, __fmaf_rn(ahy, d.y, __fmul_rn(ahz, d.z)));   // |d| = 1
    const float dlx = __fadd_rn(__fmaf_rn(-tr, d.x, ahx), alx);
    const float dly = __fadd_rn(__fmaf_rn(-tr, d.y, ahy), aly);
    const float dlz = __fadd_rn(__fmaf_rn(-tr, d.z, ahz), alz);
    const float den = __fmaf_rn(r3.x, d.x, __fmaf_rn(r3.y, d.y, __fmul_rn(r3.z, d.z)));
    if (!(fabsf(den) >= 1e-8f)) return false;
    const float num = __fmaf_rn(r3.x, dlx, __fmaf_rn(r3.y, dly, __fmul_rn(r3.z, dlz)));
    const float tp = __fdiv_rn(num, den);
    tau = tr + tp;
    if (!(tau > 0.f)) return false;
    const float ex = __fmaf_rn(tp, d.x, -dlx), ey = __fmaf_rn(tp, d.y, -dly), ez = __fmaf_rn(tp, d.z, -dlz);
    const float u = __fmaf_rn(ex, r1.x, __fmaf_rn(ey, r1.y, __fmul_rn(ez, r1.z)));
    const float v = __fmaf_rn(ex, r2.x, __fmaf_rn(ey, r2.y, __fmul_rn(ez, r2.z)));
    rho2 = __fmaf_rn(u, u, __fmul_rn(v, v));
    return true;
}

template <int FB>
__global__ void __launch_bounds__(kTilePix) k_raster_render(SceneView S, RasterCam c, irgs_camera cam,
                                                            TraceParams P, const int2* __restrict__ range,
                                                            const int32_t* __restrict__ order,
                                                            const int32_t* __restrict__ slot,
                                                            float* __restrict__ feat, float* __restrict__ depth,
                                                            float* __restrict__ opac, int32_t* __restrict__ nhits) {
    __shared__ float4 s_rec[4][kTilePix];
    __shared__ float2 s_ctr[kTilePix];
    __shared__ float s_feat[FB][kTilePix];
    const int tile = blockIdx.x;
    const int tx = tile % c.tiles_x, ty = tile / c.tiles_x;
    const int px = tx * kTileSide + (threadIdx.x % kTileSide), py = ty * kTileSide + (threadIdx.x / kTileSide);
    const bool inside = px < c.W && py < c.H;
    const f3 d = camera_dir(cam, (float)px, (float)py);
    const float fpx = (float)px, fpy = (float)py;
    float C[FB];
#pragma unroll
    for (int k = 0; k < FB; ++k) C[k] = 0.f;
    float D = 0.f, T = 1.f;
    int nh = 0;
    bool done = !inside;
    const int2 rg = range[tile];
    for (int base = rg.x; base < rg.y; base += kTilePix) {
        if (__syncthreads_count(!done) == 0) break;
        const int j = base + (int)threadIdx.x;
        if (j < rg.y) {
            const int32_t m = slot[order[j]];
            const float4* Rp = S.rec + (int64_t)m * kRecF4;
#pragma unroll
            for (int k = 0; k < 4; ++k) s_rec[k][threadIdx.x] = __ldg(Rp + k);
            float zc, pxc, pyc;
            project(c, mk3(s_rec[0][threadIdx.x].x, s_rec[0][threadIdx.x].y, s_rec[0][threadIdx.x].z), zc, pxc, pyc);
            s_ctr[threadIdx.x] = make_float2(pxc, pyc);
            const float* f = S.feat + (int64_t)m * S.F + P.off;
#pragma unroll
            for (int k = 0; k < FB; ++k) s_feat[k][threadIdx.x] = k < P.fc ? __ldg(f + k) : 0.f;
        }
        __syncthreads();
        const int cnt = min(kTilePix, rg.y - base);
        for (int i = 0; i < cnt && !done; ++i) {
            const float4 r0 = s_rec[0][i], r1 = s_rec[1][i], r2 = s_rec[2][i], r3 = s_rec[3][i];
            float rho3 = INFINITY, tau = 0.f;
            const bool hit3 = ray_term(r0, r1, r2, r3, c.o, d, rho3, tau);
            const float2 ctr = s_ctr[i];
            const float dx = fpx - ctr.x, dy = fpy - ctr.y;
            const float rho2d = (dx * dx + dy * dy) / kFilterSigma2;
            const float rho2 = hit3 ? fminf(rho3, rho2d) : rho2d;
            if (!(rho2 <= r1.w)) continue;
            const float alpha = fminf(r0.w * __expf(-0.5f * rho2), P.alpha_max);
            if (!(alpha >= P.alpha_min)) continue;
            const float dep = (hit3 && rho3 <= rho2d) ? tau : dot3(sub3(mk3(r0.x, r0.y, r0.z), c.o), d);
            const float w = T * alpha;
#pragma unroll
            for (int k = 0; k < FB; ++k) C[k] = fmaf(w, s_feat[k][i], C[k]);
            D = fmaf(w, dep, D);
            T *= 1.f - alpha;
            ++nh;
            if (T < P.T_min) done = true;
        }
    }
    if (!inside) return;
    const int64_t p = (int64_t)py * c.W + px;
#pragma unroll
    for (int k = 0; k < FB; ++k)
        if (k < P.fc) feat[p * P.fc + k] = C[k];
    depth[p] = D;
    opac[p] = 1.f - T;
    if (nhits != nullptr) nhits[p] = nh;
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

}  // namespace

irgs_status launch_rasterize(const SceneView& S, const float* leaf_box, const irgs_camera& cam,
                             const irgs_trace_params& p, float* feat, float* depth, float* opac, int32_t* nhits,
                             cudaStream_t st) {
    const TraceParams P = to_params(p);
    RasterCam c;
    const auto v3 = [](const float* a) { f3 r; r.x = a[0]; r.y = a[1]; r.z = a[2]; return r; };
    c.o = v3(cam.origin);
    c.fw = v3(cam.forward);
    c.rt = v3(cam.right);
    c.up = v3(cam.up);
    c.tan_half = cam.tan_half_fov;
    c.aspect = (float)cam.width / (float)cam.height;
    c.W = cam.width;
    c.H = cam.height;
    c.tiles_x = (cam.width + kTileSide - 1) / kTileSide;
    c.tiles_y = (cam.height + kTileSide - 1) / kTileSide;
    const int64_t n_tiles = (int64_t)c.tiles_x * c.tiles_y;
    const int64_t n = S.n;
    // per-surfel scratch + per-tile ranges
    const int64_t nn = n > 0 ? n : 1;
    unsigned char* base = nullptr;
    const size_t b_z = 4 * nn, b_rect = 16 * nn, b_cnt = 4 * nn, b_off = 4 * nn, b_rng = 8 * n_tiles, b_tot = 16;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t total_bytes = al(b_z) + al(b_rect) + al(b_cnt) + al(b_off) + al(b_rng) + al(b_tot);
    cudaError_t e = scratch_alloc(reinterpret_cast<void**>(&base), total_bytes, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? IRGS_ERR_OOM : IRGS_ERR_CUDA;
    size_t off = 0;
    auto take = [&](size_t b) { unsigned char* q = base + off; off += al(b); return q; };
    uint32_t* zkey = reinterpret_cast<uint32_t*>(take(b_z));
    int4* rect = reinterpret_cast<int4*>(take(b_rect));
    uint32_t* count = reinterpret_cast<uint32_t*>(take(b_cnt));
    uint32_t* offset = reinterpret_cast<uint32_t*>(take(b_off));
    int2* range = reinterpret_cast<int2*>(take(b_rng));
    uint64_t* d_total = reinterpret_cast<uint64_t*>(take(b_tot));
    unsigned char* pairs = nullptr;
    uint64_t total = 0;
    if (n > 0) {
        k_raster_prep<<<grid_for(n, 256), 256, 0, st>>>(S, leaf_box, c, P.t_min, zkey, rect, count);
        e = cudaMemcpyAsync(offset, count, 4 * n, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = scan_exclusive(offset, n, st);
        k_raster_total<<<1, 1, 0, st>>>(offset, count, n, d_total);
        count_launches(2);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&total, d_total, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(range, 0, b_rng, st);
    if (e == cudaSuccess && total > (uint64_t)INT32_MAX) e = cudaErrorInvalidValue;
    if (e == cudaSuccess && total > 0) {
        const int64_t T = (int64_t)total;
        const int64_t hw = sort_hist_words(T);
        const size_t b4 = 4 * (size_t)T;
        const size_t pb = al(b4) * 7 + al(4 * (size_t)hw);
        e = scratch_alloc(reinterpret_cast<void**>(&pairs), pb, st);
        if (e == cudaSuccess) {
            size_t o2 = 0;
            auto take2 = [&](size_t b) { unsigned char* q = pairs + o2; o2 += al(b); return q; };
            uint32_t* depth_key = reinterpret_cast<uint32_t*>(take2(b4));
            uint32_t* tile_key = reinterpret_cast<uint32_t*>(take2(b4));
            int32_t* slot = reinterpret_cast<int32_t*>(take2(b4));
            int32_t* order = reinterpret_cast<int32_t*>(take2(b4));
            uint32_t* ktmp = reinterpret_cast<uint32_t*>(take2(b4));
            int32_t* vtmp = reinterpret_cast<int32_t*>(take2(b4));
            uint32_t* tiles_sorted = reinterpret_cast<uint32_t*>(take2(b4));
            uint32_t* hist = reinterpret_cast<uint32_t*>(take2(4 * (size_t)hw));
            k_raster_emit<<<grid_for(n, 256), 256, 0, st>>>(S, c, zkey, rect, count, offset, depth_key, tile_key,
                                                            slot, order);
            // by depth (stable: equal depths keep user order), then by tile (stable)
            e = sort_pairs(depth_key, order, ktmp, vtmp, hist, T, st, 32);
            k_raster_gather_tiles<<<grid_for(T, 256), 256, 0, st>>>(tile_key, order, T, tiles_sorted);
            int bits = 1;
            while (bits < 32 && ((int64_t)1 << bits) < n_tiles) ++bits;
            if (e == cudaSuccess) e = sort_pairs(tiles_sorted, order, ktmp, vtmp, hist, T, st, bits);
            k_raster_ranges<<<grid_for(T, 256), 256, 0, st>>>(tiles_sorted, T, range);
            count_launches(3);
        }
    }
    if (e == cudaSuccess) {
        const unsigned g = (unsigned)n_tiles;
        int32_t* order = nullptr;
        int32_t* slot = nullptr;
        if (pairs != nullptr) {
            const size_t b4 = al(4 * (size_t)total);
            slot = reinterpret_cast<int32_t*>(pairs + 2 * b4);
            order = reinterpret_cast<int32_t*>(pairs + 3 * b4);
        }
        if (P.fc <= 3)
            k_raster_render<3><<<g, kTilePix, 0, st>>>(S, c, cam, P, range, order, slot, feat, depth, opac, nhits);
        else if (P.fc <= 10)
            k_raster_render<10><<<g, kTilePix, 0, st>>>(S, c, cam, P, range, order, slot, feat, depth, opac, nhits);
        else
            k_raster_render<kRasterFB><<<g, kTilePix, 0, st>>>(S, c, cam, P, range, order, slot, feat, depth, opac,
                                                               nhits);
        count_launches(1);
        e = cudaGetLastError();
    }
    const cudaError_t e1 = pairs ? cudaFreeAsync(pairs, st) : cudaSuccess;
    const cudaError_t e2 = cudaFreeAsync(base, st);
    if (e == cudaErrorMemoryAllocation) return IRGS_ERR_OOM;
    if (e == cudaErrorInvalidValue) return IRGS_ERR_UNSUPPORTED;
    return (e == cudaSuccess && e1 == cudaSuccess && e2 == cudaSuccess) ? IRGS_OK : IRGS_ERR_CUDA;
}

}  // namespace irgs
