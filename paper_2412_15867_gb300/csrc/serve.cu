// Serving: one persistent launch per scheduling step processes the trace
// tiles of many requests over several resident scenes. Blocks pull tiles
// from the step's tile table with an atomic counter until it is exhausted; a
// tile is up to a few thousand camera rays. The step (staging copy, counter
// reset, kernel) can be captured once into a CUDA graph and replayed with new
// table contents. The shading tiles of the step then run, one request's range
// of G-buffer points at a time, through the wavefront shading path (secondary
// rays regrouped by direction and origin, traced in that order, estimated
// per point), keyed by pixel index, so a pixel's estimate is the one
// irgs_shade_mc gives for it.
//
// Work per tile kind (IRGS Eq. 8 for the traces, Eq. 13-15 for shading):
//   render  : camera rays (or the request's own rays) -> Trace -> feat /
//             depth / opacity per pixel;
//   gbuffer : camera rays -> Trace of the material channels (albedo,
//             roughness, normal) -> per-pixel G-buffer normalised by the
//             opacity (Eq. 9): x = o + (D/O) d, n, a, r, w_o = -d;
//   shade   : G-buffer points -> Monte Carlo rendering equation.
// Each result depends only on its own request (camera, seed, pixel index),
// never on what else shares the step.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>

#include "../../include/irgs.h"
#include "camera.cuh"
#include "scene.h"
#include "shade.cuh"
#include "trace.cuh"

struct irgs_server_s {
    int device = 0;
    int n_scenes = 0;
    int max_jobs = 0, max_tiles = 0;
    size_t stage_bytes = 0;
    unsigned char* host_stage = nullptr;   // pinned: [header 16 B][jobs][tiles]
    unsigned char* dev_stage = nullptr;
    irgs::SceneView* dev_scenes = nullptr;
    int* dev_next = nullptr;
    int grid = 0;
    irgs::TraceParams render{}, gbuf{};
    irgs_trace_params shade_params{};          // the shading calls' trace parameters
    irgs::SceneView* host_views = nullptr;     // [n_scenes] the scenes' views and bounds, for the shading calls
    const uint32_t** host_bounds = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph = nullptr;
};

namespace irgs {
namespace {

constexpr int kServeThreads = 128;
constexpr int kServeK = 16;
constexpr size_t kHeaderBytes = 16;

struct ServeArgs {
    const SceneView* scenes;
    const int32_t* header;   // [0] jobs, [1] tiles
    const irgs_job* jobs;
    const irgs_tile* tiles;
    int* next_tile;
    TraceParams render, gbuf;
};

// Pixel p of a camera (tile by tile when tile_w x tile_h > 1) -> ray.
__device__ __forceinline__ void camera_ray(const irgs_camera& c, int64_t p, f3& o, f3& d) {
    const int tw = c.tile_w, th = c.tile_h;
    const int64_t per = (int64_t)tw * th;
    const int64_t tile = p / per, within = p - tile * per;
    const int64_t tiles_x = c.width / tw;
    const int64_t ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const float px = (float)(tx * tw + within % tw), py = (float)(ty * th + within / tw);
    d = camera_dir(c, px, py);
    o = mk3(c.origin[0], c.origin[1], c.origin[2]);
}

__global__ void k_camera_rays(irgs_camera c, int64_t first, int64_t count, float* __restrict__ ro,
                              float* __restrict__ rd) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    f3 o, d;
    camera_ray(c, first + i, o, d);
    ro[3 * i] = o.x; ro[3 * i + 1] = o.y; ro[3 * i + 2] = o.z;
    rd[3 * i] = d.x; rd[3 * i + 1] = d.y; rd[3 * i + 2] = d.z;
}

__global__ void __launch_bounds__(kServeThreads) k_serve(ServeArgs A) {
    static_assert(kServeThreads == trace_threads<kServeK>(), "k-buffer slots are laid out per block thread");
    __shared__ int s_tile;
    const int n_tiles = A.header[1];
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(A.next_tile, 1);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= n_tiles) return;
        const irgs_tile tile = A.tiles[t];
        const irgs_job& job = A.jobs[tile.job];
        const SceneView S = A.scenes[job.scene];
        if (tile.kind == IRGS_TILE_RENDER || tile.kind == IRGS_TILE_GBUFFER) {
            const bool render = tile.kind == IRGS_TILE_RENDER;
            const TraceParams& P = render ? A.render : A.gbuf;
            for (int i0 = 0; i0 < tile.count; i0 += kServeThreads) {
                const int i = i0 + threadIdx.x;
                const bool live = i < tile.count;
                const int64_t p = (int64_t)tile.first + (live ? i : 0);
                f3 o, d;
                if (job.ray_o != nullptr) {
                    o = mk3(job.ray_o[3 * p], job.ray_o[3 * p + 1], job.ray_o[3 * p + 2]);
                    d = mk3(job.ray_d[3 * p], job.ray_d[3 * p + 1], job.ray_d[3 * p + 2]);
                } else {
                    camera_ray(job.cam, p, o, d);
                }
                const Ray ray = make_ray(o, d);
                MarchState<kServeK, 10> st;
                const bool ok = march_forward<kServeK, 10, true>(S, ray, P, st, nullptr, 0, live);
                if (!live) continue;
                if (!ok) atomicOr(S.status, kErrStackOverflow);
                if (render) {
#pragma unroll
                    for (int c = 0; c < 10; ++c)
                        if (c < P.fc) job.feat[p * P.fc + c] = st.C[c];
                    job.depth[p] = st.D;
                    job.opacity[p] = 1.f - st.T;
                } else {
                    // Eq. 9 normalisation by the accumulated opacity, into the
                    // planar G-buffer of P = width x height pixels
                    const int64_t Pj = (int64_t)job.cam.width * job.cam.height;
                    const float O = 1.f - st.T;
                    float* g = job.gbuffer;
                    const bool valid = O > 0.5f;
                    const float inv = valid ? 1.f / O : 0.f;
                    const f3 x = add3(o, mul3(d, st.D * inv));
                    f3 nn = mk3(st.C[4], st.C[5], st.C[6]);
                    const float nl = sqrtf(dot3(nn, nn));
                    nn = nl > 0.f ? mul3(nn, 1.f / nl) : mk3(0.f, 0.f, 1.f);
                    float* gx = g + 3 * p;
                    float* gn = g + 3 * Pj + 3 * p;
                    float* ga = g + 6 * Pj + 3 * p;
                    float* gw = g + 10 * Pj + 3 * p;
                    gx[0] = x.x; gx[1] = x.y; gx[2] = x.z;
                    gn[0] = nn.x; gn[1] = nn.y; gn[2] = nn.z;
                    ga[0] = st.C[0] * inv; ga[1] = st.C[1] * inv; ga[2] = st.C[2] * inv;
                    g[9 * Pj + p] = st.C[3] * inv;
                    gw[0] = -d.x; gw[1] = -d.y; gw[2] = -d.z;
                    g[13 * Pj + p] = valid ? 1.f : 0.f;
                    g[14 * Pj + p] = O;
                    g[15 * Pj + p] = 0.f;
                }
            }
        }
        // shading tiles run after this kernel through the wavefront path
    }
}

void server_free(irgs_server s) {
    if (!s) return;
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    if (s->ev_out) cudaEventDestroy(s->ev_out);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->host_stage) cudaFreeHost(s->host_stage);
    if (s->dev_stage) cudaFree(s->dev_stage);
    if (s->dev_scenes) cudaFree(s->dev_scenes);
    if (s->dev_next) cudaFree(s->dev_next);
    delete[] s->host_views;
    delete[] s->host_bounds;
    delete s;
}

ServeArgs args_of(irgs_server s) {
    ServeArgs A;
    A.scenes = s->dev_scenes;
    A.header = reinterpret_cast<const int32_t*>(s->dev_stage);
    A.jobs = reinterpret_cast<const irgs_job*>(s->dev_stage + kHeaderBytes);
    A.tiles = reinterpret_cast<const irgs_tile*>(s->dev_stage + kHeaderBytes + sizeof(irgs_job) * s->max_jobs);
    A.next_tile = s->dev_next;
    A.render = s->render;
    A.gbuf = s->gbuf;
    return A;
}

// The step's device work on the server stream: staging copy, counter reset,
// persistent kernel.
cudaError_t enqueue_step(irgs_server s) {
    cudaError_t e = cudaMemcpyAsync(s->dev_stage, s->host_stage, s->stage_bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->dev_next, 0, sizeof(int), s->stream);
    if (e == cudaSuccess) {
        k_serve<<<s->grid, kServeThreads, 0, s->stream>>>(args_of(s));
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace
}  // namespace irgs

extern "C" {

irgs_status irgs_server_create(const irgs_scene* scenes, int32_t n_scenes, int32_t max_jobs, int32_t max_tiles,
                               int32_t material_offset, const irgs_trace_params* render,
                               const irgs_trace_params* shade, irgs_server* out) {
    using namespace irgs;
    if (!scenes || n_scenes <= 0 || max_jobs <= 0 || max_tiles <= 0 || !render || !shade || !out)
        return IRGS_ERR_INVALID_ARG;
    if (render->k != kServeK || shade->k != kServeK) return IRGS_ERR_UNSUPPORTED;
    if (render->feat_count < 0 || render->feat_count > 10 || shade->feat_count != 3 || !(shade->t_min > 0.f) ||
        shade->flags != 0u)
        return IRGS_ERR_INVALID_ARG;
    for (int i = 0; i < n_scenes; ++i) {
        if (!scenes[i]) return IRGS_ERR_INVALID_ARG;
        const irgs_scene sc = scenes[i];
        if (render->feat_offset + render->feat_count > sc->F || material_offset < 0 || material_offset + 7 > sc->F ||
            shade->feat_offset + 3 > sc->F || render->alpha_min < sc->alpha_min || shade->alpha_min < sc->alpha_min)
            return IRGS_ERR_INVALID_ARG;
        if (sc->device != scenes[0]->device) return IRGS_ERR_INVALID_ARG;
    }
    irgs_server s = new (std::nothrow) irgs_server_s();
    if (!s) return IRGS_ERR_OOM;
    s->device = scenes[0]->device;
    irgs::DeviceGuard dg;
    if (!dg.set(s->device)) {
        delete s;
        return IRGS_ERR_CUDA;
    }
    s->n_scenes = n_scenes;
    s->max_jobs = max_jobs;
    s->max_tiles = max_tiles;
    s->stage_bytes = kHeaderBytes + sizeof(irgs_job) * (size_t)max_jobs + sizeof(irgs_tile) * (size_t)max_tiles;
    s->render = to_params(*render);
    s->shade_params = *shade;
    s->host_views = new (std::nothrow) SceneView[n_scenes];
    s->host_bounds = new (std::nothrow) const uint32_t*[n_scenes];
    if (!s->host_views || !s->host_bounds) {
        server_free(s);
        return IRGS_ERR_OOM;
    }
    for (int i = 0; i < n_scenes; ++i) {
        s->host_views[i] = scenes[i]->view();
        s->host_bounds[i] = scenes[i]->bounds;
    }
    s->gbuf = s->render;
    s->gbuf.off = material_offset;
    s->gbuf.fc = 7;
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&s->host_stage), s->stage_bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->dev_stage), s->stage_bytes);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->dev_scenes), sizeof(SceneView) * n_scenes);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->dev_next), sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        memset(s->host_stage, 0, s->stage_bytes);
        SceneView views[64];
        int done = 0;
        while (e == cudaSuccess && done < n_scenes) {
            const int m = n_scenes - done < 64 ? n_scenes - done : 64;
            for (int i = 0; i < m; ++i) views[i] = scenes[done + i]->view();
            e = cudaMemcpy(s->dev_scenes + done, views, sizeof(SceneView) * m, cudaMemcpyHostToDevice);
            done += m;
        }
    }
    int per_sm = 0, sms = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve, kServeThreads, 0);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess || per_sm <= 0) {
        cudaGetLastError();
        server_free(s);
        return e == cudaErrorMemoryAllocation ? IRGS_ERR_OOM : IRGS_ERR_CUDA;
    }
    s->grid = per_sm * sms;
    *out = s;
    return IRGS_OK;
}

irgs_status irgs_server_staging(irgs_server s, irgs_job** jobs, irgs_tile** tiles) {
    if (!s) return IRGS_ERR_INVALID_ARG;
    if (jobs) *jobs = reinterpret_cast<irgs_job*>(s->host_stage + irgs::kHeaderBytes);
    if (tiles) *tiles = reinterpret_cast<irgs_tile*>(s->host_stage + irgs::kHeaderBytes + sizeof(irgs_job) * s->max_jobs);
    return IRGS_OK;
}

irgs_status irgs_server_step(irgs_server s, int32_t n_jobs, int32_t n_tiles, int32_t use_graph, void* stream) {
    using namespace irgs;
    if (!s || n_jobs < 0 || n_jobs > s->max_jobs || n_tiles < 0 || n_tiles > s->max_tiles) return IRGS_ERR_INVALID_ARG;
    const irgs_job* jobs = reinterpret_cast<const irgs_job*>(s->host_stage + kHeaderBytes);
    const irgs_tile* tiles = reinterpret_cast<const irgs_tile*>(s->host_stage + kHeaderBytes + sizeof(irgs_job) * s->max_jobs);
    for (int t = 0; t < n_tiles; ++t) {   // validate the tables before any device work
        const irgs_tile& tl = tiles[t];
        if (tl.job < 0 || tl.job >= n_jobs || tl.count < 0 || tl.first < 0 || tl.kind < 0 || tl.kind > 2)
            return IRGS_ERR_INVALID_ARG;
        const irgs_job& jb = jobs[tl.job];
        if (jb.scene < 0 || jb.scene >= s->n_scenes) return IRGS_ERR_INVALID_ARG;
        const int64_t P = (int64_t)jb.cam.width * jb.cam.height;
        if (jb.cam.tile_w <= 0 || jb.cam.tile_h <= 0 || jb.cam.width % jb.cam.tile_w || jb.cam.height % jb.cam.tile_h ||
            (int64_t)tl.first + tl.count > P)
            return IRGS_ERR_INVALID_ARG;
        if ((jb.ray_o == nullptr) != (jb.ray_d == nullptr)) return IRGS_ERR_INVALID_ARG;
        if (tl.kind == IRGS_TILE_RENDER && (!jb.depth || !jb.opacity || (s->render.fc > 0 && !jb.feat)))
            return IRGS_ERR_INVALID_ARG;
        if (tl.kind == IRGS_TILE_GBUFFER && !jb.gbuffer) return IRGS_ERR_INVALID_ARG;
        if (tl.kind == IRGS_TILE_SHADE &&
            (!jb.gbuffer || !jb.rgb || !jb.env || jb.env_h <= 0 || jb.env_w <= 0 || jb.n_diffuse < 0 || jb.n_spec < 0 ||
             jb.n_diffuse + jb.n_spec <= 0 || jb.n_diffuse + jb.n_spec > (1 << 24)))
            return IRGS_ERR_INVALID_ARG;
    }
    int32_t* hdr = reinterpret_cast<int32_t*>(s->host_stage);
    hdr[0] = n_jobs;
    hdr[1] = n_tiles;
    irgs::DeviceGuard dg;
    if (!dg.set(s->device)) return IRGS_ERR_CUDA;
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaEventRecord(s->ev_in, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev_in, 0);
    if (e == cudaSuccess && use_graph && !s->graph) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue_step(s);
            e = cudaStreamEndCapture(s->stream, &g);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&s->graph, g, 0);
        if (g) cudaGraphDestroy(g);
    }
    if (e == cudaSuccess) {
        if (use_graph) {
            e = cudaGraphLaunch(s->graph, s->stream);
        } else {
            e = enqueue_step(s);
        }
    }
    count_launches(1);
    // shading tiles: each maximal run of consecutive tiles of one job over
    // consecutive points is one wavefront call on its G-buffer range
    irgs_status ss = IRGS_OK;
    for (int t = 0; t < n_tiles && e == cudaSuccess && ss == IRGS_OK;) {
        const irgs_tile& tl = tiles[t];
        if (tl.kind != IRGS_TILE_SHADE) {
            ++t;
            continue;
        }
        int64_t first = tl.first, count = tl.count;
        int u = t + 1;
        while (u < n_tiles && tiles[u].kind == IRGS_TILE_SHADE && tiles[u].job == tl.job &&
               tiles[u].first == first + count) {
            count += tiles[u].count;
            ++u;
        }
        const irgs_job& jb = jobs[tl.job];
        const int64_t Pj = (int64_t)jb.cam.width * jb.cam.height;
        const float* g = jb.gbuffer;
        ss = launch_shade_wave(s->host_views[jb.scene], s->host_bounds[jb.scene], g + 3 * first, g + 3 * Pj + 3 * first,
                               g + 6 * Pj + 3 * first, g + 9 * Pj + first, g + 10 * Pj + 3 * first, count, jb.env,
                               jb.env_h, jb.env_w, jb.n_diffuse, jb.n_spec, jb.seed, kModeSplit, s->shade_params,
                               jb.rgb + 3 * first, nullptr, nullptr, s->stream, (uint64_t)first, g + 13 * Pj + first);
        t = u;
    }
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_out, s->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, s->ev_out, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return IRGS_ERR_CUDA;
    }
    return ss;
}

irgs_status irgs_server_destroy(irgs_server s) {
    if (!s) return IRGS_OK;
    irgs::DeviceGuard dg;
    dg.set(s->device);
    cudaStreamSynchronize(s->stream);
    irgs::server_free(s);
    return IRGS_OK;
}

irgs_status irgs_camera_rays(const irgs_camera* cam, int64_t first, int64_t count, float* ray_o, float* ray_d,
                             void* stream) {
    if (!cam || first < 0 || count < 0 || (count > 0 && (!ray_o || !ray_d))) return IRGS_ERR_INVALID_ARG;
    if (cam->width <= 0 || cam->height <= 0 || cam->tile_w <= 0 || cam->tile_h <= 0 ||
        cam->width % cam->tile_w || cam->height % cam->tile_h || first + count > (int64_t)cam->width * cam->height)
        return IRGS_ERR_INVALID_ARG;
    if (count == 0) return IRGS_OK;
    const int T = 256;
    irgs::k_camera_rays<<<(unsigned)((count + T - 1) / T), T, 0, static_cast<cudaStream_t>(stream)>>>(*cam, first, count,
                                                                                                     ray_o, ray_d);
    irgs::count_launches(1);
    return cudaGetLastError() == cudaSuccess ? IRGS_OK : IRGS_ERR_CUDA;
}

}  // extern "C"
