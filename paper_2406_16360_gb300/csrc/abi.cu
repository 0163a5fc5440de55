// abi.cu -- the extern "C" entry points of libmirres (include/mirres.h): argument checks,
// workspace management and the launch sequences of the plain and batched paths.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "render.h"

static thread_local std::string g_err;

void mr_set_error(const std::string& msg) { g_err = msg; }

mirres_status mr_cuda_status(cudaError_t e, const char* what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MIRRES_ERR_OOM : MIRRES_ERR_CUDA;
}

static mirres_status arg_error(const std::string& msg)
{
    g_err = msg;
    return MIRRES_ERR_ARG;
}

#define MR_TRY(x)                            \
    do {                                     \
        mirres_status s__ = (x);             \
        if (s__ != MIRRES_OK) return s__;    \
    } while (0)

static cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// samples per chunk of the plain wavefront path (queue capacity)
static const uint32_t kChunk = 1u << 22;
static const size_t kQueueCnt = 1024;

SceneDev mr_scene_dev(const mirres_scene* s)
{
    SceneDev d;
    d.nodes = MR_DFS_NODES ? s->dnodes : s->nodes;
    d.ptri = s->ptri;
    d.leaf_of = s->leaf_of;
    d.tris = s->desc.tris;
    d.tri_uv = s->desc.tri_uv;
    d.albedo = s->desc.albedo;
    d.rough = s->desc.roughness;
    d.metal = s->desc.metallic;
    d.env_texel = s->env_texel;
    d.env_row = s->env_row;
    d.env_col = s->env_col;
    d.env_fine = (s->desc.env_w >= 64 && s->desc.env_h >= 32) ? 1 : 0;
    d.env_flat = s->env_flat;
    d.env_gflat = s->env_gflat;
    d.gf_shift = s->gf_shift;
    d.n_tris = s->desc.n_tris;
    d.n_verts = s->desc.n_verts;
    d.tw = s->desc.tex_w;
    d.th = s->desc.tex_h;
    d.ew = s->desc.env_w;
    d.eh = s->desc.env_h;
    d.env_ok_dev = s->env_ok;
    d.tmin_dev = s->tmin;
    d.vnrm = s->normals ? s->vnrm : nullptr;
    d.gvn = s->normals ? s->gvn : nullptr;
    d.err = s->ctx->counters + CNT_ERROR;
    d.trav_cap = 0;
    d.wnodes = (s->traversal == MIRRES_TRAVERSAL_WIDE && s->built) ? s->wnodes : nullptr;
    d.wtri = (s->traversal == MIRRES_TRAVERSAL_WIDE && s->built) ? s->wtri : nullptr;
    return d;
}

// ---- workspace --------------------------------------------------------------------------
static mirres_status ws_reserve(mirres_context* ctx, size_t bytes)
{
    if (bytes <= ctx->ws.bytes) return MIRRES_OK;
    if (ctx->ws.ptr) {
        MR_CUDA(cudaDeviceSynchronize());
        cudaFree(ctx->ws.ptr);
        ctx->ws.ptr = nullptr;
        ctx->ws.bytes = 0;
    }
    const size_t want = bytes + bytes / 4 + (1u << 20);
    cudaError_t e = cudaMalloc(&ctx->ws.ptr, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&ctx->ws.ptr, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->ws.ptr = nullptr;
            g_err = "workspace allocation of " + std::to_string(bytes) + " bytes failed";
            return MIRRES_ERR_OOM;
        }
        ctx->ws.bytes = bytes;
        return MIRRES_OK;
    }
    ctx->ws.bytes = want;
    return MIRRES_OK;
}

struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* p) : base(static_cast<char*>(p)) {}
    template <typename T>
    T* take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += sizeof(T) * count;
        return p;
    }
};

// ---- argument checks ----------------------------------------------------------------------
static mirres_status check_views(const mirres_view* views, int32_t n_views, int32_t n_scenes,
                                 std::vector<ViewDev>& out, uint64_t& total, uint64_t& max_view)
{
    if (n_views < 1 || n_views > 65535) return arg_error("n_views must be in [1, 65535]");
    if (!views) return arg_error("views is NULL");
    out.resize((size_t)n_views);
    total = 0;
    max_view = 0;
    for (int i = 0; i < n_views; ++i) {
        const mirres_view& v = views[i];
        if (v.width < 1 || v.height < 1 || v.spp < 1 || v.bounces < 1 || v.bounces > 255)
            return arg_error("view " + std::to_string(i) + ": width, height, spp >= 1 and bounces in [1, 255]");
        const uint64_t n = (uint64_t)v.width * (uint64_t)v.height * (uint64_t)v.spp;
        if (n > 0xFFFFFFFFull) return arg_error("view " + std::to_string(i) + ": width*height*spp exceeds 2^32-1");
        if (v.scene < 0 || v.scene >= n_scenes) return arg_error("view " + std::to_string(i) + ": bad scene index");
        if (!(v.K[0] != 0.0f) || !(v.K[1] != 0.0f)) return arg_error("view " + std::to_string(i) + ": fx, fy == 0");
        ViewDev& d = out[(size_t)i];
        std::memcpy(d.K, v.K, sizeof(d.K));
        std::memcpy(d.c2w, v.c2w, sizeof(d.c2w));
        d.width = v.width;
        d.height = v.height;
        d.spp = v.spp;
        d.bounces = v.bounces;
        d.scene = v.scene;
        d.index = i;
        d.offset = total;
        total += n;
        max_view = std::max(max_view, n);
    }
    return MIRRES_OK;
}

static mirres_status check_scenes(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                                  std::vector<SceneDev>& out, int32_t trav_cap = 0)
{
    if (n_scenes < 1 || !scenes) return arg_error("need at least one scene");
    out.resize((size_t)n_scenes);
    for (int i = 0; i < n_scenes; ++i) {
        if (!scenes[i]) return arg_error("scene " + std::to_string(i) + " is NULL");
        if (scenes[i]->ctx != ctx) return arg_error("scene " + std::to_string(i) + " belongs to another context");
        if (!scenes[i]->built) {
            g_err = "scene " + std::to_string(i) + ": call mirres_bvh_build first";
            return MIRRES_ERR_STATE;
        }
        out[(size_t)i] = mr_scene_dev(scenes[i]);
        out[(size_t)i].trav_cap = trav_cap;

    }
    return MIRRES_OK;
}

static mirres_status check_params(const mirres_params* p)
{
    if (!p) return arg_error("params is NULL");
    if (p->ris_m < 1) return arg_error("ris_m must be >= 1");
    if (p->grad_mode != 0 && p->grad_mode != 1) return arg_error("grad_mode must be 0 (PRIMARY) or 1 (FULL)");
    if (p->launch < 0 || p->launch > 2)
        return arg_error("launch must be 0 (plain), 1 (batched wavefront) or 2 (persistent kernel)");
    if (p->block != 0 && (p->block < 32 || p->block > 1024 || p->block % 32))
        return arg_error("block must be 0 or a multiple of 32 in [32, 1024]");
    if (p->blocks_per_sm < 0) return arg_error("blocks_per_sm must be >= 0");
    if (p->reuse_k < 0 || p->reuse_k > MIRRES_REUSE_MAX_K) return arg_error("reuse_k must be in [0, 64]");
    if (p->reuse_k > 0 && (p->reuse_radius < 1 || p->reuse_radius > 1024))
        return arg_error("reuse_radius must be in [1, 1024] when reuse_k > 0");
    if (p->temporal < 0 || p->temporal > 2) return arg_error("temporal must be 0, 1 or 2");
    if (p->temporal == 2 && (p->temporal_cap < 1 || p->temporal_cap > 1 << 20))
        return arg_error("temporal_cap must be in [1, 2^20] when temporal = 2");
    if (p->max_visits < 0) return arg_error("max_visits must be >= 0 (0 = 4 n_tris + 64)");
    return MIRRES_OK;
}

// ---- lifetime -------------------------------------------------------------------------------
extern "C" mirres_status mirres_context_create(int32_t device, mirres_context** out)
{
    if (!out) return arg_error("out is NULL");
    *out = nullptr;
    int n = 0;
    MR_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return arg_error("device index out of range");
    MR_CUDA(cudaSetDevice(device));
    mirres_context* c = new mirres_context();
    c->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->counters, sizeof(unsigned long long) * CNT_N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->queue_cnt, sizeof(unsigned int) * kQueueCnt);
    if (e == cudaSuccess) e = cudaMemset(c->counters, 0, sizeof(unsigned long long) * CNT_N);
    if (e != cudaSuccess) {
        if (c->counters) cudaFree(c->counters);
        if (c->queue_cnt) cudaFree(c->queue_cnt);
        delete c;
        return mr_cuda_status(e, "mirres_context_create");
    }
    *out = c;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_context_destroy(mirres_context* ctx)
{
    if (!ctx) return arg_error("ctx is NULL");
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    for (int i = 0; i < ctx->n_stage_events; ++i) cudaEventDestroy(ctx->stage_events[i]);
    delete[] ctx->stage_events;
    delete[] ctx->stage_kind;
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    for (int b = 0; b < 4; ++b) {
        if (ctx->branch_stream[b]) cudaStreamDestroy(ctx->branch_stream[b]);
        if (ctx->branch_event[b]) cudaEventDestroy(ctx->branch_event[b]);
    }
    if (ctx->ws.ptr) cudaFree(ctx->ws.ptr);
    if (ctx->counters) cudaFree(ctx->counters);
    if (ctx->queue_cnt) cudaFree(ctx->queue_cnt);
    delete ctx;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_scene_create(mirres_context* ctx, const mirres_scene_desc* d, mirres_scene** out)
{
    if (!ctx || !d || !out) return arg_error("ctx, desc and out must not be NULL");
    *out = nullptr;
    if (d->n_tris < 0 || d->n_verts < 0) return arg_error("n_tris and n_verts must be >= 0");
    if (d->n_tris > 0 && (d->n_verts < 1 || !d->verts || !d->tris || !d->tri_uv))
        return arg_error("a scene with triangles needs verts, tris and tri_uv");
    if (d->n_tris > (1 << 30)) return arg_error("n_tris must be < 2^30");
    if (d->tex_w < 1 || d->tex_h < 1 || !d->albedo || !d->roughness || !d->metallic)
        return arg_error("textures: tex_w, tex_h >= 1 and non-NULL albedo, roughness, metallic");
    if ((int64_t)d->tex_w * d->tex_h > (1ll << 30)) return arg_error("texture too large");
    if (d->env_w < 1 || d->env_h < 1 || !d->env) return arg_error("env: env_w, env_h >= 1 and non-NULL env");
    if ((int64_t)d->env_w * d->env_h > (1ll << 28)) return arg_error("env map too large");
    MR_CUDA(cudaSetDevice(ctx->device));
    mirres_scene* s = new mirres_scene();
    s->ctx = ctx;
    s->desc = *d;
    mirres_status st = mr_bvh_alloc(s);
    if (st == MIRRES_OK) st = mr_env_alloc(s);
    if (st == MIRRES_OK) {
        st = mr_check_indices(s, nullptr);
        if (st == MIRRES_ERR_ARG) g_err = "mirres_scene_create: " + g_err;
    }
    if (st != MIRRES_OK) {
        mr_bvh_free(s);
        mr_env_free(s);
        delete s;
        return st;
    }
    *out = s;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_scene_validate(mirres_scene* s, void* stream)
{
    if (!s) return arg_error("scene is NULL");
    MR_CUDA(cudaSetDevice(s->ctx->device));
    const mirres_status st = mr_check_indices(s, as_stream(stream));
    if (st == MIRRES_ERR_ARG) g_err = "mirres_scene_validate: " + g_err;
    return st;
}

extern "C" mirres_status mirres_scene_destroy(mirres_scene* s)
{
    if (!s) return arg_error("scene is NULL");
    cudaSetDevice(s->ctx->device);
    cudaDeviceSynchronize();
    mr_bvh_free(s);
    mr_env_free(s);
    mr_edges_free(s);
    delete s;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_scene_set_normals(mirres_scene* s, int32_t mode)
{
    if (!s) return arg_error("scene is NULL");
    if (mode != MIRRES_NORMALS_FACE && mode != MIRRES_NORMALS_INTERPOLATED) return arg_error("unknown normals mode");
    MR_CUDA(cudaSetDevice(s->ctx->device));
    if (mode == MIRRES_NORMALS_INTERPOLATED) {
        MR_TRY(mr_normals_alloc(s));
        s->normals = mode;
        if (s->built) {
            MR_TRY(mr_vertex_normals(s, nullptr));
            MR_CUDA(cudaStreamSynchronize(nullptr));
        }
    } else {
        s->normals = mode;
    }
    return MIRRES_OK;
}

extern "C" mirres_status mirres_scene_set_traversal(mirres_scene* s, int32_t mode)
{
    if (!s) return arg_error("scene is NULL");
    if (mode != MIRRES_TRAVERSAL_BINARY && mode != MIRRES_TRAVERSAL_WIDE) return arg_error("unknown traversal");
    MR_CUDA(cudaSetDevice(s->ctx->device));
    s->traversal = mode;
    if (mode == MIRRES_TRAVERSAL_WIDE && s->built) {
        MR_TRY(mr_wide_build(s, nullptr));
        MR_CUDA(cudaStreamSynchronize(nullptr));
    }
    return MIRRES_OK;
}

extern "C" mirres_status mirres_bvh_set_builder(mirres_scene* s, int32_t builder)
{
    if (!s) return arg_error("scene is NULL");
    if (builder != MIRRES_BVH_LBVH && builder != MIRRES_BVH_PLOC) return arg_error("unknown BVH builder");
    s->builder = builder;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_bvh_build(mirres_scene* s, void* stream)
{
    if (!s) return arg_error("scene is NULL");
    MR_CUDA(cudaSetDevice(s->ctx->device));
    const cudaStream_t st = as_stream(stream);
    MR_TRY(mr_bvh_build(s, st));
    MR_TRY(mr_env_build(s, st));
    s->ctx->host_launches += 24;
    s->built = true;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_bvh_refit(mirres_scene* s, void* stream)
{
    if (!s) return arg_error("scene is NULL");
    if (!s->built) {
        g_err = "mirres_bvh_refit: call mirres_bvh_build first";
        return MIRRES_ERR_STATE;
    }
    MR_CUDA(cudaSetDevice(s->ctx->device));
    const cudaStream_t st = as_stream(stream);
    MR_TRY(mr_bvh_refit(s, st));
    MR_TRY(mr_env_build(s, st));
    s->ctx->host_launches += 6;
    return MIRRES_OK;
}

// FULL mode records vertices 1 .. max_bounces - 1 of every sample after the primary words
static int full_vertices(const mirres_view* views, int32_t n_views, int32_t grad_mode)
{
    if (grad_mode != 1) return 0;
    int max_b = 1;
    for (int i = 0; i < n_views; ++i) max_b = std::max(max_b, views[i].bounces);
    return max_b - 1;
}

static uint64_t tape_bytes_per_sample(int nvx)
{
    return (uint64_t)MIRRES_TAPE_BYTES_PER_SAMPLE + (uint64_t)MIRRES_TAPE_BYTES_PER_VERTEX * (uint64_t)nvx;
}

extern "C" size_t mirres_tape_bytes_mode(const mirres_view* views, int32_t n_views, int32_t grad_mode)
{
    if (!views || n_views < 1) return 0;
    uint64_t n = 0;
    for (int i = 0; i < n_views; ++i)
        n += (uint64_t)std::max(views[i].width, 0) * (uint64_t)std::max(views[i].height, 0) *
             (uint64_t)std::max(views[i].spp, 0);
    return (size_t)(tape_bytes_per_sample(full_vertices(views, n_views, grad_mode)) * n);
}

extern "C" size_t mirres_reuse_history_bytes(const mirres_view* views, int32_t n_views)
{
    if (!views || n_views < 1) return 0;
    uint64_t n = 0;
    for (int i = 0; i < n_views; ++i)
        n += (uint64_t)std::max(views[i].width, 0) * (uint64_t)std::max(views[i].height, 0) *
             (uint64_t)std::max(views[i].spp, 0);
    return (size_t)(20 * n);
}

extern "C" size_t mirres_tape_bytes(const mirres_view* views, int32_t n_views)
{
    return mirres_tape_bytes_mode(views, n_views, 0);
}

// FULL mode walks at most MIRRES_FULL_MAX_BOUNCES vertices per path
static mirres_status check_full(const mirres_params* p, const mirres_view* views, int32_t n_views)
{
    if (p->grad_mode != 1) return MIRRES_OK;
    for (int i = 0; i < n_views; ++i)
        if (views[i].bounces > MIRRES_FULL_MAX_BOUNCES)
            return arg_error("grad_mode 1 (FULL) supports at most " + std::to_string(MIRRES_FULL_MAX_BOUNCES) +
                             " bounces (view " + std::to_string(i) + ")");
    return MIRRES_OK;
}

// ---- forward ---------------------------------------------------------------------------------
static Rng make_rng(const mirres_params* p)
{
    Rng r;
    r.set(p->seed_lo, p->seed_hi);
    return r;
}

// the default wavefront shape (mirres_wave_shape): 2^25 samples per wave (the queues take 256
// bytes per sample of a wave), 256 threads and 8 blocks per SM for every stage, one chain
// any scene traversed through its 8-wide BVH (the persistent kernel then runs its wide variant)
static bool any_wide(const std::vector<SceneDev>& sdev)
{
    for (const SceneDev& d : sdev)
        if (d.wnodes) return true;
    return false;
}

static mirres_wave_shape default_wave_shape() { return mirres_wave_shape{25, {256, 256, 256, 256}, {8, 8, 8, 8}, 1}; }

static mirres_status check_wave_shape(const mirres_wave_shape& w)
{
    if (w.wave_log2 < 16 || w.wave_log2 > 28) return arg_error("wave_log2 must be in [16, 28]");
    for (int k = 0; k < 4; ++k) {
        if (w.block[k] != 64 && w.block[k] != 128 && w.block[k] != 256)
            return arg_error("block[" + std::to_string(k) + "] must be 64, 128 or 256");
        if (w.blocks_per_sm[k] < 1 || w.blocks_per_sm[k] > 64)
            return arg_error("blocks_per_sm[" + std::to_string(k) + "] must be in [1, 64]");
    }
    if (w.branches < 1 || w.branches > 4) return arg_error("branches must be in [1, 4]");
    return MIRRES_OK;
}

struct GraphKey {
    uint64_t total, total_pix, wave;
    uint64_t layout;  // digest of what the capture decides on the host (layout_digest)
    int32_t n_views, n_scenes, max_b, M, sms, flags, nvx, reuse_k, reuse_radius, temporal, temporal_cap;
    uint32_t k0, k1;
    const void* history;
    const void* tape;
    const void* ws;
    size_t ws_bytes;
    mirres_wave_shape shape;
};

// The host-side choices baked into a captured forward: every view's size, samples, bounces and
// scene (the wave partition, which views a rasterising wave covers) and every scene's triangle
// count and normal mode (raster grids, the interpolated-normal shading kernels). FNV-1a over
// those fields; the cameras and the scenes' device buffers are read from the tables at run time
// and stay out of it.
static uint64_t layout_digest(const std::vector<ViewDev>& vdev, const std::vector<SceneDev>& sdev)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](uint64_t x) {
        for (int k = 0; k < 8; ++k) {
            h ^= (x >> (8 * k)) & 0xffu;
            h *= 1099511628211ull;
        }
    };
    for (const ViewDev& v : vdev) {
        mix(((uint64_t)(uint32_t)v.width << 32) | (uint32_t)v.height);
        mix(((uint64_t)(uint32_t)v.spp << 32) | (uint32_t)v.bounces);
        mix((uint64_t)(uint32_t)v.scene);
    }
    for (const SceneDev& sc : sdev)
        mix(((uint64_t)(uint32_t)sc.n_tris << 2) | (sc.wnodes != nullptr ? 2u : 0u) | (sc.vnrm != nullptr ? 1u : 0u));
    return h;
}

// Batched wavefront: tables uploaded to the workspace, then the whole forward replayed from a
// CUDA graph captured on the context's capture stream (re-captured when the shape, the layout
// digest, the tape, the seed or the workspace changes).
static mirres_status stage_events(mirres_context* ctx, int pairs)
{
    if (ctx->n_stage_events >= 2 * pairs) return MIRRES_OK;
    for (int i = 0; i < ctx->n_stage_events; ++i) cudaEventDestroy(ctx->stage_events[i]);
    delete[] ctx->stage_events;
    delete[] ctx->stage_kind;
    ctx->stage_events = new cudaEvent_t[(size_t)2 * pairs];
    ctx->stage_kind = new int[(size_t)pairs];
    ctx->n_stage_events = 0;
    for (int i = 0; i < 2 * pairs; ++i) {
        MR_CUDA(cudaEventCreate(&ctx->stage_events[i]));
        ctx->n_stage_events = i + 1;
    }
    return MIRRES_OK;
}

static mirres_status render_wave(mirres_context* ctx, const std::vector<SceneDev>& sdev,
                                 const std::vector<ViewDev>& vdev, uint64_t total, float* const* images, void* tape,
                                 int M, Rng rng, int flags, int nvx, int reuse_k, int reuse_radius, int temporal,
                                 int temporal_cap, void* history, cudaStream_t st)
{
    const bool reuse = reuse_k > 0 || temporal > 0;
    const int n_views = (int)vdev.size(), n_scenes = (int)sdev.size();
    int max_b = 1;
    uint64_t total_pix = 0;
    std::vector<uint64_t> pixoff((size_t)n_views);
    for (int i = 0; i < n_views; ++i) {
        max_b = std::max(max_b, vdev[(size_t)i].bounces);
        pixoff[(size_t)i] = total_pix;
        total_pix += (uint64_t)vdev[(size_t)i].width * vdev[(size_t)i].height;
    }
    uint64_t kWave = 1ull << ctx->wave_shape.wave_log2;
    if (reuse) {
        // waves hold whole views (a pixel's neighbours must have been shaded in the same wave):
        // a view larger than the shape's wave gets a wave of its own size
        for (const ViewDev& v : vdev) kWave = std::max<uint64_t>(kWave, (uint64_t)v.width * v.height * v.spp);
    }
    const uint64_t wave = std::min<uint64_t>(total, kWave);
    // wave boundaries: every kWave samples, or with spatial reuse whole views per wave
    std::vector<uint64_t> wave_first;
    if (reuse) {
        uint64_t in_wave = 0;
        for (int i = 0; i < n_views; ++i) {
            const ViewDev& v = vdev[(size_t)i];
            const uint64_t nv = (uint64_t)v.width * v.height * v.spp;
            if (wave_first.empty() || in_wave + nv > kWave) {
                wave_first.push_back(v.offset);
                in_wave = 0;
            }
            in_wave += nv;
        }
    } else {
        for (uint64_t f = 0; f < total; f += wave) wave_first.push_back(f);
    }
    const int n_waves = (int)wave_first.size();
    const int nb = std::min(ctx->wave_shape.branches, n_waves);  // chains of waves
    Carver plan(nullptr);
    plan.take<char>(tape ? 0 : tape_bytes_per_sample(nvx) * total);
    plan.take<ViewDev>((size_t)n_views);
    plan.take<SceneDev>((size_t)n_scenes);
    plan.take<float*>((size_t)n_views);
    plan.take<uint64_t>((size_t)n_views);
    const bool bin = (flags & 8) != 0 && max_b > 1;
    for (int b = 0; b < nb; ++b) {
        plan.take<unsigned int>(5 * (size_t)max_b + 3);
        for (int k = 0; k < 16; ++k) plan.take<float4>(wave);
        plan.take<uint16_t>(bin ? wave : 0);
        plan.take<unsigned int>(bin ? 4096 : 0);
    }
    for (int k = 0; k < 6; ++k) plan.take<uint32_t>(reuse ? total : 0);
    MR_TRY(ws_reserve(ctx, plan.off));
    Carver cv(ctx->ws.ptr);
    void* internal_tape = cv.take<char>(tape ? 0 : tape_bytes_per_sample(nvx) * total);
    void* tp = tape ? tape : internal_tape;
    ViewDev* d_views = cv.take<ViewDev>((size_t)n_views);
    SceneDev* d_scenes = cv.take<SceneDev>((size_t)n_scenes);
    float** d_images = cv.take<float*>((size_t)n_views);
    uint64_t* d_pixoff = cv.take<uint64_t>((size_t)n_views);
    WaveBranch br[4];
    for (int b = 0; b < nb; ++b) {
        br[b].qc = cv.take<unsigned int>(5 * (size_t)max_b + 3);
        br[b].qa = QueueDev{cv.take<float4>(wave), cv.take<float4>(wave), cv.take<float4>(wave), cv.take<float4>(wave)};
        br[b].qb = QueueDev{cv.take<float4>(wave), cv.take<float4>(wave), cv.take<float4>(wave), cv.take<float4>(wave)};
        br[b].hq = QueueDev{cv.take<float4>(wave), cv.take<float4>(wave), cv.take<float4>(wave), cv.take<float4>(wave)};
        br[b].sq = ShadowDev{cv.take<float4>(wave), cv.take<float4>(wave), cv.take<float4>(wave), cv.take<float4>(wave)};
        br[b].bkey = cv.take<uint16_t>(bin ? wave : 0);
        br[b].bhist = cv.take<unsigned int>(bin ? 4096 : 0);
    }
    ResDev res{};
    if (reuse) {
        res.ytex = reinterpret_cast<int32_t*>(cv.take<uint32_t>(total));
        res.sel = reinterpret_cast<int32_t*>(cv.take<uint32_t>(total));
        res.ysub = cv.take<uint32_t>(total);
        res.wsum = reinterpret_cast<float*>(cv.take<uint32_t>(total));
        res.phat = reinterpret_cast<float*>(cv.take<uint32_t>(total));
        res.m = reinterpret_cast<float*>(cv.take<uint32_t>(total));
    }
    HistDev hist{};
    if (temporal > 0) {
        uint32_t* h = reinterpret_cast<uint32_t*>(history);
        hist.ytex = reinterpret_cast<int32_t*>(h);
        hist.ysub = h + total;
        hist.wsum = reinterpret_cast<float*>(h + 2 * total);
        hist.phat = reinterpret_cast<float*>(h + 3 * total);
        hist.m = reinterpret_cast<float*>(h + 4 * total);
    }
    MR_CUDA(cudaMemcpyAsync(d_views, vdev.data(), sizeof(ViewDev) * vdev.size(), cudaMemcpyHostToDevice, st));
    MR_CUDA(cudaMemcpyAsync(d_scenes, sdev.data(), sizeof(SceneDev) * sdev.size(), cudaMemcpyHostToDevice, st));
    MR_CUDA(cudaMemcpyAsync(d_images, images, sizeof(float*) * (size_t)n_views, cudaMemcpyHostToDevice, st));
    MR_CUDA(cudaMemcpyAsync(d_pixoff, pixoff.data(), sizeof(uint64_t) * pixoff.size(), cudaMemcpyHostToDevice, st));

    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.total = total;
    key.total_pix = total_pix;
    key.wave = wave;
    key.layout = layout_digest(vdev, sdev);
    key.n_views = n_views;
    key.n_scenes = n_scenes;
    key.max_b = max_b;
    key.M = M;
    key.sms = ctx->sm_count;
    key.flags = flags & 15;
    key.nvx = nvx;
    key.reuse_k = reuse_k;
    key.reuse_radius = reuse_radius;
    key.temporal = temporal;
    key.temporal_cap = temporal_cap;
    key.history = history;
    key.k0 = rng.rk0[0];
    key.k1 = rng.rk1[0];
    key.tape = tp;
    key.ws = ctx->ws.ptr;
    key.ws_bytes = ctx->ws.bytes;
    key.shape = ctx->wave_shape;
    static_assert(sizeof(GraphKey) <= sizeof(ctx->graph_key), "graph key too large");
    if (!ctx->graph || std::memcmp(ctx->graph_key, &key, sizeof(key)) != 0) {
        if (ctx->graph) {
            cudaGraphExecDestroy(ctx->graph);
            ctx->graph = nullptr;
        }
        if (!ctx->capture_stream) MR_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        br[0].st = ctx->capture_stream;
        for (int b = 0; b < nb; ++b) {
            if (b > 0 && !ctx->branch_stream[b])
                MR_CUDA(cudaStreamCreateWithFlags(&ctx->branch_stream[b], cudaStreamNonBlocking));
            if (nb > 1 && !ctx->branch_event[b])
                MR_CUDA(cudaEventCreateWithFlags(&ctx->branch_event[b], cudaEventDisableTiming));
            if (b > 0) br[b].st = ctx->branch_stream[b];
        }
        const int pairs = mr_wave_stage_pairs(n_waves, max_b);
        if (flags & 1) MR_TRY(stage_events(ctx, pairs));
        MR_CUDA(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        mr_wave_record(d_scenes, d_views, n_views, total, max_b, rng, M, wave_first.data(), n_waves, br, nb,
                       ctx->branch_event[0], ctx->branch_event, tp, ctx->counters, d_pixoff, total_pix, d_images,
                       ctx->sm_count, (flags & 1) ? ctx->stage_events : nullptr,
                       (flags & 1) ? ctx->stage_kind : nullptr, nvx, (flags & 2) != 0, reuse_k, reuse_radius, res,
                       temporal, temporal_cap, hist, vdev.data(), sdev.data(), (flags & 4) != 0, bin,
                       ctx->wave_shape);
        ctx->stage_pairs = (flags & 1) ? pairs : 0;
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(ctx->capture_stream, &g);
        if (ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return mr_cuda_status(ec, "mirres_render: graph capture");
        }
        const cudaError_t ei = cudaGraphInstantiate(&ctx->graph, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            ctx->graph = nullptr;
            return mr_cuda_status(ei, "mirres_render: graph instantiation");
        }
        std::memcpy(ctx->graph_key, &key, sizeof(key));
        int raster_launches = 0;
        if (flags & 4) {
            for (int wv = 0; wv < n_waves; ++wv) {
                const uint64_t f0 = wave_first[(size_t)wv];
                const uint64_t f1 = wv + 1 < n_waves ? wave_first[(size_t)wv + 1] : total;
                for (const ViewDev& v : vdev) {
                    const uint64_t vn = (uint64_t)v.width * v.height * v.spp;
                    if (v.offset < f1 && v.offset + vn > f0 && sdev[(size_t)v.scene].n_tris > 0) raster_launches += 2;
                }
            }
        }
        ctx->graph_launches =
            (unsigned long long)mr_wave_launches(n_waves, max_b, reuse, temporal, raster_launches, bin);
    }
    MR_CUDA(cudaGraphLaunch(ctx->graph, st));
    ctx->host_launches += ctx->graph_launches;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_render(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                                       const mirres_view* views, int32_t n_views, const mirres_params* params,
                                       float* const* images, void* tape, size_t tape_bytes, void* stream)
{
    if (!ctx) return arg_error("ctx is NULL");
    MR_TRY(check_params(params));
    std::vector<SceneDev> sdev;
    MR_TRY(check_scenes(ctx, scenes, n_scenes, sdev, params ? params->max_visits : 0));
    std::vector<ViewDev> vdev;
    uint64_t total = 0, max_view = 0;
    MR_TRY(check_views(views, n_views, n_scenes, vdev, total, max_view));
    if (!images) return arg_error("images is NULL");
    for (int i = 0; i < n_views; ++i)
        if (!images[i]) return arg_error("images[" + std::to_string(i) + "] is NULL");
    MR_TRY(check_full(params, views, n_views));
    const int nvx = full_vertices(views, n_views, params->grad_mode);
    if (tape && tape_bytes < tape_bytes_per_sample(nvx) * total)
        return arg_error("tape_bytes is smaller than mirres_tape_bytes_mode(views, grad_mode)");
    if (tape && (reinterpret_cast<uintptr_t>(tape) & 15)) return arg_error("tape must be 16-byte aligned");
    MR_CUDA(cudaSetDevice(ctx->device));
    const cudaStream_t st = as_stream(stream);
    ctx->last_stream = st;
    const Rng rng = make_rng(params);
    const int M = params->ris_m;
    const int sms = ctx->sm_count;

    if ((params->reuse_k > 0 || params->temporal > 0) && params->launch != 1)
        return arg_error("reservoir reuse (reuse_k > 0 or temporal > 0) is implemented for the batched launch");
    if (params->temporal > 0) {
        if (!params->reuse_history) return arg_error("temporal reuse needs reuse_history");
        if (params->reuse_history_bytes < mirres_reuse_history_bytes(views, n_views))
            return arg_error("reuse_history_bytes is smaller than mirres_reuse_history_bytes(views)");
        if (reinterpret_cast<uintptr_t>(params->reuse_history) & 15)
            return arg_error("reuse_history must be 16-byte aligned");
    }
    if (params->launch == 1)
        return render_wave(ctx, sdev, vdev, total, images, tape, M, rng, params->flags, nvx, params->reuse_k,
                           params->reuse_radius, params->temporal, params->temporal_cap, params->reuse_history, st);

    // workspace layout
    const bool batched = params->launch == 2;
    const uint32_t chunk = (uint32_t)std::min<uint64_t>(max_view, kChunk);
    Carver plan(nullptr);
    plan.take<char>(tape ? 0 : tape_bytes_per_sample(nvx) * total);
    plan.take<ViewDev>((size_t)n_views);
    plan.take<SceneDev>((size_t)n_scenes);
    plan.take<float*>((size_t)n_views);
    plan.take<uint64_t>((size_t)n_views);
    plan.take<unsigned long long>(1);
    if (!batched) plan.take<float4>(16ull * chunk);
    MR_TRY(ws_reserve(ctx, plan.off));
    Carver cv(ctx->ws.ptr);
    void* internal_tape = cv.take<char>(tape ? 0 : tape_bytes_per_sample(nvx) * total);
    void* tp = tape ? tape : internal_tape;
    ViewDev* d_views = cv.take<ViewDev>((size_t)n_views);
    SceneDev* d_scenes = cv.take<SceneDev>((size_t)n_scenes);
    float** d_images = cv.take<float*>((size_t)n_views);
    uint64_t* d_pixoff = cv.take<uint64_t>((size_t)n_views);
    unsigned long long* d_work = cv.take<unsigned long long>(1);

    if (batched) {
        std::vector<uint64_t> pixoff((size_t)n_views);
        uint64_t tp_pix = 0;
        for (int i = 0; i < n_views; ++i) {
            pixoff[(size_t)i] = tp_pix;
            tp_pix += (uint64_t)vdev[(size_t)i].width * vdev[(size_t)i].height;
        }
        MR_CUDA(cudaMemcpyAsync(d_views, vdev.data(), sizeof(ViewDev) * vdev.size(), cudaMemcpyHostToDevice, st));
        MR_CUDA(cudaMemcpyAsync(d_scenes, sdev.data(), sizeof(SceneDev) * sdev.size(), cudaMemcpyHostToDevice, st));
        MR_CUDA(cudaMemcpyAsync(d_images, images, sizeof(float*) * (size_t)n_views, cudaMemcpyHostToDevice, st));
        MR_CUDA(cudaMemcpyAsync(d_pixoff, pixoff.data(), sizeof(uint64_t) * pixoff.size(), cudaMemcpyHostToDevice, st));
        MR_CUDA(cudaMemsetAsync(d_work, 0, sizeof(unsigned long long), st));
        int var = mr_persistent_pick(params->block, params->blocks_per_sm);
        unsigned int chunk_w = 256;
        if (params->block == 0 && ctx->tuned_variant >= 0) {
            var = ctx->tuned_variant;
            chunk_w = ctx->tuned_chunk;
        }
        const int per_sm = params->blocks_per_sm ? params->blocks_per_sm : mr_persistent_occupancy_v(var);
        MR_CUDA(mr_launch_persistent_v(var, d_scenes, d_views, n_views, total, rng, M, d_work, chunk_w, tp,
                                       ctx->counters, per_sm * sms, st, nvx, any_wide(sdev)));
        mr_launch_resolve_all(d_views, n_views, d_pixoff, tp_pix, d_images, tp, total, sms, st);
        MR_CUDA(cudaGetLastError());
        ctx->host_launches += 2;
        return MIRRES_OK;
    }

    // plain: per view, per chunk of at most kChunk samples, one wavefront per bounce
    QueueDev qa{cv.take<float4>(chunk), cv.take<float4>(chunk), cv.take<float4>(chunk), cv.take<float4>(chunk)};
    QueueDev qb{cv.take<float4>(chunk), cv.take<float4>(chunk), cv.take<float4>(chunk), cv.take<float4>(chunk)};
    QueueDev hq{cv.take<float4>(chunk), cv.take<float4>(chunk), cv.take<float4>(chunk), cv.take<float4>(chunk)};
    ShadowDev sq{cv.take<float4>(chunk), cv.take<float4>(chunk), cv.take<float4>(chunk), cv.take<float4>(chunk)};
    for (int vi = 0; vi < n_views; ++vi) {
        const ViewDev& v = vdev[(size_t)vi];
        const SceneDev& s = sdev[(size_t)v.scene];
        const uint64_t nv = (uint64_t)v.width * v.height * v.spp;
        for (uint64_t first = 0; first < nv; first += chunk) {
            const uint32_t n = (uint32_t)std::min<uint64_t>(chunk, nv - first);
            unsigned int* qc = ctx->queue_cnt;
            MR_CUDA(cudaMemsetAsync(qc, 0, sizeof(unsigned int) * (3 * v.bounces + 3), st));
            mr_launch_raygen(v, rng, (uint32_t)first, n, qa, tp, total, sms, st, nvx);
            QueueDev cur = qa, nxt = qb;
            for (int b = 0; b < v.bounces; ++b) {
                // ray queue of bounce b: the raygen output, then the continuations of bounce b-1
                const unsigned int* cnt_in = b == 0 ? nullptr : qc + 3 * (b - 1) + 1;
                mr_launch_closest(s, v, b, cur, cnt_in, n, n, hq, qc + 3 * b, tp, total, sms, st);
                mr_launch_shade(s, v, rng, b, M, hq, qc + 3 * b, n, nxt, qc + 3 * b + 1, sq, qc + 3 * b + 2, tp,
                                total, ctx->counters, sms, st, nvx);
                mr_launch_shadow(s, v, b, sq, qc + 3 * b + 2, n, tp, total, sms, st, nvx);
                std::swap(cur, nxt);
            }
            mr_launch_account(ctx->counters, qc, v.bounces, n, st);
            ctx->host_launches += 2 + 3 * (unsigned long long)v.bounces;
        }
        mr_launch_resolve(v, tp, total, images[vi], sms, st);
        ctx->host_launches += 1;
    }
    MR_CUDA(cudaGetLastError());
    return MIRRES_OK;
}

// ---- autotuning of the persistent launch -----------------------------------------------------
extern "C" mirres_status mirres_autotune(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                                         const mirres_view* views, int32_t n_views, const mirres_params* params,
                                         void* tape, size_t tape_bytes, uint64_t budget_samples,
                                         int32_t* out_block, int32_t* out_blocks_per_sm, int32_t* out_chunk,
                                         float* out_ms, void* stream)
{
    if (!ctx) return arg_error("ctx is NULL");
    MR_TRY(check_params(params));
    std::vector<SceneDev> sdev;
    MR_TRY(check_scenes(ctx, scenes, n_scenes, sdev, params ? params->max_visits : 0));
    std::vector<ViewDev> vdev;
    uint64_t total = 0, max_view = 0;
    MR_TRY(check_views(views, n_views, n_scenes, vdev, total, max_view));
    if (!tape || tape_bytes < (uint64_t)MIRRES_TAPE_BYTES_PER_SAMPLE * total) return arg_error("mirres_autotune needs the full tape of these views");
    MR_CUDA(cudaSetDevice(ctx->device));
    const cudaStream_t st = as_stream(stream);
    const uint64_t n = std::max<uint64_t>(1, std::min<uint64_t>(budget_samples ? budget_samples : total, total));
    Carver plan(nullptr);
    plan.take<ViewDev>((size_t)n_views);
    plan.take<SceneDev>((size_t)n_scenes);
    plan.take<unsigned long long>(1);
    MR_TRY(ws_reserve(ctx, plan.off));
    Carver cv(ctx->ws.ptr);
    ViewDev* d_views = cv.take<ViewDev>((size_t)n_views);
    SceneDev* d_scenes = cv.take<SceneDev>((size_t)n_scenes);
    unsigned long long* d_work = cv.take<unsigned long long>(1);
    MR_CUDA(cudaMemcpyAsync(d_views, vdev.data(), sizeof(ViewDev) * vdev.size(), cudaMemcpyHostToDevice, st));
    MR_CUDA(cudaMemcpyAsync(d_scenes, sdev.data(), sizeof(SceneDev) * sdev.size(), cudaMemcpyHostToDevice, st));
    cudaEvent_t e0, e1;
    MR_CUDA(cudaEventCreate(&e0));
    MR_CUDA(cudaEventCreate(&e1));
    const unsigned int chunks[] = {64u, 256u, 1024u};
    float best = 1e30f;
    int best_v = mr_persistent_pick(0, 0);
    unsigned int best_c = 256u;
    const Rng rng = make_rng(params);
    mirres_status status = MIRRES_OK;
    for (int v = 0; v < mr_persistent_variants() && status == MIRRES_OK; ++v) {
        const int blocks = mr_persistent_occupancy_v(v) * ctx->sm_count;
        for (unsigned int c : chunks) {
            float ms = 0.0f;
            for (int rep = 0; rep < 2; ++rep) {  // the first run warms caches and clocks
                cudaError_t e = cudaMemsetAsync(d_work, 0, sizeof(unsigned long long), st);
                if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                if (e == cudaSuccess)
                    e = mr_launch_persistent_v(v, d_scenes, d_views, n_views, n, rng, params->ris_m, d_work, c, tape,
                                               ctx->counters, blocks, st, 0, any_wide(sdev));
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    status = mr_cuda_status(e, "mirres_autotune");
                    break;
                }
            }
            if (status != MIRRES_OK) break;
            if (ms < best) {
                best = ms;
                best_v = v;
                best_c = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != MIRRES_OK) return status;
    ctx->tuned_variant = best_v;
    ctx->tuned_chunk = best_c;
    int blk, minb;
    mr_persistent_variant_shape(best_v, &blk, &minb);
    if (out_block) *out_block = blk;
    if (out_blocks_per_sm) *out_blocks_per_sm = minb;
    if (out_chunk) *out_chunk = (int32_t)best_c;
    if (out_ms) *out_ms = best;
    ctx->host_launches += (unsigned long long)mr_persistent_variants() * 6;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_set_launch(mirres_context* ctx, int32_t block, int32_t blocks_per_sm, int32_t chunk)
{
    if (!ctx) return arg_error("ctx is NULL");
    if (block == 0) {
        ctx->tuned_variant = -1;
        ctx->tuned_chunk = 256;
        return MIRRES_OK;
    }
    if (chunk < 1) return arg_error("chunk must be >= 1");
    ctx->tuned_variant = mr_persistent_pick(block, blocks_per_sm);
    ctx->tuned_chunk = (unsigned int)chunk;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_set_wave_shape(mirres_context* ctx, const mirres_wave_shape* shape)
{
    if (!ctx) return arg_error("ctx is NULL");
    const mirres_wave_shape w = shape ? *shape : default_wave_shape();
    MR_TRY(check_wave_shape(w));
    ctx->wave_shape = w;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_get_wave_shape(mirres_context* ctx, mirres_wave_shape* out)
{
    if (!ctx || !out) return arg_error("ctx and out must not be NULL");
    *out = ctx->wave_shape;
    return MIRRES_OK;
}

// per-stage times (0 closest, 1 shade, 2 shadow, 3 raygen) of the last render captured with
// stage events
static mirres_status stage_sums(mirres_context* ctx, double ms[4])
{
    for (int k = 0; k < 4; ++k) ms[k] = 0.0;
    for (int p = 0; p < ctx->stage_pairs; ++p) {
        MR_CUDA(cudaEventSynchronize(ctx->stage_events[2 * p + 1]));
        float t = 0.0f;
        MR_CUDA(cudaEventElapsedTime(&t, ctx->stage_events[2 * p], ctx->stage_events[2 * p + 1]));
        ms[ctx->stage_kind[p] & 15] += t;
    }
    return MIRRES_OK;
}

extern "C" mirres_status mirres_autotune_wave(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                                              const mirres_view* views, int32_t n_views, const mirres_params* params,
                                              void* tape, size_t tape_bytes, uint64_t budget_samples,
                                              mirres_wave_shape* out, float* out_ms, void* stream)
{
    if (!ctx) return arg_error("ctx is NULL");
    MR_TRY(check_params(params));
    std::vector<SceneDev> sdev;
    MR_TRY(check_scenes(ctx, scenes, n_scenes, sdev, params->max_visits));
    std::vector<ViewDev> vdev;
    uint64_t total = 0, max_view = 0;
    MR_TRY(check_views(views, n_views, n_scenes, vdev, total, max_view));
    MR_TRY(check_full(params, views, n_views));
    const int nvx = full_vertices(views, n_views, params->grad_mode);
    // the first views up to the budget (at least one)
    const uint64_t budget = budget_samples ? budget_samples : total;
    uint64_t sub_total = 0;
    size_t nv = 0;
    while (nv < vdev.size()) {
        const ViewDev& v = vdev[nv];
        const uint64_t n = (uint64_t)v.width * v.height * v.spp;
        if (nv > 0 && sub_total + n > budget) break;
        sub_total += n;
        ++nv;
    }
    vdev.resize(nv);
    if (!tape || tape_bytes < tape_bytes_per_sample(nvx) * sub_total)
        return arg_error("mirres_autotune_wave needs a tape of the tuned views");
    if (reinterpret_cast<uintptr_t>(tape) & 15) return arg_error("tape must be 16-byte aligned");
    MR_CUDA(cudaSetDevice(ctx->device));
    const cudaStream_t st = as_stream(stream);
    ctx->last_stream = st;
    // temporary images of the tuned views
    std::vector<float*> imgs(nv, nullptr);
    float* img_buf = nullptr;
    uint64_t pix = 0;
    for (size_t i = 0; i < nv; ++i) pix += (uint64_t)vdev[i].width * vdev[i].height;
    if (cudaMalloc((void**)&img_buf, sizeof(float) * 3 * pix) != cudaSuccess) {
        cudaGetLastError();
        g_err = "mirres_autotune_wave: image allocation failed";
        return MIRRES_ERR_OOM;
    }
    for (size_t i = 0, off = 0; i < nv; ++i) {
        imgs[i] = img_buf + 3 * off;
        off += (uint64_t)vdev[i].width * vdev[i].height;
    }
    const Rng rng = make_rng(params);
    const mirres_wave_shape keep = ctx->wave_shape;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mirres_status status = MIRRES_OK;
    // one render that captures the graph and warms caches and clocks, then `timed` renders of
    // which the fastest counts (the stage times are those of the last)
    auto run = [&](const mirres_wave_shape& w, double stage_ms[4], float* total_ms, int timed) -> mirres_status {
        ctx->wave_shape = w;
        *total_ms = 1e30f;
        for (int rep = 0; rep <= timed; ++rep) {
            MR_CUDA(cudaEventRecord(e0, st));
            MR_TRY(render_wave(ctx, sdev, vdev, sub_total, imgs.data(), tape, params->ris_m, rng, 1, nvx, 0, 1, 0, 1,
                               nullptr, st));
            MR_CUDA(cudaEventRecord(e1, st));
            if (rep > 0) {
                float ms = 0.0f;
                MR_CUDA(cudaEventSynchronize(e1));
                MR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                *total_ms = std::min(*total_ms, ms);
            }
        }
        return stage_sums(ctx, stage_ms);
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        status = mr_cuda_status(cudaErrorMemoryAllocation, "mirres_autotune_wave: events");
    }
    // (threads per block, blocks per SM) pairs tried for every stage at once
    static const int kCand[][2] = {{256, 4}, {256, 8}, {256, 16}, {128, 8}, {128, 16}, {128, 32}, {64, 32}};
    const int n_cand = (int)(sizeof(kCand) / sizeof(kCand[0]));
    mirres_wave_shape best = default_wave_shape();
    // the largest tried wave that the tuned views fill
    int wave_top = 23;
    while (wave_top < 25 && (1ull << wave_top) < sub_total) ++wave_top;
    best.wave_log2 = wave_top;
    double best_stage[4] = {1e300, 1e300, 1e300, 1e300};
    for (int c = 0; c < n_cand && status == MIRRES_OK; ++c) {
        mirres_wave_shape w = best;
        for (int k = 0; k < 4; ++k) {
            w.block[k] = kCand[c][0];
            w.blocks_per_sm[k] = kCand[c][1];
        }
        double ms[4];
        float tot = 0.0f;
        status = run(w, ms, &tot, 1);
        if (status != MIRRES_OK) break;
        for (int k = 0; k < 4; ++k) {
            if (ms[k] < best_stage[k]) {
                best_stage[k] = ms[k];
                best.block[k] = kCand[c][0];
                best.blocks_per_sm[k] = kCand[c][1];
            }
        }
    }
    float best_ms = 1e30f;
    int best_wave = wave_top;
    for (int wl = 23; wl <= wave_top && status == MIRRES_OK; ++wl) {
        mirres_wave_shape w = best;
        w.wave_log2 = wl;
        double ms[4];
        float tot = 0.0f;
        status = run(w, ms, &tot, 2);
        if (status == MIRRES_OK && tot < best_ms) {
            best_ms = tot;
            best_wave = wl;
        }
    }
    best.wave_log2 = best_wave;
    // then two and three concurrent chains of waves, at the chosen wave size and at half of it
    // (only where the tuned views fill at least as many waves as chains)
    const int one_chain_wave = best_wave;
    for (int nb = 2; nb <= 3 && status == MIRRES_OK; ++nb) {
        for (int wl = one_chain_wave - 1; wl <= one_chain_wave && status == MIRRES_OK; ++wl) {
            if (wl < 23 || ((uint64_t)(nb - 1) << wl) >= sub_total) continue;
            mirres_wave_shape w = best;
            w.wave_log2 = wl;
            w.branches = nb;
            double ms[4];
            float tot = 0.0f;
            status = run(w, ms, &tot, 2);
            if (status == MIRRES_OK && tot < best_ms) {
                best_ms = tot;
                best.wave_log2 = wl;
                best.branches = nb;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(img_buf);
    if (status != MIRRES_OK) {
        ctx->wave_shape = keep;
        return status;
    }
    ctx->wave_shape = best;
    if (out) *out = best;
    if (out_ms) *out_ms = best_ms;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_stage_times(mirres_context* ctx, double out_ms[4], int32_t out_launches[4])
{
    if (!ctx || !out_ms) return arg_error("ctx and out_ms must not be NULL");
    for (int k = 0; k < 4; ++k) {
        out_ms[k] = 0.0;
        if (out_launches) out_launches[k] = 0;
    }
    if (ctx->stage_pairs == 0) {
        g_err = "mirres_stage_times: no batched render with params.flags bit 0 was captured";
        return MIRRES_ERR_STATE;
    }
    MR_CUDA(cudaSetDevice(ctx->device));
    for (int p = 0; p < ctx->stage_pairs; ++p) {
        MR_CUDA(cudaEventSynchronize(ctx->stage_events[2 * p + 1]));
        float ms = 0.0f;
        MR_CUDA(cudaEventElapsedTime(&ms, ctx->stage_events[2 * p], ctx->stage_events[2 * p + 1]));
        out_ms[ctx->stage_kind[p] & 15] += ms;
        if (out_launches) out_launches[ctx->stage_kind[p] & 15] += 1;
    }
    return MIRRES_OK;
}

extern "C" mirres_status mirres_stage_trace(mirres_context* ctx, int32_t cap, float* out_ms, int32_t* out_stage,
                                            int32_t* out_bounce, int32_t* out_n)
{
    if (!ctx || !out_n || cap < 0 || (cap > 0 && (!out_ms || !out_stage || !out_bounce)))
        return arg_error("ctx and out_n required; out_ms, out_stage and out_bounce when cap > 0");
    *out_n = ctx->stage_pairs;
    if (ctx->stage_pairs == 0) {
        g_err = "mirres_stage_trace: no batched render with params.flags bit 0 was captured";
        return MIRRES_ERR_STATE;
    }
    MR_CUDA(cudaSetDevice(ctx->device));
    for (int p = 0; p < ctx->stage_pairs && p < cap; ++p) {
        MR_CUDA(cudaEventSynchronize(ctx->stage_events[2 * p + 1]));
        MR_CUDA(cudaEventElapsedTime(&out_ms[p], ctx->stage_events[2 * p], ctx->stage_events[2 * p + 1]));
        out_stage[p] = ctx->stage_kind[p] & 15;
        out_bounce[p] = (ctx->stage_kind[p] >> 4) - 1;
    }
    return MIRRES_OK;
}

// ---- adjoint ---------------------------------------------------------------------------------
// demod = false: mirres_backward; true: mirres_light_backward (the demodulated lighting of the
// primary vertex, PRIMARY mode whatever params->grad_mode says)
static mirres_status backward_impl(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                                   const mirres_view* views, int32_t n_views, const mirres_params* params,
                                   const float* const* d_images, const void* tape, size_t tape_bytes,
                                   const mirres_grads* grads, void* stream, bool demod)
{
    if (!ctx) return arg_error("ctx is NULL");
    MR_TRY(check_params(params));
    std::vector<SceneDev> sdev;
    MR_TRY(check_scenes(ctx, scenes, n_scenes, sdev, params ? params->max_visits : 0));
    std::vector<ViewDev> vdev;
    uint64_t total = 0, max_view = 0;
    MR_TRY(check_views(views, n_views, n_scenes, vdev, total, max_view));
    if (!d_images || !grads) return arg_error("d_images and grads must not be NULL");
    for (int i = 0; i < n_views; ++i)
        if (!d_images[i]) return arg_error("d_images[" + std::to_string(i) + "] is NULL");
    if (!tape) return arg_error("mirres_backward needs the tape written by mirres_render");
    MR_TRY(check_full(params, views, n_views));
    const int tape_nvx = full_vertices(views, n_views, params->grad_mode);
    if (tape_bytes < tape_bytes_per_sample(tape_nvx) * total)
        return arg_error("tape_bytes is smaller than mirres_tape_bytes_mode(views, grad_mode)");
    const int nvx = demod ? 0 : tape_nvx;
    MR_CUDA(cudaSetDevice(ctx->device));
    const cudaStream_t st = as_stream(stream);
    ctx->last_stream = st;
    std::vector<GradDev> gdev((size_t)n_scenes);
    for (int i = 0; i < n_scenes; ++i)
        gdev[(size_t)i] = GradDev{grads[i].albedo, grads[i].roughness, grads[i].metallic, grads[i].env, grads[i].verts};
    Carver plan(nullptr);
    plan.take<ViewDev>((size_t)n_views);
    plan.take<SceneDev>((size_t)n_scenes);
    plan.take<const float*>((size_t)n_views);
    plan.take<GradDev>((size_t)n_scenes);
    plan.take<char>(nvx > 0 ? mr_full_scratch_bytes() : 0);
    MR_TRY(ws_reserve(ctx, plan.off));
    Carver cv(ctx->ws.ptr);
    ViewDev* d_views = cv.take<ViewDev>((size_t)n_views);
    SceneDev* d_scenes = cv.take<SceneDev>((size_t)n_scenes);
    const float** d_dimg = cv.take<const float*>((size_t)n_views);
    GradDev* d_grads = cv.take<GradDev>((size_t)n_scenes);
    void* full_scratch = cv.take<char>(nvx > 0 ? mr_full_scratch_bytes() : 0);
    MR_CUDA(cudaMemcpyAsync(d_views, vdev.data(), sizeof(ViewDev) * vdev.size(), cudaMemcpyHostToDevice, st));
    MR_CUDA(cudaMemcpyAsync(d_scenes, sdev.data(), sizeof(SceneDev) * sdev.size(), cudaMemcpyHostToDevice, st));
    MR_CUDA(cudaMemcpyAsync(d_dimg, d_images, sizeof(float*) * (size_t)n_views, cudaMemcpyHostToDevice, st));
    MR_CUDA(cudaMemcpyAsync(d_grads, gdev.data(), sizeof(GradDev) * gdev.size(), cudaMemcpyHostToDevice, st));
    int normals_passes = 0;
    for (int i = 0; i < n_scenes; ++i)
        if (scenes[i]->normals && grads[i].verts && scenes[i]->gvn)
            MR_CUDA(cudaMemsetAsync(scenes[i]->gvn, 0, sizeof(float) * 3 * (size_t)scenes[i]->desc.n_verts, st));
    bool interp = false;
    for (int i = 0; i < n_scenes; ++i) interp = interp || scenes[i]->normals != 0;
    if (demod)
        mr_launch_light_backward(d_scenes, d_views, n_views, total, make_rng(params), d_dimg, d_grads, tape,
                                 ctx->counters, ctx->sm_count, st, interp);
    else
        mr_launch_backward(d_scenes, d_views, n_views, total, make_rng(params), d_dimg, d_grads, tape, ctx->counters,
                           ctx->sm_count, st, nvx, full_scratch, interp);
    // interpolated normals: d loss / d vertex normal to the vertices of the incident faces
    for (int i = 0; i < n_scenes; ++i)
        if (scenes[i]->normals && grads[i].verts && scenes[i]->gvn) {
            mr_launch_normals_adjoint(scenes[i], grads[i].verts, ctx->sm_count, st);
            ++normals_passes;
        }
    MR_CUDA(cudaGetLastError());
    const uint64_t full_chunk = mr_full_chunk();
    ctx->host_launches += 1 + (unsigned long long)normals_passes +
                          ((nvx > 0 && full_chunk) ? 4 * ((total + full_chunk - 1) / full_chunk) : 0);
    return MIRRES_OK;
}

extern "C" mirres_status mirres_backward(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                                         const mirres_view* views, int32_t n_views, const mirres_params* params,
                                         const float* const* d_images, const void* tape, size_t tape_bytes,
                                         const mirres_grads* grads, void* stream)
{
    return backward_impl(ctx, scenes, n_scenes, views, n_views, params, d_images, tape, tape_bytes, grads, stream,
                         false);
}

// ---- monochrome light regulariser (Appendix A, L_light) --------------------------------------
static std::vector<uint64_t> pixel_offsets(const std::vector<ViewDev>& vdev, uint64_t& total_pix)
{
    std::vector<uint64_t> off(vdev.size());
    total_pix = 0;
    for (size_t i = 0; i < vdev.size(); ++i) {
        off[i] = total_pix;
        total_pix += (uint64_t)vdev[i].width * (uint64_t)vdev[i].height;
    }
    return off;
}

extern "C" mirres_status mirres_light_demod(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                                            const mirres_view* views, int32_t n_views, const mirres_params* params,
                                            const void* tape, size_t tape_bytes, float* const* demod, void* stream)
{
    if (!ctx) return arg_error("ctx is NULL");
    MR_TRY(check_params(params));
    std::vector<SceneDev> sdev;
    MR_TRY(check_scenes(ctx, scenes, n_scenes, sdev, params ? params->max_visits : 0));
    std::vector<ViewDev> vdev;
    uint64_t total = 0, max_view = 0;
    MR_TRY(check_views(views, n_views, n_scenes, vdev, total, max_view));
    if (!demod) return arg_error("demod must not be NULL");
    for (int i = 0; i < n_views; ++i) {
        if (!demod[i]) return arg_error("demod[" + std::to_string(i) + "] is NULL");
        if (reinterpret_cast<uintptr_t>(demod[i]) % 16) return arg_error("demod[" + std::to_string(i) + "] is not 16-byte aligned");
    }
    if (!tape) return arg_error("mirres_light_demod needs the tape written by mirres_render");
    MR_TRY(check_full(params, views, n_views));
    if (tape_bytes < tape_bytes_per_sample(full_vertices(views, n_views, params->grad_mode)) * total)
        return arg_error("tape_bytes is smaller than mirres_tape_bytes_mode(views, grad_mode)");
    // tiles of whole pixels per view (the kernel's work units)
    std::vector<uint64_t> tile_off((size_t)n_views + 1, 0);
    for (int i = 0; i < n_views; ++i) {
        const uint64_t npx = (uint64_t)vdev[(size_t)i].width * vdev[(size_t)i].height;
        const uint64_t P = (uint64_t)mr_light_tile_pixels(vdev[(size_t)i].spp);
        tile_off[(size_t)i + 1] = tile_off[(size_t)i] + (npx + P - 1) / P;
    }
    MR_CUDA(cudaSetDevice(ctx->device));
    const cudaStream_t st = as_stream(stream);
    ctx->last_stream = st;
    Carver plan(nullptr);
    plan.take<ViewDev>((size_t)n_views);
    plan.take<SceneDev>((size_t)n_scenes);
    plan.take<uint64_t>((size_t)n_views + 1);
    plan.take<float*>((size_t)n_views);
    MR_TRY(ws_reserve(ctx, plan.off));
    Carver cv(ctx->ws.ptr);
    ViewDev* d_views = cv.take<ViewDev>((size_t)n_views);
    SceneDev* d_scenes = cv.take<SceneDev>((size_t)n_scenes);
    uint64_t* d_tiles = cv.take<uint64_t>((size_t)n_views + 1);
    float** d_out = cv.take<float*>((size_t)n_views);
    MR_CUDA(cudaMemcpyAsync(d_views, vdev.data(), sizeof(ViewDev) * vdev.size(), cudaMemcpyHostToDevice, st));
    MR_CUDA(cudaMemcpyAsync(d_scenes, sdev.data(), sizeof(SceneDev) * sdev.size(), cudaMemcpyHostToDevice, st));
    MR_CUDA(cudaMemcpyAsync(d_tiles, tile_off.data(), sizeof(uint64_t) * tile_off.size(), cudaMemcpyHostToDevice, st));
    MR_CUDA(cudaMemcpyAsync(d_out, demod, sizeof(float*) * (size_t)n_views, cudaMemcpyHostToDevice, st));
    bool interp = false;
    for (int i = 0; i < n_scenes; ++i) interp = interp || scenes[i]->normals != 0;
    mr_launch_light_demod(d_scenes, d_views, d_tiles, n_views, tile_off[(size_t)n_views], total, make_rng(params),
                          tape, d_out, ctx->sm_count, st, interp);
    MR_CUDA(cudaGetLastError());
    ctx->host_launches += 1;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_light_loss(mirres_context* ctx, const mirres_view* views, int32_t n_views,
                                           const float* const* demod, const float* const* ref_images, float weight,
                                           float* loss, float* const* d_demod, void* stream)
{
    if (!ctx) return arg_error("ctx is NULL");
    std::vector<ViewDev> vdev;
    uint64_t total = 0, max_view = 0;
    MR_TRY(check_views(views, n_views, 0x7FFFFFFF, vdev, total, max_view));
    if (!demod || !ref_images) return arg_error("demod and ref_images must not be NULL");
    if (!(weight >= 0.0f)) return arg_error("weight must be >= 0");
    for (int i = 0; i < n_views; ++i) {
        if (!demod[i] || !ref_images[i]) return arg_error("view " + std::to_string(i) + ": NULL demod or reference");
        if (reinterpret_cast<uintptr_t>(demod[i]) % 16) return arg_error("demod[" + std::to_string(i) + "] is not 16-byte aligned");
        if (d_demod && !d_demod[i]) return arg_error("d_demod[" + std::to_string(i) + "] is NULL");
    }
    uint64_t total_pix = 0;
    const std::vector<uint64_t> pix_off = pixel_offsets(vdev, total_pix);
    MR_CUDA(cudaSetDevice(ctx->device));
    const cudaStream_t st = as_stream(stream);
    ctx->last_stream = st;
    Carver plan(nullptr);
    plan.take<uint64_t>((size_t)n_views);
    plan.take<const float*>((size_t)n_views);
    plan.take<const float*>((size_t)n_views);
    plan.take<float*>((size_t)n_views);
    plan.take<unsigned int>(1);
    MR_TRY(ws_reserve(ctx, plan.off));
    Carver cv(ctx->ws.ptr);
    uint64_t* d_pixoff = cv.take<uint64_t>((size_t)n_views);
    const float** d_c = cv.take<const float*>((size_t)n_views);
    const float** d_ref = cv.take<const float*>((size_t)n_views);
    float** d_dc = cv.take<float*>((size_t)n_views);
    unsigned int* d_count = cv.take<unsigned int>(1);
    MR_CUDA(cudaMemcpyAsync(d_pixoff, pix_off.data(), sizeof(uint64_t) * pix_off.size(), cudaMemcpyHostToDevice, st));
    MR_CUDA(cudaMemcpyAsync(d_c, demod, sizeof(float*) * (size_t)n_views, cudaMemcpyHostToDevice, st));
    MR_CUDA(cudaMemcpyAsync(d_ref, ref_images, sizeof(float*) * (size_t)n_views, cudaMemcpyHostToDevice, st));
    if (d_demod) MR_CUDA(cudaMemcpyAsync(d_dc, d_demod, sizeof(float*) * (size_t)n_views, cudaMemcpyHostToDevice, st));
    MR_CUDA(mr_launch_light_loss(d_pixoff, n_views, total_pix, d_c, d_ref, weight, d_count, loss,
                                 d_demod ? d_dc : nullptr, ctx->sm_count, st));
    ctx->host_launches += 2;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_light_backward(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                                               const mirres_view* views, int32_t n_views,
                                               const mirres_params* params, const float* const* d_demod,
                                               const void* tape, size_t tape_bytes, const mirres_grads* grads,
                                               void* stream)
{
    return backward_impl(ctx, scenes, n_scenes, views, n_views, params, d_demod, tape, tape_bytes, grads, stream,
                         true);
}

extern "C" mirres_status mirres_l2_loss(const float* image, const float* ref, int64_t n, float* d_image,
                                        float* loss, void* stream)
{
    if (!image || !ref || n < 0) return arg_error("image, ref must not be NULL and n >= 0");
    if (n == 0) return MIRRES_OK;
    int dev = 0, sms = 1;
    MR_CUDA(cudaGetDevice(&dev));
    MR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    mr_launch_l2(image, ref, n, d_image, loss, sms, as_stream(stream));
    MR_CUDA(cudaGetLastError());
    return MIRRES_OK;
}

extern "C" mirres_status mirres_trace(mirres_context* ctx, const mirres_scene* s, const float* rays,
                                      const int32_t* skip_tri, int64_t n, int32_t any, int32_t* hit_tri,
                                      float* hit_tuv, void* stream)
{
    if (!ctx || !s || !rays || !hit_tri || n < 0) return arg_error("ctx, scene, rays, hit_tri required; n >= 0");
    if (!s->built) {
        g_err = "mirres_trace: call mirres_bvh_build first";
        return MIRRES_ERR_STATE;
    }
    if (n == 0) return MIRRES_OK;
    MR_CUDA(cudaSetDevice(ctx->device));
    mr_launch_trace_rays(mr_scene_dev(s), rays, skip_tri, n, any ? 1 : 0, hit_tri, hit_tuv, ctx->sm_count,
                         as_stream(stream));
    MR_CUDA(cudaGetLastError());
    ctx->host_launches += 1;
    return MIRRES_OK;
}

// ---- denoiser (Appendix A, "Denoiser") -------------------------------------------------------
static mirres_status check_eawt(int32_t width, int32_t height, const mirres_eawt_params* p)
{
    if (width < 1 || height < 1) return arg_error("width and height must be >= 1");
    if ((int64_t)width * height > (int64_t)1 << 31) return arg_error("image larger than 2^31 pixels");
    if (!p) return arg_error("eawt params is NULL");
    if (p->levels < 1 || p->levels > MIRRES_EAWT_MAX_LEVELS)
        return arg_error("levels must be in [1, " + std::to_string(MIRRES_EAWT_MAX_LEVELS) + "]");
    if (!(p->sigma_rt > 0.0f) || !(p->sigma_n > 0.0f) || !(p->sigma_x > 0.0f))
        return arg_error("sigma_rt, sigma_n and sigma_x must be > 0");
    return MIRRES_OK;
}

extern "C" size_t mirres_eawt_record_bytes(int32_t width, int32_t height, int32_t levels)
{
    if (width < 1 || height < 1 || levels < 1 || levels > MIRRES_EAWT_MAX_LEVELS) return 0;
    return ((size_t)32 + (size_t)20 * (size_t)levels) * (size_t)width * (size_t)height;
}

extern "C" mirres_status mirres_gbuffer(mirres_context* ctx, const mirres_scene* scene, const mirres_view* view,
                                        float* normal, float* position, void* stream)
{
    if (!ctx || !scene || !view || !normal || !position) return arg_error("ctx, scene, view, normal, position required");
    if (!scene->built) {
        g_err = "mirres_gbuffer: call mirres_bvh_build first";
        return MIRRES_ERR_STATE;
    }
    mirres_view one = *view;
    one.scene = 0;
    std::vector<ViewDev> vdev;
    uint64_t total = 0, max_view = 0;
    MR_TRY(check_views(&one, 1, 1, vdev, total, max_view));
    MR_CUDA(cudaSetDevice(ctx->device));
    mr_launch_gbuffer(mr_scene_dev(scene), vdev[0], normal, position, ctx->sm_count, as_stream(stream));
    MR_CUDA(cudaGetLastError());
    ctx->host_launches += 1;
    return MIRRES_OK;
}

// record layout (16-byte aligned) for a stack of n images of npx pixels: packed normals and
// positions [n][H][W] float4, the levels' inputs c_i [levels][n][H][W] float4, their reciprocal
// normalisers 1 / k_i [levels][n][H][W] float
struct EawtRecord {
    float4 *n, *x, *c;
    float* ik;
};

static EawtRecord eawt_record(void* base, size_t npx, int L)
{
    float4* f = reinterpret_cast<float4*>(base);
    return EawtRecord{f, f + npx, f + 2 * npx, reinterpret_cast<float*>(f + (2 + (size_t)L) * npx)};
}

static mirres_status eawt_args(int32_t n_images, int32_t width, int32_t height, const mirres_eawt_params* params,
                               const void* record, size_t record_bytes)
{
    if (n_images < 1) return arg_error("n_images must be >= 1");
    MR_TRY(check_eawt(width, height, params));
    if ((int64_t)width * height * n_images > (int64_t)1 << 31) return arg_error("image stack larger than 2^31 pixels");
    if (record_bytes / (size_t)n_images < mirres_eawt_record_bytes(width, height, params->levels))
        return arg_error("record_bytes is smaller than n_images * mirres_eawt_record_bytes");
    if (reinterpret_cast<uintptr_t>(record) & 15) return arg_error("record must be 16-byte aligned");
    return MIRRES_OK;
}

extern "C" mirres_status mirres_eawt_batch(mirres_context* ctx, int32_t n_images, const float* image,
                                           const float* normal, const float* position, int32_t width, int32_t height,
                                           const mirres_eawt_params* params, float* out, void* record,
                                           size_t record_bytes, void* stream)
{
    if (!ctx || !image || !normal || !position || !out || !record)
        return arg_error("ctx, image, normal, position, out and record required");
    MR_TRY(eawt_args(n_images, width, height, params, record, record_bytes));
    MR_CUDA(cudaSetDevice(ctx->device));
    const cudaStream_t st = as_stream(stream);
    const size_t npx = (size_t)width * height * n_images;
    const int L = params->levels, sms = ctx->sm_count;
    const EawtRecord r = eawt_record(record, npx, L);
    mr_launch_eawt_pack(normal, r.n, (int64_t)npx, sms, st);
    mr_launch_eawt_pack(position, r.x, (int64_t)npx, sms, st);
    mr_launch_eawt_pack(image, r.c, (int64_t)npx, sms, st);
    const float in2 = 1.0f / (params->sigma_n * params->sigma_n), ix2 = 1.0f / (params->sigma_x * params->sigma_x);
    for (int i = 0; i < L; ++i) {
        const int step = 1 << i;
        const float srt = params->sigma_rt / (float)step;
        const bool last = i + 1 == L;
        mr_launch_eawt_level(r.c + npx * (size_t)i, r.n, r.x, n_images, width, height, step, 1.0f / (srt * srt), in2,
                             ix2, last ? nullptr : r.c + npx * (size_t)(i + 1), last ? out : nullptr,
                             r.ik + npx * (size_t)i, sms, st);
    }
    MR_CUDA(cudaGetLastError());
    ctx->host_launches += (unsigned long long)L + 3;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_eawt(mirres_context* ctx, const float* image, const float* normal,
                                     const float* position, int32_t width, int32_t height,
                                     const mirres_eawt_params* params, float* out, void* record,
                                     size_t record_bytes, void* stream)
{
    return mirres_eawt_batch(ctx, 1, image, normal, position, width, height, params, out, record, record_bytes,
                             stream);
}

extern "C" mirres_status mirres_eawt_batch_backward(mirres_context* ctx, int32_t n_images, const float* d_out,
                                                    const float* normal, const float* position, int32_t width,
                                                    int32_t height, const mirres_eawt_params* params,
                                                    const void* record, size_t record_bytes, float* d_image,
                                                    void* stream)
{
    // (normal and position are the forward's; the record holds them packed)
    if (!ctx || !d_out || !normal || !position || !record || !d_image)
        return arg_error("ctx, d_out, normal, position, record and d_image required");
    MR_TRY(eawt_args(n_images, width, height, params, record, record_bytes));
    MR_CUDA(cudaSetDevice(ctx->device));
    const cudaStream_t st = as_stream(stream);
    const size_t npx = (size_t)width * height * n_images;
    const int L = params->levels, sms = ctx->sm_count;
    MR_TRY(ws_reserve(ctx, sizeof(float4) * 2 * npx + 256));
    float4* tmp[2] = {reinterpret_cast<float4*>(ctx->ws.ptr), reinterpret_cast<float4*>(ctx->ws.ptr) + npx};
    const EawtRecord r = eawt_record(const_cast<void*>(record), npx, L);
    const float in2 = 1.0f / (params->sigma_n * params->sigma_n), ix2 = 1.0f / (params->sigma_x * params->sigma_x);
    mr_launch_eawt_pack(d_out, tmp[0], (int64_t)npx, sms, st);
    int cur = 0;
    for (int i = L - 1; i >= 0; --i) {
        const int step = 1 << i;
        const float srt = params->sigma_rt / (float)step;
        mr_launch_eawt_level_adjoint(tmp[cur], r.c + npx * (size_t)i, r.ik + npx * (size_t)i, r.n, r.x, n_images,
                                     width, height, step, 1.0f / (srt * srt), in2, ix2,
                                     i == 0 ? nullptr : tmp[cur ^ 1], i == 0 ? d_image : nullptr, sms, st);
        cur ^= 1;
    }
    MR_CUDA(cudaGetLastError());
    ctx->host_launches += (unsigned long long)L + 1;
    return MIRRES_OK;
}

extern "C" mirres_status mirres_eawt_backward(mirres_context* ctx, const float* d_out, const float* normal,
                                              const float* position, int32_t width, int32_t height,
                                              const mirres_eawt_params* params, const void* record,
                                              size_t record_bytes, float* d_image, void* stream)
{
    return mirres_eawt_batch_backward(ctx, 1, d_out, normal, position, width, height, params, record, record_bytes,
                                      d_image, stream);
}

extern "C" mirres_status mirres_mesh_regularizers(mirres_context* ctx, mirres_scene* scene,
                                                  const float* rest_verts, float w_smooth, float w_offset,
                                                  float* loss, float* grad_verts, void* stream)
{
    if (!ctx || !scene) return arg_error("ctx and scene required");
    if (!(w_smooth >= 0.0f) || !(w_offset >= 0.0f)) return arg_error("weights must be >= 0");
    if (w_offset != 0.0f && !rest_verts) return arg_error("rest_verts required when w_offset != 0");
    if (!scene->built) {
        g_err = "mirres_mesh_regularizers: call mirres_bvh_build first";
        return MIRRES_ERR_STATE;
    }
    MR_CUDA(cudaSetDevice(ctx->device));
    const cudaStream_t st = as_stream(stream);
    if (w_smooth != 0.0f) MR_TRY(mr_edges_build(scene, st));
    if (!loss && !grad_verts) return MIRRES_OK;
    mr_launch_regularizers(scene, rest_verts, w_smooth, w_offset, loss, grad_verts, ctx->sm_count, st);
    MR_CUDA(cudaGetLastError());
    ctx->host_launches += (unsigned long long)(w_smooth != 0.0f) + (unsigned long long)(w_offset != 0.0f);
    return MIRRES_OK;
}

extern "C" mirres_status mirres_material_smoothness(mirres_context* ctx, const mirres_scene* scene,
                                                    const mirres_view* view, int32_t view_index,
                                                    const mirres_lk_params* params, float* loss, float* grad_albedo,
                                                    float* grad_roughness, float* grad_verts, void* stream)
{
    if (!ctx || !scene || !view || !params) return arg_error("ctx, scene, view and params required");
    if (!(params->sigma > 0.0f) || !(params->w_albedo >= 0.0f) || !(params->w_roughness >= 0.0f) ||
        !(params->w_normal >= 0.0f))
        return arg_error("sigma must be > 0 and the weights >= 0");
    if (view_index < 0 || view_index > 65535) return arg_error("view_index outside [0, 65535]");
    if (!scene->built) {
        g_err = "mirres_material_smoothness: call mirres_bvh_build first";
        return MIRRES_ERR_STATE;
    }
    mirres_view one = *view;
    one.scene = 0;
    std::vector<ViewDev> vdev;
    uint64_t total = 0, max_view = 0;
    MR_TRY(check_views(&one, 1, 1, vdev, total, max_view));
    if (!loss && !grad_albedo && !grad_roughness && !grad_verts) return MIRRES_OK;
    MR_CUDA(cudaSetDevice(ctx->device));
    const cudaStream_t st = as_stream(stream);
    const size_t npx = (size_t)view->width * view->height;
    Carver plan(nullptr);
    plan.take<float4>(npx);
    plan.take<float2>(npx);
    plan.take<unsigned int>(1);
    MR_TRY(ws_reserve(ctx, plan.off));
    Carver cv(ctx->ws.ptr);
    float4* rec = cv.take<float4>(npx);
    float2* bary = cv.take<float2>(npx);
    unsigned int* n_hit = cv.take<unsigned int>(1);
    MR_CUDA(cudaMemsetAsync(n_hit, 0, sizeof(unsigned int), st));
    // the normal term (interpolated normals only) accumulates d loss / d vertex normal in the
    // scene's per-vertex accumulator, then takes it to the vertices of the faces around
    const bool normal = params->w_normal > 0.0f && scene->normals && scene->gvn && scene->desc.n_verts > 0;
    if (normal && grad_verts)
        MR_CUDA(cudaMemsetAsync(scene->gvn, 0, sizeof(float) * 3 * (size_t)scene->desc.n_verts, st));
    Rng rng;
    rng.set(params->seed_lo, params->seed_hi);
    mr_launch_material_smoothness(mr_scene_dev(scene), vdev[0], (uint32_t)view_index, rng, params->sigma,
                                  params->w_albedo, params->w_roughness, normal ? params->w_normal : 0.0f, rec, bary,
                                  n_hit, loss, grad_albedo, grad_roughness, normal && grad_verts, ctx->sm_count, st);
    if (normal && grad_verts) mr_launch_normals_adjoint(scene, grad_verts, ctx->sm_count, st);
    MR_CUDA(cudaGetLastError());
    ctx->host_launches += 2 + (normal && grad_verts ? 1 : 0);
    return MIRRES_OK;
}

extern "C" mirres_status mirres_bvh_export(const mirres_scene* s, uint64_t* keys, int32_t* left, int32_t* right,
                                           int32_t* parent, float* lo, float* hi, void* stream)
{
    if (!s) return arg_error("scene is NULL");
    if (!s->built) {
        g_err = "mirres_bvh_export: call mirres_bvh_build first";
        return MIRRES_ERR_STATE;
    }
    const size_t F = (size_t)s->desc.n_tris;
    if (F == 0) return MIRRES_OK;
    const cudaStream_t st = as_stream(stream);
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    if (keys) MR_CUDA(cudaMemcpyAsync(keys, s->keys, sizeof(uint64_t) * F, k, st));
    if (left && F > 1) MR_CUDA(cudaMemcpyAsync(left, s->left, sizeof(int32_t) * (F - 1), k, st));
    if (right && F > 1) MR_CUDA(cudaMemcpyAsync(right, s->right, sizeof(int32_t) * (F - 1), k, st));
    if (parent) MR_CUDA(cudaMemcpyAsync(parent, s->parent, sizeof(int32_t) * (2 * F - 1), k, st));
    if (lo) MR_CUDA(cudaMemcpyAsync(lo, s->lo, sizeof(float) * 3 * (2 * F - 1), k, st));
    if (hi) MR_CUDA(cudaMemcpyAsync(hi, s->hi, sizeof(float) * 3 * (2 * F - 1), k, st));
    return MIRRES_OK;
}

extern "C" mirres_status mirres_env_export_flat(const mirres_scene* s, uint64_t* thresholds, void* stream)
{
    if (!s || !thresholds) return arg_error("scene and thresholds required");
    if (!s->built) {
        g_err = "mirres_env_export_flat: call mirres_bvh_build first";
        return MIRRES_ERR_STATE;
    }
    const size_t n = (size_t)s->desc.env_w * s->desc.env_h + 1;
    MR_CUDA(cudaMemcpyAsync(thresholds, s->env_flat, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice,
                            as_stream(stream)));
    return MIRRES_OK;
}

extern "C" mirres_status mirres_env_export(const mirres_scene* s, uint32_t* marg, uint32_t* cond, float* texel,
                                           double* total, void* stream)
{
    if (!s) return arg_error("scene is NULL");
    if (!s->built) {
        g_err = "mirres_env_export: call mirres_bvh_build first";
        return MIRRES_ERR_STATE;
    }
    const size_t W = (size_t)s->desc.env_w, H = (size_t)s->desc.env_h;
    const cudaStream_t st = as_stream(stream);
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    if (marg) MR_CUDA(cudaMemcpyAsync(marg, s->env_marg, sizeof(uint32_t) * (H + 1), k, st));
    if (cond) MR_CUDA(cudaMemcpyAsync(cond, s->env_cond, sizeof(uint32_t) * H * (W + 1), k, st));
    if (texel) MR_CUDA(cudaMemcpyAsync(texel, s->env_texel, sizeof(float4) * H * W, k, st));
    if (total) MR_CUDA(cudaMemcpyAsync(total, s->env_total, sizeof(double), k, st));
    return MIRRES_OK;
}

extern "C" mirres_status mirres_get_counters(mirres_context* ctx, uint64_t out[8])
{
    if (!ctx || !out) return arg_error("ctx and out must not be NULL");
    MR_CUDA(cudaSetDevice(ctx->device));
    unsigned long long h[CNT_N];
    MR_CUDA(cudaStreamSynchronize(ctx->last_stream));
    MR_CUDA(cudaMemcpy(h, ctx->counters, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 8; ++i) out[i] = (uint64_t)h[i];
    out[CNT_LAUNCH] = ctx->host_launches;
    if (h[CNT_ERROR] != 0) {
        g_err = std::to_string(h[CNT_ERROR]) +
                " ray traversal(s) reached the iteration cap or overflowed the stack since the counters were "
                "reset (malformed hierarchy or a max_visits below the tree's needs); those rays reported a miss";
        return MIRRES_ERR_TIMEOUT;
    }
    return MIRRES_OK;
}

extern "C" mirres_status mirres_get_work_counters(mirres_context* ctx, uint64_t out[4])
{
    if (!ctx || !out) return arg_error("ctx and out must not be NULL");
    MR_CUDA(cudaSetDevice(ctx->device));
    unsigned long long h[CNT_N];
    MR_CUDA(cudaStreamSynchronize(ctx->last_stream));
    MR_CUDA(cudaMemcpy(h, ctx->counters, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 4; ++i) out[i] = (uint64_t)h[CNT_CBOX + i];
    return MIRRES_OK;
}

extern "C" mirres_status mirres_reset_counters(mirres_context* ctx)
{
    if (!ctx) return arg_error("ctx is NULL");
    MR_CUDA(cudaSetDevice(ctx->device));
    MR_CUDA(cudaMemset(ctx->counters, 0, sizeof(unsigned long long) * CNT_N));
    ctx->host_launches = 0;
    return MIRRES_OK;
}

extern "C" const char* mirres_last_error(void) { return g_err.c_str(); }
