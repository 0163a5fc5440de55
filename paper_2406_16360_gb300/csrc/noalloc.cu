// noalloc.cu -- mirres_render_noalloc: the batched persistent forward without any device
// allocation. Its scratch (the per-call view, scene and image tables, pixel offsets and the
// work counter that the persistent kernel pulls samples from) lives in one file-scope
// __device__ array of MIRRES_NOALLOC_SCRATCH_BYTES; every GPU that loads the library keeps
// that array until the process exits.
#include <cstring>
#include <mutex>
#include <string>

#include "render.h"

namespace {

constexpr int kMaxViews = MIRRES_NOALLOC_MAX_VIEWS;
constexpr int kMaxScenes = MIRRES_NOALLOC_MAX_SCENES;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffViews = 0;
constexpr size_t kOffScenes = align256(kOffViews + sizeof(ViewDev) * kMaxViews);
constexpr size_t kOffImages = align256(kOffScenes + sizeof(SceneDev) * kMaxScenes);
constexpr size_t kOffPixoff = align256(kOffImages + sizeof(float*) * kMaxViews);
constexpr size_t kOffWork = align256(kOffPixoff + sizeof(uint64_t) * kMaxViews);
constexpr size_t kUsed = kOffWork + sizeof(unsigned long long);
static_assert(kUsed <= MIRRES_NOALLOC_SCRATCH_BYTES, "no-alloc scratch layout exceeds its stated size");

// the scratch: shared by every call on a device, contents kept from the last call
static __device__ __align__(256) unsigned char g_scratch[MIRRES_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_addr[kMaxDevices] = {};

// host staging for the tables (reused under the mutex; pageable copies are staged by the
// runtime before cudaMemcpyAsync returns, so the buffers are free again afterwards)
ViewDev g_views[kMaxViews];
SceneDev g_scenes[kMaxScenes];
float* g_images[kMaxViews];
uint64_t g_pixoff[kMaxViews];

mirres_status fail(mirres_status s, const std::string& msg)
{
    mr_set_error("mirres_render_noalloc: " + msg);
    return s;
}

// device address of the scratch on `device` (made current by the caller): looked up once per
// device with cudaGetSymbolAddress; the host-side name of the array is not a device address
mirres_status scratch_address(int device, unsigned char** out)
{
    if (device < 0 || device >= kMaxDevices) return fail(MIRRES_ERR_ARG, "device index out of range");
    if (!g_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return mr_cuda_status(e, "mirres_render_noalloc: cudaGetSymbolAddress");
        g_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[device];
    return MIRRES_OK;
}

}  // namespace

extern "C" mirres_status mirres_render_noalloc(mirres_scene* const* scenes, int32_t n_scenes,
                                               const mirres_view* views, int32_t n_views,
                                               const mirres_params* params, float* const* images, void* tape,
                                               size_t tape_bytes, void* stream)
{
    if (!scenes || n_scenes < 1) return fail(MIRRES_ERR_ARG, "need at least one scene");
    if (n_scenes > kMaxScenes)
        return fail(MIRRES_ERR_ARG, "n_scenes = " + std::to_string(n_scenes) + " exceeds the static maximum of " +
                                        std::to_string(kMaxScenes));
    if (!views || n_views < 1) return fail(MIRRES_ERR_ARG, "need at least one view");
    if (n_views > kMaxViews)
        return fail(MIRRES_ERR_ARG, "n_views = " + std::to_string(n_views) + " exceeds the static maximum of " +
                                        std::to_string(kMaxViews));
    if (!params || params->ris_m < 1) return fail(MIRRES_ERR_ARG, "params missing or ris_m < 1");
    if (params->grad_mode != 0)
        return fail(MIRRES_ERR_ARG, "mirres_render_noalloc writes the PRIMARY-mode tape only (grad_mode 0)");
    if (params->launch < 0 || params->launch > 2)
        return fail(MIRRES_ERR_ARG, "launch must be 0, 1 or 2 (the persistent kernel runs whichever is given)");
    if (params->block != 0 && (params->block < 32 || params->block > 1024 || params->block % 32))
        return fail(MIRRES_ERR_ARG, "block must be 0 or a multiple of 32 in [32, 1024]");
    if (params->blocks_per_sm < 0) return fail(MIRRES_ERR_ARG, "blocks_per_sm must be >= 0");
    if (params->max_visits < 0) return fail(MIRRES_ERR_ARG, "max_visits must be >= 0");
    // reservoir reuse needs per-sample scratch that this entry point does not have (mirres_render
    // offers it with the batched launch only)
    if (params->reuse_k != 0 || params->temporal != 0)
        return fail(MIRRES_ERR_ARG, "reservoir reuse (reuse_k > 0 or temporal > 0) is not available here");
    if (!images) return fail(MIRRES_ERR_ARG, "images is NULL");
    if (!tape) return fail(MIRRES_ERR_ARG, "a caller-owned tape is required (this entry point allocates nothing)");
    if (reinterpret_cast<uintptr_t>(tape) & 15) return fail(MIRRES_ERR_ARG, "tape must be 16-byte aligned");
    mirres_context* ctx = scenes[0] ? scenes[0]->ctx : nullptr;
    if (!ctx) return fail(MIRRES_ERR_ARG, "scene 0 is NULL");

    std::lock_guard<std::mutex> lock(g_mutex);
    for (int i = 0; i < n_scenes; ++i) {
        if (!scenes[i]) return fail(MIRRES_ERR_ARG, "scene " + std::to_string(i) + " is NULL");
        if (scenes[i]->ctx != ctx) return fail(MIRRES_ERR_ARG, "all scenes must share one context");
        if (!scenes[i]->built) return fail(MIRRES_ERR_STATE, "scene " + std::to_string(i) + " is not built");
        g_scenes[i] = mr_scene_dev(scenes[i]);
        g_scenes[i].trav_cap = params->max_visits;
    }
    uint64_t total = 0, total_pix = 0;
    for (int i = 0; i < n_views; ++i) {
        const mirres_view& v = views[i];
        if (v.width < 1 || v.height < 1 || v.spp < 1 || v.bounces < 1 || v.bounces > 255)
            return fail(MIRRES_ERR_ARG, "view " + std::to_string(i) + ": width, height, spp >= 1, bounces in [1, 255]");
        const uint64_t n = (uint64_t)v.width * (uint64_t)v.height * (uint64_t)v.spp;
        if (n > 0xFFFFFFFFull) return fail(MIRRES_ERR_ARG, "view " + std::to_string(i) + ": more than 2^32-1 samples");
        if (v.scene < 0 || v.scene >= n_scenes) return fail(MIRRES_ERR_ARG, "view " + std::to_string(i) + ": bad scene");
        if (!(v.K[0] != 0.0f) || !(v.K[1] != 0.0f)) return fail(MIRRES_ERR_ARG, "view " + std::to_string(i) + ": fx, fy == 0");
        if (!images[i]) return fail(MIRRES_ERR_ARG, "images[" + std::to_string(i) + "] is NULL");
        ViewDev& d = g_views[i];
        std::memcpy(d.K, v.K, sizeof(d.K));
        std::memcpy(d.c2w, v.c2w, sizeof(d.c2w));
        d.width = v.width;
        d.height = v.height;
        d.spp = v.spp;
        d.bounces = v.bounces;
        d.scene = v.scene;
        d.index = i;
        d.offset = total;
        g_images[i] = images[i];
        g_pixoff[i] = total_pix;
        total += n;
        total_pix += (uint64_t)v.width * (uint64_t)v.height;
    }
    if (tape_bytes < (uint64_t)MIRRES_TAPE_BYTES_PER_SAMPLE * total) return fail(MIRRES_ERR_ARG, "tape_bytes is smaller than mirres_tape_bytes(views)");

    MR_CUDA(cudaSetDevice(ctx->device));
    unsigned char* base = nullptr;
    mirres_status st = scratch_address(ctx->device, &base);
    if (st != MIRRES_OK) return st;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ViewDev* d_views = reinterpret_cast<ViewDev*>(base + kOffViews);
    SceneDev* d_scenes = reinterpret_cast<SceneDev*>(base + kOffScenes);
    float** d_images = reinterpret_cast<float**>(base + kOffImages);
    uint64_t* d_pixoff = reinterpret_cast<uint64_t*>(base + kOffPixoff);
    unsigned long long* d_work = reinterpret_cast<unsigned long long*>(base + kOffWork);
    MR_CUDA(cudaMemcpyAsync(d_views, g_views, sizeof(ViewDev) * (size_t)n_views, cudaMemcpyHostToDevice, s));
    MR_CUDA(cudaMemcpyAsync(d_scenes, g_scenes, sizeof(SceneDev) * (size_t)n_scenes, cudaMemcpyHostToDevice, s));
    MR_CUDA(cudaMemcpyAsync(d_images, g_images, sizeof(float*) * (size_t)n_views, cudaMemcpyHostToDevice, s));
    MR_CUDA(cudaMemcpyAsync(d_pixoff, g_pixoff, sizeof(uint64_t) * (size_t)n_views, cudaMemcpyHostToDevice, s));
    MR_CUDA(cudaMemsetAsync(d_work, 0, sizeof(unsigned long long), s));  // the previous call left it spent
    Rng rng;
    rng.set(params->seed_lo, params->seed_hi);
    // the launch shape follows mirres_render's persistent launch: the compiled variant that fits
    // (block, blocks_per_sm), or the context's autotuned variant and chunk when block is 0
    int var = mr_persistent_pick(params->block, params->blocks_per_sm);
    unsigned int chunk_w = 256;
    if (params->block == 0 && ctx->tuned_variant >= 0) {
        var = ctx->tuned_variant;
        chunk_w = ctx->tuned_chunk;
    }
    const int per_sm = params->blocks_per_sm ? params->blocks_per_sm : mr_persistent_occupancy_v(var);
    bool wide = false;
    for (int i = 0; i < n_scenes; ++i) wide = wide || g_scenes[i].wnodes != nullptr;
    MR_CUDA(mr_launch_persistent_v(var, d_scenes, d_views, n_views, total, rng, params->ris_m, d_work, chunk_w, tape,
                                   ctx->counters, per_sm * ctx->sm_count, s, 0, wide));
    mr_launch_resolve_all(d_views, n_views, d_pixoff, total_pix, d_images, tape, total, ctx->sm_count, s);
    MR_CUDA(cudaGetLastError());
    return MIRRES_OK;
}
