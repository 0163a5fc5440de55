// render.h -- structures and launchers of the forward / adjoint kernels (host side).
#pragma once

#include "internal.h"

// Reservoirs of the primary vertices for spatial reuse, one per path sample (SoA): env texel of
// the selection (RES_MISS: the primary ray escaped, RES_NONE: a hit without a selection), the
// selection's index among the vertex's own candidates, its sub-texel word, the weight sum and
// p_hat of the selection at its own vertex. All null when reuse is off.
enum { RES_MISS = -1, RES_NONE = -2 };
struct ResDev {
    int32_t* ytex;
    int32_t* sel;
    uint32_t* ysub;
    float* wsum;
    float* phat;
    float* m;  // candidates behind the reservoir
};

// The caller's reservoir history for temporal reuse (SoA over the call's samples): the final
// reservoir of each sample's primary vertex (texel or RES_MISS / RES_NONE, sub-texel word, weight
// sum, p_hat of the selection, candidate count). All null when temporal reuse is off.
struct HistDev {
    int32_t* ytex;
    uint32_t* ysub;
    float* wsum;
    float* phat;
    float* m;
};

// ray queue (SoA of float4): (o, origin triangle), (d, sample id), throughput, indirect throughput
struct QueueDev {
    float4* o;
    float4* d;
    float4* b;
    float4* bi;
};

// shadow-ray queue: (o, origin triangle), (d, sample id), radiance to add, L_ind to add
struct ShadowDev {
    float4* o;
    float4* d;
    float4* add;
    float4* addi;
};

struct GradDev {
    float* albedo;
    float* rough;
    float* metal;
    float* env;
    float* verts;
};

void mr_launch_raygen(const ViewDev& v, Rng rng, uint32_t first, uint32_t n, const QueueDev& q, void* tape,
                      uint64_t ntot, int sms, cudaStream_t st, int nvx = 0);
void mr_launch_closest(const SceneDev& s, const ViewDev& v, int b, const QueueDev& q, const unsigned int* count,
                       unsigned int count_fixed, uint64_t upper, const QueueDev& hq, unsigned int* count_hit,
                       void* tape, uint64_t ntot, int sms, cudaStream_t st);
void mr_launch_shade(const SceneDev& s, const ViewDev& v, Rng rng, int b, int M, const QueueDev& hq,
                     const unsigned int* count_hit, uint64_t upper, const QueueDev& qout, unsigned int* count_out,
                     const ShadowDev& sq, unsigned int* count_sh, void* tape, uint64_t ntot,
                     unsigned long long* counters, int sms, cudaStream_t st, int nvx = 0);
void mr_launch_shadow(const SceneDev& s, const ViewDev& v, int b, const ShadowDev& sq, const unsigned int* count,
                      uint64_t upper, void* tape, uint64_t ntot, int sms, cudaStream_t st, int nvx = 0);
void mr_launch_resolve(const ViewDev& v, const void* tape, uint64_t ntot, float* img, int sms, cudaStream_t st);
void mr_launch_account(unsigned long long* counters, const unsigned int* qcnt, int bounces, uint64_t primary,
                       cudaStream_t st);
cudaError_t mr_launch_persistent(const SceneDev* scenes, const ViewDev* views, int n_views, uint64_t total, Rng rng,
                                 int M, unsigned long long* work, uint32_t chunk, void* tape,
                                 unsigned long long* counters, int block, int blocks, cudaStream_t st, int nvx = 0);
int mr_persistent_occupancy(int block);
int mr_persistent_variants();
void mr_persistent_variant_shape(int v, int* block, int* minb);
int mr_persistent_pick(int block, int per_sm);
int mr_persistent_occupancy_v(int v);
// wide: the scenes are traversed through their 8-wide BVHs (one kernel for every v)
cudaError_t mr_launch_persistent_v(int v, const SceneDev* scenes, const ViewDev* views, int n_views, uint64_t total,
                                   Rng rng, int M, unsigned long long* work, uint32_t chunk, void* tape,
                                   unsigned long long* counters, int blocks, cudaStream_t st, int nvx, bool wide);
void mr_launch_resolve_all(const ViewDev* views, int n_views, const uint64_t* pix_off, uint64_t total_pix,
                           float* const* images, const void* tape, uint64_t ntot, int sms, cudaStream_t st);
// nvx = 0: PRIMARY-mode adjoint; nvx > 0: FULL mode over vertex records 1 .. nvx
// scratch of the FULL-mode adjoint (per-class counts and one chunk's sample list), device bytes
size_t mr_full_scratch_bytes();
uint64_t mr_full_chunk();  // samples per FULL-mode pass (0: one kernel does every vertex)
void mr_launch_backward(const SceneDev* scenes, const ViewDev* views, int n_views, uint64_t total, Rng rng,
                        const float* const* d_images, const GradDev* grads, const void* tape,
                        unsigned long long* counters, int sms, cudaStream_t st, int nvx, void* full_scratch,
                        bool interp);
void mr_launch_l2(const float* img, const float* ref, int64_t n, float* dimg, float* loss, int sms, cudaStream_t st);
// monochrome light regulariser: the demodulated lighting per pixel (out[view] [h][w][4]) and
// the PRIMARY-mode adjoint of it (d_demod[view] [h][w][3])
// pixels per tile of the demodulated-lighting kernel for a view of `spp` samples per pixel; the
// launch takes tile_off [n_views + 1] = the prefix sums of each view's ceil(pixels / tile)
int mr_light_tile_pixels(int spp);
void mr_launch_light_demod(const SceneDev* scenes, const ViewDev* views, const uint64_t* tile_off, int n_views,
                           uint64_t n_tiles, uint64_t total, Rng rng, const void* tape, float* const* out, int sms,
                           cudaStream_t st, bool interp);
void mr_launch_light_backward(const SceneDev* scenes, const ViewDev* views, int n_views, uint64_t total, Rng rng,
                              const float* const* d_demod, const GradDev* grads, const void* tape,
                              unsigned long long* counters, int sms, cudaStream_t st, bool interp);
void mr_launch_trace_rays(const SceneDev& s, const float* rays, const int32_t* skip, int64_t n, int any,
                          int32_t* hit_tri, float* hit_tuv, int sms, cudaStream_t st);

// denoise.cu: EAWT levels, their adjoints, the pixel-centre G-buffer
void mr_launch_eawt_pack(const float* a, float4* out, int64_t npx, int sms, cudaStream_t st);
void mr_launch_eawt_level(const float4* cin, const float4* nrm, const float4* pos, int N, int W, int H, int step,
                          float inv_rt2, float inv_n2, float inv_x2, float4* cout, float* out3, float* ikout, int sms,
                          cudaStream_t st);
void mr_launch_eawt_level_adjoint(const float4* gin, const float4* c, const float* ikin, const float4* nrm,
                                  const float4* pos, int N, int W, int H, int step, float inv_rt2, float inv_n2,
                                  float inv_x2, float4* gout, float* out3, int sms, cudaStream_t st);
void mr_launch_gbuffer(const SceneDev& s, const ViewDev& v, float* nrm, float* pos, int sms, cudaStream_t st);
// regular.cu: mesh regularisers over the scene's edge list (built by mr_edges_build)
void mr_launch_material_smoothness(const SceneDev& s, const ViewDev& v, uint32_t view_index, const Rng& rng,
                                   float sigma, float wa, float wr, float wn, float4* rec, float2* bary,
                                   unsigned int* n_hit, float* loss, float* ga, float* gr, bool grad_normals, int sms,
                                   cudaStream_t st);
void mr_launch_regularizers(const mirres_scene* s, const float* rest, float w_smooth, float w_offset, float* loss,
                            float* grad, int sms, cudaStream_t st);
// L_light from the demodulated lighting: loss[0] += w mean |Y(c) - V(ref)| over the covered
// pixels of every view (count is device scratch), d_demod = its gradient (overwritten)
cudaError_t mr_launch_light_loss(const uint64_t* pix_off, int n_views, uint64_t total_pixels,
                          const float* const* demod, const float* const* ref, float w, unsigned int* count,
                          float* loss, float* const* d_demod, int sms, cudaStream_t st);

// wave.cu: the batched wavefront forward (recorded on a stream, captured as a graph). A chain of
// waves: its ray queues, its stage counters [5 max_bounces + 3] and the stream it is recorded on.
struct WaveBranch {
    QueueDev qa, qb, hq;
    ShadowDev sq;
    unsigned int* qc;
    uint16_t* bkey;      // [wave] binning keys (flags bit 3)
    unsigned int* bhist; // [4096] binning histogram / cursors
    cudaStream_t st;
};
void mr_wave_record(const SceneDev* scenes, const ViewDev* views, int n_views, uint64_t total, int max_bounces,
                    Rng rng, int M, const uint64_t* wave_first, int n_waves, const WaveBranch* branches,
                    int n_branches, cudaEvent_t fork, cudaEvent_t* join, void* tape, unsigned long long* counters,
                    const uint64_t* pix_off, uint64_t total_pix, float* const* images, int sms, cudaEvent_t* ev,
                    int* kind, int nvx, bool count, int reuse_k, int reuse_radius, const ResDev& res, int temporal,
                    int temporal_cap, const HistDev& hist, const ViewDev* hviews, const SceneDev* hscenes, bool raster,
                    bool bin, const mirres_wave_shape& shape);
int mr_wave_launches(int n_waves, int max_bounces, bool reuse, int temporal, int raster_launches, bool bin);
int mr_wave_stage_pairs(int n_waves, int max_bounces);
