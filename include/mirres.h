/*
 * mirres.h -- C ABI of the GB300 (sm_103a) MIRReS stage-2 hot path: forward and adjoint
 * Monte Carlo multi-bounce path tracing of a triangle mesh under an environment map, with a
 * GGX + Lambert BRDF (per-texel albedo / roughness / metallic) and weighted-reservoir RIS of
 * environment-light candidates at every shading point.
 *
 * The calls follow the paper's statement of the problem (Sec. 3.2): a mesh M = {V, F} whose
 * vertices are refined, spatially varying materials m, an HDR environment map whose texels
 * are all trainable, calibrated cameras, rendered images I_PBR and the gradient of
 * L_PBR = ||I_PBR - I_ref||^2 (Eq. loss_pbr) with respect to all of them.
 *
 * Conventions
 *   - All array arguments inside descriptors are DEVICE pointers into caller-owned memory
 *     (for example torch tensors). The library borrows them: it never frees them and keeps
 *     only the pointer; the caller keeps them alive while a scene refers to them.
 *   - Arrays of per-view / per-scene pointers (images, d_images, grads, scenes) are HOST
 *     arrays of device pointers, read during the call only.
 *   - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream)
 *     unless documented otherwise; results are ready when the stream reaches that point.
 *   - Float arrays are row-major FP32. Triangle indices are int32.
 *   - Errors: every call returns a mirres_status; mirres_last_error() returns a message for
 *     the calling thread. Sticky CUDA errors are reported as MIRRES_ERR_CUDA. Arguments are
 *     validated on the host before any work is queued; a rejected call queues nothing.
 *
 * Readings of passages the paper leaves open (estimator details, BRDF form, sampling
 * mixture, camera model, random-number layout) are documented with each call below and
 * are shared, as statements, by the independent CPU reference used in the tests.
 */
#ifndef MIRRES_H
#define MIRRES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MIRRES_OK = 0,
    MIRRES_ERR_ARG = 1,     /* invalid argument (NULL pointer, bad size, mismatched tape) */
    MIRRES_ERR_CUDA = 2,    /* a CUDA runtime call failed */
    MIRRES_ERR_OOM = 3,     /* device allocation failed */
    MIRRES_ERR_TIMEOUT = 4, /* a bounded device loop hit its iteration cap (error flag set) */
    MIRRES_ERR_STATE = 5    /* call out of order (e.g. render before mirres_bvh_build) */
} mirres_status;

typedef struct mirres_context mirres_context; /* per device / stream: workspace, counters */
typedef struct mirres_scene mirres_scene;     /* BVH, env sampling tables, borrowed inputs */

/* Scene description (Sec. 3.2: mesh M = {V, F}, material textures, env map 256x512 in the
 * paper; any size here). Every pointer is a device pointer, borrowed.
 *   verts    [n_verts][3]        world positions (y up)
 *   tris     [n_tris][3]         vertex indices, 0 <= index < n_verts (checked on the device
 *                                by mirres_scene_create and mirres_scene_validate, which then
 *                                return MIRRES_ERR_ARG; builds and refits do not check and
 *                                read an out-of-range index as vertex 0)
 *   tri_uv   [n_tris][3][2]      per-corner texture coordinates
 *   albedo   [tex_h][tex_w][3], roughness [tex_h][tex_w], metallic [tex_h][tex_w]
 *                                sampled bilinearly, texel centres at (i + 0.5) / size,
 *                                clamp to edge; row index = v * tex_h
 *   env      [env_h][env_w][3]   latitude-longitude radiance, row 0 = zenith (+y);
 *                                direction d -> u = atan2(d.x, -d.z) / 2pi + 1/2,
 *                                v = acos(d.y) / pi, nearest texel (piecewise constant)
 * n_tris may be 0 (every ray escapes). tex_w, tex_h, env_w, env_h >= 1. */
typedef struct {
    const float* verts;   int32_t n_verts;
    const int32_t* tris;  int32_t n_tris;
    const float* tri_uv;
    const float* albedo;  const float* roughness; const float* metallic;
    int32_t tex_w, tex_h;
    const float* env;     int32_t env_w, env_h;
} mirres_scene_desc;

/* One camera (pinhole, Sec. 3.2 camera ray r(t) = o + t d). K = (fx, fy, cx, cy) in pixels;
 * c2w = row-major 3x4 [R | t] whose columns are the camera x (right), y (down) and z
 * (forward) axes in world space and whose last column is the centre o. Pixel (px, py) with
 * jitter (j0, j1) in [0,1)^2 looks along normalize(R ((px + j0 - cx)/fx, (py + j1 - cy)/fy, 1)).
 * spp = samples per pixel, bounces = shading vertices per path (the paper uses three,
 * Sec. 4.2), scene = index into the call's scene array. */
typedef struct {
    float K[4];
    float c2w[12];
    int32_t width, height, spp, bounces;
    int32_t scene;
} mirres_view;

/* Render parameters.
 *   ris_m    RIS candidates per shading point (m of Eq. restir), >= 1
 *   seed     key of the Philox4x32-10 stream. Uniform number k of purpose P for sample s
 *            of pixel p of view index v at bounce b is drawn from counter
 *            (p, s, v << 16 | b << 8 | P, j) and key (seed_lo, seed_hi); u = (x >> 8) 2^-24.
 *            P = 0 camera jitter, 1 RIS candidate j, 2 continuation. v is the view's index
 *            in the call's view array (< 65536); bounces < 256.
 *   grad_mode 0 = PRIMARY (the paper: gradients of indirect rays detached, Sec. 4.2)
 *            1 = FULL: also the gradients through every later vertex (the part Sec. 4.2
 *                detaches and Appendix C names as missing); the forward then records every
 *                vertex on the tape (mirres_tape_bytes_mode) and mirres_backward walks them;
 *                at most MIRRES_FULL_MAX_BOUNCES bounces per view
 *   launch   0 = plain: per-view wavefront launches (ray generation, closest hit with hit
 *                 compaction, shade + RIS + next-bounce queue, shadow rays, resolve);
 *            1 = batched wavefront: every view of every scene flattened into waves of up to
 *                 2^wave_log2 samples (mirres_wave_shape, default 2^25, autotuned by
 *                 mirres_autotune_wave); the whole forward is one CUDA graph, captured on first use and
 *                 replayed while the shape (each view's size, samples, bounces and scene; each
 *                 scene's triangle count and normal mode), tape, seed and workspace stay the
 *                 same (cameras and scene contents may change between replays);
 *            2 = persistent kernel: one launch over every view of every scene, each warp
 *                 pulling samples from a device counter and refilling lanes by ballot.
 *            All take every discrete decision identically (hit triangles, selected
 *            candidates, lobes); values agree to FP32 rounding (the kernels may contract
 *            multiply-adds differently).
 *   reuse_k, reuse_radius  spatial reuse at the primary vertex (Appendix A, "Spatial-temporal
 *            Reuse"): each bounce-0 reservoir merges those of reuse_k neighbouring pixels (same
 *            sample index; offsets (dx, dy) = ((x >> 8) (2 r + 1) >> 24) - r of the first two
 *            words of the reuse stream P = 3, j = neighbour; the pixel itself and pixels outside
 *            the image skipped, a neighbour whose primary ray escaped has no reservoir). Each
 *            reservoir enters with weight p_hat_here(y) w_sum / p_hat_there(y), accepted iff
 *            u w_sum < weight with u from the third word; the merged reservoir counts ris_m
 *            candidates per reservoir (own and neighbours that hit), W = w_sum / (m p_hat(y)).
 *            The paper gives no MIS weights: this is the biased 1/m combination. Batched
 *            launch only (whole views per wave, a wave enlarged to hold the largest view);
 *            reuse_k in [0, 64], reuse_radius >= 1.
 *   temporal, temporal_cap, reuse_history  temporal reuse (Appendix A: reservoirs of previous
 *            frames merged): with temporal = 2 every primary vertex first merges the reservoir
 *            its sample left in reuse_history (candidate count capped at temporal_cap * ris_m,
 *            weight p_hat_here(y) w_sum / p_hat_then(y) (m_capped / m), accepted with the third
 *            word of reuse draw j = 65535), before spatial reuse; with temporal = 1 or 2 the
 *            final reservoirs are written back to reuse_history (the same views, in the same
 *            order, must come in the next call). Batched launch only.
 *   block, blocks_per_sm  launch shape of the persistent kernel (0 = autotuned / default)
 *   flags    bit 0: record CUDA events around every stage kernel of the batched wavefront
 *            (read back with mirres_stage_times); bit 1: the batched wavefront counts its
 *            traversal work (mirres_get_work_counters) -- a separately compiled variant of the
 *            traversal kernels, so that the uncounted launch keeps its register budget; bit 2: the
 *            batched wavefront resolves primary visibility by rasterisation (each triangle
 *            projected into the view, each camera sample in its screen box tested with the
 *            traversal's FP32 ray/triangle solve, closest by a 64-bit atomicMin on (t, triangle)),
 *            as the paper does with a rasteriser, instead of tracing primary rays; bit 3: the
 *            batched wavefront bins each bounce's continuation rays by origin cell (8 x 8 x 8
 *            over the scene's bounds) and direction octant before tracing them (a counting
 *            sort of the ray queue; the results are unchanged, only the rays' order in the queue)
 *   max_visits  failure detection: every ray traversal is a bounded loop of at most max_visits
 *            node visits (0 = 4 n_tris + 64, more than any well-formed tree needs) on a bounded
 *            stack; a traversal that reaches either bound ends as a miss and raises the
 *            context's error counter, which mirres_get_counters reports as MIRRES_ERR_TIMEOUT.
 *            The kernels never wait on anything, so nothing else can stall them. */
typedef struct {
    int32_t ris_m;
    uint32_t seed_lo, seed_hi;
    int32_t grad_mode;
    int32_t launch;
    int32_t block;
    int32_t blocks_per_sm;
    int32_t flags;
    int32_t reuse_k;       /* spatial reuse: neighbouring reservoirs merged per pixel (0 = off) */
    int32_t reuse_radius;  /* ... drawn from the (2 r + 1)^2 pixel square around the pixel */
    int32_t temporal;      /* temporal reuse: 0 off, 1 record the reservoir history, 2 merge it, then record */
    int32_t temporal_cap;  /* the history counts at most temporal_cap * ris_m candidates */
    void* reuse_history;   /* device, mirres_reuse_history_bytes(views) bytes, caller-owned, kept across calls */
    uint64_t reuse_history_bytes;
    int32_t max_visits;    /* iteration cap of one ray traversal in node visits (0 = 4 n_tris + 64) */
} mirres_params;
#define MIRRES_REUSE_MAX_K 64
#define MIRRES_FLAG_STAGE_EVENTS 1
#define MIRRES_FLAG_COUNT_WORK 2
#define MIRRES_FLAG_RASTER 4
#define MIRRES_FLAG_BIN 8

/* Gradient destinations for one scene (device pointers, shapes of the scene's inputs).
 * Accumulated (+=); a NULL pointer skips that parameter. */
typedef struct {
    float* albedo; float* roughness; float* metallic; float* env; float* verts;
} mirres_grads;

/* ---- lifetime ------------------------------------------------------------------------ */

/* Create a context on `device` (makes it current on the calling thread). The context owns
 * a grow-only device workspace (ray queues, per-view scratch), device counters and an error
 * flag. Calls sharing a context must be issued on one stream at a time. */
mirres_status mirres_context_create(int32_t device, mirres_context** out);
mirres_status mirres_context_destroy(mirres_context* ctx);

/* Create a scene from borrowed device arrays; validates sizes and pointers on the host and
 * every triangle index on the device (synchronises the legacy default stream once;
 * MIRRES_ERR_ARG if an index is outside [0, n_verts)). The scene owns its LBVH and
 * env-sampling tables (allocated here). */
mirres_status mirres_scene_create(mirres_context* ctx, const mirres_scene_desc* desc, mirres_scene** out);
mirres_status mirres_scene_destroy(mirres_scene* scene);

/* Check the scene's triangle indices again (for a caller that rewrote desc.tris in place):
 * synchronises `stream`; MIRRES_ERR_ARG if an index is outside [0, n_verts). */
mirres_status mirres_scene_validate(mirres_scene* scene, void* stream);

/* LBVH build (Appendix A "Visibility estimation": a linear BVH after Karras 2012): FP32
 * triangle centroids (fixed operation order, no contraction), 30-bit Morton codes in the
 * centroid box, keys code << 32 | triangle, stable radix sort, binary radix tree, bottom-up
 * boxes, traversal layout (and, with MIRRES_TRAVERSAL_WIDE, the 8-wide BVH collapsed from
 * the binary tree). Also rebuilds the env sampling tables (FP64 prefix sums of
 * Y(L) sin(theta); Y = (r+g+b)/3, Appendix A). Asynchronous: no host synchronisation (the
 * triangle indices were checked by mirres_scene_create), so it can be captured into a graph
 * with the default LBVH builder. */
mirres_status mirres_bvh_build(mirres_scene* scene, void* stream);

/* Hierarchy builder used by the next mirres_bvh_build of this scene:
 *   MIRRES_BVH_LBVH (default): Karras's binary radix tree over the Morton-sorted triangles, the
 *     linear BVH the paper names (Appendix A, "Visibility estimation");
 *   MIRRES_BVH_PLOC: parallel locally-ordered clustering (Meister and Bittner 2018) over the same
 *     Morton-sorted triangles: each cluster pairs with the cluster within 16 positions whose
 *     union box has the smallest surface area, mutual pairs merge, repeat. A lower-SAH tree
 *     (fewer nodes visited per ray) for a slower build (about log F host round trips). Not in
 *     the paper.
 * Both write the same layout (root 0, leaves by Morton position), so refit, traversal and
 * mirres_bvh_export are unchanged, and closest / any hits do not depend on the tree.
 * MIRRES_ERR_ARG for an unknown builder. */
/* Shading normals of a scene (the paper shades with "the surface normal" and does not say how
 * it is formed):
 *   MIRRES_NORMALS_FACE (default): the face normal, turned towards the viewer;
 *   MIRRES_NORMALS_INTERPOLATED: the barycentric blend of area-weighted vertex normals (the sum
 *     of the incident faces' e1 x e2, normalised), turned to the viewer's side of the face; RIS
 *     candidates, reused reservoirs and continuations below the face are then dropped. The
 *     vertex normals are recomputed by every mirres_bvh_build and mirres_bvh_refit (and here if
 *     the scene is built); the PRIMARY adjoint follows the shading normal to the barycentrics
 *     and to the vertices of every face around the hit triangle's vertices.
 * Allocates 40 bytes per vertex the first time it is enabled. MIRRES_ERR_ARG for an unknown
 * mode. */
#define MIRRES_NORMALS_FACE 0
#define MIRRES_NORMALS_INTERPOLATED 1
mirres_status mirres_scene_set_normals(mirres_scene* scene, int32_t mode);

#define MIRRES_BVH_LBVH 0
#define MIRRES_BVH_PLOC 1
mirres_status mirres_bvh_set_builder(mirres_scene* scene, int32_t builder);

/* The tree every ray traversal of this scene runs (not in the paper; both give the same hits,
 * up to rays that touch a box within rounding):
 *   MIRRES_TRAVERSAL_BINARY (default): the binary tree of mirres_bvh_build, two child boxes in
 *     one 64-byte node, a stack of 32-bit node indices;
 *   MIRRES_TRAVERSAL_WIDE: an 8-wide BVH collapsed from the binary tree after every build and
 *     refit (80-byte nodes with 8-bit child boxes quantised outwards, leaves of up to three
 *     triangles, children slotted by octant so that a ray visits them near to far; measured
 *     slower than the binary tree on the 499k-triangle scene). Allocates ~200 bytes per
 *     triangle the first time; collapses at once (synchronising) if the scene is built.
 * MIRRES_ERR_ARG for an unknown mode. */
#define MIRRES_TRAVERSAL_BINARY 0
#define MIRRES_TRAVERSAL_WIDE 1
mirres_status mirres_scene_set_traversal(mirres_scene* scene, int32_t mode);

/* Refit after the vertices moved (the paper keeps its LBVH in step with the mesh at every
 * iteration, Appendix A): topology kept, boxes and packed triangles recomputed bottom-up and the
 * wide BVH collapsed again; env tables rebuilt. Asynchronous. Requires a prior mirres_bvh_build. */
mirres_status mirres_bvh_refit(mirres_scene* scene, void* stream);

/* ---- forward / adjoint ----------------------------------------------------------------- */

/* Tape bytes per path sample: 17 32-bit words, stored as 17 arrays over the samples. */
#define MIRRES_TAPE_BYTES_PER_SAMPLE 68
/* FULL mode (grad_mode 1) adds, per sample, one record of 9 words for each vertex b = 1 ..
 * max_bounces - 1 (max over the call's views), stored as arrays after the 17 primary words:
 * word ((b - 1) * 9 + w) of sample g at index 17 * n + ((b - 1) * 9 + w) * n + g, n = samples;
 * w: 0 hit triangle (-1: the path never reached vertex b), 1-2 barycentrics (u, v), 3 selected
 * RIS candidate (-1: none), 4 V * W, 5-7 continuation direction, 8 its pdf (0: the path ended). */
#define MIRRES_TAPE_BYTES_PER_VERTEX 36
#define MIRRES_FULL_MAX_BOUNCES 16

/* Bytes of tape needed for these views: MIRRES_TAPE_BYTES_PER_SAMPLE per path sample (sum of
 * width*height*spp). The tape records, per sample (word: content): 0 primary triangle (-1 if
 * the primary ray escaped), 1 index of the selected RIS candidate at the primary vertex (-1 if
 * none), 2 V*W of that candidate, 3-5 the incident indirect radiance L_ind at the primary
 * vertex, 6-8 the sample's radiance, 9 the env texel of the selected candidate, 10-12 its
 * direction, 13-15 the continuation direction at the primary vertex, 16 its mixture pdf
 * p_ind. Words 9-16 are meaningful only where word 1 >= 0, resp. L_ind != 0. The adjoint
 * replays the primary vertex from it and the camera's random numbers; no sample is re-drawn. */
size_t mirres_tape_bytes(const mirres_view* views, int32_t n_views);

/* Bytes of the reservoir history of temporal reuse: 20 per path sample, stored as 5 arrays over
 * the samples (selection's env texel: -1 primary ray escaped, -2 no selection; sub-texel word;
 * weight sum; p_hat of the selection; candidate count). 0 for invalid arguments. */
size_t mirres_reuse_history_bytes(const mirres_view* views, int32_t n_views);

/* Tape bytes for a gradient mode: mirres_tape_bytes for grad_mode 0 (PRIMARY); for 1 (FULL)
 * MIRRES_TAPE_BYTES_PER_SAMPLE + MIRRES_TAPE_BYTES_PER_VERTEX * (max bounces - 1) per sample.
 * 0 for invalid arguments. A FULL-mode tape also serves PRIMARY-mode calls. */
size_t mirres_tape_bytes_mode(const mirres_view* views, int32_t n_views, int32_t grad_mode);

/* Forward render (Eq. pbr_render with Eq. incident: direct light by RIS over ris_m env
 * candidates streamed through a weighted reservoir, Eq. restir and Appendix A; indirect light
 * by one continuation ray per vertex from a one-sample MIS mixture of env importance sampling
 * (weight 1/4 when the env is not black), GGX visible-normal sampling and cosine sampling
 * (split by the Fresnel/diffuse luminance ratio clamped to [0.1, 0.9]), Eq. mc_indir and
 * Eq. sec_bouce). A continuation ray that escapes adds nothing (its env light is already in
 * the direct term); a primary ray that escapes sees the env.
 *   images[v]  device [height][width][3], written (mean over spp)
 *   tape       device, mirres_tape_bytes(views) bytes, or NULL (the context's workspace is
 *              used instead; mirres_backward then needs a tape from a later render)
 * Scenes must have been built. Each images[v] must not alias another. */
mirres_status mirres_render(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                            const mirres_view* views, int32_t n_views, const mirres_params* params,
                            float* const* images, void* tape, size_t tape_bytes, void* stream);

/* Autotuner of the batched launch (no counterpart in the paper; a launch-shape search):
 * times each compiled persistent-kernel variant (block size x resident blocks per SM, which
 * sets its register cap) and each per-warp work chunk (64, 256, 1024 samples) on the first
 * budget_samples samples of this batch (0 = all), keeps the fastest in the context (used by
 * later batched renders whose params.block is 0) and reports it. Synchronises `stream`.
 * The tape must be the full tape of these views (its first samples are overwritten). */
mirres_status mirres_autotune(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                              const mirres_view* views, int32_t n_views, const mirres_params* params,
                              void* tape, size_t tape_bytes, uint64_t budget_samples, int32_t* out_block,
                              int32_t* out_blocks_per_sm, int32_t* out_chunk, float* out_ms, void* stream);

/* Set the batched launch shape of the context directly (e.g. from a cache of autotuner
 * results): block 0 restores the default. */
mirres_status mirres_set_launch(mirres_context* ctx, int32_t block, int32_t blocks_per_sm, int32_t chunk);

/* Launch shape of the batched wavefront (launch = 1; no counterpart in the paper): the wave size
 * -- samples per wave, which is the capacity of every ray queue -- and, per stage kernel
 * (index = stage: 0 closest hit, 1 shade + RIS (and the reuse kernels), 2 shadow rays, 3 ray
 * generation), the threads per block and the grid of its grid-stride loop in blocks per SM.
 * The lane-refilling kernels that trace continuation rays (bounces >= 1) and shadow rays run
 * 256 threads in one resident wave of blocks whatever the shape; the shape sets the primary
 * rays' closest-hit kernel, shading and ray generation (and shadow rays on 8-wide BVHs).
 * Default: 2^25 samples, 256 threads and 8 blocks per SM for every stage, one chain. */
typedef struct {
    int32_t wave_log2;        /* samples per wave = 2^wave_log2, in [16, 28] */
    int32_t block[4];         /* 64, 128 or 256 */
    int32_t blocks_per_sm[4]; /* in [1, 64] */
    int32_t branches;         /* in [1, 4]: waves go round-robin to this many chains, each with
                                 its own ray queues (256 bytes per sample of a wave) and stream,
                                 so that the stages of different waves overlap; default 1 */
} mirres_wave_shape;

/* Set (shape = NULL: restore the default) or read the context's wavefront shape; used by every
 * later batched render of the context (a changed shape re-captures the forward's graph).
 * MIRRES_ERR_ARG for a value outside the ranges above. */
mirres_status mirres_set_wave_shape(mirres_context* ctx, const mirres_wave_shape* shape);
mirres_status mirres_get_wave_shape(mirres_context* ctx, mirres_wave_shape* out);

/* Autotuner of the batched wavefront: renders the first views of the batch (up to
 * budget_samples samples, at least one view; 0 = all) with the wavefront and CUDA events around
 * every stage, for each of a set of (threads per block, blocks per SM) pairs applied to all
 * stages at once; keeps the fastest pair per stage, then times the wave sizes 2^23, 2^24 and
 * 2^25 (those the budget fills) with the chosen stage shapes and keeps the fastest forward,
 * then two and three chains of waves (branches = 2, 3) at the chosen wave size and at half of
 * it, where the tuned views fill as many waves as chains, kept if faster still. Each shape is
 * rendered once to capture its graph, then timed (the fastest of two renders for the wave sizes
 * and chains).
 * The result becomes the context's shape (mirres_set_wave_shape) and is written to *out, the
 * tuned forward's time to *out_ms. The tape must hold these views (it is overwritten); the
 * renders write temporary images (allocated and freed here). params as for mirres_render
 * (launch, reuse and flags ignored). Synchronises `stream`. */
mirres_status mirres_autotune_wave(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                                   const mirres_view* views, int32_t n_views, const mirres_params* params,
                                   void* tape, size_t tape_bytes, uint64_t budget_samples, mirres_wave_shape* out,
                                   float* out_ms, void* stream);

/* Summed device time (ms) and launch count of each stage of the last batched-wavefront
 * render that was issued with params.flags bit 0: out_ms[0..3] = closest hit, shade (RIS),
 * shadow rays, ray generation; out_launches likewise. Synchronises on those events. */
mirres_status mirres_stage_times(mirres_context* ctx, double out_ms[4], int32_t out_launches[4]);

/* The same events one by one, in the order the render issued them: out_ms[i] the device time
 * of stage launch i (within its wave's chain), out_stage[i] its stage (index as above),
 * out_bounce[i] its bounce (-1 for ray generation); at most `cap` entries are written, *out_n
 * receives how many there are. MIRRES_ERR_STATE when no render with flags bit 0 was captured.
 * Synchronises on those events. */
mirres_status mirres_stage_trace(mirres_context* ctx, int32_t cap, float* out_ms, int32_t* out_stage,
                                 int32_t* out_bounce, int32_t* out_n);

/* ---- forward without device allocation ------------------------------------------------ */

#define MIRRES_NOALLOC_SCRATCH_BYTES (512u * 1024u) /* static scratch per GPU, held until exit */
#define MIRRES_NOALLOC_MAX_VIEWS 4096
#define MIRRES_NOALLOC_MAX_SCENES 256

/* The paper has no counterpart to this call; it exists for callers that cannot allocate
 * device memory while they render: for example a process whose device memory is entirely
 * reserved by another allocator (a framework's caching allocator), or a latency-critical
 * serving loop that must not pay the device-wide synchronisation cudaMalloc / cudaFree can
 * bring. It runs the persistent-kernel forward of mirres_render (launch = 2, whatever valid
 * launch is given; the launch shape follows params.block / blocks_per_sm, or the context's
 * autotuned shape when block is 0) with the same results, but keeps its scratch -- the per-call view,
 * scene and image tables and the work counter -- in one static device array of
 * MIRRES_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the process
 * exits. It calls no cudaMalloc, cudaFree or allocating library routine.
 *   - The tape is required (caller-owned, mirres_tape_bytes(views) bytes, 16-byte aligned).
 *   - PRIMARY-mode tape only (grad_mode 0) and no reservoir reuse: reuse_k > 0 or temporal > 0
 *     (which need per-sample scratch) is rejected with MIRRES_ERR_ARG.
 *   - n_views > MIRRES_NOALLOC_MAX_VIEWS or n_scenes > MIRRES_NOALLOC_MAX_SCENES is rejected
 *     with MIRRES_ERR_ARG and a message naming the limit; all scenes share one context.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current.
 *   - Every call shares the one array, which keeps the last call's contents; the call resets
 *     what must start at zero (the work counter). Calls whose work overlaps on the GPU (on
 *     different streams, or from several host threads without ordering) race on the array:
 *     serialise them. */
mirres_status mirres_render_noalloc(mirres_scene* const* scenes, int32_t n_scenes, const mirres_view* views,
                                    int32_t n_views, const mirres_params* params, float* const* images,
                                    void* tape, size_t tape_bytes, void* stream);

/* Adjoint, PRIMARY mode (Sec. 4.2: gradients of indirect rays detached; Appendix C: no
 * gradients of non-primary rays): for every sample, the primary vertex is replayed from the
 * tape and the camera's random numbers, and the derivatives of direct_1 + beta_1 * L_ind (RIS weight,
 * visibility, every sampling decision, p_ind and L_ind held fixed) are scattered into the
 * texels of albedo / roughness / metallic (bilinear weights), the env texel of the selected
 * candidate and of escaping primary rays, and the three vertices of the primary triangle
 * (through the intersection barycentrics and the face normal). Warp-aggregated FP32 atomics.
 *   d_images[v]  device [height][width][3] = dL/dI (e.g. 2 (I - I_ref) for Eq. loss_pbr)
 *   grads[s]     gradient destinations of scene s (host array of n_scenes structs)
 * The views, params and scenes must be those of the render that wrote `tape`. */
mirres_status mirres_backward(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                              const mirres_view* views, int32_t n_views, const mirres_params* params,
                              const float* const* d_images, const void* tape, size_t tape_bytes,
                              const mirres_grads* grads, void* stream);

/* L2 image loss of Eq. (loss_pbr) and its gradient: d_image = 2 (image - ref) and
 * loss[0] += sum (image - ref)^2 (device scalar, FP32 accumulated per block then atomically).
 * n = number of floats. Any of d_image / loss may be NULL. */
mirres_status mirres_l2_loss(const float* image, const float* ref, int64_t n, float* d_image, float* loss,
                             void* stream);

/* ---- ray queries ---------------------------------------------------------------------- */

/* Closest (any = 0) or any (any = 1) hit of n rays against the scene's LBVH: rays [n][6]
 * device (origin, direction), skip_tri [n] device or NULL (triangle to ignore, -1 none);
 * hit_tri [n] device (-1 = miss; any-hit writes 1 / -1), hit_tuv [n][3] device or NULL
 * (t, u, v with barycentric u of vertex 1, v of vertex 2). Hits need t > t_min
 * (1e-5 x scene diagonal); equal t -> smaller triangle index. */
mirres_status mirres_trace(mirres_context* ctx, const mirres_scene* scene, const float* rays,
                           const int32_t* skip_tri, int64_t n, int32_t any, int32_t* hit_tri,
                           float* hit_tuv, void* stream);

/* ---- introspection ------------------------------------------------------------------- */

/* Copy the LBVH arrays to caller device buffers (any may be NULL): keys [F] (uint64, sorted),
 * left/right [F-1] (>= 0 internal node, < 0 leaf ~position), parent [2F-1], lo/hi [2F-1][3]
 * (internal nodes first, then leaves). */
mirres_status mirres_bvh_export(const mirres_scene* scene, uint64_t* keys, int32_t* left, int32_t* right,
                                int32_t* parent, float* lo, float* hi, void* stream);

/* Copy the env sampling tables to caller device buffers (any may be NULL): the factorised
 * form of the proposal, marg [env_h + 1] and cond [env_h][env_w + 1] as uint32 thresholds
 * ceil(cdf * 2^24) (cdf <= u exactly when threshold <= u * 2^24 for a 24-bit uniform u),
 * texel [env_h][env_w][4] = (r, g, b, probability * env_w * env_h) and the FP64 total weight
 * (device double). The draw itself inverts the CDF of mirres_env_export_flat. */
mirres_status mirres_env_export(const mirres_scene* scene, uint32_t* marg, uint32_t* cond, float* texel,
                                double* total, void* stream);

/* The CDF over all env texels in row-major order that every env draw inverts (RIS candidates,
 * the env lobe of the continuation mixture): thresholds [env_h env_w + 1] = ceil(cdf 2^53),
 * cdf = (weights of the rows before + of the texels before in the row) / total, each sum in
 * order. A draw takes k = w0 2^21 + (w1 >> 11) from two random words and the texel t with
 * thresholds[t] <= k < thresholds[t + 1]. Device copy (asynchronous); for tests. */
mirres_status mirres_env_export_flat(const mirres_scene* scene, uint64_t* thresholds, void* stream);

/* ---- denoiser between the rendered image and the loss (Appendix A, "Denoiser") ------------- */

/* Edge-avoiding a-trous wavelet denoiser. Level i (i = 0 .. levels-1) smooths c_i into
 *   c_{i+1}(p) = sum_q h(q - p) w(p, q) c_i(q) / sum_q h(q - p) w(p, q)
 * over 5 x 5 B3-spline taps (1, 4, 6, 4, 1) / 16 per axis placed 2^i pixels apart (taps outside
 * the image left out), with w(p, q) = exp(-|c_i(p) - c_i(q)|^2 / (sigma_rt / 2^i)^2
 * - |n_p - n_q|^2 / sigma_n^2 - |x_p - x_q|^2 / sigma_x^2) on the colour of the level's input
 * and the G-buffer normals n and positions x. The paper uses three levels. */
#define MIRRES_EAWT_MAX_LEVELS 8
typedef struct {
    float sigma_rt, sigma_n, sigma_x;  /* > 0 */
    int32_t levels;                    /* 1 .. MIRRES_EAWT_MAX_LEVELS */
} mirres_eawt_params;

/* Bytes of the record mirres_eawt writes for mirres_eawt_backward: (32 + 20 * levels) * width *
 * height (the packed G-buffer, each level's input image and reciprocal normaliser 1 / k). 0 for
 * invalid arguments. The record must be 16-byte aligned. */
size_t mirres_eawt_record_bytes(int32_t width, int32_t height, int32_t levels);

/* G-buffer of one view: the primary hit through each pixel centre (camera as in mirres_render,
 * jitter 1/2), face normal turned towards the camera and hit position; both 0 where the ray
 * escapes. normal, position: device [height][width][3], caller-owned. view->scene is ignored
 * (the scene is `scene`). Asynchronous. */
mirres_status mirres_gbuffer(mirres_context* ctx, const mirres_scene* scene, const mirres_view* view,
                             float* normal, float* position, void* stream);

/* Denoise one image: image, normal, position [height][width][3] device (read-only), out
 * [height][width][3] device, record (mirres_eawt_record_bytes, device) receives what the
 * adjoint needs; the image may be overwritten after the call. Asynchronous.
 * MIRRES_ERR_ARG for NULL pointers, sizes < 1, sigmas <= 0, levels outside [1, 8] or a record
 * that is too small. */
mirres_status mirres_eawt(mirres_context* ctx, const float* image, const float* normal, const float* position,
                          int32_t width, int32_t height, const mirres_eawt_params* params, float* out,
                          void* record, size_t record_bytes, void* stream);

/* Adjoint of mirres_eawt with its weights held fixed (they depend on the forward's images and
 * are treated as constants): d_image = A^T d_out, A the linear filter the recorded forward
 * applied. d_out, d_image [height][width][3] device; record, normal, position, params those of
 * the forward. d_image is overwritten (not accumulated). Uses the context workspace. */
mirres_status mirres_eawt_backward(mirres_context* ctx, const float* d_out, const float* normal,
                                   const float* position, int32_t width, int32_t height,
                                   const mirres_eawt_params* params, const void* record, size_t record_bytes,
                                   float* d_image, void* stream);

/* mirres_eawt and mirres_eawt_backward over a stack of n_images images of the same size (the
 * views of a batch): image, normal, position, out, d_out and d_image are [n_images][height]
 * [width][3] device, contiguous; the record holds n_images * mirres_eawt_record_bytes(width,
 * height, levels) bytes. Every level is one launch over the whole stack; each image is filtered
 * on its own (no tap crosses into another image), with the results of one mirres_eawt call per
 * image. MIRRES_ERR_ARG as for the single-image calls, and for n_images < 1 or a stack of more
 * than 2^31 pixels. */
mirres_status mirres_eawt_batch(mirres_context* ctx, int32_t n_images, const float* image, const float* normal,
                                const float* position, int32_t width, int32_t height,
                                const mirres_eawt_params* params, float* out, void* record, size_t record_bytes,
                                void* stream);
mirres_status mirres_eawt_batch_backward(mirres_context* ctx, int32_t n_images, const float* d_out,
                                         const float* normal, const float* position, int32_t width, int32_t height,
                                         const mirres_eawt_params* params, const void* record, size_t record_bytes,
                                         float* d_image, void* stream);

/* Mesh regularisers added to the rendering loss while the geometry is refined (Appendix A,
 * "Training details"):
 *   L_smooth = sum_i sum_{j in X_i} |v_i - v_j|^2 / |X_i|   (X_i: vertices sharing an edge with i)
 *   L_offset = sum_i |v_i - v0_i|^2                         (v0 = rest_verts)
 * on the scene's current vertices (desc.verts). Adds w_smooth L_smooth + w_offset L_offset to
 * loss[0] and its gradient to grad_verts [n_verts][3] (device, both accumulated, either may be
 * NULL). rest_verts [n_verts][3] device, needed only when w_offset != 0. X_i comes from the
 * triangles' edges, each neighbour counted once; the edge list is built on the first call with
 * w_smooth != 0 and kept by the scene (the topology is fixed; allocates once). Asynchronous;
 * the loss is an FP32 sum in no fixed order. MIRRES_ERR_ARG for a NULL ctx/scene, a negative
 * weight or a missing rest_verts; MIRRES_ERR_STATE before mirres_bvh_build. */
mirres_status mirres_mesh_regularizers(mirres_context* ctx, mirres_scene* scene, const float* rest_verts,
                                       float w_smooth, float w_offset, float* loss, float* grad_verts,
                                       void* stream);

/* Material smoothness regulariser (Appendix A, "Training details"):
 *   L_k = (1 / |X|) sum_{x in X} |k(x) - k(x + eps)|,  k in {albedo, roughness, normal}
 * X = the surface points seen through the pixel centres of `view` (camera as in mirres_render,
 * jitter 1/2; escaped pixels are not in X). The materials are textures, so the small random
 * offset is taken in texture space: k(x + eps) is the bilinear lookup at the hit's texture
 * coordinates + eps, eps uniform in [-sigma, sigma]^2 from Philox4x32-10 (key = seed, counter
 * (pixel, 0, view_index << 16 | 4, 0), eps = sigma (2 u - 1) with u the 24-bit uniforms of the
 * first two words). |.| of the albedo and of the normal is the mean of the three channels'
 * absolute differences. The normal is the shading normal of interpolated vertex normals
 * (mirres_scene_set_normals), S / |S| with S = w0 VN_a + u VN_b + v VN_c; the texture-space
 * offset moves the point within the hit triangle by the barycentric offset J^-1 eps (J = the
 * triangle's texture-coordinate map [uv_b - uv_a | uv_c - uv_a]; the blend continued linearly
 * where the offset leaves the triangle; no normal term where J is singular). With face normals
 * the normal is constant on a triangle and the term is 0. Adds w_albedo L_albedo + w_roughness
 * L_roughness + w_normal L_normal to loss[0] and its gradient (sign(0) = 0) to grad_albedo
 * [tex_h][tex_w][3], grad_roughness [tex_h][tex_w] and grad_verts [n_verts][3] (the normal term,
 * with the hit point held fixed: through the vertex normals to the vertices of every face
 * around the hit triangle's vertices); all device, accumulated, any may be NULL. view->scene is
 * ignored. Uses the context workspace (24 B per pixel); asynchronous; FP32 sums in no fixed
 * order. MIRRES_ERR_ARG for NULL ctx/scene/view/params, sigma <= 0, a negative weight, a bad
 * view or view_index outside [0, 65535]; MIRRES_ERR_STATE before mirres_bvh_build. */
typedef struct {
    float sigma;                /* half-width of the texture-space offset, > 0 */
    float w_albedo, w_roughness; /* weights, >= 0 */
    uint32_t seed_lo, seed_hi;  /* Philox key */
    float w_normal;             /* weight of the normal term, >= 0 (interpolated normals only) */
} mirres_lk_params;
mirres_status mirres_material_smoothness(mirres_context* ctx, const mirres_scene* scene, const mirres_view* view,
                                         int32_t view_index, const mirres_lk_params* params, float* loss,
                                         float* grad_albedo, float* grad_roughness, float* grad_verts,
                                         void* stream);

/* Monochrome light regulariser (Appendix A, "Training details", after NVdiffrec-MC):
 *   L_light = | Y(c_d + c_s) - V(I_ref) |,  Y = (r + g + b) / 3,  V = max(r, g, b)
 * with c_d, c_s the demodulated diffuse and specular lighting. Readings: both are taken at each
 * pixel's primary vertex from the samples of the render that wrote `tape`: the primary
 * vertex's direct term V W L_env(y) Q(y) plus its continuation term Q(wc) L_ind / p_ind, with
 * the BRDF-times-cosine replaced by Q = (1 / pi + the GGX lobe) max(0, n.wi) -- the diffuse
 * lobe's reflectance (1 - metallic) albedo divided out, the specular lobe (whose Schlick F0
 * mixes albedo and metallic inside F, not as a factor) unchanged -- averaged over the pixel's
 * samples; an escaping primary ray contributes nothing. The loss is the mean over P, the pixels
 * of all the call's views with at least one sample on a surface, and the gradient takes
 * sign(0) = 0. Three calls:
 *
 * mirres_light_demod: demod[v] device [height][width][4] (16-byte aligned), overwritten with
 *   (c_d + c_s (3 channels), fraction of the pixel's samples whose primary ray hit). scenes,
 *   views, params and tape are those of the render (any launch; any grad_mode, whose tape
 *   size is checked); each pixel's samples summed in order (blocks take tiles of whole pixels and
 *   read the tape's sample-major words coalesced).
 * mirres_light_loss: loss[0] += weight L_light (device float, FP32 sums in no fixed order;
 *   may be NULL) and, if d_demod is not NULL, d_demod[v] device [height][width][3] overwritten
 *   with d(weight L_light) / d(c_d + c_s) = weight sign(Y - V) / (3 |P|) per channel (0 outside
 *   P). ref_images[v] device [height][width][3]; weight >= 0. |P| = 0 adds nothing.
 * mirres_light_backward: the PRIMARY-mode adjoint of c_d + c_s (RIS weight, visibility,
 *   directions, p_ind and L_ind held fixed, as in mirres_backward) for the upstream gradient
 *   d_demod[v] [height][width][3]: accumulated into the albedo (through F0 only), roughness,
 *   metallic and env texels and the primary triangle's vertices (and, with interpolated
 *   normals, the vertices around them), like mirres_backward; no env term for escaping rays.
 * All asynchronous on `stream` and use the context workspace. MIRRES_ERR_ARG for NULL or
 * misaligned buffers, a short tape or bad views; MIRRES_ERR_STATE for an unbuilt scene. */
mirres_status mirres_light_demod(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                                 const mirres_view* views, int32_t n_views, const mirres_params* params,
                                 const void* tape, size_t tape_bytes, float* const* demod, void* stream);
mirres_status mirres_light_loss(mirres_context* ctx, const mirres_view* views, int32_t n_views,
                                const float* const* demod, const float* const* ref_images, float weight,
                                float* loss, float* const* d_demod, void* stream);
mirres_status mirres_light_backward(mirres_context* ctx, mirres_scene* const* scenes, int32_t n_scenes,
                                    const mirres_view* views, int32_t n_views, const mirres_params* params,
                                    const float* const* d_demod, const void* tape, size_t tape_bytes,
                                    const mirres_grads* grads, void* stream);

/* Cumulative counters since the context was created or mirres_reset_counters (synchronises the
 * context's last stream): [0] primary rays, [1] continuation rays, [2] shadow rays, [3] samples
 * rendered, [4] samples differentiated, [5] RIS candidates, [6] kernel launches, [7] error
 * count: ray traversals that reached their iteration cap (params.max_visits) or overflowed their
 * stack and reported a miss. out[] is filled in either case; the call returns MIRRES_ERR_TIMEOUT
 * (with a message) while [7] is not zero, until mirres_reset_counters clears it. */
mirres_status mirres_get_counters(mirres_context* ctx, uint64_t out[8]);

/* Cumulative traversal work of the batched launches (launch 1) issued with params.flags bit 1
 * since the context was created
 * (synchronises like mirres_get_counters): [0] box tests and [1] triangle tests of closest-hit
 * rays, [2] box tests and [3] triangle tests of shadow rays. A box test is one slab test of a
 * child box (two per node visited), a triangle test one ray/triangle solve. Reset with
 * mirres_reset_counters. */
mirres_status mirres_get_work_counters(mirres_context* ctx, uint64_t out[4]);
mirres_status mirres_reset_counters(mirres_context* ctx);

/* Message of the last failed call on this thread ("" if none). */
const char* mirres_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MIRRES_H */
