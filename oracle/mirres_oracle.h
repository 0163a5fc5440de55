/*
 * MIRReS stage-2 oracle: plain, slow, FP64 CPU restatement of the forward and adjoint
 * multi-bounce path tracer with RIS/WRS environment-light sampling.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this library. The product path (the CUDA library) never calls it and shares
 * no code, header, table or constant generator with it.
 *
 * Everything here is restated from the paper's text:
 *   rendering equation and incident-light split ........ Eq. (pbr_render), Eq. (incident), Sec. 3.2
 *   direct light MC / RIS estimator ..................... Eq. (pbr_dir), Eq. (restir), Sec. 4.1
 *   weighted reservoir sampling (streaming RIS) ......... Appendix A, "Spatial-temporal Reuse"
 *   indirect light, MIS of light and GGX sampling ....... Eq. (pbr_indir), Eq. (mc_indir), Sec. 4.2
 *   recursive bounces, first three, detached gradients .. Eq. (sec_bouce), Sec. 4.2
 *   visibility by ray-mesh intersection, LBVH ........... Appendix A, "Visibility estimation"
 *   vertex offsets refined through the intersection ..... Sec. 3.2 "Mesh refinement", Eq. (loss_pbr)
 *   luminance operator Y = (r+g+b)/3 .................... Appendix A, "Training details"
 * Readings of passages the paper leaves open are listed in the repository's design notes.
 */
#ifndef MIRRES_ORACLE_H
#define MIRRES_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    const float* verts;    int32_t n_verts;   /* [V][3] */
    const int32_t* tris;   int32_t n_tris;    /* [F][3] */
    const float* tri_uv;                      /* [F][3][2] */
    const float* albedo; const float* roughness; const float* metallic;
    int32_t tex_w, tex_h;                     /* [h][w][3], [h][w], [h][w] */
    const float* env; int32_t env_w, env_h;   /* [h][w][3] lat-long, row 0 = zenith */
} orc_scene_desc;

typedef struct orc_scene orc_scene;

typedef struct {
    double K[4];        /* fx, fy, cx, cy */
    double c2w[12];     /* row-major [R | t], R columns = camera x (right), y (down), z (fwd) */
    int32_t width, height, spp, bounces;
    int32_t view_index; /* enters the random counter */
} orc_view;

typedef struct {
    int32_t ris_m;       /* RIS candidates per shading point */
    uint32_t seed_lo, seed_hi;
    int32_t brdf_kind;   /* 0 = GGX + Lambert (the method); 1 = Lambert only (furnace pin);
                          * 2 (orc_brdf_cos only) = the demodulated lobes of L_light */
    int32_t threads;     /* worker threads (>= 1) */
    int32_t want_margin; /* 1: track decision margins */
    int32_t grad_mode;   /* 0 = PRIMARY (the paper's); 1 = FULL (every vertex, at most ORC_MAXB) */
    int32_t reuse_k;      /* spatial reuse at the primary vertex: neighbouring reservoirs merged (0 = none) */
    int32_t reuse_radius; /* ... drawn from the (2 r + 1)^2 pixel square around the pixel */
    int32_t temporal;     /* 0 off; 1 write the reservoir history; 2 merge the history first, then write it */
    int32_t temporal_cap; /* the history counts at most temporal_cap * ris_m candidates */
    const double* history_in; /* [view samples][5]: texel (-1 miss, -2 none), sub word, w_sum, p_hat, m */
    double* history_out;      /* the same layout, written for every rendered sample (may alias nothing) */
} orc_params;

/* vertices per path recorded for the FULL-mode adjoint */
#define ORC_MAXB 16

/* per-pixel gradient destinations; any pointer may be NULL */
typedef struct {
    double* albedo; double* roughness; double* metallic; double* env; double* verts;
    /* absolute-value sums of the same scattered terms (a conditioning measure), may be NULL */
    double* albedo_abs; double* roughness_abs; double* metallic_abs; double* env_abs; double* verts_abs;
    /* FP32 sensitivity of the texel terms: sum over samples of |d(texel gradient)| when the
     * primary ray is perturbed by a few FP32 rounding units (bilinear weights move between
     * neighbouring texels); a bound on how far an FP32 evaluation may legitimately differ.
     * May be NULL. */
    double* albedo_sens; double* roughness_sens; double* metallic_sens;
    /* FP32 sensitivity of the vertex terms of the PRIMARY-mode adjoint: sum over samples and
     * over the adjoint's inputs (camera direction, barycentrics, light and continuation
     * directions, shading normal) of the largest change of the term when that input moves by
     * its FP32 rounding scale. May be NULL (then not computed: it costs ~28 re-evaluations of
     * the primary vertex's adjoint per sample). */
    double* verts_sens;
} orc_grads;

/* counters: [0] primary rays, [1] continuation rays, [2] shadow rays, [3] BVH nodes visited,
 * [4] triangle tests, [5] RIS candidates, [6] samples, [7] unused */
#define ORC_NCOUNT 8

orc_scene* orc_scene_new(const orc_scene_desc* d);
/* shading normals of the scene: 0 the face normal (default), 1 the barycentric blend of
 * area-weighted vertex normals, turned to the viewer's side of the face; light and
 * continuation directions below the face are then dropped */
void orc_scene_set_normals(orc_scene* s, int32_t mode);
/* the area-weighted vertex normals [V][3] (0 for a vertex without area) */
void orc_vertex_normals(const orc_scene* s, double* out);
void orc_scene_free(orc_scene* s);
double orc_scene_tmin(const orc_scene* s);

/* One sample's path record for word-by-word comparisons: out [18 + 12 ORC_MAXB] (layout in
 * mirres_oracle.c). Returns 0, or 1 for bad arguments. */
int orc_sample_record(const orc_scene* s, const orc_view* v, const orc_params* p, int32_t px, int32_t py,
                      int32_t smp, double* out);

/* Forward render of listed pixels (pixel = py*width + px; NULL = all pixels in order).
 * out_rgb [n][3]; out_margin [n][2] (min normalised decision margin over the pixel's samples
 * and the kind of that decision, may be NULL); out_prim_tri [n][spp] (primary hit triangle or -1, may be NULL). */
int orc_render(const orc_scene* s, const orc_view* v, const orc_params* p,
               const int32_t* pixels, int32_t n_pixels,
               double* out_rgb, double* out_margin, int32_t* out_prim_tri, int64_t* counts);

/* The same forward with each sample's own result: out_sample_rgb [n][spp][3] (the sample's
 * radiance, whose mean is the pixel's), out_sample_margin [n][spp] (the smallest normalised
 * decision margin of that sample, +inf when p->want_margin is 0; may be NULL) and
 * out_sample_sens [n][spp] (test tolerance only: the FP32 sensitivity of the radiance, the sum
 * over the path's vertices of each direct term's largest channel times its relative FP32
 * error -- the rounding of the RIS weights and of the throughput, whose glossy GGX lobes are
 * conditioned like 1 / alpha near the specular peak; may be NULL). */
int orc_render_samples(const orc_scene* s, const orc_view* v, const orc_params* p, const int32_t* pixels,
                       int32_t n_pixels, double* out_rgb, double* out_margin, double* out_sample_rgb,
                       double* out_sample_margin, double* out_sample_sens, int64_t* counts);

/* Adjoint. PRIMARY mode: gradients of the primary-vertex terms, indirect light, visibility,
 * the RIS weight and all sampling decisions detached. FULL mode: in addition the terms of
 * every later vertex (its direct light and the BRDF factor it puts on the light arriving from
 * the rest of the path), with the same quantities detached and the later hit points held
 * fixed on their triangles (no geometric derivative beyond the primary vertex); requires
 * bounces <= ORC_MAXB. d_rgb [n][3] = dL/dI at the listed pixels. Gradients are accumulated (+=). */
int orc_backward(const orc_scene* s, const orc_view* v, const orc_params* p,
                 const int32_t* pixels, int32_t n_pixels, const double* d_rgb,
                 const orc_grads* g, int64_t* counts);

/* Detached forward: the sample's radiance re-evaluated with the parameters of `eval`, every
 * detached quantity (sampling decisions, W, V, p_ind, hit triangles) taken from `frozen`.
 * PRIMARY mode: the primary-vertex terms with L_ind detached too. FULL mode: the whole path,
 * later hit points fixed on their triangles (geometry from `frozen`, materials and env from
 * `eval`). Its derivative w.r.t. `eval` at eval == frozen is what orc_backward returns. */
int orc_render_detached(const orc_scene* frozen, const orc_scene* eval, const orc_view* v,
                        const orc_params* p, const int32_t* pixels, int32_t n_pixels,
                        double* out_rgb);

/* Monochrome light regulariser (Appendix A, L_light), PRIMARY mode only (grad_mode 0).
 * orc_light_demod: per pixel, out[4] = the mean over its samples of the demodulated lighting
 * c_d + c_s at the primary vertex (the direct and continuation terms of the render's primary
 * vertex with the BRDF replaced by the kind-2 lobes: 1 / pi for the diffuse lobe, the GGX
 * lobe unchanged; RIS weight, visibility, directions, p_ind and L_ind as the render drew them;
 * 0 for an escaping primary ray), then the fraction of its samples whose primary ray hit.
 * out_margin as orc_render's. orc_light_backward: the adjoint of the per-pixel mean c for the
 * upstream gradient d_c [n][3] (the same scatters as orc_backward, no env term for escaping
 * rays). orc_light_demod_detached: c re-evaluated with the parameters of `eval`, everything
 * else from `frozen` ([n][3]); its derivative at eval == frozen is orc_light_backward's. */
int orc_light_demod(const orc_scene* s, const orc_view* v, const orc_params* p, const int32_t* pixels,
                    int32_t n_pixels, double* out, double* out_margin, int64_t* counts);
int orc_light_backward(const orc_scene* s, const orc_view* v, const orc_params* p, const int32_t* pixels,
                       int32_t n_pixels, const double* d_c, const orc_grads* g, int64_t* counts);
int orc_light_demod_detached(const orc_scene* frozen, const orc_scene* eval, const orc_view* v,
                             const orc_params* p, const int32_t* pixels, int32_t n_pixels, double* out);

/* Ray queries against the oracle's own BVH (mode 0 closest, 1 any) or brute force (2, 3).
 * rays [n][6] = origin, direction; skip_tri [n] (-1 none); out_tri [n]; out_tuv [n][3];
 * out_margin [n] (may be NULL). t in (t_min, inf). */
int orc_trace(const orc_scene* s, const double* rays, const int32_t* skip_tri, int32_t n, int32_t mode,
              int32_t* out_tri, double* out_tuv, double* out_margin);

/* LBVH (Karras 2012) restated top-down, FP32 Morton codes with a fixed operation order.
 * keys [F] sorted; left/right [F-1] child codes (>= 0 internal node, < 0 leaf ~pos);
 * parent [2F-1] (internal nodes first, then leaves); lo/hi [2F-1][3]. */
int orc_lbvh(const float* verts, const int32_t* tris, int32_t n_tris,
             uint64_t* keys, int32_t* left, int32_t* right, int32_t* parent, float* lo, float* hi);

/* Environment sampling tables: cond [h][w+1], marg [h+1], prob [h][w]; returns total weight. */
double orc_env_tables(const orc_scene* s, double* cond, double* marg, double* prob);
/* the CDF over all texels in row-major order that the draw inverts [h w + 1] */
void orc_env_flat(const orc_scene* s, double* flat);

/* ---- unit functions, exported for the pins ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t x);
/* f_r(wo, wi) * max(0, n.wi) per channel, GGX + Lambert */
void orc_brdf_cos(const double n[3], const double wo[3], const double wi[3], const double albedo[3],
                  double rough, double metal, int32_t kind, double out[3]);
/* gradient of sum_c g[c] * (f_r cos)[c] w.r.t. albedo[3], rough, metal, n[3] -> out[8] */
void orc_brdf_cos_grad(const double n[3], const double wo[3], const double wi[3], const double albedo[3],
                       double rough, double metal, int32_t kind, const double g[3], double out[8]);
double orc_ggx_d(double alpha, double cos_nh);
double orc_smith_g1(double alpha, double cos_nv);
void orc_vndf_sample(const double n[3], const double wo[3], double alpha, double u1, double u2, double out[3]);
double orc_vndf_pdf(const double n[3], const double wo[3], const double wi[3], double alpha);
/* continuation sampling: lobe choice + direction; returns pdf of the full mixture */
double orc_sample_continuation(const orc_scene* s, const double n[3], const double wo[3],
                               const double albedo[3], double rough, double metal, int32_t kind,
                               const uint32_t x[4], double out_dir[3]);
double orc_pdf_continuation(const orc_scene* s, const double n[3], const double wo[3],
                            const double albedo[3], double rough, double metal, int32_t kind,
                            const double wi[3]);
/* env sampling from four random words; returns direction pdf (solid angle), texel index */
double orc_env_sample(const orc_scene* s, const uint32_t x[4], double out_dir[3], int32_t* out_texel);
double orc_env_pdf(const orc_scene* s, const double dir[3]);
int32_t orc_env_texel(const orc_scene* s, const double dir[3]);
/* streaming WRS over m candidates with weights gamma and accept uniforms u:
 * returns selected index (-1 none), writes w_sum */
int32_t orc_wrs(const double* gamma, const double* u, int32_t m, double* w_sum);
/* the texels of a w x h texture whose bilinear weight a lookup at texture coordinate (su, sv)
 * computed with a fractional-position error up to (dfx, dfy) texels may change (test tolerance
 * only): writes up to 16 indices, returns their count */
int32_t orc_taps_reach(int32_t w, int32_t h, double su, double sv, double dfx, double dfy, int32_t* out);

#ifdef __cplusplus
}
#endif
#endif
