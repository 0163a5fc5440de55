/*
 * MIRReS stage-2 oracle -- TEST INFRASTRUCTURE ONLY (see mirres_oracle.h).
 *
 * A plain, slow FP64 restatement of the method, written for a reader checking it against the
 * paper by eye: one path sample at a time, no wavefronts, no blocking, no fused kernels.
 * Its own BVH is a top-down median split (not the LBVH the product builds), so the two share
 * no acceleration-structure code; the LBVH restatement at the end exists only so that the
 * product's build can be compared bit for bit.
 *
 * Compiled with -ffp-contract=off so that the FP32 Morton-code arithmetic has a fixed
 * operation order on every host.
 */
#define _GNU_SOURCE
#include "mirres_oracle.h"

#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

/* decision-margin scales: a decision whose normalised distance to its threshold is below 1
 * is one an FP32 evaluation of the same formulas may take the other way */
#define TAU_BARY 4e-6   /* barycentric distance to an edge, scaled by cos(angle) * size / (distance + size) */
#define TAU_TMIN 1e-3   /* relative distance of t to the self-intersection threshold */
#define TAU_TDEPTH 2e-6 /* relative depth difference between two hit triangles */
#define TAU_ACC 2e-5    /* WRS accept: |u w_sum - gamma| / w_sum */
#define TAU_CDF 1e-12   /* distance of a uniform to a CDF boundary */
#define TAU_LOBE 2e-6   /* distance of the lobe uniform to a material-dependent threshold */
#define TAU_FLIP 2e-5   /* |n . d| when the face normal is flipped towards the viewer */
#define TAU_ENV 3e-6    /* distance to a texel boundary of the env lookup, in u (or v) units */
#define TAU_FRAME 1e-5  /* |n.z| in the orthonormal-basis sign choice */
#define TAU_GRAZE 2e-3  /* cos of the viewing angle at the primary vertex: below it an FP32
                         * evaluation of the BRDF carries a relative error above ~3e-5 */
#define U32 (1.0 / 16777216.0) /* the FP32 unit roundoff scale 2^-24 (test tolerances) */
#define TAU_LEAK 1e-5   /* |dir . n_face| of a light or continuation direction when shading
                         * normals are interpolated (directions below the face are dropped) */

enum { MK_NONE = 0, MK_BARY, MK_TMIN, MK_TDEPTH, MK_ACC, MK_CDF, MK_LOBE, MK_FLIP, MK_ENV, MK_FRAME, MK_GRAZE,
       MK_LEAK };

/* ---------------------------------------------------------------------------------------
 * small vector algebra (FP64)
 * ------------------------------------------------------------------------------------- */
typedef struct { double x, y, z; } v3;
static v3 V3(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 vadd(v3 a, v3 b) { return V3(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 vsub(v3 a, v3 b) { return V3(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 vscale(v3 a, double s) { return V3(a.x * s, a.y * s, a.z * s); }
static double vdot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 vcross(v3 a, v3 b) { return V3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static double vlen(v3 a) { return sqrt(vdot(a, a)); }
static v3 vnorm(v3 a) { return vscale(a, 1.0 / vlen(a)); }
static v3 vload(const double* p) { return V3(p[0], p[1], p[2]); }
static void vstore(double* p, v3 a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }
static double lum(const double c[3]) { return (c[0] + c[1] + c[2]) / 3.0; } /* Y = (r+g+b)/3 */

/* ---------------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11): ten rounds of two 32x32->64 multiplies, key bumped by the Weyl constants.
 * ------------------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* top 24 bits -> exact uniform in [0, 1) */
double orc_uniform(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }
/* 16-bit sub-texel offsets, cell midpoints in (0, 1) */
static double sub_hi(uint32_t x) { return ((double)(x >> 16) + 0.5) / 65536.0; }
static double sub_lo(uint32_t x) { return ((double)(x & 0xFFFFu) + 0.5) / 65536.0; }

enum { PURPOSE_CAMERA = 0, PURPOSE_CANDIDATE = 1, PURPOSE_CONTINUE = 2, PURPOSE_REUSE = 3 };

/* ---------------------------------------------------------------------------------------
 * scene, env tables, median-split BVH
 * ------------------------------------------------------------------------------------- */
typedef struct { double lo[3], hi[3]; int32_t left, right, first, count; } Node;

struct orc_scene {
    int nv, nf;
    double* V; int32_t* F; double* UV;
    int tw, th; double* alb; double* rgh; double* met;
    int ew, eh; double* env;
    double* cond; double* marg; double* prob; double total; int env_ok;
    double* flat; /* [H W + 1] CDF over all texels in row-major order (the one the draw inverts) */
    double tmin, diag;
    int nnodes; Node* nodes; int32_t* order;
    /* shading normals: 0 face normal, 1 interpolated from area-weighted vertex normals */
    int normals;
    double* VA;  /* [V][3] sum of the incident faces' (b - a) x (c - a) */
    double* VN;  /* [V][3] VA normalised (0 for a vertex without area) */
    int32_t* vf_off; int32_t* vf;  /* incident faces of each vertex (CSR) */
};

static __thread const double* g_cent;
static __thread int g_axis;
static int cmp_cent(const void* a, const void* b)
{
    int32_t ia = *(const int32_t*)a, ib = *(const int32_t*)b;
    double ca = g_cent[3 * ia + g_axis], cb = g_cent[3 * ib + g_axis];
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return (ia > ib) - (ia < ib);
}

static void tri_verts(const orc_scene* s, int tri, v3* a, v3* b, v3* c)
{
    *a = vload(s->V + 3 * s->F[3 * tri + 0]);
    *b = vload(s->V + 3 * s->F[3 * tri + 1]);
    *c = vload(s->V + 3 * s->F[3 * tri + 2]);
}

static int bvh_build(orc_scene* s, const double* cent, int first, int count)
{
    int ni = s->nnodes++;
    Node nd;
    for (int k = 0; k < 3; ++k) { nd.lo[k] = INFINITY; nd.hi[k] = -INFINITY; }
    for (int i = first; i < first + count; ++i) {
        v3 p[3];
        tri_verts(s, s->order[i], &p[0], &p[1], &p[2]);
        for (int j = 0; j < 3; ++j) {
            const double q[3] = {p[j].x, p[j].y, p[j].z};
            for (int k = 0; k < 3; ++k) { nd.lo[k] = dmin(nd.lo[k], q[k]); nd.hi[k] = dmax(nd.hi[k], q[k]); }
        }
    }
    /* conservative inflation far above FP64 rounding */
    double pad = 1e-9 * (s->diag + 1e-30);
    for (int k = 0; k < 3; ++k) { nd.lo[k] -= pad; nd.hi[k] += pad; }
    nd.left = nd.right = -1; nd.first = first; nd.count = count;
    if (count <= 4) { s->nodes[ni] = nd; return ni; }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = first; i < first + count; ++i)
        for (int k = 0; k < 3; ++k) {
            clo[k] = dmin(clo[k], cent[3 * s->order[i] + k]);
            chi[k] = dmax(chi[k], cent[3 * s->order[i] + k]);
        }
    int axis = 0;
    for (int k = 1; k < 3; ++k) if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
    g_cent = cent; g_axis = axis;
    qsort(s->order + first, (size_t)count, sizeof(int32_t), cmp_cent);
    int half = count / 2;
    nd.count = 0;
    int l = bvh_build(s, cent, first, half);
    int r = bvh_build(s, cent, first + half, count - half);
    nd.left = l; nd.right = r;
    s->nodes[ni] = nd;
    return ni;
}

/* Environment sampling distribution, the proposal q_dir of Sec. 4.1 (proportional to L_env):
 * texel weight Y(L) * sin(theta_row); a marginal CDF over rows and a conditional CDF per row
 * (their factorisation, kept for the tables' pins), and the CDF over all texels that the draw
 * inverts, built in FP64 by sequential prefix sums. */
static void env_build(orc_scene* s)
{
    int W = s->ew, H = s->eh;
    double* w = (double*)malloc(sizeof(double) * (size_t)W * H);
    double* rowsum = (double*)malloc(sizeof(double) * (size_t)H);
    s->total = 0.0;
    for (int r = 0; r < H; ++r) {
        double st = sin(PI * (r + 0.5) / H);
        double acc = 0.0;
        for (int c = 0; c < W; ++c) {
            double y = lum(s->env + 3 * ((size_t)r * W + c)) * st;
            w[(size_t)r * W + c] = y;
            acc += y;
        }
        rowsum[r] = acc;
    }
    for (int r = 0; r < H; ++r) s->total += rowsum[r];
    s->env_ok = s->total > 0.0;
    for (int r = 0; r < H; ++r) {
        double* cr = s->cond + (size_t)r * (W + 1);
        double acc = 0.0;
        for (int c = 0; c <= W; ++c) {
            if (rowsum[r] > 0.0) cr[c] = (c == W) ? 1.0 : acc / rowsum[r];
            else cr[c] = (double)c / W;
            if (c < W) acc += w[(size_t)r * W + c];
        }
    }
    double acc = 0.0;
    for (int r = 0; r <= H; ++r) {
        if (s->env_ok) s->marg[r] = (r == H) ? 1.0 : acc / s->total;
        else s->marg[r] = (double)r / H;
        if (r < H) acc += rowsum[r];
    }
    for (size_t i = 0; i < (size_t)W * H; ++i) s->prob[i] = s->env_ok ? w[i] / s->total : 0.0;
    /* the same distribution over all texels in row-major order: entry r W + c is
     * (rows before r + texels before c in row r) / total, each sum taken in order */
    {
        double base = 0.0;
        const size_t N = (size_t)W * H;
        for (int r = 0; r < H; ++r) {
            double within = 0.0;
            for (int c = 0; c < W; ++c) {
                const size_t i = (size_t)r * W + c;
                s->flat[i] = s->env_ok ? (base + within) / s->total : (double)i / (double)N;
                within += w[i];
            }
            base += rowsum[r];
        }
        s->flat[N] = 1.0;
    }
    free(w);
    free(rowsum);
}

static double* to_double(const float* p, size_t n)
{
    double* d = (double*)malloc(sizeof(double) * (n ? n : 1));
    for (size_t i = 0; i < n; ++i) d[i] = (double)p[i];
    return d;
}

orc_scene* orc_scene_new(const orc_scene_desc* d)
{
    if (!d || d->n_tris < 0 || d->n_verts < 0 || d->tex_w < 1 || d->tex_h < 1 || d->env_w < 1 || d->env_h < 1)
        return NULL;
    orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
    s->nv = d->n_verts; s->nf = d->n_tris;
    s->V = to_double(d->verts, (size_t)3 * s->nv);
    s->F = (int32_t*)malloc(sizeof(int32_t) * (size_t)3 * (s->nf ? s->nf : 1));
    if (s->nf) memcpy(s->F, d->tris, sizeof(int32_t) * (size_t)3 * s->nf);
    s->UV = to_double(d->tri_uv, (size_t)6 * s->nf);
    s->tw = d->tex_w; s->th = d->tex_h;
    size_t tn = (size_t)s->tw * s->th;
    s->alb = to_double(d->albedo, 3 * tn);
    s->rgh = to_double(d->roughness, tn);
    s->met = to_double(d->metallic, tn);
    s->ew = d->env_w; s->eh = d->env_h;
    s->env = to_double(d->env, (size_t)3 * s->ew * s->eh);
    s->cond = (double*)malloc(sizeof(double) * (size_t)s->eh * (s->ew + 1));
    s->marg = (double*)malloc(sizeof(double) * (size_t)(s->eh + 1));
    s->prob = (double*)malloc(sizeof(double) * (size_t)s->eh * s->ew);
    s->flat = (double*)malloc(sizeof(double) * ((size_t)s->eh * s->ew + 1));
    env_build(s);
    /* scene extent: AABB of all vertices referenced by triangles */
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < 3 * s->nf; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = dmin(lo[k], s->V[3 * s->F[i] + k]);
            hi[k] = dmax(hi[k], s->V[3 * s->F[i] + k]);
        }
    s->diag = s->nf ? sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                           (hi[2] - lo[2]) * (hi[2] - lo[2])) : 0.0;
    s->tmin = 1e-5 * s->diag; /* self-intersection threshold: 1e-5 of the scene diagonal */
    /* area-weighted vertex normals and the faces around every vertex (interpolated normals) */
    s->VA = (double*)calloc((size_t)3 * (s->nv ? s->nv : 1), sizeof(double));
    s->VN = (double*)calloc((size_t)3 * (s->nv ? s->nv : 1), sizeof(double));
    s->vf_off = (int32_t*)calloc((size_t)s->nv + 1, sizeof(int32_t));
    s->vf = (int32_t*)malloc(sizeof(int32_t) * (size_t)3 * (s->nf ? s->nf : 1));
    for (int t = 0; t < s->nf; ++t) {
        v3 a, b, c;
        tri_verts(s, t, &a, &b, &c);
        v3 N = vcross(vsub(b, a), vsub(c, a));
        for (int k = 0; k < 3; ++k) {
            int vi = s->F[3 * t + k];
            vstore(s->VA + 3 * vi, vadd(vload(s->VA + 3 * vi), N));
            s->vf_off[vi + 1]++;
        }
    }
    for (int i = 0; i < s->nv; ++i) {
        s->vf_off[i + 1] += s->vf_off[i];
        double l = vlen(vload(s->VA + 3 * i));
        if (l > 0.0) vstore(s->VN + 3 * i, vscale(vload(s->VA + 3 * i), 1.0 / l));
    }
    {
        int32_t* cur = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->nv > 0 ? s->nv : 1));
        for (int i = 0; i < s->nv; ++i) cur[i] = s->vf_off[i];
        for (int t = 0; t < s->nf; ++t)
            for (int k = 0; k < 3; ++k) s->vf[cur[s->F[3 * t + k]]++] = t;
        free(cur);
    }
    /* median-split BVH */
    s->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->nf ? s->nf : 1));
    s->nodes = (Node*)malloc(sizeof(Node) * (size_t)(2 * s->nf + 1));
    s->nnodes = 0;
    if (s->nf) {
        double* cent = (double*)malloc(sizeof(double) * (size_t)3 * s->nf);
        for (int t = 0; t < s->nf; ++t) {
            v3 a, b, c;
            tri_verts(s, t, &a, &b, &c);
            v3 m = vscale(vadd(vadd(a, b), c), 1.0 / 3.0);
            vstore(cent + 3 * t, m);
            s->order[t] = t;
        }
        bvh_build(s, cent, 0, s->nf);
        free(cent);
    }
    return s;
}

void orc_scene_free(orc_scene* s)
{
    if (!s) return;
    free(s->V); free(s->F); free(s->UV); free(s->alb); free(s->rgh); free(s->met); free(s->env);
    free(s->cond); free(s->marg); free(s->prob); free(s->flat); free(s->nodes); free(s->order);
    free(s->VA); free(s->VN); free(s->vf_off); free(s->vf);
    free(s);
}

void orc_scene_set_normals(orc_scene* s, int32_t mode) { s->normals = mode ? 1 : 0; }

void orc_vertex_normals(const orc_scene* s, double* out)
{
    memcpy(out, s->VN, sizeof(double) * (size_t)3 * s->nv);
}

double orc_scene_tmin(const orc_scene* s) { return s->tmin; }

void orc_env_flat(const orc_scene* s, double* flat)
{
    memcpy(flat, s->flat, sizeof(double) * ((size_t)s->eh * s->ew + 1));
}

double orc_env_tables(const orc_scene* s, double* cond, double* marg, double* prob)
{
    if (cond) memcpy(cond, s->cond, sizeof(double) * (size_t)s->eh * (s->ew + 1));
    if (marg) memcpy(marg, s->marg, sizeof(double) * (size_t)(s->eh + 1));
    if (prob) memcpy(prob, s->prob, sizeof(double) * (size_t)s->eh * s->ew);
    return s->total;
}

/* ---------------------------------------------------------------------------------------
 * decision margins
 * ------------------------------------------------------------------------------------- */
typedef struct { double m; int kind; } Margin;
static void note(Margin* mg, double ratio, int kind)
{
    if (mg && ratio < mg->m) { mg->m = ratio; mg->kind = kind; }
}

/* ---------------------------------------------------------------------------------------
 * ray-mesh intersection (Appendix A "Visibility estimation"): Moller-Trumbore in FP64
 * ------------------------------------------------------------------------------------- */
typedef struct { int tri; double t, u, v; } Hit;

/* plane intersection of the ray with triangle `tri`; returns 0 if the ray is parallel */
static int tri_solve(const orc_scene* s, int tri, v3 o, v3 d, double* t, double* u, double* v, double* mscale)
{
    v3 a, b, c;
    tri_verts(s, tri, &a, &b, &c);
    v3 e1 = vsub(b, a), e2 = vsub(c, a);
    v3 p = vcross(d, e2);
    double det = vdot(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    v3 sv = vsub(o, a);
    *u = vdot(sv, p) * inv;
    v3 q = vcross(sv, e1);
    *v = vdot(d, q) * inv;
    *t = vdot(e2, q) * inv;
    if (mscale) {
        double area2 = vlen(vcross(e1, e2));
        double ell = sqrt(area2);
        double cosang = fabs(det) / (vlen(d) * area2);
        *mscale = cosang * ell / (vlen(sv) + ell);
    }
    return 1;
}

static int inside(double u, double v) { return u >= 0.0 && v >= 0.0 && u + v <= 1.0; }

/* the distance and size terms of tri_solve's margin scale */
static double tri_dist(const orc_scene* s, int tri, v3 o)
{
    v3 a, b, c;
    tri_verts(s, tri, &a, &b, &c);
    return vlen(vsub(o, a));
}
static double tri_size(const orc_scene* s, int tri)
{
    v3 a, b, c;
    tri_verts(s, tri, &a, &b, &c);
    return sqrt(vlen(vcross(vsub(b, a), vsub(c, a))));
}

static int slab(const Node* n, v3 o, v3 d, double tmin, double tmax)
{
    const double oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
    double t0 = tmin, t1 = tmax;
    for (int k = 0; k < 3; ++k) {
        if (dd[k] == 0.0) {
            if (oo[k] < n->lo[k] || oo[k] > n->hi[k]) return 0;
            continue;
        }
        double a = (n->lo[k] - oo[k]) / dd[k], b = (n->hi[k] - oo[k]) / dd[k];
        if (a > b) { double tt = a; a = b; b = tt; }
        t0 = dmax(t0, a);
        t1 = dmin(t1, b);
        if (t0 > t1) return 0;
    }
    return 1;
}

/* closest hit: smallest t in (tmin, inf); equal t -> smaller triangle id */
static void bvh_closest(const orc_scene* s, v3 o, v3 d, int skip, Hit* best, int64_t* cnt)
{
    best->tri = -1; best->t = INFINITY; best->u = best->v = 0.0;
    if (!s->nf) return;
    int stack[256], sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const Node* n = &s->nodes[stack[--sp]];
        if (cnt) cnt[3]++;
        if (!slab(n, o, d, 0.5 * s->tmin, best->t * (1.0 + 1e-9) + 1e-300)) continue;
        if (n->count) {
            for (int i = n->first; i < n->first + n->count; ++i) {
                int tri = s->order[i];
                if (tri == skip) continue;
                if (cnt) cnt[4]++;
                double t, u, v;
                if (!tri_solve(s, tri, o, d, &t, &u, &v, NULL)) continue;
                if (!inside(u, v) || !(t > s->tmin)) continue;
                if (t < best->t || (t == best->t && tri < best->tri)) {
                    best->tri = tri; best->t = t; best->u = u; best->v = v;
                }
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
}

/* The margin scale of a hit decision (tri_solve's ms) is cos * size / (distance + size): an FP32
 * ray moves its hit point by a few ulps of the distance. A ray that starts at an earlier hit
 * (continuation and shadow rays) carries the rounding of every segment before it as well:
 * `lever` = the path length up to the ray's origin (0 for camera rays) joins the distance. */
static double lever_scale(double ms, double dist, double size, double lever)
{
    return lever > 0.0 ? ms * (dist + size) / (dist + size + lever) : ms;
}

/* margins of a closest-hit decision: every triangle that could be the first hit */
static void closest_margins_l(const orc_scene* s, v3 o, v3 d, int skip, const Hit* best, Margin* mg, double lever)
{
    if (!mg || !s->nf) return;
    double tcut = (best->tri >= 0) ? best->t * (1.0 + 1e-6) : INFINITY;
    int stack[256], sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const Node* n = &s->nodes[stack[--sp]];
        if (!slab(n, o, d, 0.25 * s->tmin, tcut * (1.0 + 1e-9) + 1e-300)) continue;
        if (n->count) {
            for (int i = n->first; i < n->first + n->count; ++i) {
                int tri = s->order[i];
                if (tri == skip) continue;
                double t, u, v, ms;
                if (!tri_solve(s, tri, o, d, &t, &u, &v, &ms)) continue;
                if (lever > 0.0) ms = lever_scale(ms, tri_dist(s, tri, o), tri_size(s, tri), lever);
                double e = dmin(dmin(u, v), 1.0 - u - v);
                if (t > 0.5 * s->tmin && t < tcut) note(mg, fabs(e) * ms / TAU_BARY, MK_BARY);
                if (e >= 0.0 && t > 0.25 * s->tmin && t < 4.0 * s->tmin)
                    note(mg, fabs(t - s->tmin) / (s->tmin * TAU_TMIN), MK_TMIN);
                if (best->tri >= 0 && tri != best->tri && e >= 0.0 && t > s->tmin && t < tcut)
                    note(mg, fabs(t - best->t) / (dmax(t, best->t) * TAU_TDEPTH), MK_TDEPTH);
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
}

static void closest_margins(const orc_scene* s, v3 o, v3 d, int skip, const Hit* best, Margin* mg)
{
    closest_margins_l(s, o, d, skip, best, mg, 0.0);
}

/* any hit in (tmin, inf): visibility V of Eq. (incident); `lever` as for closest_margins_l */
static int bvh_any_l(const orc_scene* s, v3 o, v3 d, int skip, int64_t* cnt, Margin* mg, double lever)
{
    if (!s->nf) return 0;
    int stack[256], sp = 0;
    stack[sp++] = 0;
    int hit = 0;
    double best_in = -1.0, best_out = INFINITY; /* robustness of a hit / closeness of a miss */
    while (sp) {
        const Node* n = &s->nodes[stack[--sp]];
        if (cnt) cnt[3]++;
        if (!slab(n, o, d, 0.5 * s->tmin, INFINITY)) continue;
        if (n->count) {
            for (int i = n->first; i < n->first + n->count; ++i) {
                int tri = s->order[i];
                if (tri == skip) continue;
                if (cnt) cnt[4]++;
                double t, u, v, ms;
                if (!tri_solve(s, tri, o, d, &t, &u, &v, &ms)) continue;
                int h = inside(u, v) && t > s->tmin;
                if (mg && t > 0.5 * s->tmin) {
                    if (lever > 0.0) ms = lever_scale(ms, tri_dist(s, tri, o), tri_size(s, tri), lever);
                    double e = dmin(dmin(u, v), 1.0 - u - v);
                    double r = fabs(e) * ms / TAU_BARY;
                    if (e >= 0.0 && t > 0.25 * s->tmin && t < 4.0 * s->tmin)
                        r = dmin(r, fabs(t - s->tmin) / (s->tmin * TAU_TMIN));
                    if (h) best_in = dmax(best_in, r); else best_out = dmin(best_out, r);
                }
                if (h) {
                    hit = 1;
                    if (!mg) return 1;
                }
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
    if (mg) {
        if (hit) note(mg, best_in, MK_BARY);
        else note(mg, best_out, MK_BARY);
    }
    return hit;
}

static int bvh_any(const orc_scene* s, v3 o, v3 d, int skip, int64_t* cnt, Margin* mg)
{
    return bvh_any_l(s, o, d, skip, cnt, mg, 0.0);
}

static void brute_closest(const orc_scene* s, v3 o, v3 d, int skip, Hit* best)
{
    best->tri = -1; best->t = INFINITY; best->u = best->v = 0.0;
    for (int tri = 0; tri < s->nf; ++tri) {
        if (tri == skip) continue;
        double t, u, v;
        if (!tri_solve(s, tri, o, d, &t, &u, &v, NULL)) continue;
        if (!inside(u, v) || !(t > s->tmin)) continue;
        if (t < best->t || (t == best->t && tri < best->tri)) { best->tri = tri; best->t = t; best->u = u; best->v = v; }
    }
}

int orc_trace(const orc_scene* s, const double* rays, const int32_t* skip_tri, int32_t n, int32_t mode,
              int32_t* out_tri, double* out_tuv, double* out_margin)
{
    for (int i = 0; i < n; ++i) {
        v3 o = vload(rays + 6 * i), d = vload(rays + 6 * i + 3);
        int skip = skip_tri ? skip_tri[i] : -1;
        Margin mg = {INFINITY, 0};
        Hit h;
        if (mode == 0 || mode == 2) {
            if (mode == 0) bvh_closest(s, o, d, skip, &h, NULL);
            else brute_closest(s, o, d, skip, &h);
            if (out_margin) closest_margins(s, o, d, skip, &h, &mg);
            out_tri[i] = h.tri;
            if (out_tuv) { out_tuv[3 * i] = h.t; out_tuv[3 * i + 1] = h.u; out_tuv[3 * i + 2] = h.v; }
        } else {
            int hit = 0;
            if (mode == 1) hit = bvh_any(s, o, d, skip, NULL, out_margin ? &mg : NULL);
            else {
                for (int tri = 0; tri < s->nf && !hit; ++tri) {
                    double t, u, v;
                    if (tri == skip || !tri_solve(s, tri, o, d, &t, &u, &v, NULL)) continue;
                    hit = inside(u, v) && t > s->tmin;
                }
            }
            out_tri[i] = hit ? 1 : -1;
        }
        if (out_margin) out_margin[i] = mg.m;
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * environment map: lat-long lookup and importance sampling (Sec. 3.2 env map; Sec. 4.1 q_dir)
 * direction (theta, phi): d = (sin t sin p, cos t, -sin t cos p); u = phi/2pi + 1/2, v = theta/pi
 * ------------------------------------------------------------------------------------- */
static int env_texel_m(const orc_scene* s, v3 d, Margin* mg)
{
    double u = atan2(d.x, -d.z) / (2.0 * PI) + 0.5;
    double v = acos(dmax(-1.0, dmin(1.0, d.y))) / PI;
    double fx = u * s->ew, fy = v * s->eh;
    int c = (int)floor(fx), r = (int)floor(fy);
    if (c > s->ew - 1) c = s->ew - 1;
    if (c < 0) c = 0;
    if (r > s->eh - 1) r = s->eh - 1;
    if (r < 0) r = 0;
    if (mg) {
        double dx = fabs(fx - floor(fx + 0.5));
        double dy = (fy > 0.5 && fy < s->eh - 0.5) ? fabs(fy - floor(fy + 0.5)) : INFINITY;
        if (s->ew > 1) note(mg, dx / (TAU_ENV * s->ew), MK_ENV);
        if (s->eh > 1) note(mg, dy / (TAU_ENV * s->eh), MK_ENV);
    }
    return r * s->ew + c;
}

int32_t orc_env_texel(const orc_scene* s, const double dir[3]) { return env_texel_m(s, vload(dir), NULL); }

/* solid-angle density of the env proposal at direction d */
static double env_pdf_m(const orc_scene* s, v3 d, Margin* mg)
{
    if (!s->env_ok) return 0.0;
    int tex = env_texel_m(s, d, mg);
    double st = sqrt(dmax(0.0, 1.0 - d.y * d.y));
    if (st <= 0.0) return 0.0;
    return s->prob[tex] * s->ew * s->eh / (2.0 * PI * PI * st);
}

double orc_env_pdf(const orc_scene* s, const double dir[3]) { return env_pdf_m(s, vload(dir), NULL); }

/* largest index i in [0, n-1] with cdf[i] <= u */
static int cdf_search(const double* cdf, int n, double u)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (cdf[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* 53-bit uniform from two random words: the high 32 bits from a, the low 21 from the top of b */
static double u53(uint32_t a, uint32_t b)
{
    return (double)(((uint64_t)a << 21) | (uint64_t)(b >> 11)) * (1.0 / 9007199254740992.0);
}

/* inverse-CDF sample over all texels (row-major CDF, a 53-bit uniform from two words), a
 * uniform position inside the texel from a 16+16-bit word; returns the solid-angle pdf */
static double env_sample_m(const orc_scene* s, uint32_t xa, uint32_t xb, uint32_t sub, v3* dir, int* texel, Margin* mg)
{
    int W = s->ew, H = s->eh;
    const double u = u53(xa, xb);
    int t = cdf_search(s->flat, W * H, u);
    if (mg) note(mg, dmin(u - s->flat[t], s->flat[t + 1] - u) / TAU_CDF, MK_CDF);
    int r = t / W, c = t % W;
    double uu = (c + sub_hi(sub)) / W, vv = (r + sub_lo(sub)) / H;
    double phi = 2.0 * PI * (uu - 0.5), theta = PI * vv;
    double st = sin(theta);
    *dir = V3(st * sin(phi), cos(theta), -st * cos(phi));
    *texel = r * W + c;
    return s->prob[r * W + c] * W * H / (2.0 * PI * PI * st);
}

double orc_env_sample(const orc_scene* s, const uint32_t x[4], double out_dir[3], int32_t* out_texel)
{
    v3 d;
    int t;
    double p = env_sample_m(s, x[0], x[1], x[3], &d, &t, NULL);
    vstore(out_dir, d);
    *out_texel = t;
    return p;
}

/* ---------------------------------------------------------------------------------------
 * BRDF (Sec. 3.2 "Intrinsic decomposition": Disney-style albedo + roughness, metallic added
 * for OWL, Sec. 5.3): Lambert (1-m) a / pi + GGX D * Smith height-correlated G2 * Schlick F
 * / (4 cos_i cos_o), F0 = 0.04 (1-m) + m a, alpha = max(r^2, 1e-3)
 * ------------------------------------------------------------------------------------- */
static double alpha_of(double r) { return dmax(r * r, 1e-3); }

double orc_ggx_d(double a, double cnh)
{
    double a2 = a * a;
    double k = cnh * cnh * (a2 - 1.0) + 1.0;
    return a2 / (PI * k * k);
}

/* A(c) = sqrt(a^2 + (1 - a^2) c^2) = c * sqrt(1 + a^2 tan^2) */
static double smith_a(double a, double c) { return sqrt(a * a + (1.0 - a * a) * c * c); }

double orc_smith_g1(double a, double c) { return 2.0 * c / (c + smith_a(a, c)); }

/* f_r * max(0, n.wi): returns 0 outside the upper hemispheres. kind 0 = the method's GGX +
 * Lambert; 1 = Lambert only (furnace pin); 2 = the demodulated lobes of the monochrome light
 * regulariser (Appendix A, L_light): the diffuse lobe with its reflectance (1 - m) albedo
 * divided out, i.e. 1 / pi, plus the specular lobe unchanged (Schlick's F0 mixes albedo and
 * metallic inside F, which is not a factor that could be divided out) */
static void brdf_cos(v3 n, v3 wo, v3 wi, const double alb[3], double r, double m, int kind, double out[3])
{
    double co = vdot(n, wo), ci = vdot(n, wi);
    out[0] = out[1] = out[2] = 0.0;
    if (co <= 0.0 || ci <= 0.0) return;
    if (kind == 1) {
        for (int k = 0; k < 3; ++k) out[k] = alb[k] / PI * ci;
        return;
    }
    double a = alpha_of(r);
    v3 h = vnorm(vadd(wo, wi));
    double cnh = vdot(n, h), coh = vdot(wo, h);
    double D = orc_ggx_d(a, cnh);
    double vis = 0.5 / (ci * smith_a(a, co) + co * smith_a(a, ci)); /* G2 / (4 ci co) */
    double w5 = pow(1.0 - coh, 5.0);
    for (int k = 0; k < 3; ++k) {
        double kd = kind == 2 ? 1.0 : (1.0 - m) * alb[k];
        double f0 = 0.04 * (1.0 - m) + m * alb[k];
        double F = f0 + (1.0 - f0) * w5;
        out[k] = (kd / PI + D * vis * F) * ci;
    }
}

/* FP32 conditioning of the GGX lobe (test tolerances only). A direction rounded to single
 * precision is off by ~DTH radians; D moves by |d ln D / d theta_h| DTH of itself, with
 * |d ln D / d theta_h| = 4 (1 - a^2) cos sin / (cos^2 (a^2 - 1) + 1) for the half vector at
 * angle theta_h from the normal: up to ~2 / alpha near the specular peak. */
#define DTH 3e-7
static double ggx_slope(v3 n, v3 wo, v3 wi, double a)
{
    v3 hs = vadd(wo, wi);
    double l = vlen(hs);
    if (!(l > 0.0)) return 0.0;
    double c = vdot(n, vscale(hs, 1.0 / l));
    if (!(c > 0.0)) return 0.0;
    double sn = sqrt(dmax(0.0, 1.0 - c * c)), a2 = a * a;
    return 4.0 * (1.0 - a2) * c * sn / (c * c * (a2 - 1.0) + 1.0);
}

/* the specular lobe's share of Y(f_r cos) (0 for the Lambert-only kind) */
static double spec_share(v3 n, v3 wo, v3 wi, const double alb[3], double r, double m, int kind)
{
    if (kind == 1) return 0.0;
    double tot[3], dem[3] = {0, 0, 0};
    brdf_cos(n, wo, wi, alb, r, m, kind, tot);
    double yt = lum(tot);
    if (!(yt > 0.0)) return 0.0;
    double ci = vdot(n, wi);
    for (int k = 0; k < 3; ++k) dem[k] = (kind == 2 ? 1.0 : (1.0 - m) * alb[k]) / PI * ci;
    double ys = yt - lum(dem);
    return dmin(1.0, dmax(0.0, ys / yt));
}

void orc_brdf_cos(const double n[3], const double wo[3], const double wi[3], const double albedo[3],
                  double rough, double metal, int32_t kind, double out[3])
{
    brdf_cos(vload(n), vload(wo), vload(wi), albedo, rough, metal, kind, out);
}

/* Analytic gradient of sum_k g_k * (f_r cos)_k with respect to (albedo[3], r, m, n[3]),
 * n treated as a free 3-vector (h depends only on wo, wi). Written out term by term. */
static void brdf_cos_grad(v3 n, v3 wo, v3 wi, const double alb[3], double r, double m, int kind,
                          const double g[3], double out[8])
{
    for (int k = 0; k < 8; ++k) out[k] = 0.0;
    double co = vdot(n, wo), ci = vdot(n, wi);
    if (co <= 0.0 || ci <= 0.0) return;
    if (kind == 1) {
        double dci = 0.0;
        for (int k = 0; k < 3; ++k) { out[k] = g[k] * ci / PI; dci += g[k] * alb[k] / PI; }
        out[5] = dci * wi.x; out[6] = dci * wi.y; out[7] = dci * wi.z;
        return;
    }
    double a = alpha_of(r);
    double dadr = (r * r > 1e-3) ? 2.0 * r : 0.0;
    v3 h = vnorm(vadd(wo, wi));
    double cnh = vdot(n, h), coh = vdot(wo, h);
    double a2 = a * a;
    double kk = cnh * cnh * (a2 - 1.0) + 1.0;
    double D = a2 / (PI * kk * kk);
    double dD_da = 2.0 * a / (PI * kk * kk) - 4.0 * a * a2 * cnh * cnh / (PI * kk * kk * kk);
    double dD_dcnh = -4.0 * a2 * cnh * (a2 - 1.0) / (PI * kk * kk * kk);
    double Ao = smith_a(a, co), Ai = smith_a(a, ci);
    double den = ci * Ao + co * Ai;
    double vis = 0.5 / den;
    double dvis_dden = -0.5 / (den * den);
    double dden_dci = Ao + co * (1.0 - a2) * ci / Ai;
    double dden_dco = Ai + ci * (1.0 - a2) * co / Ao;
    double dden_da = ci * a * (1.0 - co * co) / Ao + co * a * (1.0 - ci * ci) / Ai;
    double w5 = pow(1.0 - coh, 5.0);
    /* value Q_k = (kd_k/pi + D vis F_k) ci */
    double sum_gF = 0.0, sum_gdiff = 0.0;
    double dm = 0.0;
    /* kd_k = (1 - m) alb_k (kind 0) or 1 (kind 2, demodulated): d kd / d alb, d kd / d m */
    const double dkd_da = kind == 2 ? 0.0 : 1.0 - m;
    for (int k = 0; k < 3; ++k) {
        double kd = kind == 2 ? 1.0 : (1.0 - m) * alb[k];
        double dkd_dm = kind == 2 ? 0.0 : -alb[k];
        double f0 = 0.04 * (1.0 - m) + m * alb[k];
        double F = f0 + (1.0 - f0) * w5;
        /* dQ/dalb_k = (dkd/dalb / pi + D vis m (1 - w5)) ci */
        out[k] = g[k] * (dkd_da / PI + D * vis * m * (1.0 - w5)) * ci;
        /* dQ/dm = (dkd/dm / pi + D vis (alb - 0.04)(1 - w5)) ci */
        dm += g[k] * (dkd_dm / PI + D * vis * (alb[k] - 0.04) * (1.0 - w5)) * ci;
        sum_gF += g[k] * F;
        sum_gdiff += g[k] * kd / PI;
    }
    out[4] = dm;
    /* specular part S = D vis * sum_gF * ci ; diffuse part = sum_gdiff * ci */
    double dS_da = (dD_da * vis + D * dvis_dden * dden_da) * sum_gF * ci;
    out[3] = dS_da * dadr;
    /* n enters through ci (also the trailing cos), co, cnh */
    double dS_dci = D * dvis_dden * dden_dci * sum_gF * ci + D * vis * sum_gF;
    double dS_dco = D * dvis_dden * dden_dco * sum_gF * ci;
    double dS_dcnh = dD_dcnh * vis * sum_gF * ci;
    double d_ci = dS_dci + sum_gdiff;
    out[5] = d_ci * wi.x + dS_dco * wo.x + dS_dcnh * h.x;
    out[6] = d_ci * wi.y + dS_dco * wo.y + dS_dcnh * h.y;
    out[7] = d_ci * wi.z + dS_dco * wo.z + dS_dcnh * h.z;
}

void orc_brdf_cos_grad(const double n[3], const double wo[3], const double wi[3], const double albedo[3],
                       double rough, double metal, int32_t kind, const double g[3], double out[8])
{
    brdf_cos_grad(vload(n), vload(wo), vload(wi), albedo, rough, metal, kind, g, out);
}

/* ---------------------------------------------------------------------------------------
 * continuation sampling (Sec. 4.2): one-sample MIS mixture of env (light) importance
 * sampling, GGX visible-normal sampling (Heitz 2018) and cosine sampling of the diffuse lobe
 * ------------------------------------------------------------------------------------- */
/* orthonormal basis around n (Duff, Burgess, Christensen, Hery, Kensler, Liani, Villemin 2017);
 * the branch is taken on n.z >= 0 so that +0 and -0 choose the same basis */
static void onb(v3 n, v3* t, v3* b, Margin* mg)
{
    double sg = (n.z >= 0.0) ? 1.0 : -1.0;
    double a = -1.0 / (sg + n.z);
    double bb = n.x * n.y * a;
    *t = V3(1.0 + sg * n.x * n.x * a, sg * bb, -sg * n.x);
    *b = V3(bb, sg + n.y * n.y * a, -n.y);
    if (n.z != 0.0) note(mg, fabs(n.z) / TAU_FRAME, MK_FRAME);
}

/* Heitz 2018, "Sampling the GGX distribution of visible normals": stretch the view vector,
 * sample a point on the projected hemisphere (disk warped towards the visible half), unstretch */
static v3 vndf_local(v3 ve, double a, double u1, double u2)
{
    v3 vh = vnorm(V3(a * ve.x, a * ve.y, ve.z));
    double lensq = vh.x * vh.x + vh.y * vh.y;
    v3 t1 = lensq > 0.0 ? vscale(V3(-vh.y, vh.x, 0.0), 1.0 / sqrt(lensq)) : V3(1.0, 0.0, 0.0);
    v3 t2 = vcross(vh, t1);
    double rr = sqrt(u1), ph = 2.0 * PI * u2;
    double p1 = rr * cos(ph), p2 = rr * sin(ph);
    double sblend = 0.5 * (1.0 + vh.z);
    p2 = (1.0 - sblend) * sqrt(dmax(0.0, 1.0 - p1 * p1)) + sblend * p2;
    v3 nh = vadd(vadd(vscale(t1, p1), vscale(t2, p2)), vscale(vh, sqrt(dmax(0.0, 1.0 - p1 * p1 - p2 * p2))));
    return vnorm(V3(a * nh.x, a * nh.y, dmax(0.0, nh.z)));
}

static v3 vndf_sample_m(v3 n, v3 wo, double a, double u1, double u2, Margin* mg)
{
    v3 t, b;
    onb(n, &t, &b, mg);
    v3 ve = V3(vdot(wo, t), vdot(wo, b), vdot(wo, n));
    v3 m = vndf_local(ve, a, u1, u2);
    v3 wl = vsub(vscale(m, 2.0 * vdot(ve, m)), ve); /* reflect ve about m */
    return vadd(vadd(vscale(t, wl.x), vscale(b, wl.y)), vscale(n, wl.z));
}

void orc_vndf_sample(const double n[3], const double wo[3], double alpha, double u1, double u2, double out[3])
{
    vstore(out, vndf_sample_m(vload(n), vload(wo), alpha, u1, u2, NULL));
}

/* pdf of the reflected direction: G1(wo) D(h) / (4 cos_o) */
static double vndf_pdf_v(v3 n, v3 wo, v3 wi, double a)
{
    double co = vdot(n, wo);
    if (co <= 0.0) return 0.0;
    v3 hs = vadd(wo, wi);
    double l = vlen(hs);
    if (l <= 0.0) return 0.0;
    v3 h = vscale(hs, 1.0 / l);
    if (vdot(wo, h) <= 0.0 || vdot(n, h) <= 0.0) return 0.0;
    return orc_smith_g1(a, co) * orc_ggx_d(a, vdot(n, h)) / (4.0 * co);
}

double orc_vndf_pdf(const double n[3], const double wo[3], const double wi[3], double alpha)
{
    return vndf_pdf_v(vload(n), vload(wo), vload(wi), alpha);
}

static v3 cosine_sample(v3 n, double u1, double u2, Margin* mg)
{
    v3 t, b;
    onb(n, &t, &b, mg);
    double rr = sqrt(u1), ph = 2.0 * PI * u2;
    double z = sqrt(dmax(0.0, 1.0 - u1));
    return vadd(vadd(vscale(t, rr * cos(ph)), vscale(b, rr * sin(ph))), vscale(n, z));
}

typedef struct { double c_env, c_s; } Mix;

static Mix mixture(const orc_scene* s, const double alb[3], double m)
{
    Mix x;
    x.c_env = s->env_ok ? 0.25 : 0.0;
    double f0[3], kd[3];
    for (int k = 0; k < 3; ++k) { f0[k] = 0.04 * (1.0 - m) + m * alb[k]; kd[k] = (1.0 - m) * alb[k]; }
    double ys = lum(f0), yd = lum(kd);
    x.c_s = (ys + yd > 0.0) ? dmin(0.9, dmax(0.1, ys / (ys + yd))) : 0.5;
    return x;
}

static double pdf_mix(const orc_scene* s, Mix x, v3 n, v3 wo, v3 wi, double r, Margin* mg)
{
    double a = alpha_of(r);
    double ci = vdot(n, wi);
    double pe = (x.c_env > 0.0) ? env_pdf_m(s, wi, mg) : 0.0;
    double pv = vndf_pdf_v(n, wo, wi, a);
    double pc = dmax(0.0, ci) / PI;
    return x.c_env * pe + (1.0 - x.c_env) * (x.c_s * pv + (1.0 - x.c_s) * pc);
}

static double sample_cont_m(const orc_scene* s, v3 n, v3 wo, const double alb[3], double r, double m,
                            const uint32_t x[4], v3* dir, Margin* mg)
{
    Mix mx = mixture(s, alb, m);
    double u = orc_uniform(x[0]);
    double t2 = mx.c_env + (1.0 - mx.c_env) * mx.c_s;
    note(mg, fabs(u - t2) / TAU_LOBE, MK_LOBE);
    if (u < mx.c_env) {
        int tex;
        env_sample_m(s, x[1], x[2], x[3], dir, &tex, mg);
    } else if (u < t2) {
        *dir = vndf_sample_m(n, wo, alpha_of(r), orc_uniform(x[1]), orc_uniform(x[2]), mg);
    } else {
        *dir = cosine_sample(n, orc_uniform(x[1]), orc_uniform(x[2]), mg);
    }
    return pdf_mix(s, mx, n, wo, *dir, r, mg);
}

double orc_sample_continuation(const orc_scene* s, const double n[3], const double wo[3],
                               const double albedo[3], double rough, double metal, int32_t kind,
                               const uint32_t x[4], double out_dir[3])
{
    (void)kind;
    v3 d;
    double p = sample_cont_m(s, vload(n), vload(wo), albedo, rough, metal, x, &d, NULL);
    vstore(out_dir, d);
    return p;
}

double orc_pdf_continuation(const orc_scene* s, const double n[3], const double wo[3],
                            const double albedo[3], double rough, double metal, int32_t kind,
                            const double wi[3])
{
    (void)kind;
    Mix mx = mixture(s, albedo, metal);
    return pdf_mix(s, mx, vload(n), vload(wo), vload(wi), rough, NULL);
}

/* ---------------------------------------------------------------------------------------
 * weighted reservoir sampling (Appendix A "Spatial-temporal Reuse", Chao 1982): a stream of
 * candidates, w_sum accumulated, the newcomer kept with probability gamma / w_sum
 * ------------------------------------------------------------------------------------- */
typedef struct { double wsum; int sel; } Reservoir;

static int wrs_update(Reservoir* rs, double gamma, double u, int j)
{
    rs->wsum += gamma;
    if (u * rs->wsum < gamma) { rs->sel = j; return 1; }
    return 0;
}

int32_t orc_wrs(const double* gamma, const double* u, int32_t m, double* w_sum)
{
    Reservoir rs = {0.0, -1};
    for (int j = 0; j < m; ++j) wrs_update(&rs, gamma[j], u[j], j);
    if (w_sum) *w_sum = rs.wsum;
    return rs.sel;
}

/* ---------------------------------------------------------------------------------------
 * materials: bilinear texture lookup, texel centres at (i + 0.5) / w, clamp to edge
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int idx[4]; double w[4]; double dw_dx[4], dw_dy[4];
    int w_tex, h_tex, ix0, iy0; /* texture size and the footprint's unclamped corner */
    double fx, fy;              /* fractional position inside the footprint */
} Taps;

static void taps_at(int w, int h, double su, double sv, Taps* tp)
{
    double x = su * w - 0.5, y = sv * h - 0.5;
    double x0 = floor(x), y0 = floor(y);
    double fx = x - x0, fy = y - y0;
    int ix0 = (int)x0, iy0 = (int)y0;
    int ix1 = ix0 + 1, iy1 = iy0 + 1;
    ix0 = ix0 < 0 ? 0 : (ix0 > w - 1 ? w - 1 : ix0);
    ix1 = ix1 < 0 ? 0 : (ix1 > w - 1 ? w - 1 : ix1);
    iy0 = iy0 < 0 ? 0 : (iy0 > h - 1 ? h - 1 : iy0);
    iy1 = iy1 < 0 ? 0 : (iy1 > h - 1 ? h - 1 : iy1);
    tp->idx[0] = iy0 * w + ix0; tp->idx[1] = iy0 * w + ix1;
    tp->idx[2] = iy1 * w + ix0; tp->idx[3] = iy1 * w + ix1;
    tp->w[0] = (1 - fx) * (1 - fy); tp->w[1] = fx * (1 - fy);
    tp->w[2] = (1 - fx) * fy;       tp->w[3] = fx * fy;
    /* derivatives w.r.t. the texture coordinate (su, sv) */
    tp->dw_dx[0] = -(1 - fy) * w; tp->dw_dx[1] = (1 - fy) * w; tp->dw_dx[2] = -fy * w; tp->dw_dx[3] = fy * w;
    tp->dw_dy[0] = -(1 - fx) * h; tp->dw_dy[1] = -fx * h; tp->dw_dy[2] = (1 - fx) * h; tp->dw_dy[3] = fx * h;
    tp->w_tex = w; tp->h_tex = h; tp->ix0 = (int)x0; tp->iy0 = (int)y0; tp->fx = fx; tp->fy = fy;
}

/* Texels whose bilinear weight an FP32 evaluation of this lookup may change (test tolerance
 * only): the four taps, and where the fractional position lies within (dfx, dfy) texels of a
 * texel centre, the row or column beyond it -- a single-precision lookup on the other side of
 * the centre takes its footprint one texel further. Returns the count written to idx (<= 16;
 * indices clamped to the texture as the lookup clamps them). */
static int taps_reach(const Taps* tp, double dfx, double dfy, int idx[16])
{
    int xs[4], ys[4], nx = 0, ny = 0, n = 0;
    if (tp->fx < dfx) xs[nx++] = tp->ix0 - 1;
    xs[nx++] = tp->ix0;
    xs[nx++] = tp->ix0 + 1;
    if (1.0 - tp->fx < dfx) xs[nx++] = tp->ix0 + 2;
    if (tp->fy < dfy) ys[ny++] = tp->iy0 - 1;
    ys[ny++] = tp->iy0;
    ys[ny++] = tp->iy0 + 1;
    if (1.0 - tp->fy < dfy) ys[ny++] = tp->iy0 + 2;
    for (int b = 0; b < ny; ++b) {
        int y = ys[b] < 0 ? 0 : (ys[b] > tp->h_tex - 1 ? tp->h_tex - 1 : ys[b]);
        for (int a = 0; a < nx; ++a) {
            int x = xs[a] < 0 ? 0 : (xs[a] > tp->w_tex - 1 ? tp->w_tex - 1 : xs[a]);
            int id = y * tp->w_tex + x, dup = 0;
            for (int k = 0; k < n; ++k) dup |= idx[k] == id;
            if (!dup) idx[n++] = id;
        }
    }
    return n;
}

int32_t orc_taps_reach(int32_t w, int32_t h, double su, double sv, double dfx, double dfy, int32_t* out)
{
    Taps tp;
    taps_at(w, h, su, sv, &tp);
    int idx[16];
    int n = taps_reach(&tp, dfx, dfy, idx);
    for (int k = 0; k < n; ++k) out[k] = idx[k];
    return n;
}

typedef struct {
    int tri;
    double u, v, t;
    v3 x, n, N;      /* hit point, shading normal (flipped towards -d), unflipped face normal */
    double sign;     /* face normal towards the viewer: ng = sign * N / |N| */
    v3 ng;           /* face normal towards the viewer */
    int interp;      /* 1: n is the interpolated normal nsg * S / |S| */
    v3 S;            /* w0 VN_a + u VN_b + v VN_c */
    double nsg;      /* +-1: S turned to the side of ng */
    v3 e1, e2;
    double su, sv;   /* texture coordinate */
    Taps tp;
    double alb[3], rgh, met;
} Shade;

static void shade_at(const orc_scene* s, int tri, double u, double v, double t, v3 d, Shade* sh, Margin* mg)
{
    v3 a, b, c;
    tri_verts(s, tri, &a, &b, &c);
    sh->tri = tri; sh->u = u; sh->v = v; sh->t = t;
    sh->e1 = vsub(b, a); sh->e2 = vsub(c, a);
    sh->N = vcross(sh->e1, sh->e2);
    v3 nh = vnorm(sh->N);
    double nd = vdot(nh, d);
    note(mg, fabs(nd) / TAU_FLIP, MK_FLIP);
    sh->sign = (nd > 0.0) ? -1.0 : 1.0;
    sh->n = vscale(nh, sh->sign);
    sh->ng = sh->n;
    sh->x = vadd(a, vadd(vscale(sh->e1, u), vscale(sh->e2, v)));
    const double* uv = s->UV + 6 * tri;
    double w0 = 1.0 - u - v;
    sh->interp = 0; sh->nsg = 1.0; sh->S = V3(0, 0, 0);
    if (s->normals) {
        /* interpolated shading normal: the barycentric blend of the vertex normals, turned to
         * the viewer's side of the face */
        const int32_t* f = s->F + 3 * tri;
        v3 S = vadd(vadd(vscale(vload(s->VN + 3 * f[0]), w0), vscale(vload(s->VN + 3 * f[1]), u)),
                    vscale(vload(s->VN + 3 * f[2]), v));
        double l = vlen(S);
        if (l > 0.0) {
            double cg = vdot(S, sh->ng) / l;
            note(mg, fabs(cg) / TAU_FLIP, MK_FLIP);
            sh->nsg = cg < 0.0 ? -1.0 : 1.0;
            sh->n = vscale(S, sh->nsg / l);
            sh->S = S;
            sh->interp = 1;
        }
    }
    sh->su = w0 * uv[0] + u * uv[2] + v * uv[4];
    sh->sv = w0 * uv[1] + u * uv[3] + v * uv[5];
    taps_at(s->tw, s->th, sh->su, sh->sv, &sh->tp);
    sh->alb[0] = sh->alb[1] = sh->alb[2] = sh->rgh = sh->met = 0.0;
    for (int k = 0; k < 4; ++k) {
        int i = sh->tp.idx[k];
        double w = sh->tp.w[k];
        for (int ch = 0; ch < 3; ++ch) sh->alb[ch] += w * s->alb[3 * i + ch];
        sh->rgh += w * s->rgh[i];
        sh->met += w * s->met[i];
    }
}

/* ---------------------------------------------------------------------------------------
 * one path sample (Eq. pbr_render with the split of Eq. incident, RIS of Eq. restir for the
 * direct part, Eq. mc_indir + Eq. sec_bouce for the indirect part)
 * ------------------------------------------------------------------------------------- */
typedef struct {
    const orc_scene* s;
    const orc_view* v;
    const orc_params* p;
    double R[9], o[3];
    int want_sens; /* accumulate the FP32 sensitivity of each sample's radiance (test tolerance only) */
} Ctx;

typedef struct {
    double rgb[3];
    v3 d0;
    int prim_tri;
    double pu, pv, pt;
    int bg_texel;
    int sel, y_texel;
    v3 y;
    double WV;        /* RIS weight times visibility at the primary vertex */
    int has_cont;
    v3 wc;
    double p_ind;
    double Lind[3];
    double sens;      /* FP32 sensitivity of rgb (test tolerance only): sum over the vertices of the
                       * largest channel of each direct term times its relative FP32 error */
    int nv;           /* vertices recorded below (FULL mode) */
    struct {
        int tri;
        double u, v, t;
        v3 d;         /* incoming ray direction */
        int sel, y_texel;
        v3 y;
        double WV;    /* V W of the direct term (0: none) */
        int has_cont;
        v3 wc;
        double p_ind;
    } vx[ORC_MAXB];
} Rec;

static void rng(const Ctx* c, uint32_t pixel, uint32_t sample, uint32_t bounce, uint32_t purpose, uint32_t j, uint32_t out[4])
{
    uint32_t ctr[4] = {pixel, sample, ((uint32_t)c->v->view_index << 16) | (bounce << 8) | purpose, j};
    uint32_t key[2] = {c->p->seed_lo, c->p->seed_hi};
    orc_philox4x32_10(ctr, key, out);
}

static void ctx_init(Ctx* c, const orc_scene* s, const orc_view* v, const orc_params* p)
{
    c->s = s; c->v = v; c->p = p;
    c->want_sens = 0;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) c->R[3 * i + j] = v->c2w[4 * i + j];
        c->o[i] = v->c2w[4 * i + 3];
    }
}

/* pinhole camera ray through the jittered pixel position (Sec. 3.2, r(t) = o + t d) */
static v3 camera_dir(const Ctx* c, int px, int py, int smp)
{
    uint32_t x[4];
    rng(c, (uint32_t)(py * c->v->width + px), (uint32_t)smp, 0, PURPOSE_CAMERA, 0, x);
    double jx = orc_uniform(x[0]), jy = orc_uniform(x[1]);
    double dc[3] = {(px + jx - c->v->K[2]) / c->v->K[0], (py + jy - c->v->K[3]) / c->v->K[1], 1.0};
    v3 d = V3(c->R[0] * dc[0] + c->R[1] * dc[1] + c->R[2] * dc[2],
              c->R[3] * dc[0] + c->R[4] * dc[1] + c->R[5] * dc[2],
              c->R[6] * dc[0] + c->R[7] * dc[1] + c->R[8] * dc[2]);
    return vnorm(d);
}

/* RIS at one shading point (Eq. restir, N = 1): M env candidates streamed through a weighted
 * reservoir (Appendix A). Out: the selection (sel < 0: none), its direction, texel, f_r cos,
 * p_hat, the weight sum and the number of candidates behind the reservoir (m). */
typedef struct {
    int sel, ytex; uint32_t ysub; v3 y; double f[3], phat, wsum, m;
    double werr; /* FP32 sensitivity (test tolerance only): relative error of w_sum and of f(y) / p_hat(y) */
} Ris;

/* f_r cos of a light direction at a shading point; with interpolated normals a direction
 * below the face gets nothing (its shadow ray would leave through the surface) */
static void light_brdf(const Shade* sh, v3 wo, v3 dir, int kind, double fc[3], Margin* mg)
{
    if (sh->interp) {
        double cg = vdot(dir, sh->ng);
        note(mg, fabs(cg) / TAU_LEAK, MK_LEAK);
        if (!(cg > 0.0)) {
            fc[0] = fc[1] = fc[2] = 0.0;
            return;
        }
    }
    brdf_cos(sh->n, wo, dir, sh->alb, sh->rgh, sh->met, kind, fc);
}

static void ris_at(const Ctx* c, uint32_t pix, int smp, int b, const Shade* sh, v3 wo, Margin* mg, int64_t* cnt,
                   Ris* r)
{
    const orc_scene* s = c->s;
    const int M = c->p->ris_m, kind = c->p->brdf_kind;
    Reservoir rs = {0.0, -1};
    r->sel = -1; r->ytex = -1; r->ysub = 0u; r->y = V3(0, 0, 0); r->phat = 0.0; r->m = M;
    r->f[0] = r->f[1] = r->f[2] = 0.0;
    r->werr = 0.0;
    const double a = alpha_of(sh->rgh);
    double esum = 0.0, esel = 0.0; /* FP32 error of w_sum (absolute) and of the selection's f / p_hat */
    for (int j = 0; j < M; ++j) {
        uint32_t x[4];
        rng(c, pix, (uint32_t)smp, (uint32_t)b, PURPOSE_CANDIDATE, (uint32_t)j, x);
        v3 dir;
        int tex;
        double q = env_sample_m(s, x[0], x[1], x[3], &dir, &tex, mg);
        double fc[3];
        light_brdf(sh, wo, dir, kind, fc, mg);
        double phat = lum(s->env + 3 * tex) * lum(fc); /* p_hat = Y(L_env) Y(f_r) cos */
        double gamma = phat / q;                      /* gamma_s = p_hat / q_dir */
        double ua = orc_uniform(x[2]);
        /* relative FP32 error of gamma: the glossy lobe's conditioning (test tolerance only) */
        double eg = (gamma > 0.0 && (mg || c->want_sens))
                        ? spec_share(sh->n, wo, dir, sh->alb, sh->rgh, sh->met, kind) * ggx_slope(sh->n, wo, dir, a) * DTH
                        : 0.0;
        if (cnt) cnt[5]++;
        if (wrs_update(&rs, gamma, ua, j)) {
            r->y = dir; r->ytex = tex; r->ysub = x[3]; r->phat = phat;
            for (int k = 0; k < 3; ++k) r->f[k] = fc[k];
            esel = eg;
        }
        esum += eg * gamma;
        /* the accept decision's margin: its FP32 error is the base rounding plus the rounding of
         * the weights, whose glossy lobes are conditioned like 1 / alpha (scales 10x the error) */
        if (gamma > 0.0)
            note(mg, fabs(ua * rs.wsum - gamma) / (TAU_ACC * rs.wsum + 10.0 * (ua * esum + eg * gamma)), MK_ACC);
    }
    r->sel = rs.sel;
    r->wsum = rs.wsum;
    r->werr = (rs.wsum > 0.0 ? esum / rs.wsum : 0.0) + esel;
}

/* direction of the sub-texel position `sub` of env texel `texel` (as env_sample_m draws it) */
static v3 texel_dir(const orc_scene* s, int texel, uint32_t sub)
{
    int r = texel / s->ew, cidx = texel % s->ew;
    double uu = (cidx + sub_hi(sub)) / s->ew, vv = (r + sub_lo(sub)) / s->eh;
    double phi = 2.0 * PI * (uu - 0.5), theta = PI * vv;
    double st = sin(theta);
    return V3(st * sin(phi), cos(theta), -st * cos(phi));
}

/* Temporal reuse (Appendix A, "Spatial-temporal Reuse": reservoirs of previous frames merged):
 * the sample's reservoir of the previous call, its candidate count capped at temporal_cap *
 * ris_m, enters after the fresh one with weight p_hat_here(y) w_sum / p_hat_then(y) (m_capped /
 * m), accepted with the third word of reuse draw j = 65535. Its selection code is 65 ris_m. */
static void temporal_merge(const Ctx* c, int px, int py, int smp, const Shade* sh, v3 wo, Margin* mg, Ris* r)
{
    const orc_params* p = c->p;
    if (p->temporal != 2 || !p->history_in) return;
    const orc_scene* s = c->s;
    const int M = p->ris_m;
    const uint32_t pix = (uint32_t)(py * c->v->width + px);
    const double* h = p->history_in + 5 * ((size_t)pix * c->v->spp + smp);
    const int ht = (int)h[0];
    if (ht == -1) return;  /* the primary ray escaped last time */
    const double mc = dmin(h[4], (double)p->temporal_cap * M);
    r->m += mc;
    if (ht < 0 || !(h[2] > 0.0) || !(h[3] > 0.0) || !(h[4] > 0.0)) return;
    v3 y = texel_dir(s, ht, (uint32_t)h[1]);
    double fc[3];
    light_brdf(sh, wo, y, c->p->brdf_kind, fc, mg);
    double phat = lum(s->env + 3 * ht) * lum(fc);
    double w = phat * h[2] / h[3] * (mc / h[4]);
    uint32_t x[4];
    rng(c, pix, (uint32_t)smp, 0, PURPOSE_REUSE, 65535u, x);
    double u = orc_uniform(x[2]);
    r->wsum += w;
    if (u * r->wsum < w) {
        r->sel = 65 * M;
        r->y = y; r->ytex = ht; r->ysub = (uint32_t)h[1]; r->phat = phat;
        for (int k = 0; k < 3; ++k) r->f[k] = fc[k];
    }
    if (w > 0.0) note(mg, fabs(u * r->wsum - w) / r->wsum / TAU_ACC, MK_ACC);
}

/* the primary vertex's RIS reservoir of sample smp of pixel (qx, qy), merged with its history
 * when temporal reuse is on: 0 if its ray escapes */
static int primary_reservoir(const Ctx* c, int qx, int qy, int smp, Margin* mg, int64_t* cnt, Ris* r)
{
    const orc_scene* s = c->s;
    v3 o = vload(c->o), d = camera_dir(c, qx, qy, smp);
    Hit h;
    bvh_closest(s, o, d, -1, &h, cnt);
    closest_margins(s, o, d, -1, &h, mg);
    if (h.tri < 0) return 0;
    Shade sh;
    shade_at(s, h.tri, h.u, h.v, h.t, d, &sh, mg);
    ris_at(c, (uint32_t)(qy * c->v->width + qx), smp, 0, &sh, vscale(d, -1.0), mg, cnt, r);
    temporal_merge(c, qx, qy, smp, &sh, vscale(d, -1.0), mg, r);
    return 1;
}

/* Spatial reuse at the primary vertex (Appendix A, "Spatial-temporal Reuse": reservoirs of
 * neighbouring pixels merged into the pixel's own). Reading: reuse_k neighbours of the same
 * sample index, pixel offsets drawn uniformly from the (2 r + 1)^2 square (the pixel itself
 * and pixels outside the image skipped; a neighbour whose primary ray escapes has no
 * reservoir). Reservoirs are merged by the standard resampling rule: each enters with weight
 * p_hat_here(y_i) W_i m_i, W_i = w_sum_i / (m_i p_hat_i(y_i)), i.e. p_hat_here(y_i) w_sum_i /
 * p_hat_i(y_i), streamed through a reservoir (the pixel's own first), and the merged
 * reservoir counts sum m_i candidates; W = w_sum / (m p_hat_here(y)). The paper gives no MIS
 * weights, so this is the biased 1/m combination. */
static void spatial_reuse(const Ctx* c, int px, int py, int smp, const Shade* sh, v3 wo, Margin* mg, int64_t* cnt,
                          Ris* r)
{
    const orc_scene* s = c->s;
    const int K = c->p->reuse_k, R = c->p->reuse_radius, kind = c->p->brdf_kind;
    const uint32_t pix = (uint32_t)(py * c->v->width + px);
    Ris out = *r;
    out.wsum = 0.0;
    out.sel = -1;
    out.m = r->m;
    if (r->sel >= 0 && r->wsum > 0.0 && r->phat > 0.0) {
        double w = r->phat * r->wsum / r->phat; /* own reservoir: p_hat_here = p_hat_own */
        out.wsum = w;
        out.sel = r->sel;
    }
    for (int j = 0; j < K; ++j) {
        uint32_t x[4];
        rng(c, pix, (uint32_t)smp, 0, PURPOSE_REUSE, (uint32_t)j, x);
        int dx = (int)floor(orc_uniform(x[0]) * (2 * R + 1)) - R;
        int dy = (int)floor(orc_uniform(x[1]) * (2 * R + 1)) - R;
        int qx = px + dx, qy = py + dy;
        if ((dx == 0 && dy == 0) || qx < 0 || qy < 0 || qx >= c->v->width || qy >= c->v->height) continue;
        Ris nb;
        if (!primary_reservoir(c, qx, qy, smp, mg, cnt, &nb)) continue;
        out.m += nb.m;
        if (nb.sel < 0 || !(nb.wsum > 0.0) || !(nb.phat > 0.0)) continue;
        double fc[3];
        light_brdf(sh, wo, nb.y, kind, fc, mg);
        double phat = lum(s->env + 3 * nb.ytex) * lum(fc);
        double w = phat * nb.wsum / nb.phat;
        out.wsum += w;
        double u = orc_uniform(x[2]);
        if (u * out.wsum < w) {
            out.sel = c->p->ris_m * (j + 1) + nb.sel;
            out.y = nb.y; out.ytex = nb.ytex; out.ysub = nb.ysub; out.phat = phat;
            for (int k = 0; k < 3; ++k) out.f[k] = fc[k];
        }
        if (w > 0.0) note(mg, fabs(u * out.wsum - w) / out.wsum / TAU_ACC, MK_ACC);
    }
    *r = out;
}

static void path_sample(const Ctx* c, int px, int py, int smp, Rec* rec, Margin* mg, int64_t* cnt)
{
    const orc_scene* s = c->s;
    const int M = c->p->ris_m, B = c->v->bounces, kind = c->p->brdf_kind;
    const uint32_t pix = (uint32_t)(py * c->v->width + px);
    memset(rec, 0, sizeof(*rec));
    rec->prim_tri = -1; rec->sel = -1; rec->y_texel = -1; rec->bg_texel = -1;
    v3 o = vload(c->o), d = camera_dir(c, px, py, smp);
    rec->d0 = d;
    if (cnt) { cnt[0]++; cnt[6]++; }
    Hit h;
    bvh_closest(s, o, d, -1, &h, cnt);
    closest_margins(s, o, d, -1, &h, mg);
    if (h.tri < 0) {
        /* primary miss: the environment seen directly */
        if (c->p->temporal && c->p->history_out) {
            double* ho = c->p->history_out + 5 * ((size_t)pix * c->v->spp + smp);
            ho[0] = -1; ho[1] = ho[2] = ho[3] = ho[4] = 0.0;
        }
        int tx = env_texel_m(s, d, mg);
        rec->bg_texel = tx;
        for (int k = 0; k < 3; ++k) rec->rgb[k] = s->env[3 * tx + k];
        return;
    }
    rec->prim_tri = h.tri; rec->pu = h.u; rec->pv = h.v; rec->pt = h.t;
    double beta[3] = {1, 1, 1}, beta_ind[3] = {1, 1, 1};
    double L[3] = {0, 0, 0}, Lind[3] = {0, 0, 0};
    double rel_beta = 0.0; /* relative FP32 error of the throughput (test tolerance only) */
    double plen = h.t;     /* path length to the current vertex: the lever of its rays' rounding */
    for (int b = 0; b < B; ++b) {
        Shade sh;
        shade_at(s, h.tri, h.u, h.v, h.t, d, &sh, mg);
        v3 wo = vscale(d, -1.0);
        if (b < ORC_MAXB) {
            rec->nv = b + 1;
            rec->vx[b].tri = h.tri; rec->vx[b].u = h.u; rec->vx[b].v = h.v; rec->vx[b].t = h.t;
            rec->vx[b].d = d;
            rec->vx[b].sel = -1; rec->vx[b].y_texel = -1; rec->vx[b].WV = 0.0; rec->vx[b].has_cont = 0;
        }
        if (b == 0) {
            note(mg, vdot(sh.n, wo) / TAU_GRAZE, MK_GRAZE);
            /* with interpolated normals the hit can graze the face while the shading normal
             * does not: the intersection's derivative grows as 1 / (n_face . d) all the same */
            if (sh.interp) note(mg, fabs(vdot(sh.ng, wo)) / TAU_GRAZE, MK_GRAZE);
        }
        /* ---- direct light: RIS over M env candidates, streamed through a reservoir ---- */
        double direct[3] = {0, 0, 0};
        double werr = 0.0;
        if (s->env_ok && M > 0) {
            Ris r;
            ris_at(c, pix, smp, b, &sh, wo, mg, cnt, &r);
            if (b == 0 && (c->p->reuse_k > 0 || c->p->temporal)) {
                temporal_merge(c, px, py, smp, &sh, wo, mg, &r);
                spatial_reuse(c, px, py, smp, &sh, wo, mg, cnt, &r);
                if (c->p->temporal && c->p->history_out) {
                    double* ho = c->p->history_out + 5 * ((size_t)pix * c->v->spp + smp);
                    int ok = r.sel >= 0 && r.wsum > 0.0 && r.phat > 0.0;
                    ho[0] = ok ? r.ytex : -2; ho[1] = r.ysub; ho[2] = r.wsum; ho[3] = r.phat; ho[4] = r.m;
                }
            }
            if (r.sel >= 0 && r.wsum > 0.0) {
                /* Eq. restir with N = 1: f(y) / p_hat(y) * (1/m) sum gamma */
                double W = r.wsum / (r.m * r.phat);
                if (cnt) cnt[2]++;
                int occluded = bvh_any_l(s, sh.x, r.y, sh.tri, cnt, mg, plen);
                double V = occluded ? 0.0 : 1.0;
                for (int k = 0; k < 3; ++k) direct[k] = V * W * s->env[3 * r.ytex + k] * r.f[k];
                werr = r.werr;
                if (b == 0) { rec->sel = r.sel; rec->y = r.y; rec->y_texel = r.ytex; rec->WV = V * W; }
                if (b < ORC_MAXB) {
                    rec->vx[b].sel = r.sel; rec->vx[b].y = r.y; rec->vx[b].y_texel = r.ytex; rec->vx[b].WV = V * W;
                }
            }
        }
        double dmax_c = 0.0;
        for (int k = 0; k < 3; ++k) {
            L[k] += beta[k] * direct[k];
            if (b >= 1) Lind[k] += beta_ind[k] * direct[k];
            dmax_c = dmax(dmax_c, fabs(beta[k] * direct[k]));
        }
        rec->sens += dmax_c * (rel_beta + werr);
        if (b == B - 1) break;
        /* ---- indirect light: one continuation ray from the MIS mixture ---- */
        uint32_t x[4];
        rng(c, pix, (uint32_t)smp, (uint32_t)b, PURPOSE_CONTINUE, 0, x);
        v3 wc;
        double pind = sample_cont_m(s, sh.n, wo, sh.alb, sh.rgh, sh.met, x, &wc, mg);
        if (sh.interp) {
            /* with interpolated normals a continuation below the face ends the path */
            double cg = vdot(wc, sh.ng);
            note(mg, fabs(cg) / TAU_LEAK, MK_LEAK);
            if (!(cg > 0.0)) break;
        }
        double fc[3];
        brdf_cos(sh.n, wo, wc, sh.alb, sh.rgh, sh.met, kind, fc);
        if (!(pind > 0.0) || (fc[0] <= 0.0 && fc[1] <= 0.0 && fc[2] <= 0.0)) break;
        if (b == 0) { rec->has_cont = 1; rec->wc = wc; rec->p_ind = pind; }
        if (b < ORC_MAXB) { rec->vx[b].has_cont = 1; rec->vx[b].wc = wc; rec->vx[b].p_ind = pind; }
        if (c->want_sens) {
            /* FP32 error of f cos / p_ind: the GGX D in f and in the VNDF part of the mixture pdf
             * cancel to the extent their shares agree (test tolerance only) */
            Mix mx = mixture(s, sh.alb, sh.met);
            double a = alpha_of(sh.rgh);
            double pshare = (1.0 - mx.c_env) * mx.c_s * vndf_pdf_v(sh.n, wo, wc, a) / pind;
            double fshare = spec_share(sh.n, wo, wc, sh.alb, sh.rgh, sh.met, kind);
            rel_beta += fabs(fshare - pshare) * ggx_slope(sh.n, wo, wc, a) * DTH;
        }
        for (int k = 0; k < 3; ++k) {
            double f = fc[k] / pind;
            beta[k] *= f;
            if (b >= 1) beta_ind[k] *= f;
        }
        if (cnt) cnt[1]++;
        Hit nh;
        bvh_closest(s, sh.x, wc, sh.tri, &nh, cnt);
        closest_margins_l(s, sh.x, wc, sh.tri, &nh, mg, plen);
        if (nh.tri < 0) break; /* escaped: its env light is already in the direct term */
        h = nh;
        d = wc;
        plen += nh.t;
    }
    for (int k = 0; k < 3; ++k) { rec->rgb[k] = L[k]; rec->Lind[k] = Lind[k]; }
}

/* The radiance of a recorded path re-evaluated with every decision (hit triangles, selected
 * candidates and their V W, continuation directions and pdfs) held, and the barycentrics of
 * vertex `bp` moved by (du, dv) (test tolerance only). */
static void path_value(const Ctx* c, const Rec* rec, int bp, double du, double dv, double out[3])
{
    const orc_scene* s = c->s;
    const int kind = c->p->brdf_kind;
    double beta[3] = {1, 1, 1};
    out[0] = out[1] = out[2] = 0.0;
    for (int b = 0; b < rec->nv && b < ORC_MAXB; ++b) {
        const double u = rec->vx[b].u + (b == bp ? du : 0.0), v = rec->vx[b].v + (b == bp ? dv : 0.0);
        Shade sh;
        shade_at(s, rec->vx[b].tri, u, v, rec->vx[b].t, rec->vx[b].d, &sh, NULL);
        v3 wo = vscale(rec->vx[b].d, -1.0);
        if (rec->vx[b].sel >= 0 && rec->vx[b].WV != 0.0) {
            double fc[3];
            brdf_cos(sh.n, wo, rec->vx[b].y, sh.alb, sh.rgh, sh.met, kind, fc);
            for (int k = 0; k < 3; ++k) out[k] += beta[k] * rec->vx[b].WV * s->env[3 * rec->vx[b].y_texel + k] * fc[k];
        }
        if (!rec->vx[b].has_cont) break;
        double fc[3];
        brdf_cos(sh.n, wo, rec->vx[b].wc, sh.alb, sh.rgh, sh.met, kind, fc);
        for (int k = 0; k < 3; ++k) beta[k] *= fc[k] / rec->vx[b].p_ind;
    }
}

/* FP32 sensitivity of a sample's radiance to the rounding of its hit points (test tolerance
 * only): every vertex's barycentrics moved by +- the FP32 error of a single-precision solve of
 * its ray, 8 u (|o - v0| + |o| + lever) |row of A^-1| / |det| as for the texel sensitivity,
 * whose origin carries the rounding of the path before it (the lever, its path length); the
 * material lookups, the shading normal and the shading point follow. Sum over vertices and the
 * two barycentrics of the larger change of the largest channel. */
static double path_hit_sens(const Ctx* c, const Rec* rec)
{
    if (rec->prim_tri < 0 || rec->nv < 1) return 0.0;
    const orc_scene* s = c->s;
    double base[3];
    path_value(c, rec, -1, 0.0, 0.0, base);
    v3 o = vload(c->o);
    double lever = 0.0, sens = 0.0;
    for (int b = 0; b < rec->nv && b < ORC_MAXB; ++b) {
        v3 a, bb, cc;
        tri_verts(s, rec->vx[b].tri, &a, &bb, &cc);
        v3 e1 = vsub(bb, a), e2 = vsub(cc, a), md = vscale(rec->vx[b].d, -1.0);
        v3 r0 = vcross(e2, md), r1 = vcross(md, e1);
        double det = fabs(vdot(e1, r0));
        if (det > 0.0) {
            double l = 8.0 * U32 * (vlen(vsub(o, a)) + vlen(o) + lever) / det;
            const double dbary[2] = {l * vlen(r0), l * vlen(r1)};
            for (int comp = 0; comp < 2; ++comp) {
                double worst = 0.0;
                for (int sg = -1; sg <= 1; sg += 2) {
                    double o3[3];
                    path_value(c, rec, b, comp == 0 ? sg * dbary[0] : 0.0, comp == 1 ? sg * dbary[1] : 0.0, o3);
                    for (int k = 0; k < 3; ++k) worst = dmax(worst, fabs(o3[k] - base[k]));
                }
                sens += worst;
            }
        }
        /* the next ray starts at this vertex's hit point */
        lever += rec->vx[b].t;
        o = vadd(a, vadd(vscale(e1, rec->vx[b].u), vscale(e2, rec->vx[b].v)));
        if (!rec->vx[b].has_cont) break;
    }
    return sens;
}

/* ---------------------------------------------------------------------------------------
 * adjoint of one sample (PRIMARY mode, Sec. 4.2 last sentence and Appendix C limitations)
 * ------------------------------------------------------------------------------------- */
enum { GB_ALB = 0, GB_RGH, GB_MET, GB_ENV, GB_VERT, GB_ALB_S, GB_RGH_S, GB_MET_S, GB_VERT_S, GB_N };
typedef struct { int32_t buf; int64_t idx; double val; } Entry;
typedef struct { Entry* e; size_t n, cap; } Sparse;

static void sp_add(Sparse* sp, int buf, int64_t idx, double val)
{
    if (val == 0.0) return;
    if (sp->n == sp->cap) {
        sp->cap = sp->cap ? 2 * sp->cap : 4096;
        sp->e = (Entry*)realloc(sp->e, sizeof(Entry) * sp->cap);
    }
    sp->e[sp->n].buf = buf; sp->e[sp->n].idx = idx; sp->e[sp->n].val = val;
    sp->n++;
}

/* Sparse lists of vertex terms that can be compared entry by entry: zero terms are kept (the
 * entry structure must not depend on the values) */
static void sp_put(Sparse* sp, int buf, int64_t idx, double val)
{
    if (sp->n == sp->cap) {
        sp->cap = sp->cap ? 2 * sp->cap : 256;
        sp->e = (Entry*)realloc(sp->e, sizeof(Entry) * sp->cap);
    }
    sp->e[sp->n].buf = buf; sp->e[sp->n].idx = idx; sp->e[sp->n].val = val;
    sp->n++;
}

/* FP32 sensitivity of the vertex gradient (test tolerance only): one input of the primary
 * vertex's adjoint moved by the rounding error an FP32 evaluation of it may carry. comp 0-2:
 * the camera direction; 3-4: the barycentrics (by the FP32 error of a single-precision ray's
 * intersection, du / dv); 5-7: the selected light direction; 8-10: the continuation direction;
 * 11-13: the shading normal; sgn = +1 or -1. */
typedef struct { int comp; double sgn, du, dv, dn; } Pert;

/* a unit vector with component k moved by rel, renormalised */
static v3 nudge(v3 a, int k, double rel)
{
    double q[3] = {a.x, a.y, a.z};
    q[k] += rel;
    return vnorm(V3(q[0], q[1], q[2]));
}

/* The primary vertex's adjoint of one sample (PRIMARY mode, the sample's primary triangle hit).
 * tex = 1: every term (env, textures with their FP32 sensitivity, vertices); tex = 0: only the
 * vertex terms, for the FP32 sensitivity (pt = the perturbed input, NULL = none). */
static void prim_grad(const Ctx* c, const Rec* rec, const double g[3], int kind, const Pert* pt, int tex, Sparse* sp)
{
    const orc_scene* s = c->s;
    void (*put)(Sparse*, int, int64_t, double) = tex ? sp_add : sp_put;
    v3 d0 = rec->d0, y = rec->y, wc = rec->wc;
    double pu = rec->pu, pv = rec->pv;
    if (pt) {
        const int k = pt->comp;
        if (k < 3) d0 = nudge(d0, k, pt->sgn * 4.0 * U32);
        else if (k == 3) pu += pt->sgn * pt->du;
        else if (k == 4) pv += pt->sgn * pt->dv;
        else if (k < 8) y = nudge(y, k - 5, pt->sgn * 8.0 * U32);
        else if (k < 11) wc = nudge(wc, k - 8, pt->sgn * 8.0 * U32);
    }
    Shade sh;
    shade_at(s, rec->prim_tri, pu, pv, rec->pt, d0, &sh, NULL);
    if (pt && pt->comp >= 11) sh.n = nudge(sh.n, pt->comp - 11, pt->sgn * pt->dn);
    v3 wo = vscale(d0, -1.0);
    double gm[8] = {0, 0, 0, 0, 0, 0, 0, 0}, tmp[8];
    /* direct_1 = V W L_env(y) (f_r cos)(y) */
    if (rec->sel >= 0 && rec->WV != 0.0) {
        double fc[3], gq[3];
        brdf_cos(sh.n, wo, y, sh.alb, sh.rgh, sh.met, kind, fc);
        for (int k = 0; k < 3; ++k) {
            double le = s->env[3 * rec->y_texel + k];
            if (tex) sp_add(sp, GB_ENV, 3 * (int64_t)rec->y_texel + k, g[k] * rec->WV * fc[k]);
            gq[k] = g[k] * rec->WV * le;
        }
        brdf_cos_grad(sh.n, wo, y, sh.alb, sh.rgh, sh.met, kind, gq, tmp);
        for (int k = 0; k < 8; ++k) gm[k] += tmp[k];
    }
    /* beta_1 L_ind = (f_r cos)(wc) / p_ind * L_ind */
    if (rec->has_cont) {
        double gq[3];
        for (int k = 0; k < 3; ++k) gq[k] = g[k] * rec->Lind[k] / rec->p_ind;
        brdf_cos_grad(sh.n, wo, wc, sh.alb, sh.rgh, sh.met, kind, gq, tmp);
        for (int k = 0; k < 8; ++k) gm[k] += tmp[k];
    }
    const double* uv = s->UV + 6 * sh.tri;
    v3 md = vscale(d0, -1.0);
    /* A = [e1 | e2 | -d]; rows of A^-1 are (e2 x -d, -d x e1, e1 x e2) / det */
    v3 r0 = vcross(sh.e2, md), r1 = vcross(md, sh.e1);
    double det = vdot(sh.e1, r0);
    if (tex) {
        /* FP32 sensitivity (test tolerance only): barycentric error of a single-precision primary
         * ray, ~8 u (t + |o - v0| + |o|) |row of A^-1|, mapped to the fractional texel position */
        v3 o = vload(c->o), a, b, cc;
        tri_verts(s, sh.tri, &a, &b, &cc);
        double lever = 8.0 * U32 * (sh.t + vlen(vsub(o, a)) + vlen(o)) / fabs(det);
        double du = lever * vlen(r0), dv = lever * vlen(r1);
        double dfx = s->tw * (fabs(uv[2] - uv[0]) * du + fabs(uv[4] - uv[0]) * dv);
        double dfy = s->th * (fabs(uv[3] - uv[1]) * du + fabs(uv[5] - uv[1]) * dv);
        double dw = dfx + dfy;
        int reach[16];
        int nr = taps_reach(&sh.tp, dfx, dfy, reach);
        for (int k = 0; k < nr; ++k) {
            int i = reach[k];
            for (int ch = 0; ch < 3; ++ch) sp_add(sp, GB_ALB_S, 3 * (int64_t)i + ch, dw * fabs(gm[ch]));
            sp_add(sp, GB_RGH_S, i, dw * fabs(gm[3]));
            sp_add(sp, GB_MET_S, i, dw * fabs(gm[4]));
        }
    }
    /* textures (bilinear scatter) and the texture coordinate */
    double gsu = 0.0, gsv = 0.0;
    for (int k = 0; k < 4; ++k) {
        int i = sh.tp.idx[k];
        double w = sh.tp.w[k];
        double dot = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            if (tex) sp_add(sp, GB_ALB, 3 * (int64_t)i + ch, w * gm[ch]);
            dot += gm[ch] * s->alb[3 * i + ch];
        }
        if (tex) {
            sp_add(sp, GB_RGH, i, w * gm[3]);
            sp_add(sp, GB_MET, i, w * gm[4]);
        }
        dot += gm[3] * s->rgh[i] + gm[4] * s->met[i];
        gsu += sh.tp.dw_dx[k] * dot;
        gsv += sh.tp.dw_dy[k] * dot;
    }
    /* vertices: (u, v) through the intersection, n through the face normal -- or, with
     * interpolated normals, through S = w0 VN_a + u VN_b + v VN_c to (u, v) and to the vertex
     * normals VN_i = VA_i / |VA_i|, VA_i the sum of the incident faces' e1 x e2 */
    double gu = gsu * (uv[2] - uv[0]) + gsv * (uv[3] - uv[1]);
    double gv = gsu * (uv[4] - uv[0]) + gsv * (uv[5] - uv[1]);
    v3 gn = V3(gm[5], gm[6], gm[7]);
    const int32_t* fv = s->F + 3 * sh.tri;
    double bw[3] = {1.0 - sh.u - sh.v, sh.u, sh.v};
    v3 gS = V3(0, 0, 0);
    if (sh.interp) {
        double Sl = vlen(sh.S);
        v3 sn = vscale(sh.S, 1.0 / Sl);
        v3 gsn = vscale(gn, sh.nsg);
        gS = vscale(vsub(gsn, vscale(sn, vdot(sn, gsn))), 1.0 / Sl);
        v3 na = vload(s->VN + 3 * fv[0]), nb = vload(s->VN + 3 * fv[1]), nc = vload(s->VN + 3 * fv[2]);
        gu += vdot(gS, vsub(nb, na));
        gv += vdot(gS, vsub(nc, na));
    }
    v3 z = vscale(vadd(vscale(r0, gu), vscale(r1, gv)), 1.0 / det); /* A^-T (gu, gv, 0) */
    v3 gvert[3];
    for (int k = 0; k < 3; ++k) gvert[k] = vscale(z, -bw[k]);
    if (sh.interp) {
        for (int k = 0; k < 3; ++k) {
            const int vi = fv[k];
            v3 A = vload(s->VA + 3 * vi);
            double Al = vlen(A);
            if (!(Al > 0.0)) continue;
            v3 vn = vscale(A, 1.0 / Al);
            v3 gvn = vscale(gS, bw[k]);
            v3 gA = vscale(vsub(gvn, vscale(vn, vdot(vn, gvn))), 1.0 / Al);
            for (int q = s->vf_off[vi]; q < s->vf_off[vi + 1]; ++q) {
                const int f = s->vf[q];
                v3 a, b, cc;
                tri_verts(s, f, &a, &b, &cc);
                v3 fe1 = vsub(b, a), fe2 = vsub(cc, a);
                v3 ge1 = vcross(fe2, gA), ge2 = vcross(gA, fe1);
                v3 gf[3] = {vscale(vadd(ge1, ge2), -1.0), ge1, ge2};
                for (int m = 0; m < 3; ++m) {
                    int vj = s->F[3 * f + m];
                    put(sp, GB_VERT, 3 * (int64_t)vj + 0, gf[m].x);
                    put(sp, GB_VERT, 3 * (int64_t)vj + 1, gf[m].y);
                    put(sp, GB_VERT, 3 * (int64_t)vj + 2, gf[m].z);
                }
            }
        }
    } else {
        double Nl = vlen(sh.N);
        v3 Nh = vscale(sh.N, 1.0 / Nl);
        v3 gNh = vscale(gn, sh.sign);
        v3 gN = vscale(vsub(gNh, vscale(Nh, vdot(Nh, gNh))), 1.0 / Nl);
        v3 ge1 = vcross(sh.e2, gN), ge2 = vcross(gN, sh.e1);
        gvert[0] = vsub(gvert[0], vadd(ge1, ge2));
        gvert[1] = vadd(gvert[1], ge1);
        gvert[2] = vadd(gvert[2], ge2);
    }
    for (int k = 0; k < 3; ++k) {
        int vi = s->F[3 * sh.tri + k];
        put(sp, GB_VERT, 3 * (int64_t)vi + 0, gvert[k].x);
        put(sp, GB_VERT, 3 * (int64_t)vi + 1, gvert[k].y);
        put(sp, GB_VERT, 3 * (int64_t)vi + 2, gvert[k].z);
    }
}

/* FP32 sensitivity of one sample's vertex terms (test tolerance only): for every input of
 * prim_grad, the larger change of each vertex term when that input moves by +- its FP32
 * rounding scale, summed over the inputs (a first-order bound on what a single-precision
 * evaluation of the same formulas may differ by; it also covers a texture coordinate that
 * sits within rounding of a texel centre, where the bilinear derivative jumps). */
static void vert_sens(const Ctx* c, const Rec* rec, const double g[3], int kind, Sparse* sp)
{
    const orc_scene* s = c->s;
    Shade sh;
    shade_at(s, rec->prim_tri, rec->pu, rec->pv, rec->pt, rec->d0, &sh, NULL);
    v3 md = vscale(rec->d0, -1.0);
    v3 r0 = vcross(sh.e2, md), r1 = vcross(md, sh.e1);
    double det = vdot(sh.e1, r0);
    v3 o = vload(c->o), a, b, cc;
    tri_verts(s, sh.tri, &a, &b, &cc);
    /* rounding of a single-precision Moller-Trumbore solve: a few units of |o - v0| |row| and
     * |o| |row| over det (the direction's own rounding is comp 0-2) */
    double lever = 3.0 * U32 * (vlen(vsub(o, a)) + vlen(o)) / fabs(det);
    Pert pt;
    pt.du = lever * vlen(r0);
    pt.dv = lever * vlen(r1);
    /* the face normal's FP32 direction error grows with the cross product's cancellation; the
     * interpolated normal is a blend of three FP32 unit vectors */
    pt.dn = sh.interp ? 8.0 * U32 : 4.0 * U32 * vlen(sh.e1) * vlen(sh.e2) / vlen(sh.N);
    Sparse base = {0}, pe = {0};
    /* tex = 0 keeps zero terms, so the lists of the perturbed evaluations line up entry by entry */
    prim_grad(c, rec, g, kind, NULL, 0, &base);
    double* acc = (double*)calloc(base.n ? base.n : 1, sizeof(double));
    double* mx = (double*)calloc(base.n ? base.n : 1, sizeof(double));
    const int has_y = rec->sel >= 0 && rec->WV != 0.0;
    for (int comp = 0; comp < 14; ++comp) {
        if (comp >= 5 && comp < 8 && !has_y) continue;
        if (comp >= 8 && comp < 11 && !rec->has_cont) continue;
        for (size_t e = 0; e < base.n; ++e) mx[e] = 0.0;
        for (int sg = -1; sg <= 1; sg += 2) {
            pt.comp = comp;
            pt.sgn = (double)sg;
            pe.n = 0;
            prim_grad(c, rec, g, kind, &pt, 0, &pe);
            const size_t n = pe.n < base.n ? pe.n : base.n;
            for (size_t e = 0; e < n; ++e) mx[e] = dmax(mx[e], fabs(pe.e[e].val - base.e[e].val));
        }
        for (size_t e = 0; e < base.n; ++e) acc[e] += mx[e];
    }
    for (size_t e = 0; e < base.n; ++e) sp_add(sp, GB_VERT_S, base.e[e].idx, acc[e]);
    free(acc);
    free(mx);
    free(base.e);
    free(pe.e);
}

/* demod = 0: the sample's radiance. demod = 1: its demodulated lighting at the primary vertex
 * (the same terms with the kind-2 lobes; an escaping primary ray has none). vsens = 1 also
 * accumulates the FP32 sensitivity of the vertex terms (GB_VERT_S). */
static void sample_grad(const Ctx* c, const Rec* rec, const double g[3], int demod, int vsens, Sparse* sp)
{
    const int kind = demod ? 2 : c->p->brdf_kind;
    if (rec->prim_tri < 0) {
        if (demod) return;
        for (int k = 0; k < 3; ++k) sp_add(sp, GB_ENV, 3 * (int64_t)rec->bg_texel + k, g[k]);
        return;
    }
    prim_grad(c, rec, g, kind, NULL, 1, sp);
    if (vsens) vert_sens(c, rec, g, kind, sp);
}

/* FULL mode: the vertices after the primary one (the gradients of indirect rays that Sec. 4.2
 * detaches and Appendix C lists as missing). With L = sum_b beta_b direct_b, beta_{b+1} =
 * beta_b (f_r cos)(wc_b) / p_b, direct_b = WV_b L_env(y_b) (f_r cos)(y_b), every sampling
 * decision, W, V and p_ind detached and the hit points of vertices b >= 1 held fixed on their
 * triangles, the derivative w.r.t. the material at x_b (b >= 1) is, per channel,
 *   beta_b [ WV_b L_env(y_b) d(f_r cos)(y_b) + (Lin_b / p_b) d(f_r cos)(wc_b) ]
 * and w.r.t. the env texel of y_b it is beta_b WV_b (f_r cos)(y_b); Lin_b is the radiance
 * arriving at x_b along wc_b from the rest of the path. The normal's derivative is dropped
 * (geometry detached beyond the primary vertex). */
static void sample_grad_secondary(const Ctx* c, const Rec* rec, const double g[3], Sparse* sp)
{
    const orc_scene* s = c->s;
    const int kind = c->p->brdf_kind;
    const int nv = rec->nv;
    if (rec->prim_tri < 0 || nv < 2) return;
    Shade sh[ORC_MAXB];
    double fy[ORC_MAXB][3], fc[ORC_MAXB][3], dir[ORC_MAXB][3], beta[ORC_MAXB][3], lin[ORC_MAXB][3];
    for (int b = 0; b < nv; ++b) {
        shade_at(s, rec->vx[b].tri, rec->vx[b].u, rec->vx[b].v, rec->vx[b].t, rec->vx[b].d, &sh[b], NULL);
        v3 wo = vscale(rec->vx[b].d, -1.0);
        for (int k = 0; k < 3; ++k) fy[b][k] = fc[b][k] = dir[b][k] = 0.0;
        if (rec->vx[b].sel >= 0 && rec->vx[b].WV != 0.0) {
            brdf_cos(sh[b].n, wo, rec->vx[b].y, sh[b].alb, sh[b].rgh, sh[b].met, kind, fy[b]);
            for (int k = 0; k < 3; ++k) dir[b][k] = rec->vx[b].WV * s->env[3 * rec->vx[b].y_texel + k] * fy[b][k];
        }
        if (rec->vx[b].has_cont) brdf_cos(sh[b].n, wo, rec->vx[b].wc, sh[b].alb, sh[b].rgh, sh[b].met, kind, fc[b]);
    }
    for (int k = 0; k < 3; ++k) beta[0][k] = 1.0;
    for (int b = 1; b < nv; ++b)
        for (int k = 0; k < 3; ++k) beta[b][k] = beta[b - 1][k] * fc[b - 1][k] / rec->vx[b - 1].p_ind;
    for (int k = 0; k < 3; ++k) lin[nv - 1][k] = 0.0;
    for (int b = nv - 2; b >= 0; --b)
        for (int k = 0; k < 3; ++k)
            lin[b][k] = dir[b + 1][k] +
                        (rec->vx[b + 1].has_cont ? fc[b + 1][k] / rec->vx[b + 1].p_ind * lin[b + 1][k] : 0.0);
    for (int b = 1; b < nv; ++b) {
        const Shade* h = &sh[b];
        v3 wo = vscale(rec->vx[b].d, -1.0);
        double gm[8] = {0, 0, 0, 0, 0, 0, 0, 0}, tmp[8], gq[3];
        if (rec->vx[b].sel >= 0 && rec->vx[b].WV != 0.0) {
            for (int k = 0; k < 3; ++k) {
                double le = s->env[3 * rec->vx[b].y_texel + k];
                sp_add(sp, GB_ENV, 3 * (int64_t)rec->vx[b].y_texel + k, g[k] * beta[b][k] * rec->vx[b].WV * fy[b][k]);
                gq[k] = g[k] * beta[b][k] * rec->vx[b].WV * le;
            }
            brdf_cos_grad(h->n, wo, rec->vx[b].y, h->alb, h->rgh, h->met, kind, gq, tmp);
            for (int k = 0; k < 8; ++k) gm[k] += tmp[k];
        }
        if (rec->vx[b].has_cont) {
            for (int k = 0; k < 3; ++k) gq[k] = g[k] * beta[b][k] * lin[b][k] / rec->vx[b].p_ind;
            brdf_cos_grad(h->n, wo, rec->vx[b].wc, h->alb, h->rgh, h->met, kind, gq, tmp);
            for (int k = 0; k < 8; ++k) gm[k] += tmp[k];
        }
        /* FP32 sensitivity (test tolerance only): a single-precision path reaches x_b with a
         * position error of a few FP32 units of the distances involved, amplified along the
         * path; bounded generously by 64 u (t + |x_{b-1} - v0| + |x_{b-1}|) |row of A^-1| */
        {
            const double u32 = 1.0 / 16777216.0;
            const double* uv = s->UV + 6 * h->tri;
            v3 md = vscale(rec->vx[b].d, -1.0);
            v3 r0 = vcross(h->e2, md), r1 = vcross(md, h->e1);
            double det = vdot(h->e1, r0);
            v3 a, bb, cc;
            tri_verts(s, h->tri, &a, &bb, &cc);
            v3 o = sh[b - 1].x;
            double lever = 64.0 * u32 * (h->t + vlen(vsub(o, a)) + vlen(o)) / fabs(det);
            double du = lever * vlen(r0), dv = lever * vlen(r1);
            double dfx = s->tw * (fabs(uv[2] - uv[0]) * du + fabs(uv[4] - uv[0]) * dv);
            double dfy = s->th * (fabs(uv[3] - uv[1]) * du + fabs(uv[5] - uv[1]) * dv);
            double dw = dfx + dfy;
            int reach[16];
            int nr = taps_reach(&h->tp, dfx, dfy, reach);
            for (int k = 0; k < nr; ++k) {
                int i = reach[k];
                for (int ch = 0; ch < 3; ++ch) sp_add(sp, GB_ALB_S, 3 * (int64_t)i + ch, dw * fabs(gm[ch]));
                sp_add(sp, GB_RGH_S, i, dw * fabs(gm[3]));
                sp_add(sp, GB_MET_S, i, dw * fabs(gm[4]));
            }
        }
        for (int k = 0; k < 4; ++k) {
            int i = h->tp.idx[k];
            double w = h->tp.w[k];
            for (int ch = 0; ch < 3; ++ch) sp_add(sp, GB_ALB, 3 * (int64_t)i + ch, w * gm[ch]);
            sp_add(sp, GB_RGH, i, w * gm[3]);
            sp_add(sp, GB_MET, i, w * gm[4]);
        }
    }
}

/* the material of a fixed surface point re-fetched from the textures of `ev` */
static void refetch_material(const orc_scene* ev, Shade* sh)
{
    sh->alb[0] = sh->alb[1] = sh->alb[2] = sh->rgh = sh->met = 0.0;
    for (int k = 0; k < 4; ++k) {
        int i = sh->tp.idx[k];
        double w = sh->tp.w[k];
        for (int ch = 0; ch < 3; ++ch) sh->alb[ch] += w * ev->alb[3 * i + ch];
        sh->rgh += w * ev->rgh[i];
        sh->met += w * ev->met[i];
    }
}

/* FULL mode detached evaluation: the light arriving at the primary vertex along wc_0 (Lin_0),
 * re-evaluated with the materials and env of `ev` at the recorded vertices b >= 1 */
static void detached_lin0(const Ctx* c, const orc_scene* ev, const Rec* rec, double lin0[3])
{
    const int kind = c->p->brdf_kind;
    const int nv = rec->nv;
    double lin[3] = {0, 0, 0};
    for (int b = nv - 1; b >= 1; --b) {
        Shade sh;
        shade_at(c->s, rec->vx[b].tri, rec->vx[b].u, rec->vx[b].v, rec->vx[b].t, rec->vx[b].d, &sh, NULL);
        refetch_material(ev, &sh);
        v3 wo = vscale(rec->vx[b].d, -1.0);
        double nl[3] = {0, 0, 0}, f[3];
        if (rec->vx[b].sel >= 0 && rec->vx[b].WV != 0.0) {
            brdf_cos(sh.n, wo, rec->vx[b].y, sh.alb, sh.rgh, sh.met, kind, f);
            for (int k = 0; k < 3; ++k) nl[k] += rec->vx[b].WV * ev->env[3 * rec->vx[b].y_texel + k] * f[k];
        }
        if (rec->vx[b].has_cont) {
            brdf_cos(sh.n, wo, rec->vx[b].wc, sh.alb, sh.rgh, sh.met, kind, f);
            for (int k = 0; k < 3; ++k) nl[k] += f[k] / rec->vx[b].p_ind * lin[k];
        }
        for (int k = 0; k < 3; ++k) lin[k] = nl[k];
    }
    for (int k = 0; k < 3; ++k) lin0[k] = lin[k];
}

/* detached evaluation of one sample's primary-vertex terms with the parameters of `ev` */
/* demod = 1: the demodulated lighting at the primary vertex instead (kind-2 lobes, L_ind
 * detached in either grad mode, nothing for an escaping primary ray) */
static void sample_detached(const Ctx* c, const orc_scene* ev, const Rec* rec, int demod, double out[3])
{
    const int kind = demod ? 2 : c->p->brdf_kind;
    if (rec->prim_tri < 0) {
        for (int k = 0; k < 3; ++k) out[k] = demod ? 0.0 : ev->env[3 * rec->bg_texel + k];
        return;
    }
    v3 o = vload(c->o);
    double t, u, v;
    out[0] = out[1] = out[2] = 0.0;
    if (!tri_solve(ev, rec->prim_tri, o, rec->d0, &t, &u, &v, NULL)) return;
    Shade sh;
    shade_at(ev, rec->prim_tri, u, v, t, rec->d0, &sh, NULL);
    v3 wo = vscale(rec->d0, -1.0);
    if (rec->sel >= 0 && rec->WV != 0.0) {
        double fc[3];
        brdf_cos(sh.n, wo, rec->y, sh.alb, sh.rgh, sh.met, kind, fc);
        for (int k = 0; k < 3; ++k) out[k] += rec->WV * ev->env[3 * rec->y_texel + k] * fc[k];
    }
    if (rec->has_cont) {
        double fc[3], lin[3] = {rec->Lind[0], rec->Lind[1], rec->Lind[2]};
        if (c->p->grad_mode == 1 && !demod) detached_lin0(c, ev, rec, lin);
        brdf_cos(sh.n, wo, rec->wc, sh.alb, sh.rgh, sh.met, kind, fc);
        for (int k = 0; k < 3; ++k) out[k] += fc[k] / rec->p_ind * lin[k];
    }
}

/* ---------------------------------------------------------------------------------------
 * pixel loops, threaded over contiguous chunks of the pixel list
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int mode;  /* 0 render, 1 backward, 2 detached */
    int demod; /* 1: the demodulated lighting of the primary vertex (L_light) instead of the
                * radiance; mode 0 then writes [c_d + c_s (3), fraction of samples that hit] */
    int vsens; /* mode 1: also the FP32 sensitivity of the vertex terms */
    Ctx c;
    const orc_scene* ev;
    const int32_t* pixels;
    int32_t i0, i1;
    double* out_rgb; double* out_margin; int32_t* out_prim;
    double* out_srgb; double* out_smargin; /* per sample: radiance [n][spp][3], margin [n][spp] */
    double* out_ssens;                     /* per sample: FP32 sensitivity of the radiance [n][spp] */
    const double* d_rgb;
    Sparse sp;
    int64_t cnt[ORC_NCOUNT];
} Job;

static void* job_run(void* arg)
{
    Job* jb = (Job*)arg;
    const Ctx* c = &jb->c;
    const int W = c->v->width, spp = c->v->spp;
    for (int i = jb->i0; i < jb->i1; ++i) {
        int pix = jb->pixels ? jb->pixels[i] : i;
        int px = pix % W, py = pix / W;
        double acc[3] = {0, 0, 0}, hits = 0.0;
        Margin mg = {INFINITY, 0};
        Margin* pmg = (jb->mode == 0 && jb->out_margin && c->p->want_margin) ? &mg : NULL;
        for (int smp = 0; smp < spp; ++smp) {
            Rec rec;
            Margin smg = {INFINITY, 0};
            path_sample(c, px, py, smp, &rec, pmg ? &smg : NULL, jb->cnt);
            if (pmg && smg.m < mg.m) mg = smg;
            if (jb->mode == 0 && !jb->demod && jb->out_srgb) {
                for (int k = 0; k < 3; ++k) jb->out_srgb[3 * ((size_t)i * spp + smp) + k] = rec.rgb[k];
                if (jb->out_smargin) jb->out_smargin[(size_t)i * spp + smp] = pmg ? smg.m : INFINITY;
                if (jb->out_ssens) jb->out_ssens[(size_t)i * spp + smp] = rec.sens + path_hit_sens(c, &rec);
            }
            if (jb->mode == 0 && jb->demod) {
                double o3[3];
                sample_detached(c, c->s, &rec, 1, o3);
                for (int k = 0; k < 3; ++k) acc[k] += o3[k];
                hits += rec.prim_tri >= 0 ? 1.0 : 0.0;
            } else if (jb->mode == 0) {
                for (int k = 0; k < 3; ++k) acc[k] += rec.rgb[k];
                if (jb->out_prim) jb->out_prim[(size_t)i * spp + smp] = rec.prim_tri;
            } else if (jb->mode == 1) {
                double g[3];
                for (int k = 0; k < 3; ++k) g[k] = jb->d_rgb[3 * (size_t)i + k] / spp;
                if (g[0] != 0.0 || g[1] != 0.0 || g[2] != 0.0) {
                    sample_grad(c, &rec, g, jb->demod, jb->vsens, &jb->sp);
                    if (c->p->grad_mode == 1) sample_grad_secondary(c, &rec, g, &jb->sp);
                }
            } else {
                double o3[3];
                sample_detached(c, jb->ev, &rec, jb->demod, o3);
                for (int k = 0; k < 3; ++k) acc[k] += o3[k];
            }
        }
        if (jb->mode == 0 && jb->demod) {
            for (int k = 0; k < 3; ++k) jb->out_rgb[4 * (size_t)i + k] = acc[k] / spp;
            jb->out_rgb[4 * (size_t)i + 3] = hits / spp;
        } else if (jb->mode != 1)
            for (int k = 0; k < 3; ++k) jb->out_rgb[3 * (size_t)i + k] = acc[k] / spp;
        if (jb->mode == 0 && jb->out_margin) {
            jb->out_margin[2 * (size_t)i] = mg.m;
            jb->out_margin[2 * (size_t)i + 1] = (double)mg.kind;
        }
    }
    return NULL;
}

static int run_jobs(int mode, int demod, const orc_scene* s, const orc_scene* ev, const orc_view* v,
                    const orc_params* p, const int32_t* pixels, int32_t n, double* out_rgb, double* out_margin,
                    int32_t* out_prim, const double* d_rgb, const orc_grads* g, int64_t* counts,
                    double* out_srgb, double* out_smargin, double* out_ssens)
{
    if (demod && p && p->grad_mode != 0) return 1;
    if (!s || !v || !p || v->width < 1 || v->height < 1 || v->spp < 1 || v->bounces < 1 || p->ris_m < 0) return 1;
    if (p->grad_mode != 0 && (p->grad_mode != 1 || v->bounces > ORC_MAXB)) return 1;
    if (p->reuse_k < 0 || p->reuse_radius < 0 || (p->reuse_k > 0 && p->reuse_radius < 1)) return 1;
    if (p->temporal < 0 || p->temporal > 2 || (p->temporal == 2 && (!p->history_in || p->temporal_cap < 1))) return 1;
    if (!pixels) n = v->width * v->height;
    for (int i = 0; pixels && i < n; ++i)
        if (pixels[i] < 0 || pixels[i] >= v->width * v->height) return 1;
    int nt = p->threads < 1 ? 1 : p->threads;
    if (nt > n) nt = n > 0 ? n : 1;
    Job* jobs = (Job*)calloc((size_t)nt, sizeof(Job));
    pthread_t* th = (pthread_t*)calloc((size_t)nt, sizeof(pthread_t));
    for (int t = 0; t < nt; ++t) {
        Job* jb = &jobs[t];
        jb->mode = mode;
        jb->demod = demod;
        jb->vsens = (mode == 1 && g && g->verts_sens) ? 1 : 0;
        ctx_init(&jb->c, s, v, p);
        jb->ev = ev;
        jb->pixels = pixels;
        jb->i0 = (int32_t)((int64_t)n * t / nt);
        jb->i1 = (int32_t)((int64_t)n * (t + 1) / nt);
        jb->out_rgb = out_rgb; jb->out_margin = out_margin; jb->out_prim = out_prim;
        jb->out_srgb = out_srgb; jb->out_smargin = out_smargin; jb->out_ssens = out_ssens;
        jb->c.want_sens = out_ssens != NULL;
        jb->d_rgb = d_rgb;
    }
    if (nt == 1) job_run(&jobs[0]);
    else {
        for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, job_run, &jobs[t]);
        for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    }
    for (int t = 0; t < nt; ++t) {
        if (counts) for (int k = 0; k < ORC_NCOUNT; ++k) counts[k] += jobs[t].cnt[k];
        if (mode == 1 && g) {
            double* dst[GB_N] = {g->albedo, g->roughness, g->metallic, g->env, g->verts,
                                 g->albedo_sens, g->roughness_sens, g->metallic_sens, g->verts_sens};
            double* dab[GB_N] = {g->albedo_abs, g->roughness_abs, g->metallic_abs, g->env_abs, g->verts_abs,
                                 NULL, NULL, NULL, NULL};
            for (size_t e = 0; e < jobs[t].sp.n; ++e) {
                const Entry* en = &jobs[t].sp.e[e];
                if (dst[en->buf]) dst[en->buf][en->idx] += en->val;
                if (dab[en->buf]) dab[en->buf][en->idx] += fabs(en->val);
            }
        }
        free(jobs[t].sp.e);
    }
    free(jobs);
    free(th);
    return 0;
}

int orc_render_samples(const orc_scene* s, const orc_view* v, const orc_params* p, const int32_t* pixels,
                       int32_t n_pixels, double* out_rgb, double* out_margin, double* out_sample_rgb,
                       double* out_sample_margin, double* out_sample_sens, int64_t* counts)
{
    if (!out_rgb || !out_sample_rgb) return 1;
    return run_jobs(0, 0, s, NULL, v, p, pixels, n_pixels, out_rgb, out_margin, NULL, NULL, NULL, counts,
                    out_sample_rgb, out_sample_margin, out_sample_sens);
}

/* one sample's record (for comparisons word by word): out[0] primary triangle, [1] selected
 * candidate, [2] V W, [3..5] L_ind, [6..8] radiance, [9] env texel of the selection, [10..12]
 * its direction, [13..15] the continuation direction, [16] its pdf (0: none), [17] vertices
 * recorded; then per vertex b < ORC_MAXB 12 values: triangle, u, v, selected candidate, texel,
 * V W, continuation direction (3), its pdf, has continuation, t */
int orc_sample_record(const orc_scene* s, const orc_view* v, const orc_params* p, int32_t px, int32_t py,
                      int32_t smp, double* out)
{
    if (!s || !v || !p || !out || px < 0 || py < 0 || px >= v->width || py >= v->height || smp < 0 ||
        smp >= v->spp)
        return 1;
    Ctx c;
    ctx_init(&c, s, v, p);
    Rec rec;
    path_sample(&c, px, py, smp, &rec, NULL, NULL);
    out[0] = rec.prim_tri; out[1] = rec.sel; out[2] = rec.WV;
    for (int k = 0; k < 3; ++k) { out[3 + k] = rec.Lind[k]; out[6 + k] = rec.rgb[k]; }
    out[9] = rec.y_texel; out[10] = rec.y.x; out[11] = rec.y.y; out[12] = rec.y.z;
    out[13] = rec.wc.x; out[14] = rec.wc.y; out[15] = rec.wc.z; out[16] = rec.has_cont ? rec.p_ind : 0.0;
    out[17] = rec.nv;
    for (int b = 0; b < rec.nv && b < ORC_MAXB; ++b) {
        double* o = out + 18 + 12 * b;
        o[0] = rec.vx[b].tri; o[1] = rec.vx[b].u; o[2] = rec.vx[b].v; o[3] = rec.vx[b].sel;
        o[4] = rec.vx[b].y_texel; o[5] = rec.vx[b].WV; o[6] = rec.vx[b].wc.x; o[7] = rec.vx[b].wc.y;
        o[8] = rec.vx[b].wc.z; o[9] = rec.vx[b].p_ind; o[10] = rec.vx[b].has_cont; o[11] = rec.vx[b].t;
    }
    return 0;
}

int orc_render(const orc_scene* s, const orc_view* v, const orc_params* p, const int32_t* pixels, int32_t n_pixels,
               double* out_rgb, double* out_margin, int32_t* out_prim_tri, int64_t* counts)
{
    if (!out_rgb) return 1;
    return run_jobs(0, 0, s, NULL, v, p, pixels, n_pixels, out_rgb, out_margin, out_prim_tri, NULL, NULL, counts, NULL, NULL, NULL);
}

int orc_backward(const orc_scene* s, const orc_view* v, const orc_params* p, const int32_t* pixels, int32_t n_pixels,
                 const double* d_rgb, const orc_grads* g, int64_t* counts)
{
    if (!d_rgb || !g) return 1;
    return run_jobs(1, 0, s, NULL, v, p, pixels, n_pixels, NULL, NULL, NULL, d_rgb, g, counts, NULL, NULL, NULL);
}

int orc_render_detached(const orc_scene* frozen, const orc_scene* eval, const orc_view* v, const orc_params* p,
                        const int32_t* pixels, int32_t n_pixels, double* out_rgb)
{
    if (!eval || !out_rgb) return 1;
    return run_jobs(2, 0, frozen, eval, v, p, pixels, n_pixels, out_rgb, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
}

/* ---------------------------------------------------------------------------------------
 * monochrome light regulariser (Appendix A, L_light): the demodulated diffuse and specular
 * lighting c_d + c_s of each pixel's primary vertex, estimated from the same samples as the
 * render (kind-2 lobes in place of the BRDF in the primary vertex's direct and continuation
 * terms), and the adjoint of its PRIMARY-mode dependence on the parameters
 * ------------------------------------------------------------------------------------- */
int orc_light_demod(const orc_scene* s, const orc_view* v, const orc_params* p, const int32_t* pixels,
                    int32_t n_pixels, double* out, double* out_margin, int64_t* counts)
{
    if (!out) return 1;
    return run_jobs(0, 1, s, NULL, v, p, pixels, n_pixels, out, out_margin, NULL, NULL, NULL, counts, NULL, NULL, NULL);
}

int orc_light_backward(const orc_scene* s, const orc_view* v, const orc_params* p, const int32_t* pixels,
                       int32_t n_pixels, const double* d_c, const orc_grads* g, int64_t* counts)
{
    if (!d_c || !g) return 1;
    return run_jobs(1, 1, s, NULL, v, p, pixels, n_pixels, NULL, NULL, NULL, d_c, g, counts, NULL, NULL, NULL);
}

int orc_light_demod_detached(const orc_scene* frozen, const orc_scene* eval, const orc_view* v,
                             const orc_params* p, const int32_t* pixels, int32_t n_pixels, double* out)
{
    if (!eval || !out) return 1;
    return run_jobs(2, 1, frozen, eval, v, p, pixels, n_pixels, out, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
}

/* ---------------------------------------------------------------------------------------
 * LBVH (Appendix A: a linear BVH after Karras 2012), restated top-down for comparison.
 * Morton codes of the triangle centroids in the centroid bounding box (10 bits per axis,
 * x in the highest position of each triple), key = code << 32 | triangle id, sorted.
 * The binary radix tree over the sorted keys: a node covering [first, last] splits after
 * the last key that shares more leading bits with keys[first] than keys[last] does; its
 * children are numbered by the split position (left = g, right = g + 1), which is the
 * numbering Karras's bottom-up construction produces.
 * ------------------------------------------------------------------------------------- */
static uint32_t spread10(uint32_t v)
{
    uint32_t r = 0;
    for (int b = 0; b < 10; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

static int clz64(uint64_t x) { return x ? __builtin_clzll(x) : 64; }

static int cmp_u64(const void* a, const void* b)
{
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

typedef struct { const uint64_t* k; int32_t* left; int32_t* right; int32_t* parent; int n; } Lb;

static void lb_node(Lb* L, int first, int last, int idx)
{
    int dnode = clz64(L->k[first] ^ L->k[last]);
    int g = first;
    for (int i = first; i < last; ++i)
        if (clz64(L->k[first] ^ L->k[i]) > dnode) g = i;
    if (g == first) { L->left[idx] = ~g; L->parent[(L->n - 1) + g] = idx; }
    else { L->left[idx] = g; L->parent[g] = idx; lb_node(L, first, g, g); }
    if (g + 1 == last) { L->right[idx] = ~(g + 1); L->parent[(L->n - 1) + g + 1] = idx; }
    else { L->right[idx] = g + 1; L->parent[g + 1] = idx; lb_node(L, g + 1, last, g + 1); }
}

static void lb_box(int node, int n, const int32_t* left, const int32_t* right, float* lo, float* hi)
{
    int ch[2] = {left[node], right[node]};
    for (int c = 0; c < 2; ++c) if (ch[c] >= 0) lb_box(ch[c], n, left, right, lo, hi);
    for (int k = 0; k < 3; ++k) {
        int a = ch[0] >= 0 ? ch[0] : (n - 1) + ~ch[0];
        int b = ch[1] >= 0 ? ch[1] : (n - 1) + ~ch[1];
        lo[3 * node + k] = fminf(lo[3 * a + k], lo[3 * b + k]);
        hi[3 * node + k] = fmaxf(hi[3 * a + k], hi[3 * b + k]);
    }
}

int orc_lbvh(const float* verts, const int32_t* tris, int32_t n, uint64_t* keys, int32_t* left, int32_t* right,
             int32_t* parent, float* lo, float* hi)
{
    if (n <= 0) return 0;
    float* cen = (float*)malloc(sizeof(float) * 3 * (size_t)n);
    float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const float third = 1.0f / 3.0f;
    for (int t = 0; t < n; ++t)
        for (int k = 0; k < 3; ++k) {
            float a = verts[3 * tris[3 * t] + k], b = verts[3 * tris[3 * t + 1] + k], c = verts[3 * tris[3 * t + 2] + k];
            float s = a + b;
            s = s + c;
            float m = s * third;
            cen[3 * t + k] = m;
            if (m < clo[k]) clo[k] = m;
            if (m > chi[k]) chi[k] = m;
        }
    for (int t = 0; t < n; ++t) {
        uint32_t q[3];
        for (int k = 0; k < 3; ++k) {
            float ext = chi[k] - clo[k];
            float f = 0.0f;
            if (ext > 0.0f) {
                float num = cen[3 * t + k] - clo[k];
                float r = num / ext;
                f = r * 1024.0f;
            }
            float fl = floorf(f);
            int qi = (int)fl;
            if (qi < 0) qi = 0;
            if (qi > 1023) qi = 1023;
            q[k] = (uint32_t)qi;
        }
        uint32_t code = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
        keys[t] = ((uint64_t)code << 32) | (uint32_t)t;
    }
    qsort(keys, (size_t)n, sizeof(uint64_t), cmp_u64);
    for (int i = 0; i < 2 * n - 1; ++i) parent[i] = -1;
    /* leaf boxes: exact min / max of the three vertices */
    for (int i = 0; i < n; ++i) {
        int t = (int)(uint32_t)keys[i];
        for (int k = 0; k < 3; ++k) {
            float a = verts[3 * tris[3 * t] + k], b = verts[3 * tris[3 * t + 1] + k], c = verts[3 * tris[3 * t + 2] + k];
            lo[3 * ((n - 1) + i) + k] = fminf(fminf(a, b), c);
            hi[3 * ((n - 1) + i) + k] = fmaxf(fmaxf(a, b), c);
        }
    }
    if (n >= 2) {
        Lb L = {keys, left, right, parent, n};
        lb_node(&L, 0, n - 1, 0);
        lb_box(0, n, left, right, lo, hi);
    }
    free(cen);
    return 0;
}
