// path.cuh -- per-path device code shared by the plain wavefront, the batched wavefront and
// the persistent kernels: the tape layout, one shading vertex (RIS + shadow ray + continuation)
// and warp-aggregated queue appends.
#pragma once

#include "../../include/mirres.h"
#include "device.cuh"

namespace {

constexpr int kCandUnroll = MR_CAND_UNROLL;

// The tape: TAPE_WORDS 32-bit words per path sample, structure of arrays over the samples.
// It holds what the PRIMARY-mode adjoint needs to replay the primary vertex without
// re-drawing any sample: the hit triangle, the RIS selection, the continuation and the
// radiance the rest of the path brought back.
enum { TAPE_WORDS = MIRRES_TAPE_BYTES_PER_SAMPLE / 4 };
static_assert(TAPE_WORDS == 17, "tape_of lays out 17 words");

struct TapeDev {
    int32_t* tri;    // primary triangle, -1 when the primary ray escaped
    int32_t* cand;   // index of the selected RIS candidate at the primary vertex, -1 if none
    float* wv;       // V * W of that candidate (0 when occluded)
    float* lind[3];  // L_ind arriving at the primary vertex along the continuation
    float* rad[3];   // radiance of the whole sample
    int32_t* ytex;   // env texel of the selected candidate (valid when cand >= 0)
    float* y[3];     // its direction (valid when cand >= 0)
    float* wc[3];    // continuation direction at the primary vertex (valid when L_ind != 0)
    float* pind;     // its mixture pdf (valid when L_ind != 0)
    // FULL-mode vertex records of vertices 1 .. nvx, VX_WORDS words each, after the primary
    // words: vx[((b - 1) * VX_WORDS + w) * n + g]; nvx = 0 in PRIMARY mode
    uint32_t* vx;
    int nvx;
    uint64_t n;
};

// words of a FULL-mode vertex record: hit triangle (-1: the path never reached the vertex),
// barycentrics, selected RIS candidate (-1: none), V * W, continuation direction and pdf
// (0: the path ended here)
enum { VX_TRI = 0, VX_U, VX_V, VX_CAND, VX_WV, VX_WC, VX_P = VX_WC + 3, VX_WORDS };

__device__ __forceinline__ uint32_t* vx_at(const TapeDev& t, int b, int w, uint64_t g)
{
    return t.vx + ((uint64_t)(b - 1) * VX_WORDS + (uint64_t)w) * t.n + g;
}

__device__ __forceinline__ TapeDev tape_of(void* base, uint64_t n, int nvx = 0)
{
    TapeDev t;
    t.n = n;
    t.nvx = nvx;
    t.vx = reinterpret_cast<uint32_t*>(base) + (uint64_t)TAPE_WORDS * n;
    uint32_t* w = reinterpret_cast<uint32_t*>(base);
    t.tri = reinterpret_cast<int32_t*>(w);
    t.cand = reinterpret_cast<int32_t*>(w + n);
    t.wv = reinterpret_cast<float*>(w + 2 * n);
    for (int k = 0; k < 3; ++k) t.lind[k] = reinterpret_cast<float*>(w + (3 + k) * n);
    for (int k = 0; k < 3; ++k) t.rad[k] = reinterpret_cast<float*>(w + (6 + k) * n);
    t.ytex = reinterpret_cast<int32_t*>(w + 9 * n);
    for (int k = 0; k < 3; ++k) t.y[k] = reinterpret_cast<float*>(w + (10 + k) * n);
    for (int k = 0; k < 3; ++k) t.wc[k] = reinterpret_cast<float*>(w + (13 + k) * n);
    t.pind = reinterpret_cast<float*>(w + 16 * n);
    return t;
}

// ---------------------------------------------------------------------------------------
// one shading vertex: RIS over M env candidates (Eq. restir, streamed through a weighted
// reservoir), the shadow ray that tests the selected candidate, and the continuation ray
// drawn from the MIS mixture (Eq. mc_indir). Shared by the wavefront and persistent kernels.
// ---------------------------------------------------------------------------------------
struct VertexOut {
    bool shadow;
    float3 sh_o, sh_d;
    float3 add_rad, add_lind;
    bool cont;
    float3 c_d, c_beta, c_bind;
    float3 x;
    int cand, ytex;
    float W, c_pind;
    // the vertex's RIS reservoir (for spatial reuse): selected candidate's sub-texel word,
    // weight sum and target p_hat of the selection
    uint32_t ysub;
    float wsum, phat;
};

// FULL mode: no later vertex reached yet (written when the sample starts)
__device__ __forceinline__ void tape_vx_init(const TapeDev& tp, uint64_t g)
{
    for (int b = 1; b <= tp.nvx; ++b) *vx_at(tp, b, VX_TRI, g) = 0xFFFFFFFFu;
}

// FULL mode: the record of vertex b >= 1 (V * W is cleared later if the shadow ray is blocked)
__device__ __forceinline__ void tape_vx_record(const TapeDev& tp, uint64_t g, int b, const Hit& h,
                                               const VertexOut& out)
{
    if (b < 1 || b > tp.nvx) return;
    *vx_at(tp, b, VX_TRI, g) = (uint32_t)h.tri;
    *vx_at(tp, b, VX_U, g) = __float_as_uint(h.u);
    *vx_at(tp, b, VX_V, g) = __float_as_uint(h.v);
    *vx_at(tp, b, VX_CAND, g) = (uint32_t)out.cand;
    *vx_at(tp, b, VX_WV, g) = __float_as_uint(out.W);
    *vx_at(tp, b, VX_WC, g) = __float_as_uint(out.c_d.x);
    *vx_at(tp, b, VX_WC + 1, g) = __float_as_uint(out.c_d.y);
    *vx_at(tp, b, VX_WC + 2, g) = __float_as_uint(out.c_d.z);
    *vx_at(tp, b, VX_P, g) = __float_as_uint(out.c_pind);
}

__device__ __forceinline__ void tape_vx_occluded(const TapeDev& tp, uint64_t g, int b)
{
    if (b >= 1 && b <= tp.nvx) *vx_at(tp, b, VX_WV, g) = 0u;
}

// the directions the primary vertex drew, for the adjoint's replay (written at bounce 0)
__device__ __forceinline__ void tape_directions(const TapeDev& tp, uint64_t g, const VertexOut& out)
{
    tp.ytex[g] = out.ytex;
    tp.y[0][g] = out.sh_d.x;
    tp.y[1][g] = out.sh_d.y;
    tp.y[2][g] = out.sh_d.z;
    tp.wc[0][g] = out.c_d.x;
    tp.wc[1][g] = out.c_d.y;
    tp.wc[2][g] = out.c_d.z;
    tp.pind[g] = out.c_pind;
}

template <bool INTERP = true>
__device__ __forceinline__ void shade_vertex(const SceneDev& s, int env_ok, const Rng& rng, uint32_t pixel,
                                             uint32_t smp, uint32_t view, int b, int B, int M, const Hit& h,
                                             float3 d, float3 beta, float3 bind, VertexOut& out)
{
    Shade sh;
    shade_at<INTERP>(s, h.tri, h.u, h.v, d, sh);
    const float3 wo = f3(-d.x, -d.y, -d.z);
    out.x = sh.x;
    out.shadow = false;
    out.cont = false;
    out.cand = -1;
    out.ytex = -1;
    out.W = 0.0f;
    out.ysub = 0u;
    out.wsum = 0.0f;
    out.phat = 0.0f;
    out.c_pind = 0.0f;
    out.sh_d = f3(0.f, 0.f, 0.f);
    out.c_d = f3(0.f, 0.f, 0.f);
    if (env_ok && M > 0) {
        // per-vertex parts of the BRDF: the candidates need only the luminance of f_r cos
        // (p_hat = Y(L_env) Y(f_r) cos); the selected one's RGB is rebuilt after the loop
        const float co = dot(sh.n, wo);
        const float a = alpha_of(sh.m.rough), a2 = a * a;
        const float Ao = smith_a(a2, co);
        const float3 kd = mul(sh.m.alb, 1.0f - sh.m.metal);
        const float3 f0 = f3(0.04f * (1.0f - sh.m.metal) + sh.m.metal * sh.m.alb.x,
                             0.04f * (1.0f - sh.m.metal) + sh.m.metal * sh.m.alb.y,
                             0.04f * (1.0f - sh.m.metal) + sh.m.metal * sh.m.alb.z);
        const float ykd = lum(kd) * MR_INV_PI, yf0 = lum(f0);
        float wsum = 0.0f, yfc_sel = 0.0f;
        float dv_sel = 0.0f, w5_sel = 0.0f, ci_sel = 0.0f;
        int sel = -1, ytex = 0;
        uint32_t ysub = 0u;
        float3 ysel = f3(0.f, 0.f, 0.f);
        // candidate j with direction dir, texel tex and gq = Y(L_env) / q_dir into the reservoir
        auto consider = [&](int j, const uint4& x, float3 dir, int tex, float gq) {
            const float ci = dot(sh.n, dir);
            float yfc = 0.0f, dv = 0.0f, w5 = 0.0f;
            if (co > 0.0f && ci > 0.0f && above_face(sh, dir)) {
                const float3 h = normalize(add(wo, dir));
                const float cnh = dot(sh.n, h), coh = dot(wo, h);
                const float k = ggx_k(sh.n, h, cnh, a2);
                const float D = __fdividef(a2, MR_PI * k * k);
                dv = D * __fdividef(0.5f, ci * Ao + co * smith_a(a2, ci));
                const float om = 1.0f - coh;
                w5 = (om * om) * (om * om) * om;
                yfc = (ykd + dv * (yf0 * (1.0f - w5) + w5)) * ci;  // Y(f_r) cos
            }
            const float gamma = yfc * gq;  // gamma = p_hat / q_dir, p_hat = Y(L_env) Y(f_r) cos
            wsum += gamma;
            if (u24(x.z) * wsum < gamma) {
                sel = j;
                ytex = tex;
                ysub = x.w;
                ysel = dir;
                yfc_sel = yfc;
                dv_sel = dv;
                w5_sel = w5;
                ci_sel = ci;
            }
        };
        int j = 0;
#if MR_CAND_PAIR
        // two candidates per round: both env searches and row loads in flight together, then
        // the reservoir takes them in order (the same arithmetic as one at a time)
        for (; j + 1 < M; j += 2) {
            const uint4 x0 = rng.draw(pixel, smp, view, (uint32_t)b, PURPOSE_CANDIDATE, (uint32_t)j);
            const uint4 x1 = rng.draw(pixel, smp, view, (uint32_t)b, PURPOSE_CANDIDATE, (uint32_t)(j + 1));
            int r0, c0, r1, c1;
            env_texel_draw2(s, x0.x, x0.y, x1.x, x1.y, r0, c0, r1, c1);
            float3 d0, d1;
            float4 rv0, rv1;
            const float st0 = env_dir(s, r0, c0, x0.w, d0, rv0);
            const float st1 = env_dir(s, r1, c1, x1.w, d1, rv1);
            consider(j, x0, d0, r0 * s.ew + c0, st0 * rv0.z);
            consider(j + 1, x1, d1, r1 * s.ew + c1, st1 * rv1.z);
        }
#endif
#pragma unroll kCandUnroll
        for (; j < M; ++j) {
            const uint4 x = rng.draw(pixel, smp, view, (uint32_t)b, PURPOSE_CANDIDATE, (uint32_t)j);
            float3 dir;
            int tex;
            const float gq = env_candidate(s, x.x, x.y, x.w, dir, tex);
            consider(j, x, dir, tex, gq);
        }
        const float4 L = (sel >= 0) ? __ldg(s.env_texel + ytex) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float phat_sel = lum(xyz(L)) * yfc_sel;
        out.wsum = wsum;
        out.phat = phat_sel;
        out.ysub = ysub;
        if (sel >= 0 && wsum > 0.0f && phat_sel > 0.0f) {
            const float W = wsum / ((float)M * phat_sel);
            const float3 fsel = f3((kd.x * MR_INV_PI + dv_sel * (f0.x * (1.0f - w5_sel) + w5_sel)) * ci_sel,
                                   (kd.y * MR_INV_PI + dv_sel * (f0.y * (1.0f - w5_sel) + w5_sel)) * ci_sel,
                                   (kd.z * MR_INV_PI + dv_sel * (f0.z * (1.0f - w5_sel) + w5_sel)) * ci_sel);
            const float3 contrib = mul(hmul(xyz(L), fsel), W);
            out.add_rad = hmul_rn(beta, contrib);
            out.add_lind = (b >= 1) ? hmul_rn(bind, contrib) : f3(0.f, 0.f, 0.f);
            out.shadow = true;
            out.sh_o = sh.x;
            out.sh_d = ysel;
            out.cand = sel;
            out.ytex = ytex;
            out.W = W;
        }
    }
    if (b < B - 1) {
        const uint4 x = rng.draw(pixel, smp, view, (uint32_t)b, PURPOSE_CONTINUE, 0u);
        float3 wc;
        const float pind = sample_continuation(s, env_ok, sh.n, wo, sh.m, x, wc);
        const float3 fc = brdf_cos(sh.n, wo, wc, sh.m);
        if (pind > 0.0f && (fc.x > 0.0f || fc.y > 0.0f || fc.z > 0.0f) && above_face(sh, wc)) {
            const float3 f = f3(fc.x / pind, fc.y / pind, fc.z / pind);
            out.cont = true;
            out.c_d = wc;
            out.c_pind = pind;
            out.c_beta = hmul_rn(beta, f);
            out.c_bind = (b >= 1) ? hmul_rn(bind, f) : bind;
        }
    }
}

__device__ __forceinline__ const ViewDev& view_of(const ViewDev* views, int n, uint64_t g, int& vi)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].offset <= g) lo = mid;
        else hi = mid - 1;
    }
    vi = lo;
    return views[lo];
}


// warp-aggregated append: returns the slot of this lane (valid only if want)
__device__ __forceinline__ unsigned int warp_append(bool want, unsigned int* counter)
{
    const unsigned m = __ballot_sync(MR_FULL, want);
    if (!m) return 0u;
    const int leader = __ffs(m) - 1;
    unsigned int base = 0;
    if (lane_id() == leader) base = atomicAdd(counter, (unsigned)__popc(m));
    base = __shfl_sync(MR_FULL, base, leader);
    return base + __popc(m & lanemask_lt());
}

}  // namespace
