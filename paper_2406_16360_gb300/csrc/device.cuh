// device.cuh -- sm_103a device code shared by the kernels of the MIRReS hot path.
//
// FP32 throughout (FP64 only in the env CDF build). Everything here is __forceinline__ so
// that each translation unit is self-contained (no relocatable device code).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define MR_PI 3.14159265358979323846f
#define MR_INV_PI 0.31830988618379067154f
#define MR_FULL 0xffffffffu

// launch tuning knobs (overridable with -D at build time): minimum resident blocks of 256
// threads per SM for the shading, adjoint and traversal kernels, and the RIS candidate loop's
// unroll
#ifndef MR_SHADE_MINB
#define MR_SHADE_MINB 4
#endif
#ifndef MR_BWD_MINB
#define MR_BWD_MINB 4
#endif
#ifndef MR_TRACE_MINB
#define MR_TRACE_MINB 0  // the batched closest-hit and shadow-ray kernels (0: no minimum)
#endif
#if MR_TRACE_MINB > 0
#define MR_TRACE_BOUNDS __launch_bounds__(256, MR_TRACE_MINB)
#else
#define MR_TRACE_BOUNDS __launch_bounds__(256)
#endif
#ifndef MR_REFILL
#define MR_REFILL 1  // batched wavefront: shadow rays traced by lane-refilling warps
#endif
#ifndef MR_REFILL_CLOSEST
#define MR_REFILL_CLOSEST 1  // ... and continuation rays (at 64 registers: 6-8% faster than k_wclosest)
#endif
#ifndef MR_DFS_NODES
#define MR_DFS_NODES 1  // traversal nodes in depth-first preorder (else the builders' order)
#endif
#ifndef MR_NODE_LD256
#define MR_NODE_LD256 1  // traversal nodes read with two 256-bit loads (2.5% faster traversal stages)
#endif
#ifndef MR_TRI_LD256
#define MR_TRI_LD256 0  // packed triangles padded to 64 bytes and read with two 256-bit loads
#endif
#define MR_TRI_STRIDE (MR_TRI_LD256 ? 4 : 3)  // float4 per packed triangle
#ifndef MR_CLOSEST_REFILL_MINB
#define MR_CLOSEST_REFILL_MINB 4  // its register cap: four 256-thread blocks per SM (64 registers)
#endif
#ifndef MR_REFILL_STEPS
#define MR_REFILL_STEPS 16  // node visits between refill checks
#endif
#ifndef MR_REFILL_MIN
#define MR_REFILL_MIN 8  // idle lanes that trigger a refill
#endif
#ifndef MR_CAND_UNROLL
#define MR_CAND_UNROLL 1
#endif
#ifndef MR_CAND_PAIR
#define MR_CAND_PAIR 1  // RIS candidates drawn two at a time (interleaved env searches)
#endif

// traversal stack: the first MR_SSTACK entries live in shared memory (column per thread),
// deeper entries in a small local array; an LBVH over 64-bit unique keys is at most 63 deep
// (a clustering tree deeper than the stack is not used)
#ifndef MR_SSTACK
#define MR_SSTACK 32
#endif
#define MR_LSTACK (64 - MR_SSTACK)
static_assert(MR_SSTACK >= 8 && MR_SSTACK <= 56, "MR_SSTACK out of range");
// the wide traversal's stack of 8-byte node groups: the first MR_SSTACK / 2 in the same shared
// memory column, the rest local; a wide tree is at most as deep as its binary tree (<= 63)
#define MR_WSSTACK (MR_SSTACK / 2)
#define MR_WLSTACK (64 - MR_WSSTACK)
// launches of the wide-BVH collapse (one per level of the wide tree)
#define MR_WIDE_LEVELS 64

// ---------------------------------------------------------------------------------------
// scene as seen by the kernels
// ---------------------------------------------------------------------------------------
struct SceneDev {
    const float4* nodes;      // [F-1][4]: (lmin.xyz, lmax.x) (lmax.yz, rmin.xy) (rmin.z, rmax.xyz) (l, r, -, -)
    const float4* ptri;       // [F][3] by leaf position: (v0, tri) (e1, 0) (e2, 0)
    const int32_t* leaf_of;   // [F] triangle -> leaf position
    const int32_t* tris;      // [F][3] caller's vertex indices
    const float* tri_uv;      // [F][3][2]
    const float* albedo;      // [th][tw][3]
    const float* rough;       // [th][tw]
    const float* metal;       // [th][tw]
    const float4* env_texel;  // [eh][ew]: (r, g, b, prob * ew * eh)
    const float4* env_row;    // [eh]: (cos th_r, sin th_r, 2 pi^2 total / (ew eh sin th_r), 0) at row centres
    const float2* env_col;    // [ew]: (cos psi_c, sin psi_c), psi = 2 pi u - pi at column centres
    int32_t env_fine;         // 1 when a texel spans at most pi/32 in both angles (tables used)
    const unsigned long long* env_flat; // [eh ew + 1] ceil(cdf 2^53) of the CDF over all texels
    const uint32_t* env_gflat;          // [gf + 1] guide: answer of the search at bucket starts
    int32_t gf_shift;
    int32_t n_tris, n_verts, tw, th, ew, eh;
    const int32_t* env_ok_dev; // device-written: total env weight > 0
    const float* tmin_dev;     // device-written: 1e-5 x scene diagonal
    // interpolated shading normals (null: face normals): unit area-weighted vertex normals,
    // and the adjoint's per-vertex accumulator of d loss / d vertex normal [V][3]
    const float4* vnrm;
    float* gvn;
    // failure detection: a traversal that reaches its iteration cap (trav_cap node visits, 0 =
    // 4 n_tris + 64) or overflows its stack ends as a miss and adds 1 to *err (the context's
    // error counter, read back by mirres_get_counters)
    unsigned long long* err;
    int32_t trav_cap;
    // the 8-wide BVH the traversal runs (null: the binary tree's traversal); see wbvh.cu
    const uint4* wnodes;   // [][5] 80-byte nodes
    const float4* wtri;    // [F][3] packed triangles in the wide leaves' order
};

// iteration cap of one traversal
__device__ __forceinline__ int trav_cap_of(const SceneDev& s)
{
    return s.trav_cap > 0 ? s.trav_cap : 4 * s.n_tris + 64;
}
__device__ __forceinline__ void trav_fail(const SceneDev& s)
{
    if (s.err) atomicAdd(s.err, 1ull);
}

struct ViewDev {
    float K[4];
    float c2w[12];
    int32_t width, height, spp, bounces;
    int32_t scene;
    int32_t index;            // the view's index in the call (enters the random counter)
    uint64_t offset;          // first global sample index of this view
};

// ---------------------------------------------------------------------------------------
// small vector algebra
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 add(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 sub(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 mul(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 hmul(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b)
{
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize(float3 a) { return mul(a, 1.0f / sqrtf(dot(a, a))); }
__device__ __forceinline__ float lum(float3 c) { return (c.x + c.y + c.z) * (1.0f / 3.0f); }
__device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }
// explicitly rounded operations at the boundaries between stages, so that a product formed
// in one kernel and summed in another rounds exactly like the fused persistent kernel
__device__ __forceinline__ float3 hmul_rn(float3 a, float3 b)
{
    return f3(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y), __fmul_rn(a.z, b.z));
}
__device__ __forceinline__ float3 add_rn(float3 a, float3 b)
{
    return f3(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z));
}

// ---------------------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon et al., SC'11)
// ---------------------------------------------------------------------------------------
enum { PURPOSE_CAMERA = 0, PURPOSE_CANDIDATE = 1, PURPOSE_CONTINUE = 2, PURPOSE_REUSE = 3, PURPOSE_SMOOTH = 4 };

// The key schedule (k += Weyl constants each round) depends on the seed only, so the ten round
// keys are computed once on the host and travel in the kernel parameters, where each round
// reads its keys as constant operands.
struct Rng {
    uint32_t rk0[10], rk1[10];
    __host__ __device__ void set(uint32_t k0, uint32_t k1)
    {
        for (int i = 0; i < 10; ++i) {
            rk0[i] = k0 + (uint32_t)i * 0x9E3779B9u;
            rk1[i] = k1 + (uint32_t)i * 0xBB67AE85u;
        }
    }
    __device__ __forceinline__ uint4 philox(uint4 c) const
    {
#pragma unroll
        for (int i = 0; i < 10; ++i) {
            const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
            const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
            c = make_uint4(hi1 ^ c.y ^ rk0[i], lo1, hi0 ^ c.w ^ rk1[i], lo0);
        }
        return c;
    }
    __device__ __forceinline__ uint4 draw(uint32_t pixel, uint32_t sample, uint32_t view, uint32_t bounce,
                                          uint32_t purpose, uint32_t j) const
    {
        return philox(make_uint4(pixel, sample, (view << 16) | (bounce << 8) | purpose, j));
    }
};

// 24-bit uniform in [0, 1), exact in FP32
__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-8f; }
__device__ __forceinline__ float sub_hi(uint32_t x) { return ((float)(x >> 16) + 0.5f) * 1.52587890625e-5f; }
__device__ __forceinline__ float sub_lo(uint32_t x) { return ((float)(x & 0xFFFFu) + 0.5f) * 1.52587890625e-5f; }

// ---------------------------------------------------------------------------------------
// environment map: lookup and inverse-CDF sampling over uint32 thresholds
// ---------------------------------------------------------------------------------------
// largest i in [0, n-1] with a[i] <= k (a[0] == 0 <= k)
__device__ __forceinline__ int search_le(const uint32_t* __restrict__ a, int n, uint32_t k)
{
    int lo = 0, len = n;
    while (len > 1) {
        const int half = len >> 1;
        const int mid = lo + half;
        if (__ldg(a + mid) <= k) lo = mid;
        len -= half;
    }
    return lo;
}

__device__ __forceinline__ int env_texel_of(const SceneDev& s, float3 d)
{
    const float u = atan2f(d.x, -d.z) * (0.5f * MR_INV_PI) + 0.5f;
    // the polar angle from atan2(sin, cos): acos of d.y loses most of its digits near the poles
    const float v = atan2f(sqrtf(d.x * d.x + d.z * d.z), d.y) * MR_INV_PI;
    int c = (int)floorf(u * (float)s.ew), r = (int)floorf(v * (float)s.eh);
    c = min(max(c, 0), s.ew - 1);
    r = min(max(r, 0), s.eh - 1);
    return r * s.ew + c;
}

__device__ __forceinline__ float env_pdf_dir(const SceneDev& s, float3 d, int texel)
{
    // sin(theta) of a unit direction as |(x, z)|: sqrt(1 - y^2) cancels catastrophically near
    // the poles, where the pdf grows like 1 / sin(theta)
    const float st = sqrtf(d.x * d.x + d.z * d.z);
    if (!(st > 0.0f)) return 0.0f;
    return __ldg(&s.env_texel[texel].w) / (2.0f * MR_PI * MR_PI * st);
}

// sin and cos of a small angle by their Taylor series; for |x| <= pi/64 the truncation error
// is below 2e-13, far under FP32 rounding
__device__ __forceinline__ void sincos_small(float x, float& sn, float& cs)
{
    const float x2 = x * x;
    sn = x * (1.0f - x2 * (1.0f / 6.0f) * (1.0f - x2 * (1.0f / 20.0f)));
    cs = 1.0f - x2 * 0.5f * (1.0f - x2 * (1.0f / 12.0f) * (1.0f - x2 * (1.0f / 30.0f)));
}

// direction of the sub-texel position (c + s_hi, r + s_lo) of texel (r, c) of the y-up
// lat-long map: theta = pi v, psi = 2 pi u - pi, dir = (sin theta sin psi, cos theta,
// -sin theta cos psi). On fine maps each angle is its texel centre (tabulated) plus an offset
// of at most half a texel, combined by the angle-sum formulas; coarse maps use sincospi.
// Returns sin theta; rowv = the row's table entry.
__device__ __forceinline__ float env_dir(const SceneDev& s, int r, int c, uint32_t sub, float3& dir, float4& rowv)
{
    rowv = __ldg(s.env_row + r);
    float st, ct, sp, cp;
    if (s.env_fine) {
        const float2 cv = __ldg(s.env_col + c);
        float sdt, cdt, sdp, cdp;
        sincos_small((sub_lo(sub) - 0.5f) * (MR_PI / (float)s.eh), sdt, cdt);
        sincos_small((sub_hi(sub) - 0.5f) * ((2.0f * MR_PI) / (float)s.ew), sdp, cdp);
        st = rowv.y * cdt + rowv.x * sdt;
        ct = rowv.x * cdt - rowv.y * sdt;
        sp = cv.y * cdp + cv.x * sdp;
        cp = cv.x * cdp - cv.y * sdp;
    } else {
        const float uu = ((float)c + sub_hi(sub)) / (float)s.ew;
        const float vv = ((float)r + sub_lo(sub)) / (float)s.eh;
        sincospif(2.0f * uu - 1.0f, &sp, &cp);
        sincospif(vv, &st, &ct);
    }
    dir = f3(st * sp, ct, -st * cp);
    return st;
}

// inverse-CDF texel draw: row from the marginal, column from the row's conditional. The
// searches start from guide tables (cut-point method): the answer at the start of the
// uniform's bucket and at the next bucket bound the answer, so the search is the same
// function of the uniform as a full binary search, over a range of ~1-2 entries.
// the texel of the CDF over all texels (row-major) at the 53-bit uniform k 2^-53,
// k = xa 2^21 + (xb >> 11): the largest t with threshold[t] <= k, searched inside the range
// the guide gives for k's bucket
__device__ __forceinline__ void env_texel_draw(const SceneDev& s, uint32_t xa, uint32_t xb, int& r, int& c)
{
    const unsigned long long k = ((unsigned long long)xa << 21) | (unsigned long long)(xb >> 11);
    const uint32_t b = (uint32_t)(k >> s.gf_shift);
    int lo = (int)__ldg(s.env_gflat + b), hi = (int)__ldg(s.env_gflat + b + 1);
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(s.env_flat + mid) <= k) lo = mid;
        else hi = mid - 1;
    }
    r = lo / s.ew;
    c = lo - r * s.ew;
}

// two independent draws at once: the two guided searches step in lock-step, so each round
// issues both threshold loads before waiting on either (the same texels as two single draws)
__device__ __forceinline__ void env_texel_draw2(const SceneDev& s, uint32_t xa0, uint32_t xb0, uint32_t xa1,
                                                uint32_t xb1, int& r0, int& c0, int& r1, int& c1)
{
    const unsigned long long k0 = ((unsigned long long)xa0 << 21) | (unsigned long long)(xb0 >> 11);
    const unsigned long long k1 = ((unsigned long long)xa1 << 21) | (unsigned long long)(xb1 >> 11);
    const uint32_t b0 = (uint32_t)(k0 >> s.gf_shift), b1 = (uint32_t)(k1 >> s.gf_shift);
    int lo0 = (int)__ldg(s.env_gflat + b0), hi0 = (int)__ldg(s.env_gflat + b0 + 1);
    int lo1 = (int)__ldg(s.env_gflat + b1), hi1 = (int)__ldg(s.env_gflat + b1 + 1);
    while (lo0 < hi0 || lo1 < hi1) {
        const int m0 = (lo0 + hi0 + 1) >> 1, m1 = (lo1 + hi1 + 1) >> 1;
        const bool a0 = lo0 < hi0, a1 = lo1 < hi1;
        const unsigned long long t0 = a0 ? __ldg(s.env_flat + m0) : 0ull;
        const unsigned long long t1 = a1 ? __ldg(s.env_flat + m1) : 0ull;
        if (a0) {
            if (t0 <= k0) lo0 = m0;
            else hi0 = m0 - 1;
        }
        if (a1) {
            if (t1 <= k1) lo1 = m1;
            else hi1 = m1 - 1;
        }
    }
    r0 = lo0 / s.ew;
    c0 = lo0 - r0 * s.ew;
    r1 = lo1 / s.ew;
    c1 = lo1 - r1 * s.ew;
}

// sample a direction with probability proportional to Y(L) sin(theta_row); returns pdf.
__device__ __forceinline__ float env_sample(const SceneDev& s, uint32_t xrow, uint32_t xcol, uint32_t sub,
                                            float3& dir, int& texel)
{
    int r, c;
    env_texel_draw(s, xrow, xcol, r, c);
    float4 rowv;
    const float st = env_dir(s, r, c, sub, dir, rowv);
    texel = r * s.ew + c;
    return __ldg(&s.env_texel[texel].w) / (2.0f * MR_PI * MR_PI * st);
}

// a RIS candidate: direction and texel as env_sample, and instead of its pdf the factor
// Y(L_env) sin(theta) / q = (sin theta) 2 pi^2 total / (W H sin theta_row), so that the
// resampling weight p_hat / q = Y(f_r cos) times this factor (no texel fetch, no division)
__device__ __forceinline__ float env_candidate(const SceneDev& s, uint32_t xrow, uint32_t xcol, uint32_t sub,
                                               float3& dir, int& texel)
{
    int r, c;
    env_texel_draw(s, xrow, xcol, r, c);
    float4 rowv;
    const float st = env_dir(s, r, c, sub, dir, rowv);
    texel = r * s.ew + c;
    return st * rowv.z;
}

// ---------------------------------------------------------------------------------------
// BRDF: Lambert (1-m) a / pi + GGX D * height-correlated Smith G2 * Schlick F / (4 ci co)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float alpha_of(float r) { return fmaxf(r * r, 1e-3f); }
__device__ __forceinline__ float smith_a(float a2, float c) { return sqrtf(a2 + (1.0f - a2) * c * c); }

// GGX denominator k = cos^2 (a^2 - 1) + 1 written as |n x h|^2 + a^2 cos^2: near the specular
// peak 1 - cos^2 cancels catastrophically in FP32, the cross product does not
__device__ __forceinline__ float ggx_k(float3 n, float3 h, float cnh, float a2)
{
    const float3 c = cross(n, h);
    return dot(c, c) + a2 * cnh * cnh;
}

struct Material {
    float3 alb;
    float rough, metal;
};

// f_r(wo, wi) * max(0, n.wi), zero outside both upper hemispheres. DEMOD: the demodulated
// lobes of the monochrome light regulariser (Appendix A, L_light): the diffuse lobe's
// reflectance (1 - metallic) albedo divided out (1 / pi), the GGX lobe unchanged
template <bool DEMOD = false>
__device__ __forceinline__ float3 brdf_cos(float3 n, float3 wo, float3 wi, const Material& m)
{
    const float co = dot(n, wo), ci = dot(n, wi);
    if (co <= 0.0f || ci <= 0.0f) return f3(0.f, 0.f, 0.f);
    const float a = alpha_of(m.rough), a2 = a * a;
    const float3 h = normalize(add(wo, wi));
    const float cnh = dot(n, h), coh = dot(wo, h);
    const float k = ggx_k(n, h, cnh, a2);
    const float D = a2 / (MR_PI * k * k);
    const float vis = 0.5f / (ci * smith_a(a2, co) + co * smith_a(a2, ci));
    const float om = 1.0f - coh;
    const float w5 = (om * om) * (om * om) * om;
    const float dv = D * vis;
    float3 out;
    {
        const float kd = DEMOD ? 1.0f : (1.0f - m.metal) * m.alb.x;
        const float f0 = 0.04f * (1.0f - m.metal) + m.metal * m.alb.x;
        out.x = (kd * MR_INV_PI + dv * (f0 + (1.0f - f0) * w5)) * ci;
    }
    {
        const float kd = DEMOD ? 1.0f : (1.0f - m.metal) * m.alb.y;
        const float f0 = 0.04f * (1.0f - m.metal) + m.metal * m.alb.y;
        out.y = (kd * MR_INV_PI + dv * (f0 + (1.0f - f0) * w5)) * ci;
    }
    {
        const float kd = DEMOD ? 1.0f : (1.0f - m.metal) * m.alb.z;
        const float f0 = 0.04f * (1.0f - m.metal) + m.metal * m.alb.z;
        out.z = (kd * MR_INV_PI + dv * (f0 + (1.0f - f0) * w5)) * ci;
    }
    return out;
}

// ---------------------------------------------------------------------------------------
// continuation sampling: one-sample mixture of env, GGX visible normals (Heitz 2018), cosine
// ---------------------------------------------------------------------------------------
// orthonormal basis (Duff et al. 2017), branch on n.z >= 0 so that +0 and -0 agree
__device__ __forceinline__ void onb(float3 n, float3& t, float3& b)
{
    const float sg = (n.z >= 0.0f) ? 1.0f : -1.0f;
    const float a = -1.0f / (sg + n.z);
    const float bb = n.x * n.y * a;
    t = f3(1.0f + sg * n.x * n.x * a, sg * bb, -sg * n.x);
    b = f3(bb, sg + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ float3 vndf_local(float3 ve, float a, float u1, float u2)
{
    const float3 vh = normalize(f3(a * ve.x, a * ve.y, ve.z));
    const float lensq = vh.x * vh.x + vh.y * vh.y;
    const float3 t1 = lensq > 0.0f ? mul(f3(-vh.y, vh.x, 0.0f), rsqrtf(lensq)) : f3(1.0f, 0.0f, 0.0f);
    const float3 t2 = cross(vh, t1);
    const float r = sqrtf(u1);
    float sp, cp;
    sincospif(2.0f * u2, &sp, &cp);
    const float p1 = r * cp, p2 = r * sp;
    const float s = 0.5f * (1.0f + vh.z), s1 = 0.5f * (1.0f - vh.z);
    // The disc point (p1, p2) is warped to (p1, p2') with p2' = (1 - s) q + s p2, q = sqrt(1 - p1^2),
    // and lifted by sqrt(1 - p1^2 - p2'^2). Near the rim of the disc (u1 -> 1) both square roots
    // cancel catastrophically when taken as written; they are rewritten through om = 1 - u1 (exact
    // for a 24-bit uniform): q^2 = om + p2^2, (q - p2)(q + p2) = om, and
    // q^2 - p2'^2 = (q - p2')(q + p2') = s (q - p2) (2 (1 - s) q + s (q + p2)), every factor a sum of
    // non-negative terms or a quotient of them.
    const float om = 1.0f - u1;
    const float q = sqrtf(om + p2 * p2);
    float e, d;  // e = q + p2, d = q - p2, both >= 0 with e d = om
    if (p2 >= 0.0f) {
        e = q + p2;
        d = om / e;
    } else {
        d = q - p2;
        e = om / d;
    }
    const float p2w = s1 * q + s * p2;
    const float z = sqrtf(fmaxf(0.0f, s * d * (2.0f * s1 * q + s * e)));
    float3 nh = add(add(mul(t1, p1), mul(t2, p2w)), mul(vh, z));
    // The normal's height above the surface, len p2' + vh.z z (t1.z = 0, t2.z = len = |vh.xy|),
    // cancels near the visible horizon when p2' < 0; there it equals, with |vh| = 1 and
    // vh.z q - |p2'| = s (q + p2), s e (vh.z q + |p2'|) / (vh.z z + len |p2'|).
    const float len = sqrtf(lensq);
    if (p2w < 0.0f) {
        const float den = vh.z * z - len * p2w;
        nh.z = den > 0.0f ? s * e * (vh.z * q - p2w) / den : 0.0f;
    } else {
        nh.z = len * p2w + vh.z * z;
    }
    return normalize(f3(a * nh.x, a * nh.y, fmaxf(0.0f, nh.z)));
}

__device__ __forceinline__ float vndf_pdf(float3 n, float3 wo, float3 wi, float a)
{
    const float co = dot(n, wo);
    if (co <= 0.0f) return 0.0f;
    const float3 hs = add(wo, wi);
    const float l2 = dot(hs, hs);
    if (!(l2 > 0.0f)) return 0.0f;
    const float3 h = mul(hs, rsqrtf(l2));
    const float cnh = dot(n, h);
    if (dot(wo, h) <= 0.0f || cnh <= 0.0f) return 0.0f;
    const float a2 = a * a;
    const float k = ggx_k(n, h, cnh, a2);
    const float D = a2 / (MR_PI * k * k);
    const float g1 = 2.0f * co / (co + smith_a(a2, co));
    return g1 * D / (4.0f * co);
}

struct Mix {
    float c_env, c_s;
};

__device__ __forceinline__ Mix mixture(int env_ok, const Material& m)
{
    Mix x;
    x.c_env = env_ok ? 0.25f : 0.0f;
    const float3 f0 = f3(0.04f * (1.0f - m.metal) + m.metal * m.alb.x, 0.04f * (1.0f - m.metal) + m.metal * m.alb.y,
                         0.04f * (1.0f - m.metal) + m.metal * m.alb.z);
    const float3 kd = mul(m.alb, 1.0f - m.metal);
    const float ys = lum(f0), yd = lum(kd);
    x.c_s = (ys + yd > 0.0f) ? fminf(0.9f, fmaxf(0.1f, ys / (ys + yd))) : 0.5f;
    return x;
}

__device__ __forceinline__ float pdf_mix(const SceneDev& s, int env_ok, Mix x, float3 n, float3 wo, float3 wi,
                                         float rough)
{
    const float a = alpha_of(rough);
    const float pe = (x.c_env > 0.0f) ? env_pdf_dir(s, wi, env_texel_of(s, wi)) : 0.0f;
    const float pv = vndf_pdf(n, wo, wi, a);
    const float pc = fmaxf(0.0f, dot(n, wi)) * MR_INV_PI;
    return x.c_env * pe + (1.0f - x.c_env) * (x.c_s * pv + (1.0f - x.c_s) * pc);
}

// returns the mixture pdf of the sampled direction
__device__ __forceinline__ float sample_continuation(const SceneDev& s, int env_ok, float3 n, float3 wo,
                                                     const Material& m, uint4 x, float3& dir)
{
    const Mix mx = mixture(env_ok, m);
    const float u = u24(x.x);
    const float t2 = mx.c_env + (1.0f - mx.c_env) * mx.c_s;
    if (u < mx.c_env) {
        int tex;
        env_sample(s, x.y, x.z, x.w, dir, tex);
    } else {
        float3 t, b;
        onb(n, t, b);
        const float u1 = u24(x.y), u2 = u24(x.z);
        float3 wl;
        if (u < t2) {
            const float3 ve = f3(dot(wo, t), dot(wo, b), dot(wo, n));
            const float3 mh = vndf_local(ve, alpha_of(m.rough), u1, u2);
            wl = sub(mul(mh, 2.0f * dot(ve, mh)), ve);
        } else {
            const float r = sqrtf(u1);
            float sp, cp;
            sincospif(2.0f * u2, &sp, &cp);
            wl = f3(r * cp, r * sp, sqrtf(fmaxf(0.0f, 1.0f - u1)));
        }
        dir = add(add(mul(t, wl.x), mul(b, wl.y)), mul(n, wl.z));
    }
    return pdf_mix(s, env_ok, mx, n, wo, dir, m.rough);
}

// ---------------------------------------------------------------------------------------
// ray / triangle (Moller-Trumbore, FP32) and LBVH traversal
// ---------------------------------------------------------------------------------------
struct Hit {
    float t, u, v;
    int tri;
};

// plane intersection; returns false only when the ray is parallel (det == 0)
__device__ __forceinline__ bool tri_solve(float3 o, float3 d, float3 v0, float3 e1, float3 e2, float& t, float& u,
                                          float& v)
{
    const float3 p = cross(d, e2);
    const float det = dot(e1, p);
    if (det == 0.0f) return false;
    const float inv = 1.0f / det;
    const float3 sv = sub(o, v0);
    u = dot(sv, p) * inv;
    const float3 q = cross(sv, e1);
    v = dot(d, q) * inv;
    t = dot(e2, q) * inv;
    return true;
}

__device__ __forceinline__ void load_tri(const SceneDev& s, int leaf, float3& v0, float3& e1, float3& e2, int& tri)
{
    const float4* p = s.ptri + MR_TRI_STRIDE * (size_t)leaf;
#if MR_TRI_LD256
    float4 a, b, c, pad;
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(c.x), "=f"(c.y), "=f"(c.z), "=f"(c.w), "=f"(pad.x), "=f"(pad.y), "=f"(pad.z), "=f"(pad.w)
        : "l"(p + 2));
#else
    const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
#endif
    v0 = xyz(a);
    tri = __float_as_int(a.w);
    e1 = xyz(b);
    e2 = xyz(c);
}

// test one leaf; closest: keep smallest t, ties -> smaller id. Returns hit (any mode).
__device__ __forceinline__ bool test_leaf(const SceneDev& s, int leaf, float3 o, float3 d, int skip, float tmin,
                                          Hit& best)
{
    float3 v0, e1, e2;
    int tri;
    load_tri(s, leaf, v0, e1, e2, tri);
    if (tri == skip) return false;
    float t, u, v;
    if (!tri_solve(o, d, v0, e1, e2, t, u, v)) return false;
    if (!(u >= 0.0f && v >= 0.0f && u + v <= 1.0f && t > tmin)) return false;
    if (t < best.t || (t == best.t && tri < best.tri)) {
        best.t = t;
        best.u = u;
        best.v = v;
        best.tri = tri;
        return true;
    }
    return false;
}

__device__ __forceinline__ float safe_inv(float x)
{
    return 1.0f / (fabsf(x) > 1e-30f ? x : copysignf(1e-30f, x));
}

// slab test of one box; returns the entry distance, or NaN on a miss (NaN <= t is false).
// Plane distances as one FMA each, (plane * inv) - (o * inv) with oi = o * inv per ray.
__device__ __forceinline__ float slab(float3 lo, float3 hi, float3 oi, float3 inv, float tmin, float tmax)
{
    const float tx0 = fmaf(lo.x, inv.x, -oi.x), tx1 = fmaf(hi.x, inv.x, -oi.x);
    const float ty0 = fmaf(lo.y, inv.y, -oi.y), ty1 = fmaf(hi.y, inv.y, -oi.y);
    const float tz0 = fmaf(lo.z, inv.z, -oi.z), tz1 = fmaf(hi.z, inv.z, -oi.z);
    const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tmin));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
    // a few ulp of slack so that rounding never culls a box the ray touches
    return (tn <= tf * 1.0000005f + 1e-30f) ? tn : __int_as_float(0x7fffffff);
}

// One traversal node (64 bytes, 64-byte aligned): the two child boxes and the child codes. With
// MR_NODE_LD256 as two 32-byte loads (ld.global.nc.v8.f32, sm_100 and later) instead of four.
__device__ __forceinline__ void load_node(const float4* p, float4& n0, float4& n1, float4& n2, int2& ch)
{
#if MR_NODE_LD256
    float4 n3;
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(n0.x), "=f"(n0.y), "=f"(n0.z), "=f"(n0.w), "=f"(n1.x), "=f"(n1.y), "=f"(n1.z), "=f"(n1.w)
        : "l"(p));
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(n2.x), "=f"(n2.y), "=f"(n2.z), "=f"(n2.w), "=f"(n3.x), "=f"(n3.y), "=f"(n3.z), "=f"(n3.w)
        : "l"(p + 2));
    ch = make_int2(__float_as_int(n3.x), __float_as_int(n3.y));
#else
    n0 = __ldg(p);
    n1 = __ldg(p + 1);
    n2 = __ldg(p + 2);
    ch = *reinterpret_cast<const int2*>(p + 3);
#endif
}

// Closest (any = false) or any hit with t in (tmin, tmax). `sstk` = this thread's shared
// stack column (stride `sstride`). Returns the number of nodes visited (two box tests each),
// or -1 if the iteration cap was reached or the stack overflowed (a malformed tree: the ray
// reports a miss and the scene's error counter is raised); adds the triangle tests to *ntri
// when given.
template <bool ANY>
__device__ __forceinline__ int traverse(const SceneDev& s, float3 o, float3 d, int skip, float tmin, float tmax,
                                        Hit& best, uint32_t* sstk, int sstride, int* ntri = nullptr)
{
    best.t = tmax;
    best.tri = -1;
    best.u = best.v = 0.0f;
    const int F = s.n_tris;
    if (F <= 0) return 0;
    if (F == 1) {
        if (ntri) ++*ntri;
        test_leaf(s, 0, o, d, skip, tmin, best);
        return 0;
    }
    const float3 inv = f3(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
    const float3 oi = f3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    uint32_t lstk[MR_LSTACK];
    int sp = 0;
    int node = 0;
    int visited = 0;
    const int cap = trav_cap_of(s);
    while (true) {
        if (++visited > cap) {
            best.tri = -1;
            trav_fail(s);
            return -1;
        }
        float4 n0, n1, n2;
        int2 ch;
        load_node(s.nodes + 4 * (size_t)node, n0, n1, n2, ch);
        const float tl = slab(f3(n0.x, n0.y, n0.z), f3(n0.w, n1.x, n1.y), oi, inv, tmin, best.t);
        const float tr = slab(f3(n1.z, n1.w, n2.x), f3(n2.y, n2.z, n2.w), oi, inv, tmin, best.t);
        bool gl = tl <= best.t, gr = tr <= best.t;
        // leaves are tested on the spot
        if (gl && ch.x < 0) {
            if (ntri) ++*ntri;
            if (test_leaf(s, ~ch.x, o, d, skip, tmin, best) && ANY) return visited;
            gl = false;
        }
        if (gr && ch.y < 0) {
            if (ntri) ++*ntri;
            if (test_leaf(s, ~ch.y, o, d, skip, tmin, best) && ANY) return visited;
            gr = false;
        }
        if (gl && gr) {
            const bool lfirst = tl <= tr;
            const int nearc = lfirst ? ch.x : ch.y, farc = lfirst ? ch.y : ch.x;
            if (sp < MR_SSTACK) {
                sstk[sp * sstride] = (uint32_t)farc;
            } else if (sp < MR_SSTACK + MR_LSTACK) {
                lstk[sp - MR_SSTACK] = (uint32_t)farc;
            } else {  // deeper than any tree the builders keep: a malformed tree
                best.tri = -1;
                trav_fail(s);
                return -1;
            }
            ++sp;
            node = nearc;
        } else if (gl) {
            node = ch.x;
        } else if (gr) {
            node = ch.y;
        } else {
            if (sp == 0) break;
            --sp;
            node = (int)(sp < MR_SSTACK ? sstk[sp * sstride] : lstk[sp - MR_SSTACK]);
        }
    }
    return visited;
}

// ---------------------------------------------------------------------------------------
// traversal of the 8-wide BVH (layout in wbvh.cu)
// ---------------------------------------------------------------------------------------
// byte k of a word as a float (exact: 2^23 + q, minus 2^23)
__device__ __forceinline__ float qbyte(uint32_t word, uint32_t k)
{
    return __uint_as_float(__byte_perm(word, 0x4B000000u, 0x7540u | k)) - 8388608.0f;
}

// one triangle of the wide leaves; closest: smallest t, ties -> smaller id; returns a hit
__device__ __forceinline__ bool test_wtri(const SceneDev& s, uint32_t k, float3 o, float3 d, int skip, float tmin,
                                          Hit& best)
{
    const float4 a = __ldg(s.wtri + 3 * (size_t)k);
    const int tri = __float_as_int(a.w);
    if (tri == skip) return false;
    const float4 b = __ldg(s.wtri + 3 * (size_t)k + 1);
    const float4 c = __ldg(s.wtri + 3 * (size_t)k + 2);
    float t, u, v;
    if (!tri_solve(o, d, xyz(a), xyz(b), xyz(c), t, u, v)) return false;
    if (!(u >= 0.0f && v >= 0.0f && u + v <= 1.0f && t > tmin)) return false;
    if (t < best.t || (t == best.t && tri < best.tri)) {
        best.t = t;
        best.u = u;
        best.v = v;
        best.tri = tri;
        return true;
    }
    return false;
}

// Expand one wide node: test its eight child boxes (t entry <= best.t, the binary traversal's
// rule, with the same few-ulp slack), return the node children hit as bits in visit order
// (slot ^ oct) in bits 0-7 with the node-slot mask in bits 8-15, and the leaf triangles hit as
// bits (offset) of *tbits; *cbase / *tbase receive the node's first child and first triangle.
__device__ __forceinline__ uint32_t wide_expand(const SceneDev& s, uint32_t node, float3 o, float3 inv, uint32_t oct,
                                                float tmin, float tmax, uint32_t& cbase, uint32_t& tbase,
                                                uint32_t& tbits)
{
    const uint4* np = s.wnodes + 5 * (size_t)node;
    const uint4 w0 = __ldg(np), w1 = __ldg(np + 1), w2 = __ldg(np + 2), w3 = __ldg(np + 3), w4 = __ldg(np + 4);
    // t of a plane at p + q 2^e: q (2^e inv) + (p - o) inv
    const float ax = __uint_as_float((w0.w & 0xffu) << 23) * inv.x;
    const float ay = __uint_as_float(((w0.w >> 8) & 0xffu) << 23) * inv.y;
    const float az = __uint_as_float(((w0.w >> 16) & 0xffu) << 23) * inv.z;
    const float bx = (__uint_as_float(w0.x) - o.x) * inv.x;
    const float by = (__uint_as_float(w0.y) - o.y) * inv.y;
    const float bz = (__uint_as_float(w0.z) - o.z) * inv.z;
    // the near plane of each axis is the low one for a positive direction, the high one otherwise
    const uint32_t nx0 = (oct & 1u) ? w3.z : w2.x, nx1 = (oct & 1u) ? w3.w : w2.y;
    const uint32_t fx0 = (oct & 1u) ? w2.x : w3.z, fx1 = (oct & 1u) ? w2.y : w3.w;
    const uint32_t ny0 = (oct & 2u) ? w4.x : w2.z, ny1 = (oct & 2u) ? w4.y : w2.w;
    const uint32_t fy0 = (oct & 2u) ? w2.z : w4.x, fy1 = (oct & 2u) ? w2.w : w4.y;
    const uint32_t nz0 = (oct & 4u) ? w4.z : w3.x, nz1 = (oct & 4u) ? w4.w : w3.y;
    const uint32_t fz0 = (oct & 4u) ? w3.x : w4.z, fz1 = (oct & 4u) ? w3.y : w4.w;
    cbase = w1.x;
    tbase = w1.y;
    const uint32_t imask = w0.w >> 24;
    uint32_t hits = 0, tb = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t k = (uint32_t)(i & 3);
        const uint32_t meta = ((i < 4 ? w1.z : w1.w) >> (8 * k)) & 0xffu;
        const float tnx = fmaf(qbyte(i < 4 ? nx0 : nx1, k), ax, bx);
        const float tny = fmaf(qbyte(i < 4 ? ny0 : ny1, k), ay, by);
        const float tnz = fmaf(qbyte(i < 4 ? nz0 : nz1, k), az, bz);
        const float tfx = fmaf(qbyte(i < 4 ? fx0 : fx1, k), ax, bx);
        const float tfy = fmaf(qbyte(i < 4 ? fy0 : fy1, k), ay, by);
        const float tfz = fmaf(qbyte(i < 4 ? fz0 : fz1, k), az, bz);
        const float tn = fmaxf(fmaxf(tnx, tny), fmaxf(tnz, tmin));
        const float tf = fminf(fminf(tfx, tfy), fminf(tfz, tmax));
        if (meta != 0u && tn <= tf * 1.0000005f + 1e-30f) {
            if (meta & 0x80u) hits |= 1u << ((uint32_t)i ^ oct);
            else tb |= ((1u << (meta >> 5)) - 1u) << (meta & 31u);
        }
    }
    tbits = tb;
    return hits | (imask << 8);
}

// Closest (any = false) or any hit with t in (tmin, tmax) through the wide BVH: the same
// contract as traverse() (returns the nodes visited, -1 on a cap or stack overflow, triangle
// tests added to *ntri). `sstk` = this thread's shared column of 8-byte entries (stride
// `sstride`).
template <bool ANY>
__device__ __forceinline__ int wtraverse(const SceneDev& s, float3 o, float3 d, int skip, float tmin, float tmax,
                                         Hit& best, uint2* sstk, int sstride, int* ntri = nullptr)
{
    best.t = tmax;
    best.tri = -1;
    best.u = best.v = 0.0f;
    const int F = s.n_tris;
    if (F <= 0) return 0;
    if (F == 1) {
        if (ntri) ++*ntri;
        test_leaf(s, 0, o, d, skip, tmin, best);
        return 0;
    }
    const float3 inv = f3(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
    const uint32_t oct = (d.x < 0.0f ? 1u : 0u) | (d.y < 0.0f ? 2u : 0u) | (d.z < 0.0f ? 4u : 0u);
    uint2 lstk[MR_WLSTACK];
    int sp = 0;
    int visited = 0;
    const int cap = trav_cap_of(s);
    uint32_t node = 0;
    while (true) {
        // a wide tree has fewer than F nodes and exactly F triangles: an index outside that
        // (a malformed tree) ends the ray like the iteration cap instead of reading past it
        if (++visited > cap || node >= (uint32_t)F) {
            best.tri = -1;
            trav_fail(s);
            return -1;
        }
        uint32_t cbase, tbase, tbits;
        uint32_t group = wide_expand(s, node, o, inv, oct, tmin, best.t, cbase, tbase, tbits);
        if (tbits && tbase + (uint32_t)(31 - __clz(tbits)) >= (uint32_t)F) {
            best.tri = -1;
            trav_fail(s);
            return -1;
        }
        while (tbits) {
            const uint32_t k = (uint32_t)(__ffs(tbits) - 1);
            tbits &= tbits - 1u;
            if (ntri) ++*ntri;
            if (test_wtri(s, tbase + k, o, d, skip, tmin, best) && ANY) return visited;
        }
        if ((group & 0xffu) == 0u) {
            if (sp == 0) break;
            --sp;
            const uint2 e = sp < MR_WSSTACK ? sstk[sp * sstride] : lstk[sp - MR_WSSTACK];
            cbase = e.x;
            group = e.y;
        }
        const uint32_t bit = (uint32_t)(__ffs(group & 0xffu) - 1);
        group &= ~(1u << bit);
        const uint32_t slot = bit ^ oct;
        node = cbase + (uint32_t)__popc((group >> 8) & ((1u << slot) - 1u));
        if (group & 0xffu) {
            if (sp < MR_WSSTACK) {
                sstk[sp * sstride] = make_uint2(cbase, group);
            } else if (sp < MR_WSSTACK + MR_WLSTACK) {
                lstk[sp - MR_WSSTACK] = make_uint2(cbase, group);
            } else {
                best.tri = -1;
                trav_fail(s);
                return -1;
            }
            ++sp;
        }
    }
    return visited;
}

// the scene's traversal: the wide BVH when it has one, else the binary tree. `sstk` is the
// thread's column of MR_SSTACK 32-bit words in a shared buffer whose base is 8-byte aligned:
// sstk = base + threadIdx.x, stride blockDim.x (the wide traversal reads the same buffer as
// MR_WSSTACK 8-byte words per thread, base + threadIdx.x in 8-byte units)
template <bool ANY>
__device__ __forceinline__ int trace(const SceneDev& s, float3 o, float3 d, int skip, float tmin, float tmax, Hit& best,
                                     uint32_t* sstk, int* ntri = nullptr)
{
    if (s.wnodes)
        return wtraverse<ANY>(s, o, d, skip, tmin, tmax, best,
                              reinterpret_cast<uint2*>(sstk - threadIdx.x) + threadIdx.x, blockDim.x, ntri);
    return traverse<ANY>(s, o, d, skip, tmin, tmax, best, sstk, blockDim.x, ntri);
}

// the same with the tree chosen at compile time (WIDE: the scene must have a wide BVH), for the
// stage kernels whose registers are tight: each variant carries one traversal only
template <bool ANY, bool WIDE>
__device__ __forceinline__ int trace_as(const SceneDev& s, float3 o, float3 d, int skip, float tmin, float tmax,
                                        Hit& best, uint32_t* sstk, int* ntri = nullptr)
{
    if (WIDE)
        return wtraverse<ANY>(s, o, d, skip, tmin, tmax, best,
                              reinterpret_cast<uint2*>(sstk - threadIdx.x) + threadIdx.x, blockDim.x, ntri);
    return traverse<ANY>(s, o, d, skip, tmin, tmax, best, sstk, blockDim.x, ntri);
}

// The same traversal as a resumable state, for kernels that interleave the rays of a warp's
// lanes and hand a finished lane a new ray: trav_begin sets a ray up, trav_run advances it by
// at most `steps` node visits and returns true when it is done (result in T.best; T.visited =
// -1 when the iteration cap was reached). The stack is the thread's shared column plus `lstk`.
struct Trav {
    float3 o, d, inv, oi;
    float tmin;
    int skip, node, sp, visited;  // node < 0: done
    Hit best;
};

__device__ __forceinline__ void trav_begin(const SceneDev& s, Trav& T, float3 o, float3 d, int skip, float tmin,
                                           float tmax, int* ntri)
{
    T.best.t = tmax;
    T.best.tri = -1;
    T.best.u = T.best.v = 0.0f;
    T.o = o;
    T.d = d;
    T.inv = f3(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
    T.oi = f3(o.x * T.inv.x, o.y * T.inv.y, o.z * T.inv.z);
    T.tmin = tmin;
    T.skip = skip;
    T.sp = 0;
    T.visited = 0;
    T.node = 0;
    if (s.n_tris <= 0) {
        T.node = -1;
    } else if (s.n_tris == 1) {
        if (ntri) ++*ntri;
        test_leaf(s, 0, o, d, skip, tmin, T.best);
        T.node = -1;
    }
}

template <bool ANY>
__device__ __forceinline__ bool trav_run(const SceneDev& s, Trav& T, uint32_t* sstk, int sstride, uint32_t* lstk,
                                         int steps, int* ntri)
{
    if (T.node < 0) return true;
    const int cap = trav_cap_of(s);
    for (int k = 0; k < steps; ++k) {
        if (++T.visited > cap) {
            T.best.tri = -1;
            T.visited = -1;
            T.node = -1;
            trav_fail(s);
            return true;
        }
        const int node = T.node;
        float4 n0, n1, n2;
        int2 ch;
        load_node(s.nodes + 4 * (size_t)node, n0, n1, n2, ch);
        const float tl = slab(f3(n0.x, n0.y, n0.z), f3(n0.w, n1.x, n1.y), T.oi, T.inv, T.tmin, T.best.t);
        const float tr = slab(f3(n1.z, n1.w, n2.x), f3(n2.y, n2.z, n2.w), T.oi, T.inv, T.tmin, T.best.t);
        bool gl = tl <= T.best.t, gr = tr <= T.best.t;
        if (gl && ch.x < 0) {
            if (ntri) ++*ntri;
            if (test_leaf(s, ~ch.x, T.o, T.d, T.skip, T.tmin, T.best) && ANY) {
                T.node = -1;
                return true;
            }
            gl = false;
        }
        if (gr && ch.y < 0) {
            if (ntri) ++*ntri;
            if (test_leaf(s, ~ch.y, T.o, T.d, T.skip, T.tmin, T.best) && ANY) {
                T.node = -1;
                return true;
            }
            gr = false;
        }
        if (gl && gr) {
            const bool lfirst = tl <= tr;
            const int nearc = lfirst ? ch.x : ch.y, farc = lfirst ? ch.y : ch.x;
            if (T.sp < MR_SSTACK) {
                sstk[T.sp * sstride] = (uint32_t)farc;
            } else if (T.sp < MR_SSTACK + MR_LSTACK) {
                lstk[T.sp - MR_SSTACK] = (uint32_t)farc;
            } else {
                T.best.tri = -1;
                T.visited = -1;
                T.node = -1;
                trav_fail(s);
                return true;
            }
            ++T.sp;
            T.node = nearc;
        } else if (gl) {
            T.node = ch.x;
        } else if (gr) {
            T.node = ch.y;
        } else {
            if (T.sp == 0) {
                T.node = -1;
                return true;
            }
            --T.sp;
            T.node = (int)(T.sp < MR_SSTACK ? sstk[T.sp * sstride] : lstk[T.sp - MR_SSTACK]);
        }
    }
    return false;
}

// ---------------------------------------------------------------------------------------
// shading point
// ---------------------------------------------------------------------------------------
struct Taps {
    int idx[4];
    float w[4];
    float fx, fy;
};

__device__ __forceinline__ void taps_at(int w, int h, float su, float sv, Taps& tp)
{
    const float x = su * (float)w - 0.5f, y = sv * (float)h - 0.5f;
    const float x0 = floorf(x), y0 = floorf(y);
    tp.fx = x - x0;
    tp.fy = y - y0;
    int ix0 = (int)x0, iy0 = (int)y0;
    int ix1 = ix0 + 1, iy1 = iy0 + 1;
    ix0 = min(max(ix0, 0), w - 1);
    ix1 = min(max(ix1, 0), w - 1);
    iy0 = min(max(iy0, 0), h - 1);
    iy1 = min(max(iy1, 0), h - 1);
    tp.idx[0] = iy0 * w + ix0;
    tp.idx[1] = iy0 * w + ix1;
    tp.idx[2] = iy1 * w + ix0;
    tp.idx[3] = iy1 * w + ix1;
    tp.w[0] = (1.0f - tp.fx) * (1.0f - tp.fy);
    tp.w[1] = tp.fx * (1.0f - tp.fy);
    tp.w[2] = (1.0f - tp.fx) * tp.fy;
    tp.w[3] = tp.fx * tp.fy;
}

struct Shade {
    float3 x, n, N, e1, e2;
    float sign;
    float su, sv;
    Taps tp;
    Material m;
    // with interpolated normals: n = nsg S / |S|, S = w0 VN_a + u VN_b + v VN_c, and ng the
    // face normal towards the viewer (below it, light and continuation directions are dropped)
    bool interp;
    float3 ng, S;
    float nsg;
};

// INTERP = false compiles the interpolated-normal path out (kernels launched for scenes that
// all use face normals); INTERP = true follows the scene (s.vnrm)
template <bool INTERP = true>
__device__ __forceinline__ void shade_at(const SceneDev& s, int tri, float u, float v, float3 d, Shade& sh)
{
    float3 v0;
    int tri_chk;
    load_tri(s, __ldg(s.leaf_of + tri), v0, sh.e1, sh.e2, tri_chk);
    sh.N = cross(sh.e1, sh.e2);
    const float3 nh = normalize(sh.N);
    sh.sign = (dot(nh, d) > 0.0f) ? -1.0f : 1.0f;
    sh.n = mul(nh, sh.sign);
    sh.ng = sh.n;
    sh.interp = false;
    sh.nsg = 1.0f;
    sh.S = f3(0.f, 0.f, 0.f);
    sh.x = add(v0, add(mul(sh.e1, u), mul(sh.e2, v)));
    const float* uv = s.tri_uv + 6 * (size_t)tri;
    const float w0 = 1.0f - u - v;
    if (INTERP && s.vnrm) {
        const int ia = __ldg(s.tris + 3 * (size_t)tri), ib = __ldg(s.tris + 3 * (size_t)tri + 1),
                  ic = __ldg(s.tris + 3 * (size_t)tri + 2);
        const float3 na = xyz(__ldg(s.vnrm + ia)), nb = xyz(__ldg(s.vnrm + ib)), nc = xyz(__ldg(s.vnrm + ic));
        const float3 S = add(add(mul(na, w0), mul(nb, u)), mul(nc, v));
        const float l2 = dot(S, S);
        if (l2 > 0.0f) {
            const float il = rsqrtf(l2);
            sh.nsg = dot(S, sh.ng) < 0.0f ? -1.0f : 1.0f;
            sh.n = mul(S, sh.nsg * il);
            sh.S = S;
            sh.interp = true;
        }
    }
    sh.su = w0 * __ldg(uv + 0) + u * __ldg(uv + 2) + v * __ldg(uv + 4);
    sh.sv = w0 * __ldg(uv + 1) + u * __ldg(uv + 3) + v * __ldg(uv + 5);
    taps_at(s.tw, s.th, sh.su, sh.sv, sh.tp);
    float3 a = f3(0.f, 0.f, 0.f);
    float r = 0.0f, m = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = sh.tp.idx[k];
        const float w = sh.tp.w[k];
        a.x += w * __ldg(s.albedo + 3 * (size_t)i);
        a.y += w * __ldg(s.albedo + 3 * (size_t)i + 1);
        a.z += w * __ldg(s.albedo + 3 * (size_t)i + 2);
        r += w * __ldg(s.rough + i);
        m += w * __ldg(s.metal + i);
    }
    sh.m.alb = a;
    sh.m.rough = r;
    sh.m.metal = m;
}

// with interpolated normals, false for a direction below the face: light from it and a
// continuation along it are dropped
__device__ __forceinline__ bool above_face(const Shade& sh, float3 dir) { return !sh.interp || dot(sh.ng, dir) > 0.0f; }

// f_r cos of a light direction at a shading point (0 below the face with interpolated normals)
__device__ __forceinline__ float3 light_brdf(const Shade& sh, float3 wo, float3 dir)
{
    return above_face(sh, dir) ? brdf_cos(sh.n, wo, dir, sh.m) : f3(0.f, 0.f, 0.f);
}

// camera ray direction for pixel (px, py) with jitter from the random stream
__device__ __forceinline__ float3 camera_dir(const ViewDev& v, int px, int py, float j0, float j1)
{
    const float dcx = ((float)px + j0 - v.K[2]) / v.K[0];
    const float dcy = ((float)py + j1 - v.K[3]) / v.K[1];
    const float3 d = f3(v.c2w[0] * dcx + v.c2w[1] * dcy + v.c2w[2], v.c2w[4] * dcx + v.c2w[5] * dcy + v.c2w[6],
                        v.c2w[8] * dcx + v.c2w[9] * dcy + v.c2w[10]);
    return normalize(d);
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

// warp-aggregated scatter: lanes holding the same key add their values and the key's first
// lane issues one set of atomics. The sums are segmented suffix sums by pointer jumping along
// each key's lanes in lane order, every key at once: ceil(log2(largest group)) steps of
// NV + 1 shuffles, however many distinct keys the warp holds.
template <int NV, class Emit>
__device__ __forceinline__ void scatter_agg(int key, const float (&v)[NV], const Emit& emit)
{
    const int lane = lane_id();
    const unsigned peers = __match_any_sync(MR_FULL, key);
    const unsigned after = peers & ~((2u << lane) - 1u);  // my key's lanes above me
    int nxt = (key >= 0 && after) ? __ffs(after) - 1 : -1;
    float acc[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) acc[c] = v[c];
    while (__any_sync(MR_FULL, nxt >= 0)) {
        const int src = nxt >= 0 ? nxt : lane;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            const float o = __shfl_sync(MR_FULL, acc[c], src);
            if (nxt >= 0) acc[c] += o;
        }
        const int n2 = __shfl_sync(MR_FULL, nxt, src);
        nxt = nxt >= 0 ? n2 : -1;
    }
    if (key >= 0 && (__ffs(peers) - 1) == lane) emit(key, acc);
}
