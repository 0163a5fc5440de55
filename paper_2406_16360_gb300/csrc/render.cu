// render.cu -- forward path tracing (wavefront and persistent), adjoint replay, L2 loss.
//
// One path sample = one pixel sample of one view. Per sample the tape holds nine 32-bit
// words (SoA, N = samples of the call): primary triangle, selected RIS candidate at the
// primary vertex, V*W at the primary vertex, L_ind (3) at the primary vertex, radiance (3).
// The image is the mean of the sample radiances over spp, summed in sample order.
#include "render.h"
#include "path.cuh"

namespace {

// ---------------------------------------------------------------------------------------
// wavefront (plain) kernels: one view chunk at a time
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_raygen(ViewDev v, Rng rng, uint32_t first, uint32_t n, QueueDev q,
                                                void* tape, uint64_t ntot, int nvx)
{
    const TapeDev tp = tape_of(tape, ntot, nvx);
    const float3 o = f3(v.c2w[3], v.c2w[7], v.c2w[11]);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t sid = first + i;
        const uint32_t pixel = sid / (uint32_t)v.spp, smp = sid % (uint32_t)v.spp;
        const int px = (int)(pixel % (uint32_t)v.width), py = (int)(pixel / (uint32_t)v.width);
        const uint4 x = rng.draw(pixel, smp, (uint32_t)v.index, 0u, PURPOSE_CAMERA, 0u);
        const float3 d = camera_dir(v, px, py, u24(x.x), u24(x.y));
        q.o[i] = make_float4(o.x, o.y, o.z, __int_as_float(-1));
        q.d[i] = make_float4(d.x, d.y, d.z, __uint_as_float(sid));
        q.b[i] = make_float4(1.f, 1.f, 1.f, 0.f);
        q.bi[i] = make_float4(1.f, 1.f, 1.f, 0.f);
        const uint64_t g = v.offset + sid;
        tp.tri[g] = -1;
        tp.cand[g] = -1;
        tp.wv[g] = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            tp.lind[k][g] = 0.0f;
            tp.rad[k][g] = 0.0f;
        }
        tape_vx_init(tp, g);
    }
}



// closest hit of every queued ray. A primary ray that escapes writes the environment into
// its sample; an escaping continuation ray ends its path. Hits are compacted (warp ballot)
// into the shade queue, so that shading runs on full warps of hits.
__global__ void __launch_bounds__(256) k_closest(SceneDev s, ViewDev v, int b, QueueDev q, const unsigned int* count,
                                                 unsigned int count_fixed, QueueDev hq, unsigned int* count_hit,
                                                 void* tape, uint64_t ntot)
{
    extern __shared__ __align__(16) uint32_t sstk[];
    const TapeDev tp = tape_of(tape, ntot);
    const unsigned int n = count ? *count : count_fixed;
    const float tmin = *s.tmin_dev;
    const unsigned int stride = gridDim.x * blockDim.x;
    const unsigned int rounds = (n + stride - 1) / stride;
    for (unsigned int r = 0; r < rounds; ++r) {
        const unsigned int i = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
        Hit h;
        h.tri = -1;
        float4 qd = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < n) {
            const float4 a = q.o[i];
            qd = q.d[i];
            trace<false>(s, xyz(a), xyz(qd), __float_as_int(a.w), tmin, __int_as_float(0x7f800000), h,
                         sstk + threadIdx.x);
            if (h.tri < 0 && b == 0) {
                const uint64_t g = v.offset + __float_as_uint(qd.w);
                const float4 L = __ldg(s.env_texel + env_texel_of(s, xyz(qd)));
                tp.rad[0][g] = L.x;
                tp.rad[1][g] = L.y;
                tp.rad[2][g] = L.z;
            }
        }
        const bool hit = h.tri >= 0;
        const unsigned int slot = warp_append(hit, count_hit);
        if (hit) {
            hq.o[slot] = make_float4(h.t, h.u, h.v, __int_as_float(h.tri));
            hq.d[slot] = qd;
            hq.b[slot] = q.b[i];
            hq.bi[slot] = q.bi[i];
        }
    }
}

// shade every compacted hit: RIS + shadow ray + continuation (next-bounce queue)
__global__ void __launch_bounds__(256, MR_SHADE_MINB) k_shade(SceneDev s, ViewDev v, Rng rng, int b, int M, QueueDev hq,
                                               const unsigned int* count_hit, QueueDev qout,
                                               unsigned int* count_out, ShadowDev sq, unsigned int* count_sh,
                                               void* tape, uint64_t ntot, int nvx, unsigned long long* counters)
{
    const TapeDev tp = tape_of(tape, ntot, nvx);
    const unsigned int n = *count_hit;
    unsigned long long n_cand = 0;
    const int env_ok = *s.env_ok_dev;
    const unsigned int stride = gridDim.x * blockDim.x;
    const unsigned int rounds = (n + stride - 1) / stride;
    for (unsigned int r = 0; r < rounds; ++r) {
        const unsigned int i = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
        VertexOut out;
        out.shadow = false;
        out.cont = false;
        uint32_t sid = 0;
        int tri = -1;
        if (i < n) {
            const float4 hd = hq.o[i];
            const float4 qd = hq.d[i];
            const float3 d = xyz(qd);
            sid = __float_as_uint(qd.w);
            const uint64_t g = v.offset + sid;
            tri = __float_as_int(hd.w);
            const uint32_t pixel = sid / (uint32_t)v.spp, smp = sid % (uint32_t)v.spp;
            Hit h;
            h.t = hd.x;
            h.u = hd.y;
            h.v = hd.z;
            h.tri = tri;
            shade_vertex(s, env_ok, rng, pixel, smp, (uint32_t)v.index, b, v.bounces, M, h, d, xyz(hq.b[i]),
                         xyz(hq.bi[i]), out);
            if (env_ok) n_cand += (unsigned long long)M;
            if (b == 0) {
                tp.tri[g] = tri;
                tp.cand[g] = out.cand;
                tp.wv[g] = out.W;
                tape_directions(tp, g, out);
            } else {
                tape_vx_record(tp, g, b, h, out);
            }
        }
        const unsigned int ss = warp_append(out.shadow, count_sh);
        if (out.shadow) {
            sq.o[ss] = make_float4(out.sh_o.x, out.sh_o.y, out.sh_o.z, __int_as_float(tri));
            sq.d[ss] = make_float4(out.sh_d.x, out.sh_d.y, out.sh_d.z, __uint_as_float(sid));
            sq.add[ss] = make_float4(out.add_rad.x, out.add_rad.y, out.add_rad.z, 0.f);
            sq.addi[ss] = make_float4(out.add_lind.x, out.add_lind.y, out.add_lind.z, 0.f);
        }
        const unsigned int cs = warp_append(out.cont, count_out);
        if (out.cont) {
            qout.o[cs] = make_float4(out.x.x, out.x.y, out.x.z, __int_as_float(tri));
            qout.d[cs] = make_float4(out.c_d.x, out.c_d.y, out.c_d.z, __uint_as_float(sid));
            qout.b[cs] = make_float4(out.c_beta.x, out.c_beta.y, out.c_beta.z, 0.f);
            qout.bi[cs] = make_float4(out.c_bind.x, out.c_bind.y, out.c_bind.z, 0.f);
        }
    }
    for (int off = 16; off > 0; off >>= 1) n_cand += __shfl_xor_sync(MR_FULL, n_cand, off);
    if (lane_id() == 0 && n_cand) atomicAdd(counters + 5, n_cand);
}

// shadow rays: any hit; unoccluded rays add their contribution to the sample
__global__ void __launch_bounds__(256) k_shadow(SceneDev s, ViewDev v, int b, ShadowDev sq,
                                                const unsigned int* count, void* tape, uint64_t ntot, int nvx)
{
    extern __shared__ __align__(16) uint32_t sstk[];
    const TapeDev tp = tape_of(tape, ntot, nvx);
    const unsigned int n = *count;
    const float tmin = *s.tmin_dev;
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 a = sq.o[i], dd = sq.d[i];
        Hit h;
        trace<true>(s, xyz(a), xyz(dd), __float_as_int(a.w), tmin, __int_as_float(0x7f800000), h,
                    sstk + threadIdx.x);
        const uint64_t g = v.offset + __float_as_uint(dd.w);
        if (h.tri < 0) {
            const float4 ad = sq.add[i], ai = sq.addi[i];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float av = k == 0 ? ad.x : (k == 1 ? ad.y : ad.z);
                const float ai_ = k == 0 ? ai.x : (k == 1 ? ai.y : ai.z);
                tp.rad[k][g] = __fadd_rn(tp.rad[k][g], av);
                if (b >= 1) tp.lind[k][g] = __fadd_rn(tp.lind[k][g], ai_);
            }
        } else if (b == 0) {
            tp.wv[g] = 0.0f;
        } else {
            tape_vx_occluded(tp, g, b);
        }
    }
}

__global__ void __launch_bounds__(256) k_resolve(ViewDev v, const void* tape, uint64_t ntot, float* __restrict__ img)
{
    const TapeDev tp = tape_of(const_cast<void*>(tape), ntot);
    const uint32_t npix = (uint32_t)v.width * (uint32_t)v.height;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        const uint64_t g0 = v.offset + (uint64_t)p * (uint32_t)v.spp;
        float acc[3] = {0.f, 0.f, 0.f};
        for (int smp = 0; smp < v.spp; ++smp)
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[k] = __fadd_rn(acc[k], tp.rad[k][g0 + smp]);
#pragma unroll
        for (int k = 0; k < 3; ++k) img[3 * (size_t)p + k] = acc[k] / (float)v.spp;
    }
}

// ---------------------------------------------------------------------------------------
// persistent batched kernel: every view of every scene in one launch. Each warp pulls chunks
// of consecutive samples from a device counter. An iteration first refills and traces until
// every lane holds a ray that hit something (lanes whose ray escaped finish their sample and
// take the next one), so that the expensive part -- shading with RIS over M candidates --
// runs on full warps; then the shadow rays of those vertices are traced.
// ---------------------------------------------------------------------------------------
template <bool WIDE>
__device__ __forceinline__ void persistent_body(const SceneDev* __restrict__ scenes,
                                                const ViewDev* __restrict__ views, int n_views, uint64_t total,
                                                Rng rng, int M, unsigned long long* work, uint32_t chunk,
                                                void* tape, int nvx, unsigned long long* counters)
{
    extern __shared__ __align__(16) uint32_t sstk[];
    const TapeDev tp = tape_of(tape, total, nvx);
    const int lane = lane_id();
    uint32_t* mystk = sstk + threadIdx.x;

    bool has_path = false, has_hit = false;
    uint64_t g = 0;
    int b = 0, B = 1, origin = -1, tri0 = -1, cand0 = -1, env_ok = 0;
    uint32_t pixel = 0, smp = 0, vidx = 0;
    float3 o = f3(0.f, 0.f, 0.f), d = f3(0.f, 0.f, 1.f), beta = f3(1.f, 1.f, 1.f), bind = beta;
    float3 rad = f3(0.f, 0.f, 0.f), lind = rad;
    float wv0 = 0.0f, tmin = 0.0f;
    const SceneDev* sp = scenes;
    Hit h;
    h.tri = -1;

    uint64_t pool = 0, pool_end = 0;
    bool exhausted = false;
    unsigned long long n_cont = 0, n_shadow = 0, n_cand = 0, n_prim = 0;

    while (true) {
        // ---- refill and trace until the warp is full of hits (bounded number of passes) ----
        for (int pass = 0; pass < 8; ++pass) {
            const unsigned idle = __ballot_sync(MR_FULL, !has_path);
            if (idle && pool == pool_end && !exhausted) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(work, (unsigned long long)chunk);
                base = __shfl_sync(MR_FULL, base, 0);
                if (base >= total) exhausted = true;
                else {
                    pool = base;
                    pool_end = (base + chunk < total) ? base + chunk : total;
                }
            }
            if (idle && pool < pool_end) {
                const uint64_t avail = pool_end - pool;
                const unsigned rank = __popc(idle & lanemask_lt());
                if (!has_path && rank < avail) {
                    g = pool + rank;
                    int vi;
                    const ViewDev& v = view_of(views, n_views, g, vi);
                    sp = scenes + v.scene;
                    const uint32_t sid = (uint32_t)(g - v.offset);
                    pixel = sid / (uint32_t)v.spp;
                    smp = sid % (uint32_t)v.spp;
                    vidx = (uint32_t)v.index;
                    B = v.bounces;
                    const int px = (int)(pixel % (uint32_t)v.width), py = (int)(pixel / (uint32_t)v.width);
                    const uint4 x = rng.draw(pixel, smp, vidx, 0u, PURPOSE_CAMERA, 0u);
                    o = f3(v.c2w[3], v.c2w[7], v.c2w[11]);
                    d = camera_dir(v, px, py, u24(x.x), u24(x.y));
                    beta = bind = f3(1.f, 1.f, 1.f);
                    rad = lind = f3(0.f, 0.f, 0.f);
                    b = 0;
                    origin = -1;
                    tri0 = -1;
                    cand0 = -1;
                    wv0 = 0.0f;
                    env_ok = *sp->env_ok_dev;
                    tmin = *sp->tmin_dev;
                    tape_vx_init(tp, g);
                    has_path = true;
                    has_hit = false;
                    ++n_prim;
                }
                const uint64_t took = ((uint64_t)__popc(idle) < avail) ? (uint64_t)__popc(idle) : avail;
                pool += took;
            }
            const bool need = has_path && !has_hit;
            if (!__any_sync(MR_FULL, need)) break;
            if (need) {
                if (WIDE)  // per scene: its 8-wide BVH, or the binary tree of a scene below two triangles
                    trace<false>(*sp, o, d, origin, tmin, __int_as_float(0x7f800000), h, mystk);
                else
                    trace_as<false, false>(*sp, o, d, origin, tmin, __int_as_float(0x7f800000), h, mystk);
                if (h.tri >= 0) {
                    has_hit = true;
                } else {
                    // escaped: a primary ray sees the env; a continuation ray ends the path
                    if (b == 0) {
                        const float4 L = __ldg(sp->env_texel + env_texel_of(*sp, d));
                        rad = f3(L.x, L.y, L.z);
                    }
                    tp.tri[g] = tri0;
                    tp.cand[g] = cand0;
                    tp.wv[g] = wv0;
                    tp.lind[0][g] = lind.x;
                    tp.lind[1][g] = lind.y;
                    tp.lind[2][g] = lind.z;
                    tp.rad[0][g] = rad.x;
                    tp.rad[1][g] = rad.y;
                    tp.rad[2][g] = rad.z;
                    has_path = false;
                }
            }
            if (__all_sync(MR_FULL, has_hit || (!has_path && exhausted && pool == pool_end))) break;
        }
        if (!__any_sync(MR_FULL, has_hit)) {
            if (exhausted && pool == pool_end && !__any_sync(MR_FULL, has_path)) break;
            continue;
        }
        // ---- shade the hits: RIS, shadow ray, continuation ----
        VertexOut out;
        out.shadow = false;
        out.cont = false;
        if (has_hit) {
            const SceneDev& s = *sp;
            if (b == 0) tri0 = h.tri;
            shade_vertex(s, env_ok, rng, pixel, smp, vidx, b, B, M, h, d, beta, bind, out);
            n_cand += (env_ok && M > 0) ? (unsigned long long)M : 0ull;
            if (b == 0) {
                cand0 = out.cand;
                wv0 = out.W;
                tape_directions(tp, g, out);
            } else {
                tape_vx_record(tp, g, b, h, out);
            }
        }
        if (out.shadow) {
            ++n_shadow;
            Hit hs;
            if (WIDE)
                trace<true>(*sp, out.sh_o, out.sh_d, h.tri, tmin, __int_as_float(0x7f800000), hs, mystk);
            else
                trace_as<true, false>(*sp, out.sh_o, out.sh_d, h.tri, tmin, __int_as_float(0x7f800000), hs, mystk);
            if (hs.tri < 0) {
                rad = add_rn(rad, out.add_rad);
                if (b >= 1) lind = add_rn(lind, out.add_lind);
            } else if (b == 0) {
                wv0 = 0.0f;
            } else {
                tape_vx_occluded(tp, g, b);
            }
        }
        if (has_hit) {
            has_hit = false;
            if (out.cont) {
                ++n_cont;
                o = out.x;
                d = out.c_d;
                beta = out.c_beta;
                bind = out.c_bind;
                origin = h.tri;
                ++b;
            } else {
                tp.tri[g] = tri0;
                tp.cand[g] = cand0;
                tp.wv[g] = wv0;
                tp.lind[0][g] = lind.x;
                tp.lind[1][g] = lind.y;
                tp.lind[2][g] = lind.z;
                tp.rad[0][g] = rad.x;
                tp.rad[1][g] = rad.y;
                tp.rad[2][g] = rad.z;
                has_path = false;
            }
        }
    }
    // per-warp counter flush
    for (int off = 16; off > 0; off >>= 1) {
        n_prim += __shfl_xor_sync(MR_FULL, n_prim, off);
        n_cont += __shfl_xor_sync(MR_FULL, n_cont, off);
        n_shadow += __shfl_xor_sync(MR_FULL, n_shadow, off);
        n_cand += __shfl_xor_sync(MR_FULL, n_cand, off);
    }
    if (lane == 0) {
        atomicAdd(counters + 0, n_prim);
        atomicAdd(counters + 1, n_cont);
        atomicAdd(counters + 2, n_shadow);
        atomicAdd(counters + 5, n_cand);
    }
}

// launch-shape variants: the register cap of each (block size, resident blocks per SM)
// pair is set by __launch_bounds__; the autotuner times them on the workload. WIDE: every
// traversal through the 8-wide BVHs (one variant; the binary ones keep their register budget)
template <int BLOCK, int MINB, bool WIDE = false>
__global__ void __launch_bounds__(BLOCK, MINB)
    k_persistent(const SceneDev* __restrict__ scenes, const ViewDev* __restrict__ views, int n_views, uint64_t total,
                 Rng rng, int M, unsigned long long* work, uint32_t chunk, void* tape, int nvx,
                 unsigned long long* counters)
{
    persistent_body<WIDE>(scenes, views, n_views, total, rng, M, work, chunk, tape, nvx, counters);
}

// resolve every view of a batch in one launch: one thread per pixel over all views
__global__ void __launch_bounds__(256) k_resolve_all(const ViewDev* __restrict__ views, int n_views,
                                                     const uint64_t* __restrict__ pix_off, uint64_t total_pix,
                                                     float* const* __restrict__ images, const void* tape,
                                                     uint64_t ntot)
{
    const TapeDev tp = tape_of(const_cast<void*>(tape), ntot);
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < total_pix;
         q += (uint64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_views - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pix_off[mid] <= q) lo = mid;
            else hi = mid - 1;
        }
        const ViewDev& v = views[lo];
        const uint64_t p = q - pix_off[lo];
        const uint64_t g0 = v.offset + p * (uint32_t)v.spp;
        float acc[3] = {0.f, 0.f, 0.f};
        for (int smp = 0; smp < v.spp; ++smp)
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[k] = __fadd_rn(acc[k], tp.rad[k][g0 + smp]);
        float* img = images[lo];
#pragma unroll
        for (int k = 0; k < 3; ++k) img[3 * p + k] = acc[k] / (float)v.spp;
    }
}

// ---------------------------------------------------------------------------------------
// adjoint (PRIMARY mode): replay of the primary vertex from the tape and the random stream
// ---------------------------------------------------------------------------------------
// reverse-mode derivative of Q = f_r(wo, wi) max(0, n.wi) (per channel) for the upstream
// gradient gq: gm = (d/d albedo[3], d/d roughness, d/d metallic, d/d n[3]). DEMOD: of the
// demodulated lobes (diffuse reflectance 1: no albedo or metallic term through it)
template <bool DEMOD = false>
__device__ __forceinline__ void brdf_cos_adjoint(float3 n, float3 wo, float3 wi, const Material& m, float3 gq,
                                                 float gm[8])
{
    const float co = dot(n, wo), ci = dot(n, wi);
    if (co <= 0.0f || ci <= 0.0f) return;
    const float r = m.rough;
    const float a = alpha_of(r), a2 = a * a;
    const float3 h = normalize(add(wo, wi));
    const float cnh = dot(n, h), coh = dot(wo, h);
    const float k = ggx_k(n, h, cnh, a2);  // d k / d cnh = 2 cnh (a^2 - 1)
    const float D = a2 / (MR_PI * k * k);
    const float Ao = smith_a(a2, co), Ai = smith_a(a2, ci);
    const float den = ci * Ao + co * Ai;
    const float vis = 0.5f / den;
    const float om = 1.0f - coh;
    const float w5 = (om * om) * (om * om) * om;
    const float alb[3] = {m.alb.x, m.alb.y, m.alb.z};
    const float g[3] = {gq.x, gq.y, gq.z};
    float S = 0.0f, g_ci = 0.0f, g_m = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float kd = DEMOD ? 1.0f : (1.0f - m.metal) * alb[c];
        const float f0 = 0.04f * (1.0f - m.metal) + m.metal * alb[c];
        const float F = f0 * (1.0f - w5) + w5;
        const float gF = g[c] * D * vis * ci;
        const float gkd = DEMOD ? 0.0f : g[c] * ci * MR_INV_PI;
        gm[c] += gkd * (1.0f - m.metal) + gF * (1.0f - w5) * m.metal;
        g_m += -gkd * alb[c] + gF * (1.0f - w5) * (alb[c] - 0.04f);
        S += g[c] * F;
        g_ci += g[c] * (kd * MR_INV_PI + D * vis * F);  // the trailing cosine
    }
    const float gDV = S * ci;
    const float gD = gDV * vis, gvis = gDV * D;
    const float gden = gvis * (-0.5f / (den * den));
    const float k3 = MR_PI * k * k * k;
    float g_a = gD * (2.0f * a / (MR_PI * k * k) - 4.0f * a * a2 * cnh * cnh / k3);
    const float g_cnh = gD * (-4.0f * a2 * cnh * (a2 - 1.0f) / k3);
    g_ci += gden * (Ao + co * (1.0f - a2) * ci / Ai);
    const float g_co = gden * (Ai + ci * (1.0f - a2) * co / Ao);
    g_a += gden * (ci * a * (1.0f - co * co) / Ao + co * a * (1.0f - ci * ci) / Ai);
    gm[3] += (r * r > 1e-3f) ? g_a * 2.0f * r : 0.0f;
    gm[4] += g_m;
    gm[5] += g_ci * wi.x + g_co * wo.x + g_cnh * h.x;
    gm[6] += g_ci * wi.y + g_co * wo.y + g_cnh * h.y;
    gm[7] += g_ci * wi.z + g_co * wo.z + g_cnh * h.z;
}

struct EmitEnv {
    float* g;
    __device__ void operator()(int key, const float (&v)[3]) const
    {
        if (!g) return;
        atomicAdd(g + 3 * (size_t)key, v[0]);
        atomicAdd(g + 3 * (size_t)key + 1, v[1]);
        atomicAdd(g + 3 * (size_t)key + 2, v[2]);
    }
};
struct EmitTex {
    float* ga;
    float* gr;
    float* gm;
    __device__ void operator()(int key, const float (&v)[5]) const
    {
        if (ga) {
            atomicAdd(ga + 3 * (size_t)key, v[0]);
            atomicAdd(ga + 3 * (size_t)key + 1, v[1]);
            atomicAdd(ga + 3 * (size_t)key + 2, v[2]);
        }
        if (gr) atomicAdd(gr + key, v[3]);
        if (gm) atomicAdd(gm + key, v[4]);
    }
};
struct EmitVert {
    float* g;
    __device__ void operator()(int key, const float (&v)[3]) const
    {
        if (!g) return;
        atomicAdd(g + 3 * (size_t)key, v[0]);
        atomicAdd(g + 3 * (size_t)key + 1, v[1]);
        atomicAdd(g + 3 * (size_t)key + 2, v[2]);
    }
};

// The FULL-mode vertex loops call the heavy helpers (shading point, BRDF, its adjoint, the
// candidate redraw, the gradient scatters) through these wrappers; MR_FULL_NOINLINE=1 makes
// them single out-of-line copies. That helped while one kernel held the primary and the later
// vertices (it outgrew the instruction cache); the later-vertex kernel alone is faster inlined.
#ifndef MR_FULL_NOINLINE
#define MR_FULL_NOINLINE 0
#endif
#ifndef MR_FULL_MINB
#define MR_FULL_MINB 2  // resident blocks of 256 threads per SM for the FULL-mode adjoint
#endif
#ifndef MR_FULL_SPLIT
#define MR_FULL_SPLIT 1  // later vertices in their own kernel over samples grouped by vertex count
#endif
#define MR_FULL_CHUNK (1u << 25)  // samples classified per pass
#if MR_FULL_NOINLINE
#define MR_FULL_FN __device__ __noinline__
#else
#define MR_FULL_FN __device__ __forceinline__
#endif

MR_FULL_FN void fv_shade(const SceneDev& s, int tri, float u, float v, float3 d, Shade& sh)
{
    shade_at(s, tri, u, v, d, sh);
}

MR_FULL_FN float3 fv_brdf(float3 n, float3 wo, float3 wi, const Material& m) { return brdf_cos(n, wo, wi, m); }

MR_FULL_FN void fv_brdf_adjoint(float3 n, float3 wo, float3 wi, const Material& m, float3 gq, float* gm)
{
    brdf_cos_adjoint(n, wo, wi, m, gq, gm);
}

// the selected candidate of vertex b, redrawn from its Philox block
MR_FULL_FN void fv_candidate(const SceneDev& s, const Rng& rng, uint32_t pixel, uint32_t smp, uint32_t view,
                             uint32_t b, uint32_t cand, float3& y, int& ytex)
{
    const uint4 x = rng.draw(pixel, smp, view, b, PURPOSE_CANDIDATE, cand);
    env_candidate(s, x.x, x.y, x.w, y, ytex);
}

// one vertex's env and texture gradients; warp-collective when every lane is of one scene
MR_FULL_FN void fv_scatter(int env_key, const float* env_v, const int* tex_key, const float* tex_v, const GradDev& gd,
                           bool uniform_scene)
{
    if (uniform_scene) {
        const float ev[3] = {env_v[0], env_v[1], env_v[2]};
        scatter_agg<3>(env_key, ev, EmitEnv{gd.env});
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float tv[5] = {tex_v[5 * q], tex_v[5 * q + 1], tex_v[5 * q + 2], tex_v[5 * q + 3], tex_v[5 * q + 4]};
            scatter_agg<5>(tex_key[q], tv, EmitTex{gd.albedo, gd.rough, gd.metal});
        }
    } else {
        const float ev[3] = {env_v[0], env_v[1], env_v[2]};
        if (env_key >= 0) EmitEnv{gd.env}(env_key, ev);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float tv[5] = {tex_v[5 * q], tex_v[5 * q + 1], tex_v[5 * q + 2], tex_v[5 * q + 3], tex_v[5 * q + 4]};
            if (tex_key[q] >= 0) EmitTex{gd.albedo, gd.rough, gd.metal}(tex_key[q], tv);
        }
    }
}

// vertices per path the FULL-mode adjoint walks (primary included)
#define MR_FULL_MAXV 16
static_assert(MR_FULL_MAXV == MIRRES_FULL_MAX_BOUNCES, "FULL-mode vertex limit");

// FULL mode, forward pass over the vertices b >= 1 of one sample (the gradients of indirect
// rays, which the paper detaches in Sec. 4.2 and names as missing in Appendix C): from the
// tape records, the throughput beta_b into each vertex, its direct light V W L_env(y) f_r(y)
// and its continuation factor f_r(wc) / p_ind. Returns the number of vertices (primary
// included). beta = throughput into vertex 1, d = the primary continuation direction.
__device__ __forceinline__ int full_forward(const SceneDev& s, const Rng& rng, const TapeDev& tp, uint64_t g,
                                            uint32_t pixel, uint32_t smp, uint32_t view, int bounces, float3 beta,
                                            float3 d, float3* vbeta, float3* vdir, float3* vfcp)
{
    int nv = 1;
    const int last = min(min(bounces - 1, tp.nvx), MR_FULL_MAXV - 1);
    for (int b = 1; b <= last; ++b) {
        const int tri = (int)*vx_at(tp, b, VX_TRI, g);
        if (tri < 0) break;
        Shade sh;
        fv_shade(s, tri, __uint_as_float(*vx_at(tp, b, VX_U, g)), __uint_as_float(*vx_at(tp, b, VX_V, g)), d, sh);
        const float3 wo = f3(-d.x, -d.y, -d.z);
        float3 dir = f3(0.f, 0.f, 0.f), fcp = f3(0.f, 0.f, 0.f);
        const int cand = (int)*vx_at(tp, b, VX_CAND, g);
        const float wv = __uint_as_float(*vx_at(tp, b, VX_WV, g));
        if (cand >= 0 && wv != 0.0f) {
            float3 y;
            int ytex;
            fv_candidate(s, rng, pixel, smp, view, (uint32_t)b, (uint32_t)cand, y, ytex);
            const float3 fy = fv_brdf(sh.n, wo, y, sh.m);
            const float4 L = __ldg(s.env_texel + ytex);
            dir = f3(wv * L.x * fy.x, wv * L.y * fy.y, wv * L.z * fy.z);
        }
        const float p = __uint_as_float(*vx_at(tp, b, VX_P, g));
        const float3 wc = f3(__uint_as_float(*vx_at(tp, b, VX_WC, g)), __uint_as_float(*vx_at(tp, b, VX_WC + 1, g)),
                             __uint_as_float(*vx_at(tp, b, VX_WC + 2, g)));
        if (p > 0.0f) {
            const float3 fc = fv_brdf(sh.n, wo, wc, sh.m);
            fcp = f3(fc.x / p, fc.y / p, fc.z / p);
        }
        vbeta[b] = beta;
        vdir[b] = dir;
        vfcp[b] = fcp;
        beta = f3(beta.x * fcp.x, beta.y * fcp.y, beta.z * fcp.z);
        d = wc;
        nv = b + 1;
        if (!(p > 0.0f)) break;
    }
    return nv;
}

// FULL mode, backward pass from the last vertex to vertex 1: with Lin_b the light arriving at
// x_b along wc_b from the rest of the path (Lin = direct_{b+1} + f_r/p_{b+1} Lin_{b+1}), the
// material at x_b receives beta_b [V W L_env(y) d f_r(y) + Lin_b / p_b d f_r(wc)] and the env
// texel of y receives beta_b V W f_r(y), per channel and weighted by dL/dI. The hit point is
// held fixed on its triangle (no geometric derivative beyond the primary vertex). Every lane
// of the warp calls this (the scatters are warp-collective); lanes with nv < 2 only take part.
__device__ __forceinline__ void full_backward(const SceneDev& s, const Rng& rng, const TapeDev& tp, uint64_t g,
                                              uint32_t pixel, uint32_t smp, uint32_t view, int nv, float3 gI,
                                              const float3* vbeta, const float3* vdir, const float3* vfcp,
                                              const GradDev& gd, bool uniform_scene)
{
    const int wnv = __reduce_max_sync(MR_FULL, nv);
    float3 lin = f3(0.f, 0.f, 0.f);
    for (int b = wnv - 1; b >= 1; --b) {
        int env_key = -1, tex_key[4] = {-1, -1, -1, -1};
        float env_v[3] = {0.f, 0.f, 0.f};
        float tex_v[20];
        if (b < nv) {
            const float3 d = (b == 1) ? f3(tp.wc[0][g], tp.wc[1][g], tp.wc[2][g])
                                      : f3(__uint_as_float(*vx_at(tp, b - 1, VX_WC, g)),
                                           __uint_as_float(*vx_at(tp, b - 1, VX_WC + 1, g)),
                                           __uint_as_float(*vx_at(tp, b - 1, VX_WC + 2, g)));
            const int tri = (int)*vx_at(tp, b, VX_TRI, g);
            Shade sh;
            fv_shade(s, tri, __uint_as_float(*vx_at(tp, b, VX_U, g)), __uint_as_float(*vx_at(tp, b, VX_V, g)), d, sh);
            const float3 wo = f3(-d.x, -d.y, -d.z);
            const float3 bt = vbeta[b];
            float gm[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const int cand = (int)*vx_at(tp, b, VX_CAND, g);
            const float wv = __uint_as_float(*vx_at(tp, b, VX_WV, g));
            if (cand >= 0 && wv != 0.0f) {
                float3 y;
                int ytex;
                fv_candidate(s, rng, pixel, smp, view, (uint32_t)b, (uint32_t)cand, y, ytex);
                const float3 fy = fv_brdf(sh.n, wo, y, sh.m);
                const float4 L = __ldg(s.env_texel + ytex);
                env_key = ytex;
                env_v[0] = gI.x * bt.x * wv * fy.x;
                env_v[1] = gI.y * bt.y * wv * fy.y;
                env_v[2] = gI.z * bt.z * wv * fy.z;
                fv_brdf_adjoint(sh.n, wo, y, sh.m, f3(gI.x * bt.x * wv * L.x, gI.y * bt.y * wv * L.y, gI.z * bt.z * wv * L.z),
                                gm);
            }
            const float p = __uint_as_float(*vx_at(tp, b, VX_P, g));
            if (p > 0.0f && (lin.x != 0.0f || lin.y != 0.0f || lin.z != 0.0f)) {
                const float3 wc = f3(__uint_as_float(*vx_at(tp, b, VX_WC, g)),
                                     __uint_as_float(*vx_at(tp, b, VX_WC + 1, g)),
                                     __uint_as_float(*vx_at(tp, b, VX_WC + 2, g)));
                fv_brdf_adjoint(sh.n, wo, wc, sh.m,
                                f3(gI.x * bt.x * lin.x / p, gI.y * bt.y * lin.y / p, gI.z * bt.z * lin.z / p), gm);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                tex_key[q] = sh.tp.idx[q];
#pragma unroll
                for (int c = 0; c < 5; ++c) tex_v[5 * q + c] = sh.tp.w[q] * gm[c];
            }
            const float3 dr = vdir[b], fp = vfcp[b];
            lin = f3(dr.x + fp.x * lin.x, dr.y + fp.y * lin.y, dr.z + fp.z * lin.z);
        } else {
#pragma unroll
            for (int c = 0; c < 20; ++c) tex_v[c] = 0.0f;
        }
        fv_scatter(env_key, env_v, tex_key, tex_v, gd, uniform_scene);
    }
}

// Adjoint of every sample. PRIMARY mode (FULL = false): the primary vertex, replayed from the
// tape. FULL mode: in addition the vertices b >= 1 from their tape records (see
// full_vertices below). DEMOD (PRIMARY only): of the demodulated lighting of the monochrome
// light regulariser instead of the radiance -- the same primary-vertex terms with the
// demodulated lobes, and nothing for an escaping primary ray. All 32 lanes of a warp run the
// same number of rounds, so the warp-collective scatters see every lane.
template <bool FULL, int MINB, bool INTERP, bool DEMOD = false>
__global__ void __launch_bounds__(256, MINB) k_backward(const SceneDev* __restrict__ scenes,
                                                        const ViewDev* __restrict__ views, int n_views, uint64_t total,
                                                        Rng rng, const float* const* __restrict__ d_images,
                                                        const GradDev* __restrict__ grads, const void* tape, int nvx,
                                                        unsigned long long* counters)
{
    static_assert(!(FULL && DEMOD), "the demodulated lighting is differentiated in PRIMARY mode only");
    const TapeDev tp = tape_of(const_cast<void*>(tape), total, nvx);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t rounds = (total + stride - 1) / stride;
    unsigned long long n_diff = 0;
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t g = r * stride + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
        const bool live = g < total;
        int env_key = -1, tex_key[4] = {-1, -1, -1, -1}, vert_key[3] = {-1, -1, -1};
        float env_v[3] = {0.f, 0.f, 0.f};
        float tex_v[4][5];
        float vert_v[3][3];
        float3 gS = f3(0.f, 0.f, 0.f);  // d loss / d S of the interpolated normal
        float bw_u = 0.0f, bw_v = 0.0f;
        int scene_id = 0;
        // FULL mode: the later vertices' throughput, direct light and continuation factor
        int nv = 0;
        float3 gI_f = f3(0.f, 0.f, 0.f);
        float3 vbeta[FULL ? MR_FULL_MAXV : 1], vdir[FULL ? MR_FULL_MAXV : 1], vfcp[FULL ? MR_FULL_MAXV : 1];
        uint32_t f_pixel = 0, f_smp = 0, f_view = 0;
        if (live) {
            int vi;
            const ViewDev& v = view_of(views, n_views, g, vi);
            scene_id = v.scene;
            const SceneDev s = scenes[v.scene];
            const uint32_t sid = (uint32_t)(g - v.offset);
            const uint32_t pixel = sid / (uint32_t)v.spp, smp = sid % (uint32_t)v.spp;
            const float* dimg = d_images[vi];
            const float inv_spp = 1.0f / (float)v.spp;
            const float3 gI = f3(dimg[3 * (size_t)pixel] * inv_spp, dimg[3 * (size_t)pixel + 1] * inv_spp,
                                 dimg[3 * (size_t)pixel + 2] * inv_spp);
            if (gI.x != 0.0f || gI.y != 0.0f || gI.z != 0.0f) {
                ++n_diff;
                const int px = (int)(pixel % (uint32_t)v.width), py = (int)(pixel / (uint32_t)v.width);
                const uint4 xc = rng.draw(pixel, smp, (uint32_t)v.index, 0u, PURPOSE_CAMERA, 0u);
                const float3 o = f3(v.c2w[3], v.c2w[7], v.c2w[11]);
                const float3 d = camera_dir(v, px, py, u24(xc.x), u24(xc.y));
                const int tri = tp.tri[g];
                if (tri < 0) {
                    if (!DEMOD) {
                        env_key = env_texel_of(s, d);
                        env_v[0] = gI.x;
                        env_v[1] = gI.y;
                        env_v[2] = gI.z;
                    }
                } else {
                    float3 v0, e1, e2;
                    int tchk;
                    load_tri(s, __ldg(s.leaf_of + tri), v0, e1, e2, tchk);
                    float t, u, vv;
                    tri_solve(o, d, v0, e1, e2, t, u, vv);
                    Shade sh;
                    shade_at<INTERP>(s, tri, u, vv, d, sh);
                    const float3 wo = f3(-d.x, -d.y, -d.z);
                    float gm[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    const int cand = tp.cand[g];
                    const float wv = tp.wv[g];
                    if (cand >= 0 && wv != 0.0f) {
                        // the selected candidate's direction and texel, as the forward drew them
                        const float3 y = f3(tp.y[0][g], tp.y[1][g], tp.y[2][g]);
                        const int ytex = tp.ytex[g];
                        const float3 fc = brdf_cos<DEMOD>(sh.n, wo, y, sh.m);
                        const float4 L = __ldg(s.env_texel + ytex);
                        env_key = ytex;
                        env_v[0] = gI.x * wv * fc.x;
                        env_v[1] = gI.y * wv * fc.y;
                        env_v[2] = gI.z * wv * fc.z;
                        brdf_cos_adjoint<DEMOD>(sh.n, wo, y, sh.m, f3(gI.x * wv * L.x, gI.y * wv * L.y, gI.z * wv * L.z),
                                                gm);
                    }
                    const float3 li = f3(tp.lind[0][g], tp.lind[1][g], tp.lind[2][g]);
                    if (v.bounces > 1 && (li.x != 0.0f || li.y != 0.0f || li.z != 0.0f)) {
                        // the continuation the forward drew (L_ind != 0 implies it was taken)
                        const float3 wc = f3(tp.wc[0][g], tp.wc[1][g], tp.wc[2][g]);
                        const float pind = tp.pind[g];
                        if (FULL && pind > 0.0f) {
                            // throughput into vertex 1, then the later vertices' forward pass
                            const float3 fc0 = brdf_cos(sh.n, wo, wc, sh.m);
                            gI_f = gI;
                            f_pixel = pixel;
                            f_smp = smp;
                            f_view = (uint32_t)v.index;
                            nv = full_forward(s, rng, tp, g, pixel, smp, (uint32_t)v.index, v.bounces,
                                              f3(fc0.x / pind, fc0.y / pind, fc0.z / pind), wc, vbeta, vdir, vfcp);
                        }
                        if (pind > 0.0f)
                            brdf_cos_adjoint<DEMOD>(sh.n, wo, wc, sh.m,
                                                    f3(gI.x * li.x / pind, gI.y * li.y / pind, gI.z * li.z / pind),
                                                    gm);
                    }
                    // textures (bilinear) and the texture coordinate
                    const Taps& tpz = sh.tp;
                    float dt[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ti = tpz.idx[q];
                        const float w = tpz.w[q];
                        tex_key[q] = ti;
#pragma unroll
                        for (int c = 0; c < 5; ++c) tex_v[q][c] = w * gm[c];
                        dt[q] = gm[0] * __ldg(s.albedo + 3 * (size_t)ti) + gm[1] * __ldg(s.albedo + 3 * (size_t)ti + 1) +
                                gm[2] * __ldg(s.albedo + 3 * (size_t)ti + 2) + gm[3] * __ldg(s.rough + ti) +
                                gm[4] * __ldg(s.metal + ti);
                    }
                    // derivative of the bilinear lookup along the texture coordinate, as texel
                    // differences (exactly zero across clamped or equal texels)
                    const float gsu = (float)s.tw * ((1.0f - tpz.fy) * (dt[1] - dt[0]) + tpz.fy * (dt[3] - dt[2]));
                    const float gsv = (float)s.th * ((1.0f - tpz.fx) * (dt[2] - dt[0]) + tpz.fx * (dt[3] - dt[1]));
                    const float* uv = s.tri_uv + 6 * (size_t)tri;
                    float gu = gsu * (__ldg(uv + 2) - __ldg(uv + 0)) + gsv * (__ldg(uv + 3) - __ldg(uv + 1));
                    float gv = gsu * (__ldg(uv + 4) - __ldg(uv + 0)) + gsv * (__ldg(uv + 5) - __ldg(uv + 1));
                    int vid[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) vid[c] = __ldg(s.tris + 3 * (size_t)tri + c);
                    if (sh.interp) {
                        // n = nsg S / |S|, S = w0 VN_a + u VN_b + v VN_c: to (u, v) here, to the
                        // vertex normals through the per-vertex accumulator (a later pass
                        // takes them to the faces around each vertex)
                        const float il = rsqrtf(dot(sh.S, sh.S));
                        const float3 sn = mul(sh.S, il);
                        const float3 gsn = mul(f3(gm[5], gm[6], gm[7]), sh.nsg);
                        gS = mul(sub(gsn, mul(sn, dot(sn, gsn))), il);
                        const float3 na = xyz(__ldg(s.vnrm + vid[0])), nb = xyz(__ldg(s.vnrm + vid[1])),
                                     nc = xyz(__ldg(s.vnrm + vid[2]));
                        gu += dot(gS, sub(nb, na));
                        gv += dot(gS, sub(nc, na));
                    }
                    // (u, v) through the intersection: A = [e1 | e2 | -d], z = A^-T (gu, gv, 0)
                    const float3 md = f3(-d.x, -d.y, -d.z);
                    const float3 r0 = cross(e2, md), r1 = cross(md, e1);
                    const float det = dot(e1, r0);
                    const float3 z = mul(add(mul(r0, gu), mul(r1, gv)), 1.0f / det);
                    bw_u = u;
                    bw_v = vv;
                    const float bw[3] = {1.0f - u - vv, u, vv};
                    float3 gvx[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) gvx[c] = mul(z, -bw[c]);
                    if (!sh.interp) {
                        // n = sign * N / |N|, N = e1 x e2
                        const float Nl = sqrtf(dot(sh.N, sh.N));
                        const float3 Nh = mul(sh.N, 1.0f / Nl);
                        const float3 gNh = mul(f3(gm[5], gm[6], gm[7]), sh.sign);
                        const float3 gN = mul(sub(gNh, mul(Nh, dot(Nh, gNh))), 1.0f / Nl);
                        const float3 ge1 = cross(e2, gN), ge2 = cross(gN, e1);
                        gvx[0] = sub(gvx[0], add(ge1, ge2));
                        gvx[1] = add(gvx[1], ge1);
                        gvx[2] = add(gvx[2], ge2);
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        vert_key[c] = (vid[c] >= 0 && vid[c] < s.n_verts) ? vid[c] : -1;
                        vert_v[c][0] = gvx[c].x;
                        vert_v[c][1] = gvx[c].y;
                        vert_v[c][2] = gvx[c].z;
                    }
                }
            }
        }
        // scatters are keyed per scene; lanes of other scenes never share a key group
        // because the key is combined with the scene id in the match
        const GradDev gd = grads[scene_id];
        float* const gvn = (INTERP && gd.verts) ? scenes[scene_id].gvn : nullptr;  // interpolated normals only
        const unsigned same_scene = __match_any_sync(MR_FULL, scene_id);
        if (same_scene == MR_FULL) {
            scatter_agg<3>(env_key, env_v, EmitEnv{gd.env});
#pragma unroll
            for (int q = 0; q < 4; ++q) scatter_agg<5>(tex_key[q], tex_v[q], EmitTex{gd.albedo, gd.rough, gd.metal});
#pragma unroll
            for (int c = 0; c < 3; ++c) scatter_agg<3>(vert_key[c], vert_v[c], EmitVert{gd.verts});
            if (gvn) {
                const float bw[3] = {1.0f - bw_u - bw_v, bw_u, bw_v};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float gv3[3] = {gS.x * bw[c], gS.y * bw[c], gS.z * bw[c]};
                    scatter_agg<3>(vert_key[c], gv3, EmitVert{gvn});
                }
            }
        } else {
            if (env_key >= 0) EmitEnv{gd.env}(env_key, env_v);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (tex_key[q] >= 0) EmitTex{gd.albedo, gd.rough, gd.metal}(tex_key[q], tex_v[q]);
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (vert_key[c] >= 0) EmitVert{gd.verts}(vert_key[c], vert_v[c]);
            if (gvn) {
                const float bw[3] = {1.0f - bw_u - bw_v, bw_u, bw_v};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float gv3[3] = {gS.x * bw[c], gS.y * bw[c], gS.z * bw[c]};
                    if (vert_key[c] >= 0) EmitVert{gvn}(vert_key[c], gv3);
                }
            }
        }
        if (FULL) {
            const SceneDev* sp = scenes + scene_id;
            full_backward(*sp, rng, tp, g, f_pixel, f_smp, f_view, nv, gI_f, vbeta, vdir, vfcp, gd,
                          same_scene == MR_FULL);
        }
    }
    if (DEMOD) return;  // counters[4] counts the samples of mirres_backward
    for (int off = 16; off > 0; off >>= 1) n_diff += __shfl_xor_sync(MR_FULL, n_diff, off);
    if (lane_id() == 0 && n_diff) atomicAdd(counters + 4, n_diff);
}

// ---------------------------------------------------------------------------------------
// Monochrome light regulariser (Appendix A, L_light): the demodulated diffuse + specular
// lighting at each pixel's primary vertex, from the tape of the render: out[view][pixel] = (mean
// c_d + c_s, fraction of samples whose primary ray hit). The primary vertex is replayed as the
// adjoint does. A block takes a tile of whole pixels of one view (P = floor(256 / spp) pixels,
// one pixel in passes of 256 samples when spp > 256): its threads replay consecutive samples, so
// that every tape word is read coalesced, and each pixel's samples are then summed in order
// from shared memory. tile_off[i] is view i's first tile (tile_off[n_views] = all tiles).
// ---------------------------------------------------------------------------------------
constexpr int LD_BLOCK = 256;

__device__ __forceinline__ int light_tile_pixels(int spp) { return spp <= LD_BLOCK ? LD_BLOCK / spp : 1; }

// c_d + c_s of one sample (0 where its primary ray escaped); *hit = 1 where it hit
template <bool INTERP>
__device__ __forceinline__ float3 light_sample(const SceneDev& s, const ViewDev& v, const TapeDev& tp, Rng rng,
                                               uint32_t pixel, uint32_t smp, uint64_t g, float& hit)
{
    float3 acc = f3(0.f, 0.f, 0.f);
    hit = 0.0f;
    const int tri = tp.tri[g];
    if (tri < 0) return acc;
    hit = 1.0f;
    const int px = (int)(pixel % (uint32_t)v.width), py = (int)(pixel / (uint32_t)v.width);
    const float3 o = f3(v.c2w[3], v.c2w[7], v.c2w[11]);
    const uint4 xc = rng.draw(pixel, smp, (uint32_t)v.index, 0u, PURPOSE_CAMERA, 0u);
    const float3 d = camera_dir(v, px, py, u24(xc.x), u24(xc.y));
    float3 v0, e1, e2;
    int tchk;
    load_tri(s, __ldg(s.leaf_of + tri), v0, e1, e2, tchk);
    float t, u, vv;
    tri_solve(o, d, v0, e1, e2, t, u, vv);
    Shade sh;
    shade_at<INTERP>(s, tri, u, vv, d, sh);
    const float3 wo = f3(-d.x, -d.y, -d.z);
    const float wv = tp.wv[g];
    if (tp.cand[g] >= 0 && wv != 0.0f) {
        const float3 fc = brdf_cos<true>(sh.n, wo, f3(tp.y[0][g], tp.y[1][g], tp.y[2][g]), sh.m);
        const float4 L = __ldg(s.env_texel + tp.ytex[g]);
        acc = add(acc, f3(wv * L.x * fc.x, wv * L.y * fc.y, wv * L.z * fc.z));
    }
    const float3 li = f3(tp.lind[0][g], tp.lind[1][g], tp.lind[2][g]);
    const float pind = tp.pind[g];
    if (v.bounces > 1 && (li.x != 0.0f || li.y != 0.0f || li.z != 0.0f) && pind > 0.0f) {
        const float3 fc = brdf_cos<true>(sh.n, wo, f3(tp.wc[0][g], tp.wc[1][g], tp.wc[2][g]), sh.m);
        acc = add(acc, f3(fc.x / pind * li.x, fc.y / pind * li.y, fc.z / pind * li.z));
    }
    return acc;
}

template <bool INTERP>
__global__ void __launch_bounds__(LD_BLOCK) k_light_demod(const SceneDev* __restrict__ scenes,
                                                          const ViewDev* __restrict__ views,
                                                          const uint64_t* __restrict__ tile_off, int n_views,
                                                          uint64_t total, Rng rng, const void* tape,
                                                          float* const* __restrict__ out)
{
    __shared__ float4 part[LD_BLOCK];
    const TapeDev tp = tape_of(const_cast<void*>(tape), total, 0);
    const uint64_t n_tiles = tile_off[n_views];
    const int tid = threadIdx.x;
    // block-uniform loops: every __syncthreads below is reached by the whole block
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        int vi = 0, hi = n_views - 1;
        while (vi < hi) {
            const int mid = (vi + hi + 1) >> 1;
            if (tile_off[mid] <= tile) vi = mid;
            else hi = mid - 1;
        }
        const ViewDev& v = views[vi];
        const SceneDev s = scenes[v.scene];
        const int spp = v.spp;
        const uint32_t npx = (uint32_t)v.width * (uint32_t)v.height;
        const uint32_t P = (uint32_t)light_tile_pixels(spp);
        const uint32_t first = (uint32_t)(tile - tile_off[vi]) * P;
        const uint32_t tpx = min(P, npx - first);
        const uint32_t nsamp = tpx * (uint32_t)spp;
        const uint64_t g0 = v.offset + (uint64_t)first * (uint64_t)spp;
        float4 carry = make_float4(0.f, 0.f, 0.f, 0.f);  // thread 0, one pixel over several passes
        for (uint32_t base = 0; base < nsamp; base += LD_BLOCK) {
            const uint32_t idx = base + (uint32_t)tid;
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            if (idx < nsamp) {
                const uint32_t pixel = first + idx / (uint32_t)spp, smp = idx % (uint32_t)spp;
                float h;
                const float3 a = light_sample<INTERP>(s, v, tp, rng, pixel, smp, g0 + idx, h);
                c = make_float4(a.x, a.y, a.z, h);
            }
            part[tid] = c;
            __syncthreads();
            if (spp <= LD_BLOCK) {
                if ((uint32_t)tid < tpx) {
                    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int k = 0; k < spp; ++k) {  // the pixel's samples in order
                        const float4 q = part[tid * spp + k];
                        acc = make_float4(acc.x + q.x, acc.y + q.y, acc.z + q.z, acc.w + q.w);
                    }
                    const float inv_spp = 1.0f / (float)spp;
                    reinterpret_cast<float4*>(out[vi])[first + (uint32_t)tid] =
                        make_float4(acc.x * inv_spp, acc.y * inv_spp, acc.z * inv_spp, acc.w * inv_spp);
                }
            } else if (tid == 0) {
                const uint32_t m = min((uint32_t)LD_BLOCK, nsamp - base);
                for (uint32_t k = 0; k < m; ++k) {
                    const float4 q = part[k];
                    carry = make_float4(carry.x + q.x, carry.y + q.y, carry.z + q.z, carry.w + q.w);
                }
            }
            __syncthreads();
        }
        if (spp > LD_BLOCK && tid == 0) {
            const float inv_spp = 1.0f / (float)spp;
            reinterpret_cast<float4*>(out[vi])[first] =
                make_float4(carry.x * inv_spp, carry.y * inv_spp, carry.z * inv_spp, carry.w * inv_spp);
        }
    }
}

// ---------------------------------------------------------------------------------------
// FULL mode, later vertices: the primary vertex of every sample is differentiated by the
// PRIMARY kernel; the vertices b >= 1 run here over the samples that have any, grouped by
// their vertex count (longest first) so that the warp-uniform vertex loops keep their lanes
// busy. Per chunk of samples: count per class, scan, scatter the sample ids, walk them.
// ---------------------------------------------------------------------------------------
// vertices the FULL walk of sample g visits (primary included), 0 when it has nothing to
// walk: the same conditions and the same stopping rule as the walk itself
__device__ __forceinline__ int full_count(const ViewDev* views, int n_views, const float* const* d_images,
                                          const TapeDev& tp, uint64_t g)
{
    int vi;
    const ViewDev& v = view_of(views, n_views, g, vi);
    if (v.bounces < 2 || tp.tri[g] < 0) return 0;
    const uint32_t pixel = (uint32_t)(g - v.offset) / (uint32_t)v.spp;
    const float* dimg = d_images[vi];
    const float inv_spp = 1.0f / (float)v.spp;
    if (dimg[3 * (size_t)pixel] * inv_spp == 0.0f && dimg[3 * (size_t)pixel + 1] * inv_spp == 0.0f &&
        dimg[3 * (size_t)pixel + 2] * inv_spp == 0.0f)
        return 0;
    if (tp.lind[0][g] == 0.0f && tp.lind[1][g] == 0.0f && tp.lind[2][g] == 0.0f) return 0;
    if (!(tp.pind[g] > 0.0f)) return 0;
    int nv = 1;
    const int last = min(min(v.bounces - 1, tp.nvx), MR_FULL_MAXV - 1);
    for (int b = 1; b <= last; ++b) {
        if ((int)*vx_at(tp, b, VX_TRI, g) < 0) break;
        nv = b + 1;
        if (!(__uint_as_float(*vx_at(tp, b, VX_P, g)) > 0.0f)) break;
    }
    return nv;
}

// warp-aggregated add of 1 to counter[bin] for every lane with bin >= 0; returns the lane's
// rank within its bin's block of slots (old value + lanes of the same bin below it)
__device__ __forceinline__ unsigned int bin_append(int bin, unsigned int* counter)
{
    const unsigned peers = __match_any_sync(MR_FULL, bin);
    const int leader = __ffs(peers) - 1;
    unsigned int base = 0;
    if (bin >= 0 && lane_id() == leader) base = atomicAdd(counter + bin, (unsigned)__popc(peers));
    base = __shfl_sync(MR_FULL, base, leader);
    return base + (unsigned)__popc(peers & lanemask_lt());
}

// pass 1 (scatter = false): per-class counts; pass 3 (scatter = true): sample ids (relative to
// `first`) into their class's slots, classes ordered by decreasing vertex count
template <bool SCATTER>
__global__ void __launch_bounds__(256) k_full_classify(const ViewDev* __restrict__ views, int n_views,
                                                       const float* const* __restrict__ d_images, const void* tape,
                                                       uint64_t total, int nvx, uint64_t first, uint32_t n,
                                                       unsigned int* __restrict__ bins, uint32_t* __restrict__ list)
{
    const TapeDev tp = tape_of(const_cast<void*>(tape), total, nvx);
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t rounds = (n + stride - 1) / stride;
    for (uint32_t r = 0; r < rounds; ++r) {  // warp-uniform
        const uint32_t i = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
        const int nv = i < n ? full_count(views, n_views, d_images, tp, first + i) : 0;
        const int bin = nv >= 2 ? MR_FULL_MAXV - nv : -1;
        const unsigned int slot = bin_append(bin, SCATTER ? bins + 16 : bins);
        if (SCATTER && bin >= 0) list[slot] = i;
    }
}

// pass 2: cursors = exclusive scan of the counts, bins[32] = the number of listed samples
__global__ void k_full_scan(unsigned int* bins)
{
    if (threadIdx.x != 0) return;
    unsigned int acc = 0;
    for (int k = 0; k < 16; ++k) {
        bins[16 + k] = acc;
        acc += bins[k];
    }
    bins[32] = acc;
}

// pass 4: the later vertices of the listed samples
__global__ void __launch_bounds__(256, MR_FULL_MINB) k_full(const SceneDev* __restrict__ scenes,
                                                           const ViewDev* __restrict__ views, int n_views,
                                                           uint64_t total, Rng rng,
                                                           const float* const* __restrict__ d_images,
                                                           const GradDev* __restrict__ grads, const void* tape, int nvx,
                                                           uint64_t first, const uint32_t* __restrict__ list,
                                                           const unsigned int* __restrict__ bins, uint32_t cap)
{
    const TapeDev tp = tape_of(const_cast<void*>(tape), total, nvx);
    const uint32_t n = min(bins[32], cap);
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t rounds = (n + stride - 1) / stride;
    for (uint32_t r = 0; r < rounds; ++r) {  // warp-uniform: full_backward's scatters are warp-collective
        const uint32_t i = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
        int nv = 0, scene_id = 0;
        float3 gI = f3(0.f, 0.f, 0.f);
        float3 vbeta[MR_FULL_MAXV], vdir[MR_FULL_MAXV], vfcp[MR_FULL_MAXV];
        uint32_t pixel = 0, smp = 0, view = 0;
        uint64_t g = 0;
        if (i < n) {
            g = first + list[i];
            int vi;
            const ViewDev& v = view_of(views, n_views, g, vi);
            scene_id = v.scene;
            const SceneDev s = scenes[v.scene];
            const uint32_t sid = (uint32_t)(g - v.offset);
            pixel = sid / (uint32_t)v.spp;
            smp = sid % (uint32_t)v.spp;
            view = (uint32_t)v.index;
            const float* dimg = d_images[vi];
            const float inv_spp = 1.0f / (float)v.spp;
            gI = f3(dimg[3 * (size_t)pixel] * inv_spp, dimg[3 * (size_t)pixel + 1] * inv_spp,
                    dimg[3 * (size_t)pixel + 2] * inv_spp);
            // the primary vertex again, for the throughput into vertex 1
            const int px = (int)(pixel % (uint32_t)v.width), py = (int)(pixel / (uint32_t)v.width);
            const uint4 xc = rng.draw(pixel, smp, view, 0u, PURPOSE_CAMERA, 0u);
            const float3 o = f3(v.c2w[3], v.c2w[7], v.c2w[11]);
            const float3 d = camera_dir(v, px, py, u24(xc.x), u24(xc.y));
            const int tri = tp.tri[g];
            float3 v0, e1, e2;
            int tchk;
            load_tri(s, __ldg(s.leaf_of + tri), v0, e1, e2, tchk);
            float t, u, vv;
            tri_solve(o, d, v0, e1, e2, t, u, vv);
            Shade sh;
            shade_at(s, tri, u, vv, d, sh);
            const float3 wo = f3(-d.x, -d.y, -d.z);
            const float3 wc = f3(tp.wc[0][g], tp.wc[1][g], tp.wc[2][g]);
            const float pind = tp.pind[g];
            const float3 fc0 = brdf_cos(sh.n, wo, wc, sh.m);
            nv = full_forward(s, rng, tp, g, pixel, smp, view, v.bounces, f3(fc0.x / pind, fc0.y / pind, fc0.z / pind),
                              wc, vbeta, vdir, vfcp);
        }
        const GradDev gd = grads[scene_id];
        const unsigned same_scene = __match_any_sync(MR_FULL, scene_id);
        full_backward(scenes[scene_id], rng, tp, g, pixel, smp, view, nv, gI, vbeta, vdir, vfcp, gd,
                      same_scene == MR_FULL);
    }
}

// ---------------------------------------------------------------------------------------
// L2 loss of Eq. (loss_pbr) and its image gradient
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_l2(const float* __restrict__ img, const float* __restrict__ ref, int64_t n,
                                            float* __restrict__ dimg, float* loss)
{
    float acc = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = img[i] - ref[i];
        if (dimg) dimg[i] = 2.0f * e;
        acc += e * e;
    }
    if (!loss) return;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(MR_FULL, acc, off);
    __shared__ float ws[8];
    if (lane_id() == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
        atomicAdd(loss, s);
    }
}

// add one chunk's queue counts to the cumulative counters: per bounce b, qcnt[3b] hits,
// qcnt[3b+1] continuation rays emitted, qcnt[3b+2] shadow rays
__global__ void k_account(unsigned long long* counters, const unsigned int* __restrict__ qcnt, int bounces,
                          uint64_t primary)
{
    if (threadIdx.x != 0) return;
    unsigned long long cont = 0, shadow = 0;
    for (int b = 0; b < bounces; ++b) {
        cont += qcnt[3 * b + 1];
        shadow += qcnt[3 * b + 2];
    }
    // atomics: the accounting of concurrent wave chains may overlap
    atomicAdd(&counters[0], (unsigned long long)primary);
    atomicAdd(&counters[1], cont);
    atomicAdd(&counters[2], shadow);
}

// ray queries for mirres_trace
__global__ void __launch_bounds__(256) k_trace_rays(SceneDev s, const float* __restrict__ rays,
                                                    const int32_t* __restrict__ skip, int64_t n, int any,
                                                    int32_t* __restrict__ hit_tri, float* __restrict__ hit_tuv)
{
    extern __shared__ __align__(16) uint32_t sstk[];
    const float tmin = *s.tmin_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float3 o = f3(rays[6 * i], rays[6 * i + 1], rays[6 * i + 2]);
        const float3 d = f3(rays[6 * i + 3], rays[6 * i + 4], rays[6 * i + 5]);
        const int sk = skip ? skip[i] : -1;
        Hit h;
        if (any) trace<true>(s, o, d, sk, tmin, __int_as_float(0x7f800000), h, sstk + threadIdx.x);
        else trace<false>(s, o, d, sk, tmin, __int_as_float(0x7f800000), h, sstk + threadIdx.x);
        hit_tri[i] = any ? (h.tri >= 0 ? 1 : -1) : h.tri;
        if (hit_tuv && !any) {
            hit_tuv[3 * i] = h.tri >= 0 ? h.t : 0.0f;
            hit_tuv[3 * i + 1] = h.u;
            hit_tuv[3 * i + 2] = h.v;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------------------
static unsigned grid_cap(uint64_t n, int block, int cap)
{
    const uint64_t g = (n + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : (g > (uint64_t)cap ? (uint64_t)cap : g));
}

static size_t stack_bytes(int block) { return sizeof(uint32_t) * MR_SSTACK * (size_t)block; }

void mr_launch_raygen(const ViewDev& v, Rng rng, uint32_t first, uint32_t n, const QueueDev& q, void* tape,
                      uint64_t ntot, int sms, cudaStream_t st, int nvx)
{
    k_raygen<<<grid_cap(n, 256, sms * 8), 256, 0, st>>>(v, rng, first, n, q, tape, ntot, nvx);
}

void mr_launch_closest(const SceneDev& s, const ViewDev& v, int b, const QueueDev& q, const unsigned int* count,
                       unsigned int count_fixed, uint64_t upper, const QueueDev& hq, unsigned int* count_hit,
                       void* tape, uint64_t ntot, int sms, cudaStream_t st)
{
    k_closest<<<grid_cap(upper, 256, sms * 8), 256, stack_bytes(256), st>>>(s, v, b, q, count, count_fixed, hq,
                                                                           count_hit, tape, ntot);
}

void mr_launch_shade(const SceneDev& s, const ViewDev& v, Rng rng, int b, int M, const QueueDev& hq,
                     const unsigned int* count_hit, uint64_t upper, const QueueDev& qout, unsigned int* count_out,
                     const ShadowDev& sq, unsigned int* count_sh, void* tape, uint64_t ntot,
                     unsigned long long* counters, int sms, cudaStream_t st, int nvx)
{
    k_shade<<<grid_cap(upper, 256, sms * 8), 256, 0, st>>>(s, v, rng, b, M, hq, count_hit, qout, count_out, sq,
                                                          count_sh, tape, ntot, nvx, counters);
}

void mr_launch_shadow(const SceneDev& s, const ViewDev& v, int b, const ShadowDev& sq, const unsigned int* count,
                      uint64_t upper, void* tape, uint64_t ntot, int sms, cudaStream_t st, int nvx)
{
    k_shadow<<<grid_cap(upper, 256, sms * 8), 256, stack_bytes(256), st>>>(s, v, b, sq, count, tape, ntot, nvx);
}

void mr_launch_resolve(const ViewDev& v, const void* tape, uint64_t ntot, float* img, int sms, cudaStream_t st)
{
    k_resolve<<<grid_cap((uint64_t)v.width * v.height, 256, sms * 8), 256, 0, st>>>(v, tape, ntot, img);
}

typedef void (*PersistentFn)(const SceneDev*, const ViewDev*, int, uint64_t, Rng, int, unsigned long long*, uint32_t,
                             void*, int, unsigned long long*);

struct PersistentVariant {
    int block, minb;
    PersistentFn fn;
};

static const PersistentVariant kVariants[] = {
    {128, 2, k_persistent<128, 2>}, {128, 3, k_persistent<128, 3>}, {128, 4, k_persistent<128, 4>},
    {128, 5, k_persistent<128, 5>}, {128, 6, k_persistent<128, 6>}, {256, 2, k_persistent<256, 2>},
    {256, 3, k_persistent<256, 3>}, {64, 8, k_persistent<64, 8>},
};

int mr_persistent_variants() { return (int)(sizeof(kVariants) / sizeof(kVariants[0])); }

void mr_persistent_variant_shape(int v, int* block, int* minb)
{
    *block = kVariants[v].block;
    *minb = kVariants[v].minb;
}

// variant for a requested (block, blocks per SM): the same block size with the nearest
// register cap; block 0 (or no variant of that size) = the default (128, 3)
int mr_persistent_pick(int block, int per_sm)
{
    const int dflt = 1;
    if (block == 0) return dflt;
    const int want = per_sm ? per_sm : 3;
    int best = -1, bestd = 1 << 30;
    for (int i = 0; i < mr_persistent_variants(); ++i) {
        if (kVariants[i].block != block) continue;
        const int d = abs(kVariants[i].minb - want);
        if (d < bestd) {
            bestd = d;
            best = i;
        }
    }
    return best < 0 ? dflt : best;
}

int mr_persistent_occupancy_v(int v)
{
    const PersistentVariant& pv = kVariants[v];
    const size_t smem = stack_bytes(pv.block);
    cudaFuncSetAttribute(pv.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pv.fn, pv.block, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n < 1 ? 1 : n;
}

static const PersistentVariant kWideVariant = {128, 3, k_persistent<128, 3, true>};

cudaError_t mr_launch_persistent_v(int v, const SceneDev* scenes, const ViewDev* views, int n_views, uint64_t total,
                                   Rng rng, int M, unsigned long long* work, uint32_t chunk, void* tape,
                                   unsigned long long* counters, int blocks, cudaStream_t st, int nvx, bool wide)
{
    // (with wide BVHs the one wide variant runs; extra blocks find no work left and exit)
    const PersistentVariant& pv = wide ? kWideVariant : kVariants[v];
    const size_t smem = stack_bytes(pv.block);
    cudaError_t e = cudaFuncSetAttribute(pv.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    pv.fn<<<blocks, pv.block, smem, st>>>(scenes, views, n_views, total, rng, M, work, chunk, tape, nvx, counters);
    return cudaGetLastError();
}

// the launch used before variants existed: (block, blocks per SM) mapped to a variant
cudaError_t mr_launch_persistent(const SceneDev* scenes, const ViewDev* views, int n_views, uint64_t total, Rng rng,
                                 int M, unsigned long long* work, uint32_t chunk, void* tape,
                                 unsigned long long* counters, int block, int blocks, cudaStream_t st, int nvx)
{
    const int v = mr_persistent_pick(block, 0);
    return mr_launch_persistent_v(v, scenes, views, n_views, total, rng, M, work, chunk, tape, counters, blocks, st,
                                  nvx, false);
}

int mr_persistent_occupancy(int block) { return mr_persistent_occupancy_v(mr_persistent_pick(block, 0)); }

void mr_launch_resolve_all(const ViewDev* views, int n_views, const uint64_t* pix_off, uint64_t total_pix,
                           float* const* images, const void* tape, uint64_t ntot, int sms, cudaStream_t st)
{
    k_resolve_all<<<grid_cap(total_pix, 256, sms * 8), 256, 0, st>>>(views, n_views, pix_off, total_pix, images, tape,
                                                                     ntot);
}

size_t mr_full_scratch_bytes() { return sizeof(uint32_t) * ((size_t)MR_FULL_CHUNK + 64); }
uint64_t mr_full_chunk() { return MR_FULL_SPLIT ? MR_FULL_CHUNK : 0; }

void mr_launch_backward(const SceneDev* scenes, const ViewDev* views, int n_views, uint64_t total, Rng rng,
                        const float* const* d_images, const GradDev* grads, const void* tape,
                        unsigned long long* counters, int sms, cudaStream_t st, int nvx, void* full_scratch,
                        bool interp)
{
#if MR_FULL_SPLIT
    // the primary vertex of every sample (the tape's FULL records are read by k_full only)
    (interp ? k_backward<false, MR_BWD_MINB, true> : k_backward<false, MR_BWD_MINB, false>)<<<
        grid_cap(total, 256, sms * 8), 256, 0, st>>>(scenes, views, n_views, total, rng, d_images, grads, tape, nvx,
                                                     counters);
    if (nvx <= 0) return;
    unsigned int* bins = static_cast<unsigned int*>(full_scratch);  // [0, 16) counts, [16, 32) cursors, [32] total
    uint32_t* list = bins + 64;
    for (uint64_t first = 0; first < total; first += MR_FULL_CHUNK) {
        const uint32_t n = (uint32_t)std::min<uint64_t>(MR_FULL_CHUNK, total - first);
        const unsigned grid = grid_cap(n, 256, sms * 8);
        cudaMemsetAsync(bins, 0, sizeof(unsigned int) * 64, st);
        k_full_classify<false><<<grid, 256, 0, st>>>(views, n_views, d_images, tape, total, nvx, first, n, bins, list);
        k_full_scan<<<1, 32, 0, st>>>(bins);
        k_full_classify<true><<<grid, 256, 0, st>>>(views, n_views, d_images, tape, total, nvx, first, n, bins, list);
        k_full<<<grid, 256, 0, st>>>(scenes, views, n_views, total, rng, d_images, grads, tape, nvx, first, list, bins,
                                     n);
    }
#else
    (void)full_scratch;
    (void)interp;
    if (nvx > 0)
        k_backward<true, MR_FULL_MINB, true><<<grid_cap(total, 256, sms * 8), 256, 0, st>>>(scenes, views, n_views, total, rng,
                                                                          d_images, grads, tape, nvx, counters);
    else
        k_backward<false, MR_BWD_MINB, true><<<grid_cap(total, 256, sms * 8), 256, 0, st>>>(
            scenes, views, n_views, total, rng, d_images, grads, tape, 0, counters);
#endif
}

int mr_light_tile_pixels(int spp) { return spp <= LD_BLOCK ? LD_BLOCK / spp : 1; }

void mr_launch_light_demod(const SceneDev* scenes, const ViewDev* views, const uint64_t* tile_off, int n_views,
                           uint64_t n_tiles, uint64_t total, Rng rng, const void* tape, float* const* out, int sms,
                           cudaStream_t st, bool interp)
{
    if (n_tiles == 0) return;
    const unsigned grid = (unsigned)std::min<uint64_t>(n_tiles, (uint64_t)sms * 8);
    (interp ? k_light_demod<true> : k_light_demod<false>)<<<grid, LD_BLOCK, 0, st>>>(scenes, views, tile_off, n_views,
                                                                                   total, rng, tape, out);
}

void mr_launch_light_backward(const SceneDev* scenes, const ViewDev* views, int n_views, uint64_t total, Rng rng,
                              const float* const* d_demod, const GradDev* grads, const void* tape,
                              unsigned long long* counters, int sms, cudaStream_t st, bool interp)
{
    (interp ? k_backward<false, MR_BWD_MINB, true, true> : k_backward<false, MR_BWD_MINB, false, true>)<<<
        grid_cap(total, 256, sms * 8), 256, 0, st>>>(scenes, views, n_views, total, rng, d_demod, grads, tape, 0,
                                                     counters);
}

void mr_launch_account(unsigned long long* counters, const unsigned int* qcnt, int bounces, uint64_t primary,
                       cudaStream_t st)
{
    k_account<<<1, 32, 0, st>>>(counters, qcnt, bounces, primary);
}

void mr_launch_l2(const float* img, const float* ref, int64_t n, float* dimg, float* loss, int sms, cudaStream_t st)
{
    k_l2<<<grid_cap((uint64_t)n, 256, sms * 8), 256, 0, st>>>(img, ref, n, dimg, loss);
}

void mr_launch_trace_rays(const SceneDev& s, const float* rays, const int32_t* skip, int64_t n, int any,
                          int32_t* hit_tri, float* hit_tuv, int sms, cudaStream_t st)
{
    k_trace_rays<<<grid_cap((uint64_t)n, 256, sms * 8), 256, stack_bytes(256), st>>>(s, rays, skip, n, any, hit_tri,
                                                                                     hit_tuv);
}
