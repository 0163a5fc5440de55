// wave.cu -- batched wavefront: every view of every scene flattened into one sample space and
// processed in large waves (ray generation, then per bounce: closest hit with hit compaction,
// shading with RIS, shadow rays). Stage kernels are grid-stride loops over device-side queue
// counts, so the whole forward is one fixed launch sequence that is captured once as a CUDA
// graph and replayed. Each queued path carries its view index (in the w component of its
// throughput), through which it finds its camera, spp, bounce count and scene.
#include "path.cuh"
#include "render.h"

namespace {

// per-warp flush of a traversal stage's box and triangle test counts (counters idx, idx + 1)
__device__ __forceinline__ void flush_work(unsigned long long* counters, int idx, unsigned int box, unsigned int tri)
{
    box = __reduce_add_sync(MR_FULL, box);
    tri = __reduce_add_sync(MR_FULL, tri);
    if (lane_id() == 0) {
        atomicAdd(counters + idx, (unsigned long long)box);
        atomicAdd(counters + idx + 1, (unsigned long long)tri);
    }
}

__global__ void __launch_bounds__(256) k_wraygen(const ViewDev* __restrict__ views, int n_views, Rng rng,
                                                 uint64_t first, uint32_t n, QueueDev q, void* tape, uint64_t ntot,
                                                 int nvx, ResDev res)
{
    const TapeDev tp = tape_of(tape, ntot, nvx);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t g = first + i;
        int vi;
        const ViewDev& v = view_of(views, n_views, g, vi);
        const uint32_t sid = (uint32_t)(g - v.offset);
        const uint32_t pixel = sid / (uint32_t)v.spp, smp = sid % (uint32_t)v.spp;
        const int px = (int)(pixel % (uint32_t)v.width), py = (int)(pixel / (uint32_t)v.width);
        const uint4 x = rng.draw(pixel, smp, (uint32_t)v.index, 0u, PURPOSE_CAMERA, 0u);
        const float3 d = camera_dir(v, px, py, u24(x.x), u24(x.y));
        q.o[i] = make_float4(v.c2w[3], v.c2w[7], v.c2w[11], __int_as_float(-1));
        q.d[i] = make_float4(d.x, d.y, d.z, __uint_as_float(sid));
        q.b[i] = make_float4(1.f, 1.f, 1.f, __int_as_float(vi));
        q.bi[i] = make_float4(1.f, 1.f, 1.f, 0.f);
        tp.tri[g] = -1;
        tp.cand[g] = -1;
        tp.wv[g] = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            tp.lind[k][g] = 0.0f;
            tp.rad[k][g] = 0.0f;
        }
        tape_vx_init(tp, g);
        if (res.ytex) res.ytex[g] = RES_MISS;
    }
}

template <bool COUNT, bool RASTER, bool WIDE>
__global__ void MR_TRACE_BOUNDS k_wclosest(const SceneDev* __restrict__ scenes,
                                                  const ViewDev* __restrict__ views, int b, QueueDev q,
                                                  const unsigned int* count, unsigned int count_fixed, QueueDev hq,
                                                  unsigned int* count_hit, void* tape, uint64_t ntot,
                                                  unsigned long long* counters, const unsigned long long* raster)
{
    extern __shared__ __align__(16) uint32_t sstk[];
    const TapeDev tp = tape_of(tape, ntot);
    const unsigned int n = count ? *count : count_fixed;
    unsigned int n_box = 0;
    int n_tri = 0;
    const unsigned int stride = gridDim.x * blockDim.x;
    const unsigned int rounds = (n + stride - 1) / stride;
    for (unsigned int r = 0; r < rounds; ++r) {
        const unsigned int i = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
        Hit h;
        h.tri = -1;
        float4 qd = make_float4(0.f, 0.f, 0.f, 0.f), qb = qd;
        if (i < n) {
            const float4 a = q.o[i];
            qd = q.d[i];
            qb = q.b[i];
            const ViewDev& v = views[__float_as_int(qb.w)];
            const SceneDev& s = scenes[v.scene];
            if (RASTER) {
                // primary visibility from the rasteriser: the winning triangle, solved again
                // with the same arithmetic for its (t, u, v)
                const unsigned long long key = raster[i];
                h.t = __int_as_float(0x7f800000);
                h.u = h.v = 0.0f;
                if (key != ~0ull) {
                    const int tri = (int)(unsigned)(key & 0xffffffffull);
                    float3 v0, e1, e2;
                    int tchk;
                    load_tri(s, __ldg(s.leaf_of + tri), v0, e1, e2, tchk);
                    tri_solve(xyz(a), xyz(qd), v0, e1, e2, h.t, h.u, h.v);
                    h.tri = tri;
                }
            } else {
                // the counting variant counts the binary tree's work (the algorithmic work of the
                // path: two box tests per node visit, one solve per triangle), the timed one runs
                // the scene's wide BVH
                if (COUNT) {
                    const int nodes = traverse<false>(s, xyz(a), xyz(qd), __float_as_int(a.w), *s.tmin_dev,
                                                      __int_as_float(0x7f800000), h, sstk + threadIdx.x, blockDim.x,
                                                      &n_tri);
                    n_box += 2u * (unsigned int)max(nodes, 0);
                } else {
                    trace_as<false, WIDE>(s, xyz(a), xyz(qd), __float_as_int(a.w), *s.tmin_dev,
                                          __int_as_float(0x7f800000), h, sstk + threadIdx.x);
                }
            }
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
            hq.b[slot] = qb;
            hq.bi[slot] = q.bi[i];
        }
    }
    if (COUNT) flush_work(counters, CNT_CBOX, n_box, (unsigned int)n_tri);
}

// ---- binning of a ray queue by origin cell and direction octant ----------------------------
// A queue of secondary rays (4 float4 arrays; the third one's w holds the view index) is
// reordered so that rays whose origins share a cell of an 8 x 8 x 8 grid over their scene's
// bounds (Morton order) and whose directions share an octant sit next to each other: a warp of
// neighbouring rays then descends the same subtrees. Counting sort on the 12-bit key: a block
// histogram flushed to a global one, an exclusive scan, and a scatter whose warps reserve
// their slots per key with one atomic per distinct key. The order within a key is arbitrary
// (as the order of the queues already is); each ray's record moves unchanged.
constexpr int BIN_KEYS = 4096;

__device__ __forceinline__ uint32_t spread3(uint32_t x)  // 3 bits -> every third bit
{
    return (x & 1u) | ((x & 2u) << 2) | ((x & 4u) << 4);
}

__device__ __forceinline__ uint32_t bin_key(const SceneDev& s, float3 o, float3 d)
{
    const uint32_t oct = (d.x < 0.0f ? 1u : 0u) | (d.y < 0.0f ? 2u : 0u) | (d.z < 0.0f ? 4u : 0u);
    uint32_t cell = 0;
    if (s.n_tris >= 2) {  // the root node's two child boxes span the scene
        const float4 a = __ldg(s.nodes), b = __ldg(s.nodes + 1), c = __ldg(s.nodes + 2);
        const float lx = fminf(a.x, b.z), ly = fminf(a.y, b.w), lz = fminf(a.z, c.x);
        const float hx = fmaxf(a.w, c.y), hy = fmaxf(b.x, c.z), hz = fmaxf(b.y, c.w);
        auto q = [](float v, float lo, float hi) {
            const float f = (v - lo) / fmaxf(hi - lo, 1e-30f) * 8.0f;
            return (uint32_t)min(max((int)f, 0), 7);  // NaN -> 0
        };
        cell = (spread3(q(o.x, lx, hx)) << 2) | (spread3(q(o.y, ly, hy)) << 1) | spread3(q(o.z, lz, hz));
    }
    return (cell << 3) | oct;
}

__global__ void __launch_bounds__(256) k_bin_hist(const SceneDev* __restrict__ scenes,
                                                  const ViewDev* __restrict__ views, QueueDev q,
                                                  const unsigned int* __restrict__ count, uint16_t* __restrict__ keys,
                                                  unsigned int* __restrict__ hist)
{
    __shared__ unsigned int h[BIN_KEYS];
    for (int k = threadIdx.x; k < BIN_KEYS; k += blockDim.x) h[k] = 0;
    __syncthreads();
    const unsigned int n = *count;
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 o = q.o[i], d = q.d[i];
        const int vi = __float_as_int(q.b[i].w);
        const uint32_t k = bin_key(scenes[views[vi].scene], xyz(o), xyz(d));
        keys[i] = (uint16_t)k;
        atomicAdd(&h[k], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < BIN_KEYS; k += blockDim.x)
        if (h[k]) atomicAdd(&hist[k], h[k]);
}

// exclusive scan of the BIN_KEYS counts in place (one block of 1024 threads, 4 keys each)
__global__ void __launch_bounds__(1024) k_bin_scan(unsigned int* __restrict__ hist)
{
    __shared__ unsigned int wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint4 v = reinterpret_cast<const uint4*>(hist)[t];
    const unsigned int s = v.x + v.y + v.z + v.w;
    unsigned int x = s;
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned int y = __shfl_up_sync(MR_FULL, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned int w = wsum[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned int y = __shfl_up_sync(MR_FULL, w, off);
            if (lane >= off) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    const unsigned int base = x - s + (warp > 0 ? wsum[warp - 1] : 0u);
    reinterpret_cast<uint4*>(hist)[t] = make_uint4(base, base + v.x, base + v.x + v.y, base + v.x + v.y + v.z);
}

// every lane of every warp runs the same number of rounds (the match and shuffle need the
// full warp); `cursor` holds each key's next free slot
__global__ void __launch_bounds__(256) k_bin_scatter(QueueDev in, QueueDev out, const unsigned int* __restrict__ count,
                                                     const uint16_t* __restrict__ keys,
                                                     unsigned int* __restrict__ cursor)
{
    const unsigned int n = *count;
    const unsigned int stride = gridDim.x * blockDim.x;
    const unsigned int rounds = (n + stride - 1) / stride;
    const int lane = lane_id();
    for (unsigned int r = 0; r < rounds; ++r) {
        const unsigned int i = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
        const bool valid = i < n;
        const uint32_t k = valid ? (uint32_t)keys[i] : 0xFFFFFFFFu;
        const unsigned int peers = __match_any_sync(MR_FULL, k);
        const int leader = __ffs(peers) - 1;
        unsigned int base = 0;
        if (valid && lane == leader) base = atomicAdd(&cursor[k], (unsigned int)__popc(peers));
        base = __shfl_sync(MR_FULL, base, leader);
        if (valid) {
            const unsigned int dst = base + (unsigned int)__popc(peers & lanemask_lt());
            out.o[dst] = in.o[i];
            out.d[dst] = in.d[i];
            out.b[dst] = in.b[i];
            out.bi[dst] = in.bi[i];
        }
    }
}

template <bool REUSE, bool INTERP>
__global__ void __launch_bounds__(256, MR_SHADE_MINB) k_wshade(const SceneDev* __restrict__ scenes,
                                                const ViewDev* __restrict__ views, Rng rng, int b, int M,
                                                QueueDev hq, const unsigned int* count_hit, QueueDev qout,
                                                unsigned int* count_out, ShadowDev sq, unsigned int* count_sh,
                                                void* tape, uint64_t ntot, int nvx, ResDev res,
                                                unsigned long long* counters)
{
    const TapeDev tp = tape_of(tape, ntot, nvx);
    const unsigned int n = *count_hit;
    unsigned long long n_cand = 0;
    const unsigned int stride = gridDim.x * blockDim.x;
    const unsigned int rounds = (n + stride - 1) / stride;
    for (unsigned int r = 0; r < rounds; ++r) {
        const unsigned int i = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
        VertexOut out;
        out.shadow = false;
        out.cont = false;
        uint32_t sid = 0;
        int tri = -1, vi = 0;
        if (i < n) {
            const float4 hd = hq.o[i];
            const float4 qd = hq.d[i];
            const float4 qb = hq.b[i];
            vi = __float_as_int(qb.w);
            const ViewDev& v = views[vi];
            const SceneDev& s = scenes[v.scene];
            sid = __float_as_uint(qd.w);
            const uint64_t g = v.offset + sid;
            tri = __float_as_int(hd.w);
            const uint32_t pixel = sid / (uint32_t)v.spp, smp = sid % (uint32_t)v.spp;
            Hit h;
            h.t = hd.x;
            h.u = hd.y;
            h.v = hd.z;
            h.tri = tri;
            const int env_ok = *s.env_ok_dev;
            shade_vertex<INTERP>(s, env_ok, rng, pixel, smp, (uint32_t)v.index, b, v.bounces, M, h, xyz(qd), xyz(qb),
                         xyz(hq.bi[i]), out);
            if (env_ok) n_cand += (unsigned long long)M;
            if (b == 0) {
                tp.tri[g] = tri;
                tp.cand[g] = out.cand;
                tp.wv[g] = out.W;
                tape_directions(tp, g, out);
                if (REUSE) {
                    // spatial reuse: publish the reservoir; k_wreuse merges and traces the shadow ray
                    res.ytex[g] = out.cand >= 0 ? out.ytex : RES_NONE;
                    res.sel[g] = out.cand;
                    res.ysub[g] = out.ysub;
                    res.wsum[g] = out.wsum;
                    res.phat[g] = out.phat;
                    res.m[g] = (float)M;
                    out.shadow = false;
                }
            } else {
                tape_vx_record(tp, g, b, h, out);
            }
        }
        const unsigned int ss = warp_append(out.shadow, count_sh);
        if (out.shadow) {
            sq.o[ss] = make_float4(out.sh_o.x, out.sh_o.y, out.sh_o.z, __int_as_float(tri));
            sq.d[ss] = make_float4(out.sh_d.x, out.sh_d.y, out.sh_d.z, __uint_as_float(sid));
            sq.add[ss] = make_float4(out.add_rad.x, out.add_rad.y, out.add_rad.z, __int_as_float(vi));
            sq.addi[ss] = make_float4(out.add_lind.x, out.add_lind.y, out.add_lind.z, 0.f);
        }
        const unsigned int cs = warp_append(out.cont, count_out);
        if (out.cont) {
            qout.o[cs] = make_float4(out.x.x, out.x.y, out.x.z, __int_as_float(tri));
            qout.d[cs] = make_float4(out.c_d.x, out.c_d.y, out.c_d.z, __uint_as_float(sid));
            qout.b[cs] = make_float4(out.c_beta.x, out.c_beta.y, out.c_beta.z, __int_as_float(vi));
            qout.bi[cs] = make_float4(out.c_bind.x, out.c_bind.y, out.c_bind.z, 0.f);
        }
    }
    for (int off = 16; off > 0; off >>= 1) n_cand += __shfl_xor_sync(MR_FULL, n_cand, off);
    if (lane_id() == 0 && n_cand) atomicAdd(counters + 5, n_cand);
}

template <bool COUNT, bool WIDE>
__global__ void __launch_bounds__(256) k_wshadow(const SceneDev* __restrict__ scenes,
                                                 const ViewDev* __restrict__ views, int b, ShadowDev sq,
                                                 const unsigned int* count, void* tape, uint64_t ntot, int nvx,
                                                 unsigned long long* counters)
{
    extern __shared__ __align__(16) uint32_t sstk[];
    const TapeDev tp = tape_of(tape, ntot, nvx);
    const unsigned int n = *count;
    unsigned int n_box = 0;
    int n_tri = 0;
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 a = sq.o[i], dd = sq.d[i], ad = sq.add[i];
        const ViewDev& v = views[__float_as_int(ad.w)];
        const SceneDev& s = scenes[v.scene];
        Hit h;
        if (COUNT) {
            const int nodes = traverse<true>(s, xyz(a), xyz(dd), __float_as_int(a.w), *s.tmin_dev,
                                             __int_as_float(0x7f800000), h, sstk + threadIdx.x, blockDim.x, &n_tri);
            n_box += 2u * (unsigned int)max(nodes, 0);
        } else {
            trace_as<true, WIDE>(s, xyz(a), xyz(dd), __float_as_int(a.w), *s.tmin_dev, __int_as_float(0x7f800000), h,
                                 sstk + threadIdx.x);
        }
        const uint64_t g = v.offset + __float_as_uint(dd.w);
        if (h.tri < 0) {
            const float4 ai = sq.addi[i];
            tp.rad[0][g] = __fadd_rn(tp.rad[0][g], ad.x);
            tp.rad[1][g] = __fadd_rn(tp.rad[1][g], ad.y);
            tp.rad[2][g] = __fadd_rn(tp.rad[2][g], ad.z);
            if (b >= 1) {
                tp.lind[0][g] = __fadd_rn(tp.lind[0][g], ai.x);
                tp.lind[1][g] = __fadd_rn(tp.lind[1][g], ai.y);
                tp.lind[2][g] = __fadd_rn(tp.lind[2][g], ai.z);
            }
        } else if (b == 0) {
            tp.wv[g] = 0.0f;
        } else {
            tape_vx_occluded(tp, g, b);
        }
    }
    if (COUNT) flush_work(counters, CNT_SBOX, n_box, (unsigned int)n_tri);
}

// Temporal reuse (Appendix A, reservoirs of previous frames): every bounce-0 hit merges the
// history reservoir its sample left in the previous call, the candidate count capped at
// cap * M, after its fresh one, with weight p_hat_here(y) w_sum / p_hat_then(y) (m_capped / m)
// and accept word 65535 of the reuse stream (selection code 65 M); the merged reservoir is
// what spatial reuse sees. Reads the history and writes the reservoir of its own sample only.
__global__ void __launch_bounds__(256) k_wtemporal(const SceneDev* __restrict__ scenes,
                                                   const ViewDev* __restrict__ views, Rng rng, int M, int cap,
                                                   QueueDev hq, const unsigned int* count_hit, ResDev res,
                                                   HistDev hist)
{
    const unsigned int n = *count_hit;
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 hd = hq.o[i], qd = hq.d[i], qb = hq.b[i];
        const ViewDev& v = views[__float_as_int(qb.w)];
        const SceneDev& s = scenes[v.scene];
        const uint32_t sid = __float_as_uint(qd.w);
        const uint64_t g = v.offset + sid;
        const int ht = hist.ytex[g];
        if (ht == RES_MISS) continue;
        const float hm = hist.m[g];
        const float mc = fminf(hm, (float)cap * (float)M);
        res.m[g] += mc;
        const float hw = hist.wsum[g], hp = hist.phat[g];
        if (ht < 0 || !(hw > 0.0f) || !(hp > 0.0f) || !(hm > 0.0f)) continue;
        const float3 d = xyz(qd), wo = f3(-d.x, -d.y, -d.z);
        Shade sh;
        shade_at(s, __float_as_int(hd.w), hd.y, hd.z, d, sh);
        float4 rowv;
        float3 y;
        env_dir(s, ht / s.ew, ht % s.ew, hist.ysub[g], y, rowv);
        const float3 fc = light_brdf(sh, wo, y);
        const float ph = lum(xyz(__ldg(s.env_texel + ht))) * lum(fc);
        const float w = ph * hw / hp * (mc / hm);
        const uint32_t pixel = sid / (uint32_t)v.spp, smp = sid % (uint32_t)v.spp;
        const uint4 x = rng.draw(pixel, smp, (uint32_t)v.index, 0u, PURPOSE_REUSE, 65535u);
        const float ws = res.wsum[g] + w;  // the fresh reservoir's sum (zero when nothing had weight)
        res.wsum[g] = ws;
        if (u24(x.z) * ws < w) {
            res.ytex[g] = ht;
            res.sel[g] = 65 * M;
            res.ysub[g] = hist.ysub[g];
            res.phat[g] = ph;
        }
    }
}

// primary rays that escaped leave no reservoir in the history
__global__ void __launch_bounds__(256) k_whist_miss(uint64_t first, uint32_t n, void* tape, uint64_t ntot,
                                                    HistDev hist)
{
    const TapeDev tp = tape_of(tape, ntot);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t g = first + i;
        if (tp.tri[g] < 0) {
            hist.ytex[g] = RES_MISS;
            hist.ysub[g] = 0u;
            hist.wsum[g] = 0.0f;
            hist.phat[g] = 0.0f;
            hist.m[g] = 0.0f;
        }
    }
}

// Spatial reuse at the primary vertex (Appendix A, "Spatial-temporal Reuse"): every bounce-0
// hit merges the reservoirs of K neighbouring pixels (same sample index; offsets drawn from the
// (2R+1)^2 square by the reuse stream) into its own. Each reservoir enters with weight
// p_hat_here(y) w_sum / p_hat_there(y), the merged reservoir counts M candidates per reservoir
// whose primary ray hit, W = w_sum / (m p_hat_here(y)); then the shadow ray of the merged
// selection is queued. Reads only what k_wshade published for the whole wave (waves hold whole
// views), writes only its own sample's tape words.
__global__ void __launch_bounds__(256) k_wreuse(const SceneDev* __restrict__ scenes, const ViewDev* __restrict__ views,
                                                Rng rng, int M, int K, int R, QueueDev hq,
                                                const unsigned int* count_hit, ShadowDev sq, unsigned int* count_sh,
                                                ResDev res, HistDev hist, void* tape, uint64_t ntot, int nvx)
{
    const TapeDev tp = tape_of(tape, ntot, nvx);
    const unsigned int n = *count_hit;
    const unsigned int stride = gridDim.x * blockDim.x;
    const unsigned int rounds = (n + stride - 1) / stride;
    for (unsigned int r = 0; r < rounds; ++r) {
        const unsigned int i = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
        bool emit = false;
        float3 so = f3(0.f, 0.f, 0.f), sd = so, add = so;
        int tri = -1, vi = 0;
        uint32_t sid = 0;
        if (i < n) {
            const float4 hd = hq.o[i], qd = hq.d[i], qb = hq.b[i];
            vi = __float_as_int(qb.w);
            const ViewDev& v = views[vi];
            const SceneDev& s = scenes[v.scene];
            tri = __float_as_int(hd.w);
            sid = __float_as_uint(qd.w);
            const uint64_t g = v.offset + sid;
            const uint32_t pixel = sid / (uint32_t)v.spp, smp = sid % (uint32_t)v.spp;
            const int px = (int)(pixel % (uint32_t)v.width), py = (int)(pixel / (uint32_t)v.width);
            const float3 d = xyz(qd), wo = f3(-d.x, -d.y, -d.z);
            Shade sh;
            shade_at(s, tri, hd.y, hd.z, d, sh);
            float wsum = 0.0f, phat_sel = 0.0f, m = res.m[g];
            int sel = -1, ytex = 0;
            uint32_t ysub = 0u;
            const int own = res.ytex[g];
            if (own >= 0) {  // the vertex's own reservoir first: p_hat_here = p_hat_own
                const float ph = res.phat[g];
                wsum = ph * res.wsum[g] / ph;
                sel = res.sel[g];
                ytex = own;
                ysub = res.ysub[g];
                phat_sel = ph;
            }
            for (int j = 0; j < K; ++j) {
                const uint4 x = rng.draw(pixel, smp, (uint32_t)v.index, 0u, PURPOSE_REUSE, (uint32_t)j);
                const int dx = (int)(((uint64_t)(x.x >> 8) * (uint64_t)(2 * R + 1)) >> 24) - R;
                const int dy = (int)(((uint64_t)(x.y >> 8) * (uint64_t)(2 * R + 1)) >> 24) - R;
                const int qx = px + dx, qy = py + dy;
                if ((dx == 0 && dy == 0) || qx < 0 || qy < 0 || qx >= v.width || qy >= v.height) continue;
                const uint64_t gq = v.offset + ((uint64_t)qy * (uint64_t)v.width + (uint64_t)qx) * (uint64_t)v.spp + smp;
                const int nt = res.ytex[gq];
                if (nt == RES_MISS) continue;
                m += res.m[gq];
                if (nt < 0) continue;
                float4 rowv;
                float3 y;
                env_dir(s, nt / s.ew, nt % s.ew, res.ysub[gq], y, rowv);
                const float3 fc = light_brdf(sh, wo, y);
                const float ph = lum(xyz(__ldg(s.env_texel + nt))) * lum(fc);
                const float w = ph * res.wsum[gq] / res.phat[gq];
                wsum += w;
                if (u24(x.z) * wsum < w) {
                    sel = M * (j + 1) + res.sel[gq];
                    ytex = nt;
                    ysub = res.ysub[gq];
                    phat_sel = ph;
                }
            }
            float W = 0.0f;
            float3 y = f3(0.f, 0.f, 0.f);
            if (sel >= 0 && wsum > 0.0f && phat_sel > 0.0f) {
                float4 rowv;
                env_dir(s, ytex / s.ew, ytex % s.ew, ysub, y, rowv);
                const float3 fsel = brdf_cos(sh.n, wo, y, sh.m);
                const float4 L = __ldg(s.env_texel + ytex);
                W = wsum / (m * phat_sel);
                const float3 contrib = mul(hmul(xyz(L), fsel), W);
                add = hmul_rn(xyz(qb), contrib);
                emit = true;
                so = sh.x;
                sd = y;
            } else {
                sel = -1;
            }
            if (hist.ytex) {  // the final reservoir becomes the next call's history
                hist.ytex[g] = sel >= 0 ? ytex : RES_NONE;
                hist.ysub[g] = ysub;
                hist.wsum[g] = wsum;
                hist.phat[g] = phat_sel;
                hist.m[g] = m;
            }
            tp.cand[g] = sel;
            tp.wv[g] = W;
            tp.ytex[g] = sel >= 0 ? ytex : -1;
            tp.y[0][g] = y.x;
            tp.y[1][g] = y.y;
            tp.y[2][g] = y.z;
        }
        const unsigned int ss = warp_append(emit, count_sh);
        if (emit) {
            sq.o[ss] = make_float4(so.x, so.y, so.z, __int_as_float(tri));
            sq.d[ss] = make_float4(sd.x, sd.y, sd.z, __uint_as_float(sid));
            sq.add[ss] = make_float4(add.x, add.y, add.z, __int_as_float(vi));
            sq.addi[ss] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// Lane refill for the incoherent stages (continuation and shadow rays): each warp takes rays
// from its stage's queue 32 at a time (one atomic per 32 rays) and advances its lanes' rays
// MR_REFILL_STEPS node visits at a time; once MR_REFILL_MIN lanes are done (or all, when the
// queue is drained) they take new rays, so a warp does not wait for its longest ray. The grid
// is one resident wave of blocks; `fetch` is the stage's ray counter, zero at launch.
struct RefillPool {
    unsigned int pool, pool_end;
    bool drained;
};

// hands rays to idle lanes; returns this lane's new ray index, or -1
__device__ __forceinline__ long long refill(RefillPool& rp, bool has, unsigned int n, unsigned int* fetch)
{
    const unsigned idle = __ballot_sync(MR_FULL, !has);
    const int n_idle = __popc(idle);
    if (n_idle < MR_REFILL_MIN && idle != MR_FULL) return -1;
    if (rp.pool == rp.pool_end && !rp.drained) {
        unsigned int base = 0;
        if (lane_id() == 0) base = atomicAdd(fetch, 32u);
        base = __shfl_sync(MR_FULL, base, 0);
        if (base >= n) {
            rp.drained = true;
        } else {
            rp.pool = base;
            rp.pool_end = (n - base < 32u) ? n : base + 32u;
        }
    }
    long long mine = -1;
    if (rp.pool < rp.pool_end) {
        const unsigned avail = rp.pool_end - rp.pool;
        const unsigned rank = __popc(idle & lanemask_lt());
        if (!has && rank < avail) mine = (long long)(rp.pool + rank);
        rp.pool += ((unsigned)n_idle < avail) ? (unsigned)n_idle : avail;
    }
    return mine;
}

template <bool COUNT>
__global__ void __launch_bounds__(256, MR_CLOSEST_REFILL_MINB) k_wclosest_refill(const SceneDev* __restrict__ scenes,
                                                         const ViewDev* __restrict__ views, QueueDev q,
                                                         const unsigned int* count, QueueDev hq,
                                                         unsigned int* count_hit, unsigned int* fetch,
                                                         unsigned long long* counters)
{
    extern __shared__ __align__(16) uint32_t sstk[];
    const unsigned int n = *count;
    uint32_t lstk[MR_LSTACK];
    Trav T;
    T.node = -1;
    bool has = false;
    unsigned int i = 0;
    RefillPool rp{0u, 0u, false};
    float4 qd = make_float4(0.f, 0.f, 0.f, 0.f), qb = qd;
    const SceneDev* sp = scenes;
    unsigned int n_box = 0;
    int n_tri = 0;
    while (true) {
        const long long ni = refill(rp, has, n, fetch);
        if (ni >= 0) {
            i = (unsigned int)ni;
            const float4 a = q.o[i];
            qd = q.d[i];
            qb = q.b[i];
            sp = scenes + views[__float_as_int(qb.w)].scene;
            trav_begin(*sp, T, xyz(a), xyz(qd), __float_as_int(a.w), *sp->tmin_dev, __int_as_float(0x7f800000),
                       COUNT ? &n_tri : nullptr);
            has = true;
        }
        if (!__any_sync(MR_FULL, has)) break;
        bool done = false;
        if (has) {
            const int v0 = T.visited;
            done = trav_run<false>(*sp, T, sstk + threadIdx.x, blockDim.x, lstk, MR_REFILL_STEPS,
                                   COUNT ? &n_tri : nullptr);
            if (COUNT) n_box += 2u * (unsigned int)max(T.visited - v0, 0);
        }
        if (__any_sync(MR_FULL, done)) {
            const bool hit = done && T.best.tri >= 0;
            const unsigned int slot = warp_append(hit, count_hit);
            if (hit) {
                hq.o[slot] = make_float4(T.best.t, T.best.u, T.best.v, __int_as_float(T.best.tri));
                hq.d[slot] = qd;
                hq.b[slot] = qb;
                hq.bi[slot] = q.bi[i];
            }
            if (done) has = false;
        }
    }
    if (COUNT) flush_work(counters, CNT_CBOX, n_box, (unsigned int)n_tri);
}

template <bool COUNT>
__global__ void MR_TRACE_BOUNDS k_wshadow_refill(const SceneDev* __restrict__ scenes,
                                                        const ViewDev* __restrict__ views, int b, ShadowDev sq,
                                                        const unsigned int* count, unsigned int* fetch, void* tape,
                                                        uint64_t ntot, int nvx, unsigned long long* counters)
{
    extern __shared__ __align__(16) uint32_t sstk[];
    const TapeDev tp = tape_of(tape, ntot, nvx);
    const unsigned int n = *count;
    uint32_t lstk[MR_LSTACK];
    Trav T;
    T.node = -1;
    bool has = false;
    unsigned int i = 0;
    RefillPool rp{0u, 0u, false};
    float4 dd = make_float4(0.f, 0.f, 0.f, 0.f), ad = dd;
    const SceneDev* sp = scenes;
    unsigned int n_box = 0;
    int n_tri = 0;
    while (true) {
        const long long ni = refill(rp, has, n, fetch);
        if (ni >= 0) {
            i = (unsigned int)ni;
            const float4 a = sq.o[i];
            dd = sq.d[i];
            ad = sq.add[i];
            sp = scenes + views[__float_as_int(ad.w)].scene;
            trav_begin(*sp, T, xyz(a), xyz(dd), __float_as_int(a.w), *sp->tmin_dev, __int_as_float(0x7f800000),
                       COUNT ? &n_tri : nullptr);
            has = true;
        }
        if (!__any_sync(MR_FULL, has)) break;
        if (has) {
            const int v0 = T.visited;
            const bool done = trav_run<true>(*sp, T, sstk + threadIdx.x, blockDim.x, lstk, MR_REFILL_STEPS,
                                             COUNT ? &n_tri : nullptr);
            if (COUNT) n_box += 2u * (unsigned int)max(T.visited - v0, 0);
            if (done) {
                has = false;
                const uint64_t g = views[__float_as_int(ad.w)].offset + __float_as_uint(dd.w);
                if (T.best.tri < 0) {
                    const float4 ai = sq.addi[i];
                    tp.rad[0][g] = __fadd_rn(tp.rad[0][g], ad.x);
                    tp.rad[1][g] = __fadd_rn(tp.rad[1][g], ad.y);
                    tp.rad[2][g] = __fadd_rn(tp.rad[2][g], ad.z);
                    if (b >= 1) {
                        tp.lind[0][g] = __fadd_rn(tp.lind[0][g], ai.x);
                        tp.lind[1][g] = __fadd_rn(tp.lind[1][g], ai.y);
                        tp.lind[2][g] = __fadd_rn(tp.lind[2][g], ai.z);
                    }
                } else if (b == 0) {
                    tp.wv[g] = 0.0f;
                } else {
                    tape_vx_occluded(tp, g, b);
                }
            }
        }
    }
    if (COUNT) flush_work(counters, CNT_SBOX, n_box, (unsigned int)n_tri);
}

// ---- primary visibility by rasterisation ------------------------------------------------
// The paper resolves primary visibility with a rasteriser (nvdiffrast). Here each triangle is
// projected into every view of the wave, and each camera sample inside its conservative
// screen box is tested with the same FP32 ray/triangle solve the traversal runs, against the
// sample's own jittered direction from the ray queue; a 64-bit atomicMin on (t bits, triangle)
// keeps the smallest t, then the smallest triangle id -- the traversal's closest-hit rule. The
// closest-hit stage then reads the winner instead of traversing. Small triangles take one
// thread each; triangles whose box holds more than RASTER_SMALL samples (or that cross the
// camera plane) take a block each.
constexpr int RASTER_SMALL = 256;
constexpr unsigned long long RASTER_NONE = ~0ull;

struct RasterBox {
    int x0, y0, x1, y1;  // inclusive pixel range, empty when x0 > x1
    bool all;            // crosses the camera plane: every pixel
};

__device__ __forceinline__ RasterBox raster_box(const ViewDev& v, float3 a, float3 b, float3 c)
{
    const float3 o = f3(v.c2w[3], v.c2w[7], v.c2w[11]);
    const float3 p[3] = {sub(a, o), sub(b, o), sub(c, o)};
    float zs[3], xs[3], ys[3];
    int behind = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float cx = v.c2w[0] * p[k].x + v.c2w[4] * p[k].y + v.c2w[8] * p[k].z;
        const float cy = v.c2w[1] * p[k].x + v.c2w[5] * p[k].y + v.c2w[9] * p[k].z;
        zs[k] = v.c2w[2] * p[k].x + v.c2w[6] * p[k].y + v.c2w[10] * p[k].z;
        behind += zs[k] <= 1e-6f ? 1 : 0;
        xs[k] = v.K[0] * cx / zs[k] + v.K[2];
        ys[k] = v.K[1] * cy / zs[k] + v.K[3];
    }
    RasterBox r{0, 0, v.width - 1, v.height - 1, true};
    if (behind == 3) {  // no forward ray reaches a point on or behind the camera plane
        r.x0 = 1;
        r.x1 = 0;
        r.all = false;
        return r;
    }
    if (behind > 0) return r;
    // a sample at (X, Y) = (px + jx, py + jy) lies in pixel (floor X, floor Y); 0.01 px of slack
    // covers the rounding of the projection
    const float xmin = fminf(fminf(xs[0], xs[1]), xs[2]) - 0.01f, xmax = fmaxf(fmaxf(xs[0], xs[1]), xs[2]) + 0.01f;
    const float ymin = fminf(fminf(ys[0], ys[1]), ys[2]) - 0.01f, ymax = fmaxf(fmaxf(ys[0], ys[1]), ys[2]) + 0.01f;
    r.all = false;
    r.x0 = (int)fmaxf(floorf(xmin), 0.0f);
    r.y0 = (int)fmaxf(floorf(ymin), 0.0f);
    r.x1 = (int)fminf(floorf(xmax), (float)(v.width - 1));
    r.y1 = (int)fminf(floorf(ymax), (float)(v.height - 1));
    if (!(xmax >= 0.0f) || !(ymax >= 0.0f) || !(xmin <= (float)v.width) || !(ymin <= (float)v.height)) {
        r.x0 = 1;
        r.x1 = 0;
    }
    return r;
}

// test sample (pixel, s) of view v against triangle `tri` (samples outside the wave are skipped)
__device__ __forceinline__ void raster_sample(const ViewDev& v, float3 o, const float4* __restrict__ qd, uint64_t first,
                                              uint32_t n, uint32_t pixel, int s, float3 v0, float3 e1, float3 e2,
                                              int tri, float tmin, unsigned long long* keys, int& tests)
{
    const int64_t i = (int64_t)(v.offset + (uint64_t)pixel * (uint32_t)v.spp + (uint32_t)s) - (int64_t)first;
    if (i < 0 || i >= (int64_t)n) return;
    const float3 d = xyz(__ldg(qd + i));
    float t, u, w;
    ++tests;
    if (!tri_solve(o, d, v0, e1, e2, t, u, w)) return;
    if (!(u >= 0.0f && w >= 0.0f && u + w <= 1.0f && t > tmin)) return;
    const unsigned long long key = ((unsigned long long)__float_as_uint(t) << 32) | (unsigned)tri;
    if (key < keys[i]) atomicMin(keys + i, key);
}

template <bool COUNT>
__global__ void __launch_bounds__(256) k_raster_small(const SceneDev* __restrict__ scenes,
                                                      const ViewDev* __restrict__ views, int vi, uint64_t first,
                                                      uint32_t n, const float4* __restrict__ qd,
                                                      unsigned long long* keys, unsigned long long* counters)
{
    const ViewDev& v = views[vi];
    const SceneDev& s = scenes[v.scene];
    const float3 o = f3(v.c2w[3], v.c2w[7], v.c2w[11]);
    const float tmin = *s.tmin_dev;
    int tests = 0;
    for (int leaf = blockIdx.x * blockDim.x + threadIdx.x; leaf < s.n_tris; leaf += gridDim.x * blockDim.x) {
        float3 v0, e1, e2;
        int tri;
        load_tri(s, leaf, v0, e1, e2, tri);
        const RasterBox r = raster_box(v, v0, add(v0, e1), add(v0, e2));
        if (r.all || r.x0 > r.x1 || r.y0 > r.y1) continue;
        if ((int64_t)(r.x1 - r.x0 + 1) * (r.y1 - r.y0 + 1) * v.spp > RASTER_SMALL) continue;
        for (int py = r.y0; py <= r.y1; ++py)
            for (int px = r.x0; px <= r.x1; ++px)
                for (int k = 0; k < v.spp; ++k)
                    raster_sample(v, o, qd, first, n, (uint32_t)(py * v.width + px), k, v0, e1, e2, tri, tmin, keys,
                                  tests);
    }
    if (COUNT) flush_work(counters, CNT_CBOX, 0u, (unsigned int)tests);
}

template <bool COUNT>
__global__ void __launch_bounds__(256) k_raster_big(const SceneDev* __restrict__ scenes,
                                                    const ViewDev* __restrict__ views, int vi, uint64_t first,
                                                    uint32_t n, const float4* __restrict__ qd,
                                                    unsigned long long* keys, unsigned long long* counters)
{
    const ViewDev& v = views[vi];
    const SceneDev& s = scenes[v.scene];
    const float3 o = f3(v.c2w[3], v.c2w[7], v.c2w[11]);
    const float tmin = *s.tmin_dev;
    int tests = 0;
    for (int leaf = blockIdx.x; leaf < s.n_tris; leaf += gridDim.x) {  // block-uniform
        float3 v0, e1, e2;
        int tri;
        load_tri(s, leaf, v0, e1, e2, tri);
        const RasterBox r = raster_box(v, v0, add(v0, e1), add(v0, e2));
        if (r.x0 > r.x1 || r.y0 > r.y1) continue;
        const int bw = r.x1 - r.x0 + 1, bh = r.y1 - r.y0 + 1;
        const int64_t cnt = (int64_t)bw * bh * v.spp;
        if (!r.all && cnt <= RASTER_SMALL) continue;
        for (int64_t j = threadIdx.x; j < cnt; j += blockDim.x) {
            const int k = (int)(j % v.spp);
            const int64_t pj = j / v.spp;
            const int px = r.x0 + (int)(pj % bw), py = r.y0 + (int)(pj / bw);
            raster_sample(v, o, qd, first, n, (uint32_t)(py * v.width + px), k, v0, e1, e2, tri, tmin, keys, tests);
        }
    }
    if (COUNT) {
        // every lane of the block reaches here; reduce per warp
        flush_work(counters, CNT_CBOX, 0u, (unsigned int)tests);
    }
}

unsigned grid_cap(uint64_t n, int block, int cap)
{
    const uint64_t g = (n + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : (g > (uint64_t)cap ? (uint64_t)cap : g));
}

}  // namespace

// Record the whole batched forward on `st` (capturable: kernels, memsets, event records).
// With `ev` non-null, an event pair is recorded around every stage launch: ev[2k], ev[2k+1]
// for pair k, whose stage kind (0 closest, 1 shade, 2 shadow, 3 raygen) goes to kind[k].
void mr_wave_record(const SceneDev* scenes, const ViewDev* views, int n_views, uint64_t total, int max_bounces,
                    Rng rng, int M, const uint64_t* wave_first, int n_waves, const WaveBranch* branches,
                    int n_branches, cudaEvent_t fork, cudaEvent_t* join, void* tape, unsigned long long* counters,
                    const uint64_t* pix_off, uint64_t total_pix, float* const* images, int sms, cudaEvent_t* ev,
                    int* kind, int nvx, bool count, int reuse_k, int reuse_radius, const ResDev& res, int temporal,
                    int temporal_cap, const HistDev& hist, const ViewDev* hviews, const SceneDev* hscenes, bool raster,
                    bool bin, const mirres_wave_shape& shape)
{
    // waves go round-robin to `n_branches` chains of their own (queues, counters, stream): chain
    // 0 on the recording stream, the others forked from it and joined back before the resolve,
    // so that the stages of different waves overlap on the GPU
    const cudaStream_t st_main = branches[0].st;
    if (n_branches > 1) {
        cudaEventRecord(fork, st_main);
        for (int b = 1; b < n_branches; ++b) cudaStreamWaitEvent(branches[b].st, fork, 0);
    }
    // per stage (0 closest, 1 shade, 2 shadow, 3 raygen): threads per block and the grid cap
    const int blk_c = shape.block[0], blk_h = shape.block[1], blk_s = shape.block[2], blk_g = shape.block[3];
    const int cap_c = sms * shape.blocks_per_sm[0], cap_h = sms * shape.blocks_per_sm[1];
    const int cap_s = sms * shape.blocks_per_sm[2], cap_g = sms * shape.blocks_per_sm[3];
    bool interp = false;  // any scene with interpolated normals
    bool wide = true;     // every scene traversed through a wide BVH: no lane refill (binary only)
    for (int i = 0; i < n_views; ++i) {
        interp = interp || hscenes[hviews[i].scene].vnrm != nullptr;
        wide = wide && (hscenes[hviews[i].scene].wnodes != nullptr || hscenes[hviews[i].scene].n_tris < 2);
    }
    const size_t smem = sizeof(uint32_t) * MR_SSTACK * 256;  // the refilling kernels run 256 threads
    const size_t stack_c = sizeof(uint32_t) * MR_SSTACK * (size_t)blk_c, stack_s = sizeof(uint32_t) * MR_SSTACK * (size_t)blk_s;
    // the refilling kernels run one resident wave of blocks
    int occ_c = 0, occ_s = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, count ? k_wclosest_refill<true> : k_wclosest_refill<false>,
                                                  256, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, count ? k_wshadow_refill<true> : k_wshadow_refill<false>,
                                                  256, smem);
    const unsigned grid_c = (unsigned)(sms * (occ_c > 0 ? occ_c : 1));
    const unsigned grid_s = (unsigned)(sms * (occ_s > 0 ? occ_s : 1));
    int pair = 0, cur_b = -1;  // cur_b: the bounce being recorded (-1: ray generation)
    cudaStream_t st = st_main;
    auto mark = [&](int k, bool start) {
        if (!ev) return;
        if (start) kind[pair] = k | ((cur_b + 1) << 4);  // stage in bits 0-3, bounce + 1 above
        cudaEventRecordWithFlags(ev[2 * pair + (start ? 0 : 1)], st, cudaEventRecordExternal);
        if (!start) ++pair;
    };
    for (int wv = 0; wv < n_waves; ++wv) {
        const WaveBranch& br = branches[wv % n_branches];
        st = br.st;
        const QueueDev &qa = br.qa, &qb = br.qb, &hq = br.hq;
        const ShadowDev& sq = br.sq;
        unsigned int* qc = br.qc;
        unsigned int* fetch = qc + 3 * max_bounces + 3;  // [2 * max_bounces]: closest, shadow per bounce
        const uint64_t first = wave_first[wv];
        const uint32_t n = (uint32_t)((wv + 1 < n_waves ? wave_first[wv + 1] : total) - first);
        cudaMemsetAsync(qc, 0, sizeof(unsigned int) * (5 * max_bounces + 3), st);
        cur_b = -1;
        mark(3, true);
        k_wraygen<<<grid_cap(n, blk_g, cap_g), blk_g, 0, st>>>(views, n_views, rng, first, n, qa, tape, total, nvx,
                                                               res);
        mark(3, false);
        QueueDev cur = qa, nxt = qb;
        for (int b = 0; b < max_bounces; ++b) {
            const unsigned int* cnt_in = b == 0 ? nullptr : qc + 3 * (b - 1) + 1;
            cur_b = b;
            mark(0, true);
            if (bin && b > 0) {
                // the continuation rays shade wrote (cur) binned into the free queue (nxt),
                // which becomes this bounce's input
                cudaMemsetAsync(br.bhist, 0, sizeof(unsigned int) * BIN_KEYS, st);
                k_bin_hist<<<grid_cap(n, 256, sms * 4), 256, 0, st>>>(scenes, views, cur, cnt_in, br.bkey, br.bhist);
                k_bin_scan<<<1, 1024, 0, st>>>(br.bhist);
                k_bin_scatter<<<grid_cap(n, 256, sms * 8), 256, 0, st>>>(cur, nxt, cnt_in, br.bkey, br.bhist);
                const QueueDev t = cur;
                cur = nxt;
                nxt = t;
            }
            unsigned long long* keys = nullptr;
            if (raster && b == 0) {
                // the next-bounce queue is free until shading fills it: its last array holds
                // the per-sample depth keys (8 of its 16 bytes per entry)
                keys = reinterpret_cast<unsigned long long*>(nxt.bi);
                cudaMemsetAsync(keys, 0xFF, sizeof(unsigned long long) * n, st);
                for (int vi = 0; vi < n_views; ++vi) {
                    const ViewDev& hv = hviews[vi];
                    const uint64_t vn = (uint64_t)hv.width * hv.height * hv.spp;
                    if (hv.offset >= first + n || hv.offset + vn <= first) continue;
                    const int F = hscenes[hv.scene].n_tris;
                    if (F <= 0) continue;
                    (count ? k_raster_small<true> : k_raster_small<false>)<<<grid_cap((uint64_t)F, 256, sms * 8), 256,
                                                                            0, st>>>(scenes, views, vi, first, n,
                                                                                     cur.d, keys, counters);
                    (count ? k_raster_big<true> : k_raster_big<false>)<<<(unsigned)(sms * 2), 256, 0, st>>>(
                        scenes, views, vi, first, n, cur.d, keys, counters);
                }
            }
            if (MR_REFILL_CLOSEST && b > 0 && !wide)  // primary rays stay coherent in the plain stage kernel
                (count ? k_wclosest_refill<true> : k_wclosest_refill<false>)<<<grid_c, 256, smem, st>>>(
                    scenes, views, cur, cnt_in, hq, qc + 3 * b, fetch + 2 * b, counters);
            else
                (keys ? (count ? k_wclosest<true, true, false>
                               : (wide ? k_wclosest<false, true, true> : k_wclosest<false, true, false>))
                      : (count ? k_wclosest<true, false, false>
                               : (wide ? k_wclosest<false, false, true> : k_wclosest<false, false, false>)))<<<
                    grid_cap(n, blk_c, cap_c), blk_c, stack_c, st>>>(
                    scenes, views, b, cur, cnt_in, n, hq, qc + 3 * b, tape, total, counters, keys);
            mark(0, false);
            mark(1, true);
            const bool reuse_b = b == 0 && res.ytex != nullptr;
            (reuse_b ? (interp ? k_wshade<true, true> : k_wshade<true, false>)
                     : (interp ? k_wshade<false, true> : k_wshade<false, false>))<<<grid_cap(n, blk_h, cap_h), blk_h, 0, st>>>(
                scenes, views, rng, b, M, hq, qc + 3 * b, nxt, qc + 3 * b + 1, sq, qc + 3 * b + 2, tape, total, nvx,
                res, counters);
            if (reuse_b && temporal == 2)
                k_wtemporal<<<grid_cap(n, blk_h, cap_h), blk_h, 0, st>>>(scenes, views, rng, M, temporal_cap, hq, qc,
                                                                         res, hist);
            if (reuse_b)
                k_wreuse<<<grid_cap(n, blk_h, cap_h), blk_h, 0, st>>>(scenes, views, rng, M, reuse_k, reuse_radius, hq,
                                                                      qc, sq, qc + 2, res, hist, tape, total, nvx);
            if (reuse_b && temporal)
                k_whist_miss<<<grid_cap(n, blk_h, cap_h), blk_h, 0, st>>>(first, n, tape, total, hist);
            mark(1, false);
            mark(2, true);
            if (MR_REFILL && !wide)
                (count ? k_wshadow_refill<true> : k_wshadow_refill<false>)<<<grid_s, 256, smem, st>>>(
                    scenes, views, b, sq, qc + 3 * b + 2, fetch + 2 * b + 1, tape, total, nvx, counters);
            else
                (count ? k_wshadow<true, false> : (wide ? k_wshadow<false, true> : k_wshadow<false, false>))<<<
                    grid_cap(n, blk_s, cap_s), blk_s, stack_s, st>>>(
                    scenes, views, b, sq, qc + 3 * b + 2, tape, total, nvx, counters);
            mark(2, false);
            QueueDev t = cur;
            cur = nxt;
            nxt = t;
        }
        mr_launch_account(counters, qc, max_bounces, n, st);
    }
    for (int b = 1; b < n_branches; ++b) {
        cudaEventRecord(join[b], branches[b].st);
        cudaStreamWaitEvent(st_main, join[b], 0);
    }
    mr_launch_resolve_all(views, n_views, pix_off, total_pix, images, tape, total, sms, st_main);
}

int mr_wave_stage_pairs(int n_waves, int max_bounces) { return n_waves * (1 + 3 * max_bounces); }

int mr_wave_launches(int n_waves, int max_bounces, bool reuse, int temporal, int raster_launches, bool bin)
{
    const int extra = (reuse ? 1 : 0) + (temporal == 2 ? 1 : 0) + (temporal ? 1 : 0) + (bin ? 3 * (max_bounces - 1) : 0);
    return n_waves * (2 + 3 * max_bounces + extra) + 1 + raster_launches;
}
