// regular.cu -- the mesh regularisers added to the rendering loss (Appendix A, "Training
// details"): Laplacian smoothness of the refined vertices,
//   L_smooth = sum_i sum_{j in X_i} |v_i - v_j|^2 / |X_i|,
// X_i the vertices sharing an edge with i, and the offset penalty L_offset = sum_i |v_i - v0_i|^2.
// Each undirected edge (a, b) appears in X_a and X_b, so L_smooth = sum over edges of
// |v_a - v_b|^2 (1/|X_a| + 1/|X_b|): one thread per edge. The edge list is built once per scene
// (the topology is fixed) by inserting every triangle edge into an open-addressing hash table.
//
// Also the material smoothness term L_k = (1/|X|) sum_{x in X} |k(x) - k(x + eps)| for the
// albedo and roughness textures: X is the set of surface points seen through one view's pixel
// centres, the offset eps is taken in texture space (uniform in [-sigma, sigma]^2, Philox
// purpose 4), |.| of the albedo is the mean of its channels' absolute differences, and the
// gradient (sign(0) = 0) is scattered to the eight bilinear taps by warp-aggregated atomics.
#include "render.h"

namespace {

constexpr unsigned long long kEmpty = ~0ull;

__device__ __forceinline__ unsigned long long mix64(unsigned long long k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

__global__ void __launch_bounds__(256) k_edges_insert(const int32_t* __restrict__ tris, int F, int V,
                                                      unsigned long long* table, unsigned long long mask, int2* edges,
                                                      unsigned int* n_edges, unsigned int* deg)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)F; t += (int64_t)gridDim.x * blockDim.x) {
        int v[3];
        for (int c = 0; c < 3; ++c) v[c] = __ldg(tris + 3 * t + c);
        for (int c = 0; c < 3; ++c) {
            int a = v[c], b = v[(c + 1) % 3];
            if (a == b || a < 0 || b < 0 || a >= V || b >= V) continue;
            if (a > b) {
                const int x = a;
                a = b;
                b = x;
            }
            const unsigned long long key = ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
            unsigned long long h = mix64(key) & mask;
            for (unsigned long long probe = 0; probe <= mask; ++probe) {  // the table is never full
                const unsigned long long prev = atomicCAS(table + h, kEmpty, key);
                if (prev == kEmpty) {
                    const unsigned int i = atomicAdd(n_edges, 1u);
                    edges[i] = make_int2(a, b);
                    atomicAdd(deg + a, 1u);
                    atomicAdd(deg + b, 1u);
                    break;
                }
                if (prev == key) break;
                h = (h + 1) & mask;
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_inv_deg(const unsigned int* __restrict__ deg, int V, float* inv_deg)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x)
        inv_deg[i] = deg[i] ? 1.0f / (float)deg[i] : 0.0f;
}

__device__ __forceinline__ void flush_loss(float* loss, float x)
{
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(MR_FULL, x, off);
    if (lane_id() == 0 && x != 0.0f) atomicAdd(loss, x);
}

// w |v_a - v_b|^2 (1/|X_a| + 1/|X_b|) per edge, and its gradient
__global__ void __launch_bounds__(256) k_smooth(const int2* __restrict__ edges, const unsigned int* __restrict__ n_edges,
                                                const float* __restrict__ inv_deg, const float* __restrict__ verts,
                                                float w, float* loss, float* grad)
{
    const unsigned int n = *n_edges;
    const unsigned int stride = gridDim.x * blockDim.x;
    float acc = 0.0f;
    // uniform trip count per warp (the loss is reduced across the warp at the end)
    for (unsigned int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const unsigned int e = base + threadIdx.x;
        if (e < n) {
            const int2 ab = edges[e];
            const float3 va = f3(verts[3 * (size_t)ab.x], verts[3 * (size_t)ab.x + 1], verts[3 * (size_t)ab.x + 2]);
            const float3 vb = f3(verts[3 * (size_t)ab.y], verts[3 * (size_t)ab.y + 1], verts[3 * (size_t)ab.y + 2]);
            const float3 d = sub(va, vb);
            const float c = w * (__ldg(inv_deg + ab.x) + __ldg(inv_deg + ab.y));
            acc += c * dot(d, d);
            if (grad) {
                const float3 g = mul(d, 2.0f * c);
                atomicAdd(grad + 3 * (size_t)ab.x, g.x);
                atomicAdd(grad + 3 * (size_t)ab.x + 1, g.y);
                atomicAdd(grad + 3 * (size_t)ab.x + 2, g.z);
                atomicAdd(grad + 3 * (size_t)ab.y, -g.x);
                atomicAdd(grad + 3 * (size_t)ab.y + 1, -g.y);
                atomicAdd(grad + 3 * (size_t)ab.y + 2, -g.z);
            }
        }
    }
    if (loss) flush_loss(loss, acc);
}

// w |v_i - v0_i|^2 per vertex, and its gradient
__global__ void __launch_bounds__(256) k_offset(const float* __restrict__ verts, const float* __restrict__ rest, int V,
                                                float w, float* loss, float* grad)
{
    const unsigned int stride = gridDim.x * blockDim.x;
    float acc = 0.0f;
    for (unsigned int base = blockIdx.x * blockDim.x; base < (unsigned)V; base += stride) {
        const unsigned int i = base + threadIdx.x;
        if (i < (unsigned)V) {
            const float3 d = f3(verts[3 * (size_t)i] - rest[3 * (size_t)i], verts[3 * (size_t)i + 1] - rest[3 * (size_t)i + 1],
                                verts[3 * (size_t)i + 2] - rest[3 * (size_t)i + 2]);
            acc += w * dot(d, d);
            if (grad) {
                grad[3 * (size_t)i] += 2.0f * w * d.x;
                grad[3 * (size_t)i + 1] += 2.0f * w * d.y;
                grad[3 * (size_t)i + 2] += 2.0f * w * d.z;
            }
        }
    }
    if (loss) flush_loss(loss, acc);
}

// one closest-hit ray through each pixel centre: (triangle, s, t) of its hit; triangle -1 where
// the ray escapes. Hits are counted per warp (one atomic per warp and iteration).
__global__ void __launch_bounds__(256) k_lk_hits(SceneDev s, ViewDev v, float4* __restrict__ rec,
                                                 float2* __restrict__ bary, unsigned int* __restrict__ n_hit)
{
    extern __shared__ __align__(16) uint32_t sstk[];
    const int64_t npx = (int64_t)v.width * v.height;
    const float3 o = f3(v.c2w[3], v.c2w[7], v.c2w[11]);
    const float tmin = *s.tmin_dev;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // uniform trip count per warp (the hit count is taken with a ballot)
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < npx; base += stride) {
        const int64_t p = base + threadIdx.x;
        bool hit = false;
        if (p < npx) {
            const int px = (int)(p % v.width), py = (int)(p / v.width);
            const float3 d = camera_dir(v, px, py, 0.5f, 0.5f);
            Hit h;
            trace<false>(s, o, d, -1, tmin, __int_as_float(0x7f800000), h, sstk + threadIdx.x);
            float4 r = make_float4(__int_as_float(-1), 0.0f, 0.0f, 0.0f);
            if (h.tri >= 0) {
                const float* uv = s.tri_uv + 6 * (size_t)h.tri;
                const float w0 = 1.0f - h.u - h.v;
                r = make_float4(__int_as_float(h.tri), w0 * __ldg(uv + 0) + h.u * __ldg(uv + 2) + h.v * __ldg(uv + 4),
                                w0 * __ldg(uv + 1) + h.u * __ldg(uv + 3) + h.v * __ldg(uv + 5), 0.0f);
                hit = true;
            }
            rec[p] = r;
            bary[p] = make_float2(h.u, h.v);
        }
        const unsigned b = __ballot_sync(MR_FULL, hit);
        if (lane_id() == 0 && b) atomicAdd(n_hit, (unsigned)__popc(b));
    }
}

struct EmitLk {
    float* ga;
    float* gr;
    __device__ void operator()(int key, const float (&v)[4]) const
    {
        if (ga) {
            atomicAdd(ga + 3 * (size_t)key, v[0]);
            atomicAdd(ga + 3 * (size_t)key + 1, v[1]);
            atomicAdd(ga + 3 * (size_t)key + 2, v[2]);
        }
        if (gr) atomicAdd(gr + key, v[3]);
    }
};

__device__ __forceinline__ float sgn(float x) { return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f); }

struct EmitVn {
    float* g;
    __device__ void operator()(int key, const float (&v)[3]) const
    {
        atomicAdd(g + 3 * (size_t)key, v[0]);
        atomicAdd(g + 3 * (size_t)key + 1, v[1]);
        atomicAdd(g + 3 * (size_t)key + 2, v[2]);
    }
};

// the normal term of one hit (interpolated vertex normals): n0 = S0 / |S0| at the hit's
// barycentrics, n1 = S1 / |S1| at those moved by J^-1 eps (J the triangle's texture map);
// returns sum_c |n0_c - n1_c| and, scaled by cn, the gradient with respect to the three vertex
// normals (vid -1 where the term is absent: singular texture map or a vanishing blend)
__device__ __forceinline__ float lk_normal(const SceneDev& s, int tri, float u, float v, float es, float et, float cn,
                                           bool grad, int (&vid)[3], float (&gvn)[3][3])
{
    const float* uv = s.tri_uv + 6 * (size_t)tri;
    const float j00 = __ldg(uv + 2) - __ldg(uv + 0), j01 = __ldg(uv + 4) - __ldg(uv + 0);
    const float j10 = __ldg(uv + 3) - __ldg(uv + 1), j11 = __ldg(uv + 5) - __ldg(uv + 1);
    const float det = j00 * j11 - j01 * j10;
    if (!(det != 0.0f)) return 0.0f;
    const float du = (j11 * es - j01 * et) / det, dv = (j00 * et - j10 * es) / det;
    int ix[3];
    float3 vn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        ix[c] = __ldg(s.tris + 3 * (size_t)tri + c);
        vn[c] = xyz(__ldg(s.vnrm + ix[c]));
    }
    const float w0 = 1.0f - u - v;
    const float b0[3] = {w0, u, v}, b1[3] = {w0 - du - dv, u + du, v + dv};
    const float3 S0 = add(add(mul(vn[0], b0[0]), mul(vn[1], b0[1])), mul(vn[2], b0[2]));
    const float3 S1 = add(add(mul(vn[0], b1[0]), mul(vn[1], b1[1])), mul(vn[2], b1[2]));
    const float l0 = sqrtf(dot(S0, S0)), l1 = sqrtf(dot(S1, S1));
    if (!(l0 > 0.0f) || !(l1 > 0.0f)) return 0.0f;
    const float3 n0 = mul(S0, 1.0f / l0), n1 = mul(S1, 1.0f / l1);
    const float3 df = sub(n0, n1);
    if (grad) {
        const float3 g = f3(cn * sgn(df.x), cn * sgn(df.y), cn * sgn(df.z));
        const float3 gS0 = mul(sub(g, mul(n0, dot(n0, g))), 1.0f / l0);
        const float3 gS1 = mul(sub(mul(n1, dot(n1, g)), g), 1.0f / l1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            vid[c] = ix[c];
            gvn[c][0] = b0[c] * gS0.x + b1[c] * gS1.x;
            gvn[c][1] = b0[c] * gS0.y + b1[c] * gS1.y;
            gvn[c][2] = b0[c] * gS0.z + b1[c] * gS1.z;
        }
    }
    return fabsf(df.x) + fabsf(df.y) + fabsf(df.z);
}

__global__ void __launch_bounds__(256) k_lk_apply(SceneDev s, const float4* __restrict__ rec,
                                                  const float2* __restrict__ bary, int64_t npx,
                                                  const unsigned int* __restrict__ n_hit, Rng rng, uint32_t view_index,
                                                  float sigma, float wa, float wr, float wn, float* loss, float* ga,
                                                  float* gr, float* gvn_out)
{
    const unsigned int n = *n_hit;
    if (n == 0) return;  // uniform
    const float inv = 1.0f / (float)n;
    const float ca = wa * inv * (1.0f / 3.0f), cr = wr * inv, cn = wn * inv * (1.0f / 3.0f);
    const bool normal = wn > 0.0f && s.vnrm != nullptr;
    const bool want_grad = ga || gr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float acc = 0.0f;
    // uniform trip count per warp (the scatter and the loss reduction use every lane)
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < npx; base += stride) {
        const int64_t p = base + threadIdx.x;
        int tri = -1;
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < npx) {
            r = __ldg(rec + p);
            tri = __float_as_int(r.x);
        }
        Taps t[2] = {};
        float sa[3] = {0.f, 0.f, 0.f}, sr = 0.0f;
        int vid[3] = {-1, -1, -1};
        float gvn[3][3] = {};
        if (tri >= 0) {
            const uint4 x = rng.draw((uint32_t)p, 0u, view_index, 0u, PURPOSE_SMOOTH, 0u);
            const float es = sigma * (2.0f * u24(x.x) - 1.0f), et = sigma * (2.0f * u24(x.y) - 1.0f);
            if (normal) {
                const float2 b = __ldg(bary + p);
                acc += cn * lk_normal(s, tri, b.x, b.y, es, et, cn, gvn_out != nullptr, vid, gvn);
            }
            taps_at(s.tw, s.th, r.y, r.z, t[0]);
            taps_at(s.tw, s.th, r.y + es, r.z + et, t[1]);
            float da[3] = {0.f, 0.f, 0.f}, dr = 0.0f;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float sj = j ? -1.0f : 1.0f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = t[j].idx[k];
                    const float w = sj * t[j].w[k];
                    da[0] += w * __ldg(s.albedo + 3 * (size_t)i);
                    da[1] += w * __ldg(s.albedo + 3 * (size_t)i + 1);
                    da[2] += w * __ldg(s.albedo + 3 * (size_t)i + 2);
                    dr += w * __ldg(s.rough + i);
                }
            }
            acc += ca * (fabsf(da[0]) + fabsf(da[1]) + fabsf(da[2])) + cr * fabsf(dr);
            for (int c = 0; c < 3; ++c) sa[c] = ca * sgn(da[c]);
            sr = cr * sgn(dr);
        }
        if (want_grad) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float w = (j ? -1.0f : 1.0f) * t[j].w[k];
                    const float vals[4] = {sa[0] * w, sa[1] * w, sa[2] * w, sr * w};
                    scatter_agg<4>(tri >= 0 ? t[j].idx[k] : -1, vals, EmitLk{ga, gr});
                }
            }
        }
        if (normal && gvn_out) {
#pragma unroll
            for (int c = 0; c < 3; ++c) scatter_agg<3>(vid[c], gvn[c], EmitVn{gvn_out});
        }
    }
    if (loss) flush_loss(loss, acc);
}

// ---------------------------------------------------------------------------------------
// monochrome light regulariser (Appendix A, L_light): mean over the covered pixels of
// |Y(c_d + c_s) - V(I_ref)|, Y = channel mean, V = channel maximum; sign(0) = 0
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int view_of_pixel(const uint64_t* __restrict__ pix_off, int n_views, uint64_t q)
{
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pix_off[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// |P|: pixels whose demodulated lighting has coverage > 0
__global__ void __launch_bounds__(256) k_light_count(const uint64_t* __restrict__ pix_off, int n_views,
                                                     uint64_t total_pixels, const float* const* __restrict__ demod,
                                                     unsigned int* count)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < total_pixels; base += stride) {
        const uint64_t q = base + threadIdx.x;
        bool in = false;
        if (q < total_pixels) {
            const int vi = view_of_pixel(pix_off, n_views, q);
            in = demod[vi][4 * (q - pix_off[vi]) + 3] > 0.0f;
        }
        const unsigned b = __ballot_sync(MR_FULL, in);
        if (lane_id() == 0 && b) atomicAdd(count, (unsigned)__popc(b));
    }
}

__global__ void __launch_bounds__(256) k_light_apply(const uint64_t* __restrict__ pix_off, int n_views,
                                                     uint64_t total_pixels, const float* const* __restrict__ demod,
                                                     const float* const* __restrict__ ref, float w,
                                                     const unsigned int* __restrict__ count, float* loss,
                                                     float* const* __restrict__ d_demod)
{
    const unsigned int n = *count;
    const float inv = n ? 1.0f / (float)n : 0.0f;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    float acc = 0.0f;
    // uniform trip count per warp (the loss reduction uses every lane)
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < total_pixels; base += stride) {
        const uint64_t q = base + threadIdx.x;
        if (q < total_pixels) {
            const int vi = view_of_pixel(pix_off, n_views, q);
            const uint64_t p = q - pix_off[vi];
            const float4 c = __ldg(reinterpret_cast<const float4*>(demod[vi]) + p);
            float g = 0.0f;
            if (c.w > 0.0f && n) {
                const float* r = ref[vi] + 3 * p;
                const float diff = (c.x + c.y + c.z) * (1.0f / 3.0f) - fmaxf(fmaxf(__ldg(r), __ldg(r + 1)), __ldg(r + 2));
                acc += fabsf(diff);
                g = w * inv * (1.0f / 3.0f) * sgn(diff);
            }
            if (d_demod) {
                float* d = d_demod[vi] + 3 * p;
                d[0] = g;
                d[1] = g;
                d[2] = g;
            }
        }
    }
    if (loss) flush_loss(loss, acc * w * inv);
}

unsigned grid_of(int64_t n, int sms)
{
    const int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

mirres_status mr_edges_build(mirres_scene* s, cudaStream_t st)
{
    if (s->edges) return MIRRES_OK;
    const int F = s->desc.n_tris, V = s->desc.n_verts;
    const size_t cap = (size_t)3 * (F > 0 ? F : 1);
    size_t tsize = 1;
    while (tsize < 2 * cap) tsize <<= 1;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc((void**)&s->edges, sizeof(int2) * cap);
    e = e ? e : cudaMalloc((void**)&s->inv_deg, sizeof(float) * (size_t)(V > 0 ? V : 1));
    e = e ? e : cudaMalloc((void**)&s->n_edges, sizeof(unsigned int));
    e = e ? e : cudaMalloc((void**)&s->deg, sizeof(unsigned int) * (size_t)(V > 0 ? V : 1));
    e = e ? e : cudaMalloc((void**)&s->ehash, sizeof(unsigned long long) * tsize);
    if (e != cudaSuccess) {
        cudaGetLastError();
        mr_edges_free(s);
        mr_set_error(std::string("edge table allocation failed: ") + cudaGetErrorString(e));
        return MIRRES_ERR_OOM;
    }
    int dev = 0, sms = 1;
    MR_CUDA(cudaGetDevice(&dev));
    MR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MR_CUDA(cudaMemsetAsync(s->ehash, 0xFF, sizeof(unsigned long long) * tsize, st));
    MR_CUDA(cudaMemsetAsync(s->n_edges, 0, sizeof(unsigned int), st));
    MR_CUDA(cudaMemsetAsync(s->deg, 0, sizeof(unsigned int) * (size_t)(V > 0 ? V : 1), st));
    if (F > 0)
        k_edges_insert<<<grid_of(F, sms), 256, 0, st>>>(s->desc.tris, F, V, s->ehash, (unsigned long long)(tsize - 1),
                                                        s->edges, s->n_edges, s->deg);
    if (V > 0) k_inv_deg<<<grid_of(V, sms), 256, 0, st>>>(s->deg, V, s->inv_deg);
    MR_CUDA(cudaGetLastError());
    return MIRRES_OK;
}

void mr_edges_free(mirres_scene* s)
{
    void* ptrs[] = {s->edges, s->inv_deg, s->n_edges, s->deg, s->ehash};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    s->edges = nullptr;
    s->inv_deg = nullptr;
    s->n_edges = nullptr;
    s->deg = nullptr;
    s->ehash = nullptr;
}

void mr_launch_material_smoothness(const SceneDev& s, const ViewDev& v, uint32_t view_index, const Rng& rng,
                                   float sigma, float wa, float wr, float wn, float4* rec, float2* bary,
                                   unsigned int* n_hit, float* loss, float* ga, float* gr, bool grad_normals, int sms,
                                   cudaStream_t st)
{
    const int64_t npx = (int64_t)v.width * v.height;
    k_lk_hits<<<grid_of(npx, sms), 256, sizeof(uint32_t) * MR_SSTACK * 256, st>>>(s, v, rec, bary, n_hit);
    k_lk_apply<<<grid_of(npx, sms), 256, 0, st>>>(s, rec, bary, npx, n_hit, rng, view_index, sigma, wa, wr, wn, loss,
                                                  ga, gr, grad_normals ? s.gvn : nullptr);
}

void mr_launch_regularizers(const mirres_scene* s, const float* rest, float w_smooth, float w_offset, float* loss,
                            float* grad, int sms, cudaStream_t st)
{
    const int F = s->desc.n_tris, V = s->desc.n_verts;
    if (w_smooth != 0.0f && F > 0)
        k_smooth<<<grid_of(3 * (int64_t)F, sms), 256, 0, st>>>(s->edges, s->n_edges, s->inv_deg, s->desc.verts, w_smooth,
                                                               loss, grad);
    if (w_offset != 0.0f && V > 0)
        k_offset<<<grid_of(V, sms), 256, 0, st>>>(s->desc.verts, rest, V, w_offset, loss, grad);
}

cudaError_t mr_launch_light_loss(const uint64_t* pix_off, int n_views, uint64_t total_pixels,
                                 const float* const* demod, const float* const* ref, float w, unsigned int* count,
                                 float* loss, float* const* d_demod, int sms, cudaStream_t st)
{
    // |P| is counted from zero: a failed reset would scale the loss and its gradient wrongly
    const cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess || total_pixels == 0) return e;
    k_light_count<<<grid_of((int64_t)total_pixels, sms), 256, 0, st>>>(pix_off, n_views, total_pixels, demod, count);
    k_light_apply<<<grid_of((int64_t)total_pixels, sms), 256, 0, st>>>(pix_off, n_views, total_pixels, demod, ref, w,
                                                                       count, loss, d_demod);
    return cudaGetLastError();
}
