// bvh.cu -- LBVH build and refit on the GPU (Appendix A of the paper: a linear BVH after
// Karras 2012, kept up to date with the refined mesh at every optimisation iteration).
//
// build:  bounds (triangle centroids, centroid box, vertex box) -> 30-bit Morton codes ->
//         stable LSD radix sort of the codes with the triangle id as payload (the initial
//         order is by id, so the result is sorted by key = code << 32 | id) -> Karras's
//         per-node hierarchy construction -> bottom-up boxes with arrival counters, which
//         also writes the traversal layout (both child boxes in the parent, 64 bytes) and
//         the packed triangles (v0, e1, e2; 48 bytes) in leaf order.
//         With the PLOC builder selected the Karras step is replaced by locally-ordered
//         clustering over the same Morton-sorted leaves (a lower-SAH tree, same layout).
// refit:  bounds (vertex box only) -> bottom-up boxes, topology kept.
#include <algorithm>

#include "internal.h"

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__device__ __forceinline__ unsigned int f2o(float f)
{
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(unsigned int u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// bounds[0..2] centroid lo, [3..5] centroid hi, [6..8] vertex lo, [9..11] vertex hi
__global__ void k_init_bounds(unsigned int* bounds, int32_t* bad)
{
    const int i = threadIdx.x;
    if (i < 12) {
        const bool is_lo = (i < 3) || (i >= 6 && i < 9);
        bounds[i] = is_lo ? f2o(__int_as_float(0x7f800000)) : f2o(__int_as_float(0xff800000));
    }
    if (i == 0) *bad = 0;
}

__device__ __forceinline__ int checked_index(const int32_t* tris, size_t k, int V, int32_t* bad)
{
    const int i = __ldg(tris + k);
    if (i < 0 || i >= V) {
        *bad = 1;
        return 0;
    }
    return i;
}

__global__ void __launch_bounds__(256) k_bounds(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                                                int F, int V, float* __restrict__ cent, unsigned int* bounds,
                                                int32_t* bad, int with_centroids)
{
    const float INF = __int_as_float(0x7f800000);
    float b[12] = {INF, INF, INF, -INF, -INF, -INF, INF, INF, INF, -INF, -INF, -INF};
    const float third = 1.0f / 3.0f;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < F; t += gridDim.x * blockDim.x) {
        const int i0 = checked_index(tris, 3 * (size_t)t, V, bad);
        const int i1 = checked_index(tris, 3 * (size_t)t + 1, V, bad);
        const int i2 = checked_index(tris, 3 * (size_t)t + 2, V, bad);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float a = __ldg(verts + 3 * (size_t)i0 + k), c1 = __ldg(verts + 3 * (size_t)i1 + k),
                        c2 = __ldg(verts + 3 * (size_t)i2 + k);
            b[6 + k] = fminf(b[6 + k], fminf(fminf(a, c1), c2));
            b[9 + k] = fmaxf(b[9 + k], fmaxf(fmaxf(a, c1), c2));
            if (with_centroids) {
                // fixed order, no contraction: ((a + b) + c) * (1/3)
                const float m = __fmul_rn(__fadd_rn(__fadd_rn(a, c1), c2), third);
                cent[(size_t)k * F + t] = m;
                b[k] = fminf(b[k], m);
                b[3 + k] = fmaxf(b[3 + k], m);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        float v = b[k];
        const bool is_lo = (k < 3) || (k >= 6 && k < 9);
        for (int off = 16; off > 0; off >>= 1) {
            const float o = __shfl_xor_sync(MR_FULL, v, off);
            v = is_lo ? fminf(v, o) : fmaxf(v, o);
        }
        if ((threadIdx.x & 31) == 0) {
            if (is_lo) atomicMin(bounds + k, f2o(v));
            else atomicMax(bounds + k, f2o(v));
        }
    }
}

__global__ void __launch_bounds__(256) k_check_indices(const int32_t* __restrict__ tris, int64_t n, int V,
                                                       int32_t* bad)
{
    bool b = false;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int i = __ldg(tris + k);
        b = b || i < 0 || i >= V;
    }
    if (__any_sync(MR_FULL, b) && (threadIdx.x & 31) == 0) *bad = 1;
}

__global__ void k_finish_bounds(const unsigned int* bounds, int F, float* tmin)
{
    if (threadIdx.x != 0) return;
    if (F <= 0) {
        *tmin = 0.0f;
        return;
    }
    const float dx = o2f(bounds[9]) - o2f(bounds[6]);
    const float dy = o2f(bounds[10]) - o2f(bounds[7]);
    const float dz = o2f(bounds[11]) - o2f(bounds[8]);
    *tmin = 1e-5f * sqrtf(dx * dx + dy * dy + dz * dz);
}

__device__ __forceinline__ uint32_t expand10(uint32_t x)
{
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void k_morton(const float* __restrict__ cent, const unsigned int* __restrict__ bounds, int F,
                         uint32_t* __restrict__ codes, int32_t* __restrict__ vals)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= F) return;
    uint32_t q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = o2f(bounds[k]), hi = o2f(bounds[3 + k]);
        const float ext = __fsub_rn(hi, lo);
        float f = 0.0f;
        if (ext > 0.0f) f = __fmul_rn(__fdiv_rn(__fsub_rn(cent[(size_t)k * F + t], lo), ext), 1024.0f);
        int qi = (int)floorf(f);
        qi = min(max(qi, 0), 1023);
        q[k] = (uint32_t)qi;
    }
    codes[t] = (expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]);
    vals[t] = t;
}

// ---- stable LSD radix sort, 8-bit digits --------------------------------------------------
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t* __restrict__ keys, int n, int shift,
                                                        uint32_t* __restrict__ hist, int nb)
{
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * RS_TILE;
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const int idx = base + i * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of `total` entries in place, one block of 1024 threads
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t* __restrict__ a, int total)
{
    __shared__ uint32_t wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int seg = (total + 1023) / 1024;
    const int start = tid * seg, end = min(start + seg, total);
    uint32_t s = 0;
    for (int i = start; i < end; ++i) s += a[i];
    // inclusive scan of the per-thread sums
    uint32_t x = s;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(MR_FULL, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(MR_FULL, w, off);
            if (lane >= off) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    uint32_t run = x - s + (warp > 0 ? wsum[warp - 1] : 0u);
    for (int i = start; i < end; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t* __restrict__ kin,
                                                           const int32_t* __restrict__ vin,
                                                           uint32_t* __restrict__ kout, int32_t* __restrict__ vout,
                                                           int n, int shift, const uint32_t* __restrict__ offs,
                                                           int nb)
{
    constexpr int NW = RS_THREADS / 32;
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[NW][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = offs[(size_t)tid * nb + blockIdx.x];
#pragma unroll
    for (int w = 0; w < NW; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const int tile = blockIdx.x * RS_TILE;
    for (int round = 0; round < RS_ITEMS; ++round) {
        const int idx = tile + round * RS_THREADS + tid;
        const bool valid = idx < n;
        const uint32_t k = valid ? kin[idx] : 0u;
        const int32_t v = valid ? vin[idx] : 0;
        const uint32_t dig = valid ? ((k >> shift) & 255u) : 0x1000u;
        const unsigned peers = __match_any_sync(MR_FULL, dig);
        const int rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wcnt[warp][dig] = __popc(peers);
        __syncthreads();
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t c = wcnt[w][tid];
            wcnt[w][tid] = acc;
            acc += c;
        }
        __syncthreads();
        if (valid) {
            const uint32_t dst = base[dig] + wcnt[warp][dig] + (uint32_t)rank;
            kout[dst] = k;
            vout[dst] = v;
        }
        __syncthreads();
        base[tid] += acc;
#pragma unroll
        for (int w = 0; w < NW; ++w) wcnt[w][tid] = 0;
        __syncthreads();
    }
}

__global__ void k_keys(const uint32_t* __restrict__ codes, const int32_t* __restrict__ vals, int F,
                       uint64_t* __restrict__ keys, int32_t* __restrict__ perm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= F) return;
    keys[i] = ((uint64_t)codes[i] << 32) | (uint32_t)vals[i];
    perm[i] = vals[i];
}

// ---- Karras 2012 hierarchy: one thread per internal node ---------------------------------
__device__ __forceinline__ int delta(const uint64_t* __restrict__ k, int F, int i, int j)
{
    if (j < 0 || j >= F) return -1;
    return __clzll(k[i] ^ k[j]);
}

__global__ void k_karras(const uint64_t* __restrict__ k, int F, int32_t* __restrict__ left,
                         int32_t* __restrict__ right, int32_t* __restrict__ parent)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= F - 1) return;
    if (i == 0) parent[0] = -1;
    const int d = (delta(k, F, i, i + 1) - delta(k, F, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(k, F, i, i - d);
    int lmax = 2;
    while (delta(k, F, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(k, F, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(k, F, i, j);
    int s = 0;
    for (int div = 2;; div <<= 1) {
        const int t = (l + div - 1) / div;
        if (delta(k, F, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
    }
    const int g = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    if (lo == g) {
        left[i] = ~g;
        parent[(F - 1) + g] = i;
    } else {
        left[i] = g;
        parent[g] = i;
    }
    if (hi == g + 1) {
        right[i] = ~(g + 1);
        parent[(F - 1) + g + 1] = i;
    } else {
        right[i] = g + 1;
        parent[g + 1] = i;
    }
}

// ---- bottom-up boxes, traversal layout, packed triangles ---------------------------------
__global__ void k_bottom_up(const float* __restrict__ verts, const int32_t* __restrict__ tris, int F, int V,
                            const int32_t* __restrict__ perm, const int32_t* __restrict__ left,
                            const int32_t* __restrict__ right, const int32_t* __restrict__ parent,
                            float* lo, float* hi, int32_t* flags, float4* __restrict__ nodes,
                            float4* __restrict__ ptri, int32_t* __restrict__ leaf_of, int2* __restrict__ range)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= F) return;
    const int t = perm[j];
    int idx[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int v = __ldg(tris + 3 * (size_t)t + c);
        idx[c] = (v >= 0 && v < V) ? v : 0;
    }
    const float3 a = f3(verts[3 * (size_t)idx[0]], verts[3 * (size_t)idx[0] + 1], verts[3 * (size_t)idx[0] + 2]);
    const float3 b = f3(verts[3 * (size_t)idx[1]], verts[3 * (size_t)idx[1] + 1], verts[3 * (size_t)idx[1] + 2]);
    const float3 c = f3(verts[3 * (size_t)idx[2]], verts[3 * (size_t)idx[2] + 1], verts[3 * (size_t)idx[2] + 2]);
    const size_t L = (size_t)(F - 1) + j;
    lo[3 * L] = fminf(fminf(a.x, b.x), c.x);
    lo[3 * L + 1] = fminf(fminf(a.y, b.y), c.y);
    lo[3 * L + 2] = fminf(fminf(a.z, b.z), c.z);
    hi[3 * L] = fmaxf(fmaxf(a.x, b.x), c.x);
    hi[3 * L + 1] = fmaxf(fmaxf(a.y, b.y), c.y);
    hi[3 * L + 2] = fmaxf(fmaxf(a.z, b.z), c.z);
    float4* pt = ptri + MR_TRI_STRIDE * (size_t)j;
    pt[0] = make_float4(a.x, a.y, a.z, __int_as_float(t));
    pt[1] = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, 0.0f);
    pt[2] = make_float4(c.x - a.x, c.y - a.y, c.z - a.z, 0.0f);
    if (MR_TRI_STRIDE == 4) pt[3] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    leaf_of[t] = j;
    int p = parent[L];
    while (p >= 0) {
        __threadfence();
        if (atomicAdd(&flags[p], 1) == 0) return;  // the sibling's thread finishes this node
        __threadfence();
        const int cl = left[p], cr = right[p];
        const size_t il = cl >= 0 ? (size_t)cl : (size_t)(F - 1) + ~cl;
        const size_t ir = cr >= 0 ? (size_t)cr : (size_t)(F - 1) + ~cr;
        float bl[6], br[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            bl[k] = __ldcg(lo + 3 * il + k);
            bl[3 + k] = __ldcg(hi + 3 * il + k);
            br[k] = __ldcg(lo + 3 * ir + k);
            br[3 + k] = __ldcg(hi + 3 * ir + k);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            __stcg(lo + 3 * (size_t)p + k, fminf(bl[k], br[k]));
            __stcg(hi + 3 * (size_t)p + k, fmaxf(bl[3 + k], br[3 + k]));
        }
        nodes[4 * (size_t)p] = make_float4(bl[0], bl[1], bl[2], bl[3]);
        nodes[4 * (size_t)p + 1] = make_float4(bl[4], bl[5], br[0], br[1]);
        nodes[4 * (size_t)p + 2] = make_float4(br[2], br[3], br[4], br[5]);
        nodes[4 * (size_t)p + 3] = make_float4(__int_as_float(cl), __int_as_float(cr), 0.0f, 0.0f);
        // (first leaf position, leaf count) under p: the count is exact for every builder, the
        // first position delimits the subtree only for the Karras tree (clustering may pair
        // clusters that are not neighbours)
        const int2 rl = cl >= 0 ? __ldcg(range + cl) : make_int2(~cl, 1);
        const int2 rr = cr >= 0 ? __ldcg(range + cr) : make_int2(~cr, 1);
        __stcg(range + p, make_int2(min(rl.x, rr.x), rl.y + rr.y));
        p = parent[p];
    }
}

// ---- depth-first traversal layout -------------------------------------------------------------
// The traversal reads the internal nodes in depth-first preorder, left child first: a node's
// left child is the next node in memory, so a ray that descends left reads the 64 bytes after
// the ones it just read, and every subtree is one contiguous block. Preorder position of a node:
// its parent's plus 1 when it is the left child, plus 1 + (internal nodes of the left sibling's
// subtree) = the left sibling's leaf count (1 for a leaf) when it is the right child; each
// thread sums these up its path to the root. The boxes are copied unchanged, the children's
// node ids mapped to their positions (leaf children keep their leaf positions).
__global__ void k_dfs_index(const int32_t* __restrict__ parent, const int32_t* __restrict__ left,
                            const int2* __restrict__ range, int F, int32_t* __restrict__ dfs)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= F - 1) return;
    int idx = 0, c = n;
    for (int depth = 0; c != 0 && depth < 2 * F; ++depth) {  // every kept tree is at most 64 deep
        const int p = parent[c];
        if (p < 0) break;
        const int l = left[p];
        idx += (l == c) ? 1 : (l >= 0 ? range[l].y : 1);
        c = p;
    }
    dfs[n] = idx;
}

__global__ void k_dfs_gather(const float4* __restrict__ nodes, const int32_t* __restrict__ dfs, int F,
                             float4* __restrict__ dnodes)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= F - 1) return;
    const int q = dfs[n];
    if (q < 0 || q >= F - 1) return;  // (not for a well-formed tree: its positions are a permutation)
    dnodes[4 * (size_t)q] = nodes[4 * (size_t)n];
    dnodes[4 * (size_t)q + 1] = nodes[4 * (size_t)n + 1];
    dnodes[4 * (size_t)q + 2] = nodes[4 * (size_t)n + 2];
    const float4 ch = nodes[4 * (size_t)n + 3];
    int cl = __float_as_int(ch.x), cr = __float_as_int(ch.y);
    if (cl >= 0) cl = dfs[cl];
    if (cr >= 0) cr = dfs[cr];
    dnodes[4 * (size_t)q + 3] = make_float4(__int_as_float(cl), __int_as_float(cr), 0.0f, 0.0f);
}

// ---- PLOC hierarchy: parallel locally-ordered clustering (Meister and Bittner 2018) ------
// The clusters start as the leaves in Morton order. In every iteration each cluster finds,
// among the PLOC_R clusters on either side of it, the one whose union box has the smallest
// surface area; pairs are ordered by (area, smaller position, larger position), a total order,
// so the least pair of the array is always mutual and every iteration merges at least once.
// Mutual pairs merge into a new node that takes the lower position, and the array is compacted
// in order (a block scan of (kept, merged) flags). Node ids are handed out downwards from F - 2,
// so the last merge -- the root -- gets id 0, and the left / right / parent arrays have the
// layout the Karras build writes (leaves as ~position): bottom_up and refit work unchanged.
constexpr int PLOC_R = 16;
constexpr int PLOC_T = 256;
constexpr int PLOC_ITEMS = 4;
constexpr int PLOC_TILE = PLOC_T * PLOC_ITEMS;

__global__ void __launch_bounds__(256) k_ploc_leaves(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                                                     int F, int V, const int32_t* __restrict__ perm, float4* lo,
                                                     float4* hi, int32_t* node, int32_t* state)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) {
        state[0] = F;
        state[1] = F;
        state[2] = F - 2;
        state[3] = F - 2;
    }
    if (j >= F) return;
    const int t = perm[j];
    float3 p[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        int v = __ldg(tris + 3 * (size_t)t + c);
        v = (v >= 0 && v < V) ? v : 0;
        p[c] = f3(verts[3 * (size_t)v], verts[3 * (size_t)v + 1], verts[3 * (size_t)v + 2]);
    }
    lo[j] = make_float4(fminf(fminf(p[0].x, p[1].x), p[2].x), fminf(fminf(p[0].y, p[1].y), p[2].y),
                        fminf(fminf(p[0].z, p[1].z), p[2].z), 0.0f);
    hi[j] = make_float4(fmaxf(fmaxf(p[0].x, p[1].x), p[2].x), fmaxf(fmaxf(p[0].y, p[1].y), p[2].y),
                        fmaxf(fmaxf(p[0].z, p[1].z), p[2].z), 0.0f);
    node[j] = ~j;
}

// half the surface area of the union of two boxes; symmetric bit for bit, non-finite -> +inf
__device__ __forceinline__ float union_area(float4 alo, float4 ahi, float4 blo, float4 bhi)
{
    const float dx = fmaxf(ahi.x, bhi.x) - fminf(alo.x, blo.x);
    const float dy = fmaxf(ahi.y, bhi.y) - fminf(alo.y, blo.y);
    const float dz = fmaxf(ahi.z, bhi.z) - fminf(alo.z, blo.z);
    const float a = dx * dy + dy * dz + dz * dx;
    return (a <= 3.402823466e38f) ? a : __int_as_float(0x7f800000);
}

__global__ void __launch_bounds__(PLOC_T) k_ploc_nn(const int32_t* __restrict__ state, int par,
                                                    const float4* __restrict__ lo, const float4* __restrict__ hi,
                                                    int32_t* __restrict__ nn)
{
    __shared__ float4 slo[PLOC_T + 2 * PLOC_R], shi[PLOC_T + 2 * PLOC_R];
    const int n = state[par];
    for (int base = blockIdx.x * PLOC_T; base < n; base += gridDim.x * PLOC_T) {  // block-uniform
        for (int k = threadIdx.x; k < PLOC_T + 2 * PLOC_R; k += PLOC_T) {
            const int g = base - PLOC_R + k;
            if (g >= 0 && g < n) {
                slo[k] = lo[g];
                shi[k] = hi[g];
            }
        }
        __syncthreads();
        const int i = base + (int)threadIdx.x;
        if (i < n) {
            const float4 alo = slo[threadIdx.x + PLOC_R], ahi = shi[threadIdx.x + PLOC_R];
            float best = __int_as_float(0x7f800000);
            int bj = -1;
            const int j0 = max(0, i - PLOC_R), j1 = min(n - 1, i + PLOC_R);
            for (int j = j0; j <= j1; ++j) {
                if (j == i) continue;
                const int k = j - base + PLOC_R;
                const float d = union_area(alo, ahi, slo[k], shi[k]);
                // equal areas: the pair with the smaller (min, max) positions wins
                bool take = d < best;
                if (d == best) {
                    if (bj < 0) {
                        take = true;
                    } else {
                        const int a0 = min(i, j), a1 = max(i, j), b0 = min(i, bj), b1 = max(i, bj);
                        take = (a0 < b0) || (a0 == b0 && a1 < b1);
                    }
                }
                if (take) {
                    best = d;
                    bj = j;
                }
            }
            nn[i] = bj;
        }
        __syncthreads();
    }
}

// (kept, merged) of cluster i: a mutual pair keeps its lower position, which also merges
__device__ __forceinline__ uint2 ploc_flags(const int32_t* __restrict__ nn, int i)
{
    const int j = nn[i];
    const bool mutual = j >= 0 && nn[j] == i;
    return make_uint2((mutual && j < i) ? 0u : 1u, (mutual && i < j) ? 1u : 0u);
}

__device__ __forceinline__ uint2 add2(uint2 a, uint2 b) { return make_uint2(a.x + b.x, a.y + b.y); }

// exclusive scan of one uint2 per thread over a block of PLOC_T threads; returns the total
__device__ __forceinline__ uint2 block_scan2(uint2 v, uint2& excl)
{
    __shared__ uint2 warp_sum[PLOC_T / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint2 inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned ox = __shfl_up_sync(0xffffffffu, inc.x, off), oy = __shfl_up_sync(0xffffffffu, inc.y, off);
        if (lane >= off) inc = add2(inc, make_uint2(ox, oy));
    }
    if (lane == 31) warp_sum[w] = inc;
    __syncthreads();
    uint2 before = make_uint2(0u, 0u), total = make_uint2(0u, 0u);
#pragma unroll
    for (int k = 0; k < PLOC_T / 32; ++k) {
        if (k < w) before = add2(before, warp_sum[k]);
        total = add2(total, warp_sum[k]);
    }
    __syncthreads();
    excl = add2(before, make_uint2(inc.x - v.x, inc.y - v.y));
    return total;
}

__global__ void __launch_bounds__(PLOC_T) k_ploc_count(const int32_t* __restrict__ state, int par,
                                                       const int32_t* __restrict__ nn, uint2* __restrict__ part)
{
    const int n = state[par];
    const int nb = (n + PLOC_TILE - 1) / PLOC_TILE;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {  // block-uniform
        uint2 c = make_uint2(0u, 0u);
#pragma unroll
        for (int k = 0; k < PLOC_ITEMS; ++k) {
            const int i = b * PLOC_TILE + (int)threadIdx.x * PLOC_ITEMS + k;
            if (i < n) c = add2(c, ploc_flags(nn, i));
        }
        uint2 excl;
        const uint2 tot = block_scan2(c, excl);
        if (threadIdx.x == 0) part[b] = tot;
    }
}

// one block: exclusive scan of the per-block counts in place; the next iteration's cluster
// count and node-id base go to the other parity's slots
__global__ void __launch_bounds__(PLOC_T) k_ploc_scan(int32_t* __restrict__ state, int par, uint2* __restrict__ part)
{
    const int n = state[par];
    const int nb = (n + PLOC_TILE - 1) / PLOC_TILE;
    uint2 carry = make_uint2(0u, 0u);
    for (int base = 0; base < nb; base += PLOC_T) {  // block-uniform
        const int b = base + (int)threadIdx.x;
        const uint2 v = b < nb ? part[b] : make_uint2(0u, 0u);
        uint2 excl;
        const uint2 tot = block_scan2(v, excl);
        if (b < nb) part[b] = add2(carry, excl);
        carry = add2(carry, tot);
    }
    if (threadIdx.x == 0) {
        state[1 - par] = (int32_t)carry.x;
        state[3 - par] = state[2 + par] - (int32_t)carry.y;
    }
}

__global__ void __launch_bounds__(PLOC_T) k_ploc_compact(const int32_t* __restrict__ state, int par, int F,
                                                         const int32_t* __restrict__ nn, const uint2* __restrict__ part,
                                                         const float4* __restrict__ lo, const float4* __restrict__ hi,
                                                         const int32_t* __restrict__ node, float4* __restrict__ olo,
                                                         float4* __restrict__ ohi, int32_t* __restrict__ onode,
                                                         int32_t* __restrict__ left, int32_t* __restrict__ right,
                                                         int32_t* __restrict__ parent)
{
    const int n = state[par];
    const int idb = state[2 + par];
    const int nb = (n + PLOC_TILE - 1) / PLOC_TILE;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {  // block-uniform
        const int i0 = b * PLOC_TILE + (int)threadIdx.x * PLOC_ITEMS;
        uint2 f[PLOC_ITEMS];
        uint2 c = make_uint2(0u, 0u);
#pragma unroll
        for (int k = 0; k < PLOC_ITEMS; ++k) {
            f[k] = (i0 + k < n) ? ploc_flags(nn, i0 + k) : make_uint2(0u, 0u);
            c = add2(c, f[k]);
        }
        uint2 excl;
        block_scan2(c, excl);
        uint2 pos = add2(part[b], excl);
#pragma unroll
        for (int k = 0; k < PLOC_ITEMS; ++k) {
            const int i = i0 + k;
            if (i >= n || !f[k].x) continue;
            if (f[k].y) {
                const int j = nn[i];
                const int id = idb - (int)pos.y;
                const int cl = node[i], cr = node[j];
                left[id] = cl;
                right[id] = cr;
                parent[cl >= 0 ? cl : (F - 1) + ~cl] = id;
                parent[cr >= 0 ? cr : (F - 1) + ~cr] = id;
                const float4 al = lo[i], ah = hi[i], bl = lo[j], bh = hi[j];
                olo[pos.x] = make_float4(fminf(al.x, bl.x), fminf(al.y, bl.y), fminf(al.z, bl.z), 0.0f);
                ohi[pos.x] = make_float4(fmaxf(ah.x, bh.x), fmaxf(ah.y, bh.y), fmaxf(ah.z, bh.z), 0.0f);
                onode[pos.x] = id;
            } else {
                olo[pos.x] = lo[i];
                ohi[pos.x] = hi[i];
                onode[pos.x] = node[i];
            }
            pos = add2(pos, f[k]);
        }
    }
}

// depth of every leaf (edges to the root), maximum into *depth; the walk stops after 1024 steps
__global__ void __launch_bounds__(256) k_leaf_depth(const int32_t* __restrict__ parent, int F, int32_t* depth)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= F) return;
    int d = 0, p = parent[(F - 1) + j];
    while (p >= 0 && d < 1024) {
        ++d;
        p = parent[p];
    }
    atomicMax(depth, d);
}

// ---- area-weighted vertex normals for interpolated shading normals ------------------------
__global__ void __launch_bounds__(256) k_vn_accumulate(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                                                       int F, int V, float* vacc)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < F; t += gridDim.x * blockDim.x) {
        int idx[3];
        float3 p[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int v = __ldg(tris + 3 * (size_t)t + c);
            idx[c] = (v >= 0 && v < V) ? v : 0;
            p[c] = f3(verts[3 * (size_t)idx[c]], verts[3 * (size_t)idx[c] + 1], verts[3 * (size_t)idx[c] + 2]);
        }
        const float3 N = cross(sub(p[1], p[0]), sub(p[2], p[0]));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicAdd(vacc + 3 * (size_t)idx[c], N.x);
            atomicAdd(vacc + 3 * (size_t)idx[c] + 1, N.y);
            atomicAdd(vacc + 3 * (size_t)idx[c] + 2, N.z);
        }
    }
}

__global__ void __launch_bounds__(256) k_vn_normalize(const float* __restrict__ vacc, int V, float4* vnrm)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
        const float3 A = f3(vacc[3 * (size_t)i], vacc[3 * (size_t)i + 1], vacc[3 * (size_t)i + 2]);
        const float l2 = dot(A, A);
        const float il = l2 > 0.0f ? rsqrtf(l2) : 0.0f;
        vnrm[i] = make_float4(A.x * il, A.y * il, A.z * il, 0.0f);
    }
}

// VN_i = A_i / |A_i|, A_i = sum over the faces f around vertex i of N_f = e1 x e2: per face,
// d loss / d N_f = sum over its vertices of (I - VN VN^T) gvn_i / |A_i|, then to its vertices
__global__ void __launch_bounds__(256) k_vn_adjoint(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                                                    int F, int V, const float* __restrict__ vacc,
                                                    const float* __restrict__ gvn, float* grad)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < F; t += gridDim.x * blockDim.x) {
        int idx[3];
        float3 gN = f3(0.f, 0.f, 0.f);
        bool any = false;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int v = __ldg(tris + 3 * (size_t)t + c);
            idx[c] = (v >= 0 && v < V) ? v : 0;
            const float3 g = f3(gvn[3 * (size_t)idx[c]], gvn[3 * (size_t)idx[c] + 1], gvn[3 * (size_t)idx[c] + 2]);
            if (g.x == 0.0f && g.y == 0.0f && g.z == 0.0f) continue;
            const float3 A = f3(vacc[3 * (size_t)idx[c]], vacc[3 * (size_t)idx[c] + 1], vacc[3 * (size_t)idx[c] + 2]);
            const float l2 = dot(A, A);
            if (!(l2 > 0.0f)) continue;
            const float il = rsqrtf(l2);
            const float3 n = mul(A, il);
            gN = add(gN, mul(sub(g, mul(n, dot(n, g))), il));
            any = true;
        }
        if (!any) continue;
        float3 p[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            p[c] = f3(verts[3 * (size_t)idx[c]], verts[3 * (size_t)idx[c] + 1], verts[3 * (size_t)idx[c] + 2]);
        const float3 e1 = sub(p[1], p[0]), e2 = sub(p[2], p[0]);
        const float3 ge1 = cross(e2, gN), ge2 = cross(gN, e1);
        const float3 gv[3] = {f3(-(ge1.x + ge2.x), -(ge1.y + ge2.y), -(ge1.z + ge2.z)), ge1, ge2};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicAdd(grad + 3 * (size_t)idx[c], gv[c].x);
            atomicAdd(grad + 3 * (size_t)idx[c] + 1, gv[c].y);
            atomicAdd(grad + 3 * (size_t)idx[c] + 2, gv[c].z);
        }
    }
}

int grid_for(int n, int block) { return (n + block - 1) / block; }

}  // namespace

template <typename T>
static mirres_status mr_alloc(T** p, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        mr_set_error(std::string("device allocation failed: ") + cudaGetErrorString(e));
        return MIRRES_ERR_OOM;
    }
    return MIRRES_OK;
}

#define MR_TRY(x)                            \
    do {                                     \
        mirres_status s__ = (x);             \
        if (s__ != MIRRES_OK) return s__;    \
    } while (0)

mirres_status mr_bvh_alloc(mirres_scene* s)
{
    const size_t F = (size_t)s->desc.n_tris;
    const size_t nb = (F + RS_TILE - 1) / RS_TILE;
    MR_TRY(mr_alloc(&s->keys, F));
    MR_TRY(mr_alloc(&s->perm, F));
    MR_TRY(mr_alloc(&s->left, F > 1 ? F - 1 : 1));
    MR_TRY(mr_alloc(&s->right, F > 1 ? F - 1 : 1));
    MR_TRY(mr_alloc(&s->parent, F > 0 ? 2 * F - 1 : 1));
    MR_TRY(mr_alloc(&s->lo, 3 * (F > 0 ? 2 * F - 1 : 1)));
    MR_TRY(mr_alloc(&s->hi, 3 * (F > 0 ? 2 * F - 1 : 1)));
    MR_TRY(mr_alloc(&s->flags, F > 1 ? F - 1 : 1));
    MR_TRY(mr_alloc(&s->nodes, 4 * (F > 1 ? F - 1 : 1)));
    MR_TRY(mr_alloc(&s->dnodes, 4 * (F > 1 ? F - 1 : 1)));
    MR_TRY(mr_alloc(&s->dfs, F > 1 ? F - 1 : 1));
    MR_TRY(mr_alloc(&s->ptri, MR_TRI_STRIDE * F));
    MR_TRY(mr_alloc(&s->leaf_of, F));
    MR_TRY(mr_alloc(&s->range, F > 1 ? F - 1 : 1));
    MR_TRY(mr_alloc(&s->cent, 3 * F));
    MR_TRY(mr_alloc(&s->codes[0], F));
    MR_TRY(mr_alloc(&s->codes[1], F));
    MR_TRY(mr_alloc(&s->vals[0], F));
    MR_TRY(mr_alloc(&s->vals[1], F));
    MR_TRY(mr_alloc(&s->hist, 256 * (nb ? nb : 1)));
    MR_TRY(mr_alloc(&s->bounds, 12));
    MR_TRY(mr_alloc(&s->tmin, 1));
    MR_TRY(mr_alloc(&s->bad, 1));
    return MIRRES_OK;
}

void mr_bvh_free(mirres_scene* s)
{
    void* ptrs[] = {s->keys, s->perm, s->left, s->right, s->parent, s->lo, s->hi, s->flags, s->nodes, s->ptri,
                    s->leaf_of, s->cent, s->codes[0], s->codes[1], s->vals[0], s->vals[1], s->hist, s->bounds,
                    s->tmin, s->bad, s->ploc_box, s->ploc_node, s->ploc_nn, s->ploc_part, s->ploc_state,
                    s->vacc, s->vnrm, s->gvn, s->range, s->dnodes, s->dfs};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    mr_wide_free(s);
}

static mirres_status bottom_up(mirres_scene* s, cudaStream_t st)
{
    const int F = s->desc.n_tris;
    if (F <= 0) return MIRRES_OK;
    if (F > 1) MR_CUDA(cudaMemsetAsync(s->flags, 0, sizeof(int32_t) * (size_t)(F - 1), st));
    k_bottom_up<<<grid_for(F, 256), 256, 0, st>>>(s->desc.verts, s->desc.tris, F, s->desc.n_verts, s->perm, s->left,
                                                 s->right, s->parent, s->lo, s->hi, s->flags, s->nodes, s->ptri,
                                                 s->leaf_of, s->range);
    if (F > 1) {
        k_dfs_index<<<grid_for(F - 1, 256), 256, 0, st>>>(s->parent, s->left, s->range, F, s->dfs);
        k_dfs_gather<<<grid_for(F - 1, 256), 256, 0, st>>>(s->nodes, s->dfs, F, s->dnodes);
    }
    MR_CUDA(cudaGetLastError());
    return MIRRES_OK;
}

static mirres_status bounds(mirres_scene* s, cudaStream_t st, int with_centroids)
{
    const int F = s->desc.n_tris;
    k_init_bounds<<<1, 32, 0, st>>>(s->bounds, s->bad);
    if (F > 0) {
        int grid = grid_for(F, 256);
        if (grid > 4096) grid = 4096;
        k_bounds<<<grid, 256, 0, st>>>(s->desc.verts, s->desc.tris, F, s->desc.n_verts, s->cent, s->bounds, s->bad,
                                       with_centroids);
    }
    k_finish_bounds<<<1, 32, 0, st>>>(s->bounds, F, s->tmin);
    MR_CUDA(cudaGetLastError());
    return MIRRES_OK;
}

static mirres_status ploc_alloc(mirres_scene* s)
{
    if (s->ploc_box) return MIRRES_OK;
    const size_t F = (size_t)s->desc.n_tris;
    MR_TRY(mr_alloc(&s->ploc_box, 4 * F));
    MR_TRY(mr_alloc(&s->ploc_node, 2 * F));
    MR_TRY(mr_alloc(&s->ploc_nn, F));
    MR_TRY(mr_alloc(&s->ploc_part, (F + PLOC_TILE - 1) / PLOC_TILE));
    MR_TRY(mr_alloc(&s->ploc_state, 4));
    return MIRRES_OK;
}

// PLOC hierarchy over the Morton-sorted leaves (F >= 2): batches of 16 iterations between
// host checks of the cluster count; every iteration merges at least one pair
static mirres_status ploc_build(mirres_scene* s, cudaStream_t st, bool& too_deep)
{
    too_deep = false;
    MR_TRY(ploc_alloc(s));
    const int F = s->desc.n_tris;
    int dev = 0, sms = 1;
    MR_CUDA(cudaGetDevice(&dev));
    MR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float4* lo[2] = {s->ploc_box, s->ploc_box + 2 * (size_t)F};
    float4* hi[2] = {s->ploc_box + (size_t)F, s->ploc_box + 3 * (size_t)F};
    int32_t* node[2] = {s->ploc_node, s->ploc_node + (size_t)F};
    int32_t* state = s->ploc_state;
    k_ploc_leaves<<<grid_for(F, 256), 256, 0, st>>>(s->desc.verts, s->desc.tris, F, s->desc.n_verts, s->perm, lo[0],
                                                    hi[0], node[0], state);
    const int g_nn = std::min(grid_for(F, PLOC_T), sms * 8), g_t = std::min(grid_for(F, PLOC_TILE), sms * 8);
    int par = 0, n_prev = F;
    int32_t h[5] = {F, F, 0, 0, -1};
    while (h[par] > 1) {
        for (int k = 0; k < 16; ++k) {
            k_ploc_nn<<<g_nn, PLOC_T, 0, st>>>(state, par, lo[par], hi[par], s->ploc_nn);
            k_ploc_count<<<g_t, PLOC_T, 0, st>>>(state, par, s->ploc_nn, s->ploc_part);
            k_ploc_scan<<<1, PLOC_T, 0, st>>>(state, par, s->ploc_part);
            k_ploc_compact<<<g_t, PLOC_T, 0, st>>>(state, par, F, s->ploc_nn, s->ploc_part, lo[par], hi[par], node[par],
                                                   lo[par ^ 1], hi[par ^ 1], node[par ^ 1], s->left, s->right,
                                                   s->parent);
            par ^= 1;
        }
        MR_CUDA(cudaGetLastError());
        MR_CUDA(cudaMemcpyAsync(h, state, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, st));
        MR_CUDA(cudaMemcpyAsync(h + 4, node[par], sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        MR_CUDA(cudaStreamSynchronize(st));
        if (h[par] > 1 && h[par] >= n_prev) {
            mr_set_error("mirres_bvh_build: PLOC made no progress");
            return MIRRES_ERR_STATE;
        }
        n_prev = h[par];
    }
    if (h[4] != 0 || h[2 + par] != -1) {
        mr_set_error("mirres_bvh_build: PLOC did not end at the root");
        return MIRRES_ERR_STATE;
    }
    // the traversal stack holds MR_SSTACK + MR_LSTACK entries, at most one per level below the
    // root: a deeper clustering tree is replaced by the Karras tree (at most 63 deep)
    MR_CUDA(cudaMemsetAsync(state, 0, sizeof(int32_t), st));
    k_leaf_depth<<<grid_for(F, 256), 256, 0, st>>>(s->parent, F, state);
    MR_CUDA(cudaMemcpyAsync(h, state, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MR_CUDA(cudaStreamSynchronize(st));
    too_deep = h[0] > MR_SSTACK + MR_LSTACK;
    return MIRRES_OK;
}

mirres_status mr_bvh_build(mirres_scene* s, cudaStream_t st)
{
    const int F = s->desc.n_tris;
    MR_TRY(bounds(s, st, 1));
    if (F > 0) {
        const int nb = (F + RS_TILE - 1) / RS_TILE;
        k_morton<<<grid_for(F, 256), 256, 0, st>>>(s->cent, s->bounds, F, s->codes[0], s->vals[0]);
        int cur = 0;
        for (int shift = 0; shift < 32; shift += 8) {
            k_rs_hist<<<nb, RS_THREADS, 0, st>>>(s->codes[cur], F, shift, s->hist, nb);
            k_rs_scan<<<1, 1024, 0, st>>>(s->hist, 256 * nb);
            k_rs_scatter<<<nb, RS_THREADS, 0, st>>>(s->codes[cur], s->vals[cur], s->codes[cur ^ 1], s->vals[cur ^ 1],
                                                    F, shift, s->hist, nb);
            cur ^= 1;
        }
        k_keys<<<grid_for(F, 256), 256, 0, st>>>(s->codes[cur], s->vals[cur], F, s->keys, s->perm);
        MR_CUDA(cudaMemsetAsync(s->parent, 0xFF, sizeof(int32_t) * (size_t)(2 * F - 1), st));
        bool karras = F > 1;
        if (F > 1 && s->builder == MIRRES_BVH_PLOC) {
            bool too_deep = false;
            MR_TRY(ploc_build(s, st, too_deep));
            karras = too_deep;
            if (too_deep) MR_CUDA(cudaMemsetAsync(s->parent, 0xFF, sizeof(int32_t) * (size_t)(2 * F - 1), st));
        }
        if (karras) k_karras<<<grid_for(F - 1, 256), 256, 0, st>>>(s->keys, F, s->left, s->right, s->parent);
        MR_CUDA(cudaGetLastError());
        MR_TRY(bottom_up(s, st));
        if (s->traversal == MIRRES_TRAVERSAL_WIDE) MR_TRY(mr_wide_build(s, st));
    }
    if (s->normals) MR_TRY(mr_vertex_normals(s, st));
    return MIRRES_OK;
}

// Triangle indices are checked once, when the scene is created (and again on request), not
// by every build: the build would have to wait for the check on the host. The build kernels
// read an out-of-range index as vertex 0.
mirres_status mr_check_indices(mirres_scene* s, cudaStream_t st)
{
    const int F = s->desc.n_tris;
    if (F <= 0) return MIRRES_OK;
    MR_CUDA(cudaMemsetAsync(s->bad, 0, sizeof(int32_t), st));
    k_check_indices<<<std::min(grid_for(3 * F, 256), 4096), 256, 0, st>>>(s->desc.tris, 3 * (int64_t)F,
                                                                         s->desc.n_verts, s->bad);
    MR_CUDA(cudaGetLastError());
    int32_t bad = 0;
    MR_CUDA(cudaMemcpyAsync(&bad, s->bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MR_CUDA(cudaStreamSynchronize(st));
    if (bad) {
        mr_set_error("a triangle index is outside [0, n_verts)");
        return MIRRES_ERR_ARG;
    }
    return MIRRES_OK;
}

mirres_status mr_bvh_refit(mirres_scene* s, cudaStream_t st)
{
    MR_TRY(bounds(s, st, 0));
    MR_TRY(bottom_up(s, st));
    if (s->desc.n_tris > 0 && s->traversal == MIRRES_TRAVERSAL_WIDE) MR_TRY(mr_wide_build(s, st));
    if (s->normals) MR_TRY(mr_vertex_normals(s, st));
    return MIRRES_OK;
}

mirres_status mr_normals_alloc(mirres_scene* s)
{
    if (s->vnrm) return MIRRES_OK;
    const size_t V = (size_t)(s->desc.n_verts > 0 ? s->desc.n_verts : 1);
    MR_TRY(mr_alloc(&s->vacc, 3 * V));
    MR_TRY(mr_alloc(&s->vnrm, V));
    MR_TRY(mr_alloc(&s->gvn, 3 * V));
    return MIRRES_OK;
}

mirres_status mr_vertex_normals(mirres_scene* s, cudaStream_t st)
{
    const int F = s->desc.n_tris, V = s->desc.n_verts;
    if (V <= 0) return MIRRES_OK;
    MR_TRY(mr_normals_alloc(s));
    MR_CUDA(cudaMemsetAsync(s->vacc, 0, sizeof(float) * 3 * (size_t)V, st));
    if (F > 0)
        k_vn_accumulate<<<std::min(grid_for(F, 256), 4096), 256, 0, st>>>(s->desc.verts, s->desc.tris, F, V, s->vacc);
    k_vn_normalize<<<std::min(grid_for(V, 256), 4096), 256, 0, st>>>(s->vacc, V, s->vnrm);
    MR_CUDA(cudaGetLastError());
    return MIRRES_OK;
}

void mr_launch_normals_adjoint(const mirres_scene* s, float* grad_verts, int sms, cudaStream_t st)
{
    const int F = s->desc.n_tris, V = s->desc.n_verts;
    if (F <= 0 || V <= 0 || !grad_verts) return;
    k_vn_adjoint<<<std::min(grid_for(F, 256), sms * 8), 256, 0, st>>>(s->desc.verts, s->desc.tris, F, V, s->vacc,
                                                                      s->gvn, grad_verts);
}
