// wbvh.cu -- the 8-wide BVH the ray traversal runs, collapsed from the binary tree (LBVH or
// PLOC) after every build and refit.
//
// Layout (80 bytes per node, five 16-byte words; after the compressed wide BVH of Ylitie,
// Karras and Laine 2017, own encoding):
//   w0  origin p (3 floats: the node box's low corner), then bytes ex, ey, ez (biased exponents
//       e + 127 of the per-axis quantisation steps 2^e) and imask (bit i: slot i holds a node)
//   w1  index of the first child node, index of the first triangle, meta bytes of slots 0..7
//       (0 empty; 0x80 node; leaf: (count << 5) | offset, count 1..3 triangles at wtri
//       [first triangle + offset ...])
//   w2..w4  per slot, 8-bit child boxes in steps of 2^e from p: qlo x, y, z, then qhi x, y, z
//       (one byte per slot, slots 0..3 in the first 32-bit word of each pair)
// The children of a node that are nodes occupy consecutive indices in slot order; the leaf
// triangles of a node are consecutive in `wtri` (the packed triangles copied in that order; a
// leaf's triangles are gathered from its subtree, whose leaves need not be consecutive in the
// binary tree's leaf order when it was built by clustering).
// Child boxes are rounded outwards by one step on every side, so the quantised box contains
// the exact one and its FP32 reconstruction; a ray therefore enters every leaf it would enter
// in the binary tree, and the hits do not depend on the tree.
//
// Collapse, top down, one thread per wide node, one launch per level: a node's children start as
// the two binary children; the child subtree with the largest surface area that holds more
// than three triangles is replaced by its two children until there are eight or none is left to
// open; subtrees of at most three triangles (contiguous in leaf order) become leaves. Children
// are placed in slots so that slot i holds the child lying furthest along the octant direction
// (-1)^i (greedy assignment of the smallest projection of the child's centre offset onto that
// direction): a ray whose direction signs form octant `oct` visits slots in the order i ^ oct.
#include "internal.h"

namespace {

constexpr int kBlock = 128;

__device__ __forceinline__ float half_area(const float* __restrict__ lo, const float* __restrict__ hi, size_t i)
{
    const float dx = hi[3 * i] - lo[3 * i], dy = hi[3 * i + 1] - lo[3 * i + 1], dz = hi[3 * i + 2] - lo[3 * i + 2];
    return dx * dy + dy * dz + dz * dx;
}

__global__ void k_wide_init(int2* q, unsigned int* cnt)
{
    if (threadIdx.x == 0) {
        q[0] = make_int2(0, 0);  // binary root -> wide root
        cnt[0] = 1;              // wide nodes handed out (the root)
        cnt[1] = 0;              // triangles handed out
        cnt[2] = 1;              // queue length of level 0
    }
}

// quantisation exponent of one axis: the smallest step 2^e with (hi - p) / 2^e <= 253, no finer
// than 2^-22 of the largest coordinate magnitude (so p + q 2^e is reconstructed to ~an ulp)
__device__ __forceinline__ int quant_exp(float p, float hi)
{
    const float ext = __fsub_ru(hi, p);
    int e = 0;
    if (ext > 0.0f) frexpf(__fdiv_ru(ext, 253.0f), &e);
    int km = 0;
    frexpf(fmaxf(fabsf(p), fabsf(hi)), &km);
    e = max(e, km - 22);
    return min(max(e, -126), 126);
}

__global__ void __launch_bounds__(kBlock) k_wide_level(const int32_t* __restrict__ left,
                                                       const int32_t* __restrict__ right,
                                                       const int2* __restrict__ range, const float* __restrict__ lo,
                                                       const float* __restrict__ hi, const float4* __restrict__ ptri,
                                                       int F, const int2* __restrict__ qin,
                                                       const unsigned int* __restrict__ nin, int2* __restrict__ qout,
                                                       unsigned int* nout, uint4* __restrict__ wnodes,
                                                       float4* __restrict__ wtri, unsigned int* alloc)
{
    const unsigned int n = *nin;
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int2 item = qin[k];
        const int b = item.x, w = item.y;
        // children: open the largest subtree of more than three triangles until there are eight
        int c[8];
        int nc = 2;
        c[0] = left[b];
        c[1] = right[b];
        while (nc < 8) {
            int best = -1;
            float ba = -1.0f;
            for (int i = 0; i < nc; ++i) {
                const int ci = c[i];
                if (ci >= 0 && range[ci].y > 3) {
                    const float a = half_area(lo, hi, (size_t)ci);
                    if (a > ba || best < 0) {
                        ba = a;
                        best = i;
                    }
                }
            }
            if (best < 0) break;
            const int cb = c[best];
            c[best] = left[cb];
            c[nc++] = right[cb];
        }
        // child boxes, kinds, triangle ranges
        float clo[8][3], chi[8][3];
        int count[8];
        bool inner[8];
        for (int i = 0; i < nc; ++i) {
            const int ci = c[i];
            const size_t bi = ci >= 0 ? (size_t)ci : (size_t)(F - 1) + (size_t)(~ci);
            for (int a = 0; a < 3; ++a) {
                clo[i][a] = lo[3 * bi + a];
                chi[i][a] = hi[3 * bi + a];
            }
            count[i] = ci >= 0 ? range[ci].y : 1;
            inner[i] = ci >= 0 && count[i] > 3;
        }
        float p[3], ph[3];
        for (int a = 0; a < 3; ++a) {
            p[a] = lo[3 * (size_t)b + a];
            ph[a] = hi[3 * (size_t)b + a];
        }
        // slots: greedy assignment of the smallest projection onto the slot's octant direction
        float pc[3];
        for (int a = 0; a < 3; ++a) pc[a] = 0.5f * (p[a] + ph[a]);
        int slot_child[8];
        for (int sl = 0; sl < 8; ++sl) slot_child[sl] = -1;
        unsigned int used_slots = 0, used_children = 0;
        for (int it = 0; it < nc; ++it) {
            float bc = 0.0f;
            int bi = -1, bs = -1;
            for (int i = 0; i < nc; ++i) {
                if (used_children & (1u << i)) continue;
                const float ox = 0.5f * (clo[i][0] + chi[i][0]) - pc[0];
                const float oy = 0.5f * (clo[i][1] + chi[i][1]) - pc[1];
                const float oz = 0.5f * (clo[i][2] + chi[i][2]) - pc[2];
                for (int sl = 0; sl < 8; ++sl) {
                    if (used_slots & (1u << sl)) continue;
                    const float cost = ((sl & 1) ? -ox : ox) + ((sl & 2) ? -oy : oy) + ((sl & 4) ? -oz : oz);
                    if (bi < 0 || cost < bc) {
                        bc = cost;
                        bi = i;
                        bs = sl;
                    }
                }
            }
            slot_child[bs] = bi;
            used_slots |= 1u << bs;
            used_children |= 1u << bi;
        }
        // allocation: child nodes and leaf triangles, each block consecutive
        int n_inner = 0, n_tri = 0;
        for (int i = 0; i < nc; ++i) {
            if (inner[i]) ++n_inner;
            else n_tri += count[i];
        }
        const unsigned int node_base = n_inner ? atomicAdd(alloc, (unsigned int)n_inner) : 0u;
        const unsigned int tri_base = n_tri ? atomicAdd(alloc + 1, (unsigned int)n_tri) : 0u;
        // quantisation
        int e[3];
        float inv_step[3];
        for (int a = 0; a < 3; ++a) {
            e[a] = quant_exp(p[a], ph[a]);
            inv_step[a] = __int_as_float((127 - e[a]) << 23);
        }
        uint32_t meta[2] = {0u, 0u}, q[6][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}};
        uint32_t imask = 0;
        int rank = 0, offset = 0;
        for (int sl = 0; sl < 8; ++sl) {
            const int i = slot_child[sl];
            if (i < 0) continue;
            uint32_t m;
            if (inner[i]) {
                m = 0x80u;
                imask |= 1u << sl;
                const unsigned int slot_k = atomicAdd(nout, 1u);
                qout[slot_k] = make_int2(c[i], (int)(node_base + (unsigned int)rank));
                ++rank;
            } else {
                // the leaves of the (at most three-triangle) subtree, in left-to-right order: a
                // clustering tree's subtree need not cover consecutive leaf positions
                int leaf[3], nl = 0, stk[4], sp = 0;
                stk[sp++] = c[i];
                while (sp > 0 && nl < 3) {
                    const int x = stk[--sp];
                    if (x < 0) {
                        leaf[nl++] = ~x;
                    } else if (sp < 3) {
                        stk[sp++] = right[x];
                        stk[sp++] = left[x];
                    }
                }
                m = ((uint32_t)nl << 5) | (uint32_t)offset;
                for (int t = 0; t < nl; ++t) {
                    const size_t src = MR_TRI_STRIDE * (size_t)leaf[t], dst = 3 * ((size_t)tri_base + offset + t);
                    wtri[dst] = ptri[src];
                    wtri[dst + 1] = ptri[src + 1];
                    wtri[dst + 2] = ptri[src + 2];
                }
                offset += nl;
            }
            meta[sl >> 2] |= m << (8 * (sl & 3));
            for (int a = 0; a < 3; ++a) {
                const float ql = floorf(__fsub_rd(clo[i][a], p[a]) * inv_step[a]) - 1.0f;
                const float qh = ceilf(__fsub_ru(chi[i][a], p[a]) * inv_step[a]) + 1.0f;
                const uint32_t bl = (uint32_t)fminf(fmaxf(ql, 0.0f), 255.0f);
                const uint32_t bh = (uint32_t)fminf(fmaxf(qh, 0.0f), 255.0f);
                q[a][sl >> 2] |= bl << (8 * (sl & 3));
                q[3 + a][sl >> 2] |= bh << (8 * (sl & 3));
            }
        }
        uint4* dst = wnodes + 5 * (size_t)w;
        dst[0] = make_uint4(__float_as_uint(p[0]), __float_as_uint(p[1]), __float_as_uint(p[2]),
                            (uint32_t)(e[0] + 127) | ((uint32_t)(e[1] + 127) << 8) | ((uint32_t)(e[2] + 127) << 16) |
                                (imask << 24));
        dst[1] = make_uint4(node_base, tri_base, meta[0], meta[1]);
        dst[2] = make_uint4(q[0][0], q[0][1], q[1][0], q[1][1]);
        dst[3] = make_uint4(q[2][0], q[2][1], q[3][0], q[3][1]);
        dst[4] = make_uint4(q[4][0], q[4][1], q[5][0], q[5][1]);
    }
}

int grid_cap_w(int n, int block, int cap) { return std::max(1, std::min((n + block - 1) / block, cap)); }

}  // namespace

static mirres_status wide_alloc(mirres_scene* s)
{
    if (s->wnodes) return MIRRES_OK;
    const size_t F = (size_t)std::max(s->desc.n_tris, 1);
    cudaError_t e = cudaMalloc((void**)&s->wnodes, sizeof(uint4) * 5 * F);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->wtri, sizeof(float4) * 3 * F);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->wqueue, sizeof(int2) * 2 * F);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->wcnt, sizeof(unsigned int) * (3 + MR_WIDE_LEVELS));
    if (e != cudaSuccess) {
        cudaGetLastError();
        mr_wide_free(s);
        mr_set_error(std::string("device allocation failed: ") + cudaGetErrorString(e));
        return MIRRES_ERR_OOM;
    }
    return MIRRES_OK;
}

void mr_wide_free(mirres_scene* s)
{
    void* ptrs[] = {s->wnodes, s->wtri, s->wqueue, s->wcnt};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    s->wnodes = nullptr;
    s->wtri = nullptr;
    s->wqueue = nullptr;
    s->wcnt = nullptr;
}

// Collapse the binary tree (left / right / range / boxes of the last build or refit) into the
// wide tree: MR_WIDE_LEVELS launches, each over the queue the previous one filled (the binary
// tree is at most 63 deep, and every wide level consumes at least one binary level, so the
// last launches find empty queues). Asynchronous; a scene of one triangle needs no tree.
mirres_status mr_wide_build(mirres_scene* s, cudaStream_t st)
{
    const int F = s->desc.n_tris;
    if (F < 2) return MIRRES_OK;
    if (s->wnodes == nullptr) {
        const mirres_status a = wide_alloc(s);
        if (a != MIRRES_OK) return a;
    }
    int dev = 0, sms = 1;
    MR_CUDA(cudaGetDevice(&dev));
    MR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MR_CUDA(cudaMemsetAsync(s->wcnt, 0, sizeof(unsigned int) * (3 + MR_WIDE_LEVELS), st));
    k_wide_init<<<1, 32, 0, st>>>(s->wqueue, s->wcnt);
    const int grid = grid_cap_w(F / 4 + 1, kBlock, sms * 16);
    int2* q[2] = {s->wqueue, s->wqueue + (size_t)F};
    for (int lvl = 0; lvl < MR_WIDE_LEVELS; ++lvl) {
        k_wide_level<<<grid, kBlock, 0, st>>>(s->left, s->right, s->range, s->lo, s->hi, s->ptri, F, q[lvl & 1],
                                              s->wcnt + 2 + lvl, q[(lvl + 1) & 1], s->wcnt + 3 + lvl, s->wnodes,
                                              s->wtri, s->wcnt);
    }
    MR_CUDA(cudaGetLastError());
    return MIRRES_OK;
}
