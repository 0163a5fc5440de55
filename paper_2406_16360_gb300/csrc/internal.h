// internal.h -- host-side declarations shared by the translation units of libmirres.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/mirres.h"
#include "device.cuh"

// error handling: a thread-local message behind mirres_last_error()
void mr_set_error(const std::string& msg);
mirres_status mr_cuda_status(cudaError_t e, const char* what);
#define MR_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e__ = (call);                                                      \
        if (e__ != cudaSuccess) return mr_cuda_status(e__, #call);                     \
    } while (0)

// device workspace owned by a context (grow-only)
struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
};

enum { CNT_PRIMARY = 0, CNT_CONT, CNT_SHADOW, CNT_SAMPLES, CNT_DIFF, CNT_CAND, CNT_LAUNCH, CNT_ERROR,
       // traversal work of the batched wavefront: box tests and triangle tests of closest-hit
       // rays, then of shadow rays
       CNT_CBOX, CNT_CTRI, CNT_SBOX, CNT_STRI, CNT_N };

struct mirres_context {
    int device = 0;
    int sm_count = 0;
    Workspace ws;
    unsigned long long* counters = nullptr;  // device [CNT_N]
    unsigned int* queue_cnt = nullptr;       // device scratch counters [64]
    cudaStream_t last_stream = nullptr;
    unsigned long long host_launches = 0;
    int tuned_variant = -1;     // persistent-kernel launch shape chosen by mirres_autotune
    unsigned int tuned_chunk = 256;
    // batched wavefront: the captured forward and the arguments it was captured for
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    unsigned char graph_key[192] = {};
    mirres_wave_shape wave_shape = {25, {256, 256, 256, 256}, {8, 8, 8, 8}, 1};  // batched wavefront launch shape
    cudaStream_t branch_stream[4] = {};  // [1..3]: the streams of wave chains 1..3 during capture
    cudaEvent_t branch_event[4] = {};    // [0]: fork, [1..3]: join of chains 1..3
    unsigned long long graph_launches = 0;  // kernel launches inside the graph
    cudaEvent_t* stage_events = nullptr;     // [n_stage_events]: (start, end) pairs per stage launch
    int n_stage_events = 0;
    int stage_pairs = 0;                     // pairs recorded by the current graph
    int* stage_kind = nullptr;               // [n_stage_events / 2]: bits 0-3 the stage (0 closest, 1 shade,
                                             // 2 shadow, 3 raygen), above them the bounce + 1
};

struct mirres_scene {
    mirres_context* ctx = nullptr;
    mirres_scene_desc desc{};
    bool built = false;
    // LBVH
    uint64_t* keys = nullptr;        // [F]
    int32_t* perm = nullptr;         // [F] leaf position -> triangle
    int32_t* left = nullptr;         // [F-1]
    int32_t* right = nullptr;        // [F-1]
    int32_t* parent = nullptr;       // [2F-1]
    float* lo = nullptr;             // [2F-1][3]
    float* hi = nullptr;             // [2F-1][3]
    int32_t* flags = nullptr;        // [F-1] bottom-up arrival counters
    float4* nodes = nullptr;         // [F-1][4] by internal node id (the builders' layout)
    float4* dnodes = nullptr;        // [F-1][4] the same nodes in depth-first preorder (traversal)
    int32_t* dfs = nullptr;          // [F-1] internal node id -> its position in dnodes
    float4* ptri = nullptr;          // [F][3]
    int32_t* leaf_of = nullptr;      // [F]
    int2* range = nullptr;           // [F-1] (first leaf position, leaf count) under each internal node
    // the 8-wide BVH the traversal runs (collapsed from the binary tree after every build / refit)
    uint4* wnodes = nullptr;         // [F][5] 80-byte nodes with quantised child boxes
    float4* wtri = nullptr;          // [F][3] packed triangles in the wide leaves' order
    int2* wqueue = nullptr;          // [2][F] collapse work queues (binary node, wide node)
    unsigned int* wcnt = nullptr;    // [2 + MR_WIDE_LEVELS + 1] allocation counters, queue lengths
    float* cent = nullptr;           // [3][F] centroids (build scratch)
    uint32_t* codes[2] = {nullptr, nullptr};
    int32_t* vals[2] = {nullptr, nullptr};
    uint32_t* hist = nullptr;        // radix histograms
    unsigned int* bounds = nullptr;  // [12] ordered-uint bounds: centroid lo/hi, vertex lo/hi
    float* tmin = nullptr;           // [1]
    int32_t* bad = nullptr;          // [1] invalid index flag
    // shading normals: MIRRES_NORMALS_FACE or MIRRES_NORMALS_INTERPOLATED (area-weighted vertex
    // normals, recomputed by every build and refit)
    int32_t normals = 0;
    float* vacc = nullptr;   // [V][3] sum of the incident faces' e1 x e2
    float4* vnrm = nullptr;  // [V] vacc normalised
    float* gvn = nullptr;    // [V][3] adjoint accumulator of d loss / d vertex normal
    // hierarchy builder: MIRRES_BVH_LBVH (Karras) or MIRRES_BVH_PLOC (clustering); PLOC scratch
    int32_t builder = 0;
    // the tree the traversal runs: MIRRES_TRAVERSAL_BINARY (default) or MIRRES_TRAVERSAL_WIDE
    // (the 8-wide BVH, collapsed after every build and refit)
    int32_t traversal = 0;
    float4* ploc_box = nullptr;      // [2][2][F] cluster boxes (lo, hi), ping-pong
    int32_t* ploc_node = nullptr;    // [2][F] cluster node ids, ping-pong
    int32_t* ploc_nn = nullptr;      // [F] nearest neighbour of each cluster
    uint2* ploc_part = nullptr;      // [ceil(F / 1024)] per-block (kept, merged) counts, then offsets
    int32_t* ploc_state = nullptr;   // [4]: cluster count and next free node id, by iteration parity
    // env tables
    double* env_w = nullptr;         // [eh][ew]
    double* env_rowsum = nullptr;    // [eh]
    double* env_total = nullptr;     // [1]
    int32_t* env_ok = nullptr;       // [1]
    uint32_t* env_marg = nullptr;    // [eh+1]
    uint32_t* env_cond = nullptr;    // [eh][ew+1]
    float4* env_texel = nullptr;     // [eh][ew]
    uint32_t* env_gmarg = nullptr;   // [gm+1]
    uint32_t* env_gcond = nullptr;   // [eh][gc+1]
    float4* env_row = nullptr;       // [eh]: (cos, sin of the row centre, RIS weight factor, 0)
    float2* env_col = nullptr;       // [ew]: (cos, sin of the column centre angle)
    int gm_shift = 0, gc_shift = 0, gm = 1, gc = 1;
    // the CDF over all texels (row-major) that the draw inverts: 53-bit thresholds, its guide
    // and the FP64 sums of the rows before each row
    unsigned long long* env_flat = nullptr;  // [eh ew + 1] ceil(cdf 2^53)
    uint32_t* env_gflat = nullptr;           // [gf + 1]
    double* env_rowbase = nullptr;           // [eh]
    int gf = 1, gf_shift = 0;
    // mesh edges for the regularisers (built on first use; the topology is fixed per scene)
    int2* edges = nullptr;              // [<= 3F] unique undirected edges (a < b)
    float* inv_deg = nullptr;           // [V] 1 / neighbour count (0 for isolated vertices)
    unsigned int* n_edges = nullptr;    // [1] device count
    unsigned int* deg = nullptr;        // [V] neighbour counts (build scratch)
    unsigned long long* ehash = nullptr;  // open-addressing table of edge keys (build scratch)
};

SceneDev mr_scene_dev(const mirres_scene* s);

// bvh.cu
mirres_status mr_bvh_alloc(mirres_scene* s);
void mr_bvh_free(mirres_scene* s);
mirres_status mr_bvh_build(mirres_scene* s, cudaStream_t st);
// checks every triangle index against n_verts (synchronises st); MIRRES_ERR_ARG if one is out of range
mirres_status mr_check_indices(mirres_scene* s, cudaStream_t st);
// interpolated normals: allocate (idempotent), recompute from the current vertices, and the
// adjoint pass taking d loss / d vertex normal to the vertices of every incident face
mirres_status mr_normals_alloc(mirres_scene* s);
mirres_status mr_vertex_normals(mirres_scene* s, cudaStream_t st);
void mr_launch_normals_adjoint(const mirres_scene* s, float* grad_verts, int sms, cudaStream_t st);
mirres_status mr_bvh_refit(mirres_scene* s, cudaStream_t st);
// wbvh.cu: the 8-wide BVH collapsed from the binary tree (allocated on first use)
mirres_status mr_wide_build(mirres_scene* s, cudaStream_t st);
void mr_wide_free(mirres_scene* s);
// regular.cu
mirres_status mr_edges_build(mirres_scene* s, cudaStream_t st);
void mr_edges_free(mirres_scene* s);
// env.cu
mirres_status mr_env_alloc(mirres_scene* s);
void mr_env_free(mirres_scene* s);
mirres_status mr_env_build(mirres_scene* s, cudaStream_t st);
