// env.cu -- environment-map importance-sampling tables (the paper's proposal
// q_dir proportional to L_env, drawn from the environment map itself, Sec. 4.1).
//
// Texel weight w = Y(L) sin(theta_row), Y = (r + g + b) / 3 (Appendix A). Per-row conditional
// CDFs and the marginal CDF over rows are FP64 prefix sums (one thread per row, sequential
// over the row, so every sum has a fixed order), converted to uint32 thresholds
// ceil(cdf * 2^24): for a 24-bit uniform u = k 2^-24, cdf <= u exactly when threshold <= k,
// so the search needs no FP64 arithmetic. The texel table packs (r, g, b, P * W * H).
// The draw inverts the CDF over all texels in row-major order, (rows before + texels before in
// the row) / total, as 53-bit thresholds ceil(cdf * 2^53) for a 53-bit uniform made of two
// random words, through a guide with about eight buckets per texel: one short search instead of
// a row search followed by a column search.
#include "internal.h"

namespace {

__device__ __forceinline__ uint32_t threshold(double cdf)
{
    const double x = ceil(cdf * 16777216.0);
    return x <= 0.0 ? 0u : (x >= 16777216.0 ? 16777216u : (uint32_t)x);
}

__global__ void k_env_rows(const float* __restrict__ env, int W, int H, double* __restrict__ w,
                           double* __restrict__ rowsum, uint32_t* __restrict__ cond)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    const double st = sin(3.14159265358979323846 * ((double)r + 0.5) / (double)H);
    double acc = 0.0;
    for (int c = 0; c < W; ++c) {
        const float* p = env + 3 * ((size_t)r * W + c);
        const double y = (((double)p[0] + (double)p[1]) + (double)p[2]) / 3.0 * st;
        w[(size_t)r * W + c] = y;
        acc += y;
    }
    rowsum[r] = acc;
    uint32_t* cr = cond + (size_t)r * (W + 1);
    double run = 0.0;
    for (int c = 0; c <= W; ++c) {
        double v;
        if (acc > 0.0) v = (c == W) ? 1.0 : run / acc;
        else v = (double)c / (double)W;
        cr[c] = threshold(v);
        if (c < W) run += w[(size_t)r * W + c];
    }
}

__global__ void k_env_marg(const double* __restrict__ rowsum, int H, double* total_out, int32_t* ok_out,
                           uint32_t* __restrict__ marg, double* __restrict__ rowbase)
{
    if (threadIdx.x != 0) return;
    double total = 0.0;
    for (int r = 0; r < H; ++r) total += rowsum[r];
    const int ok = total > 0.0;
    double run = 0.0;
    for (int r = 0; r <= H; ++r) {
        double v;
        if (ok) v = (r == H) ? 1.0 : run / total;
        else v = (double)r / (double)H;
        marg[r] = threshold(v);
        if (r < H) {
            rowbase[r] = run;
            run += rowsum[r];
        }
    }
    *total_out = total;
    *ok_out = ok;
}

__device__ __forceinline__ unsigned long long threshold53(double cdf)
{
    const double x = ceil(cdf * 9007199254740992.0);
    return x <= 0.0 ? 0ull : (x >= 9007199254740992.0 ? 9007199254740992ull : (unsigned long long)x);
}

// one thread per row: thresholds of the CDF over all texels, (rows before + texels before in
// the row) / total, each sum in order
__global__ void k_env_flat(const double* __restrict__ w, const double* __restrict__ rowbase,
                           const double* __restrict__ total, int W, int H, unsigned long long* __restrict__ flat)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    const double tot = *total, base = rowbase[r];
    const double n = (double)W * (double)H;
    double within = 0.0;
    for (int c = 0; c < W; ++c) {
        const size_t i = (size_t)r * W + c;
        flat[i] = threshold53(tot > 0.0 ? (base + within) / tot : (double)i / n);
        within += w[i];
    }
    if (r == H - 1) flat[(size_t)W * H] = 9007199254740992ull;
}

// guide of the flat CDF: bucket b answers the search at k = b << shift; entry g is n - 1
__global__ void k_env_flat_guide(const unsigned long long* __restrict__ flat, int n, int g, int shift,
                                 uint32_t* __restrict__ guide)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > g) return;
    if (b == g) {
        guide[b] = (uint32_t)(n - 1);
        return;
    }
    const unsigned long long k = (unsigned long long)b << shift;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (flat[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    guide[b] = (uint32_t)lo;
}

__global__ void k_env_texels(const float* __restrict__ env, const double* __restrict__ w, int W, int H,
                             const double* __restrict__ total, float4* __restrict__ texel)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)W * H) return;
    const double tot = *total;
    const float p = tot > 0.0 ? (float)(w[i] / tot * ((double)W * (double)H)) : 0.0f;
    texel[i] = make_float4(env[3 * i], env[3 * i + 1], env[3 * i + 2], p);
}

// angle tables for drawing directions inside a texel without a full-range sin/cos: the row
// centre theta_r = pi (r + 1/2) / H and the column centre psi_c = 2 pi (c + 1/2) / W - pi, plus
// the per-row RIS weight factor. With q = P W H / (2 pi^2 sin theta) and P = Y(L) sin theta_r /
// total, the candidate weight p_hat / q = Y(f_r cos) sin theta 2 pi^2 total / (W H sin theta_r):
// Y(L) cancels, so a candidate needs no texel fetch.
__global__ void k_env_angles(int W, int H, const double* __restrict__ total, float4* __restrict__ row,
                             float2* __restrict__ col)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double pi = 3.14159265358979323846;
    if (i < H) {
        const double th = pi * ((double)i + 0.5) / (double)H;
        const double st = sin(th), tot = *total;
        const double g = tot > 0.0 ? 2.0 * pi * pi * tot / ((double)W * (double)H * st) : 0.0;
        row[i] = make_float4((float)cos(th), (float)st, (float)g, 0.0f);
    }
    if (i < W) {
        const double ps = 2.0 * pi * ((double)i + 0.5) / (double)W - pi;
        col[i] = make_float2((float)cos(ps), (float)sin(ps));
    }
}

// largest i in [0, n-1] with a[i] <= k
__device__ __forceinline__ uint32_t search_all(const uint32_t* a, int n, uint32_t k)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return (uint32_t)lo;
}

// guide tables: for bucket b of the 24-bit uniform, the search answer at u = b << shift;
// entry g (one past the last bucket) is n - 1
__global__ void k_env_guide(const uint32_t* __restrict__ cdf, int rows, int stride, int n, int g, int shift,
                            uint32_t* __restrict__ guide)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)rows * (g + 1)) return;
    const int row = (int)(i / (size_t)(g + 1)), b = (int)(i % (size_t)(g + 1));
    const uint32_t* a = cdf + (size_t)row * stride;
    guide[i] = (b == g) ? (uint32_t)(n - 1) : search_all(a, n, (uint32_t)b << shift);
}

}  // namespace

static void guide_shape(int n, int& g, int& shift)
{
    int lg = 0;
    while ((1 << lg) < n && lg < 24) ++lg;
    g = 1 << lg;
    shift = 24 - lg;
}

// guide buckets per texel of the flat CDF: with 8 only ~12% of the draws on config 3's env land
// in a bucket that holds a CDF boundary (and so read a threshold), against ~36% with 2; the
// shade stage measured 85.3 / 82.1 / 80.0 / 81.5 / 85.8 ms per 20-view render at 2 / 4 / 8 / 16 / 32
#ifndef MR_GUIDE_PER_TEXEL
#define MR_GUIDE_PER_TEXEL 8
#endif

mirres_status mr_env_alloc(mirres_scene* s)
{
    const size_t W = (size_t)s->desc.env_w, H = (size_t)s->desc.env_h;
    guide_shape((int)H, s->gm, s->gm_shift);
    guide_shape((int)W, s->gc, s->gc_shift);
    {
        // about MR_GUIDE_PER_TEXEL guide buckets per texel over the 53-bit uniform
        int lg = 1;
        while (((size_t)1 << lg) < (size_t)MR_GUIDE_PER_TEXEL * W * H && lg < 30) ++lg;
        s->gf = 1 << lg;
        s->gf_shift = 53 - lg;
    }
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc((void**)&s->env_gmarg, sizeof(uint32_t) * (size_t)(s->gm + 1));
    e = e ? e : cudaMalloc((void**)&s->env_gcond, sizeof(uint32_t) * H * (size_t)(s->gc + 1));
    e = e ? e : cudaMalloc((void**)&s->env_w, sizeof(double) * W * H);
    e = e ? e : cudaMalloc((void**)&s->env_rowsum, sizeof(double) * H);
    e = e ? e : cudaMalloc((void**)&s->env_total, sizeof(double));
    e = e ? e : cudaMalloc((void**)&s->env_ok, sizeof(int32_t));
    e = e ? e : cudaMalloc((void**)&s->env_marg, sizeof(uint32_t) * (H + 1));
    e = e ? e : cudaMalloc((void**)&s->env_cond, sizeof(uint32_t) * H * (W + 1));
    e = e ? e : cudaMalloc((void**)&s->env_texel, sizeof(float4) * W * H);
    e = e ? e : cudaMalloc((void**)&s->env_row, sizeof(float4) * H);
    e = e ? e : cudaMalloc((void**)&s->env_col, sizeof(float2) * W);
    e = e ? e : cudaMalloc((void**)&s->env_flat, sizeof(unsigned long long) * (W * H + 1));
    e = e ? e : cudaMalloc((void**)&s->env_gflat, sizeof(uint32_t) * ((size_t)s->gf + 1));
    e = e ? e : cudaMalloc((void**)&s->env_rowbase, sizeof(double) * H);
    if (e != cudaSuccess) {
        cudaGetLastError();
        mr_set_error(std::string("env table allocation failed: ") + cudaGetErrorString(e));
        return MIRRES_ERR_OOM;
    }
    return MIRRES_OK;
}

void mr_env_free(mirres_scene* s)
{
    void* ptrs[] = {s->env_w,    s->env_rowsum, s->env_total, s->env_ok,   s->env_marg,
                    s->env_cond, s->env_texel,  s->env_gmarg, s->env_gcond, s->env_row, s->env_col,
                    s->env_flat, s->env_gflat,  s->env_rowbase};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

mirres_status mr_env_build(mirres_scene* s, cudaStream_t st)
{
    const int W = s->desc.env_w, H = s->desc.env_h;
    k_env_rows<<<(H + 63) / 64, 64, 0, st>>>(s->desc.env, W, H, s->env_w, s->env_rowsum, s->env_cond);
    k_env_marg<<<1, 32, 0, st>>>(s->env_rowsum, H, s->env_total, s->env_ok, s->env_marg, s->env_rowbase);
    k_env_flat<<<(H + 63) / 64, 64, 0, st>>>(s->env_w, s->env_rowbase, s->env_total, W, H, s->env_flat);
    k_env_flat_guide<<<(unsigned)((s->gf + 1 + 255) / 256), 256, 0, st>>>(s->env_flat, W * H + 1, s->gf,
                                                                         s->gf_shift, s->env_gflat);
    const size_t n = (size_t)W * H;
    k_env_texels<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->desc.env, s->env_w, W, H, s->env_total,
                                                             s->env_texel);
    const int na = W > H ? W : H;
    k_env_angles<<<(na + 127) / 128, 128, 0, st>>>(W, H, s->env_total, s->env_row, s->env_col);
    k_env_guide<<<(unsigned)((s->gm + 1 + 255) / 256), 256, 0, st>>>(s->env_marg, 1, H + 1, H, s->gm, s->gm_shift,
                                                                     s->env_gmarg);
    const size_t ng = (size_t)H * (s->gc + 1);
    k_env_guide<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(s->env_cond, H, W + 1, W, s->gc, s->gc_shift,
                                                              s->env_gcond);
    MR_CUDA(cudaGetLastError());
    return MIRRES_OK;
}
