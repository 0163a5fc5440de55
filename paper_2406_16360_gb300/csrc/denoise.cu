// denoise.cu -- the edge-avoiding a-trous wavelet denoiser between the rendered image and the
// loss (Appendix A, "Denoiser"), its adjoint, and the G-buffer it stops at.
//
// Level i smooths c_i into c_{i+1}(p) = sum_q h(q - p) w(p, q) c_i(q) / k(p) over the 5 x 5
// B3-spline taps (1, 4, 6, 4, 1) / 16 placed 2^i pixels apart, with
// w(p, q) = exp(-|c_i(p) - c_i(q)|^2 / sigma_rt_i^2 - |n_p - n_q|^2 / sigma_n^2 - |x_p - x_q|^2 / sigma_x^2),
// sigma_rt_i = sigma_rt / 2^i and k(p) = sum_q h w; taps outside the image are left out. The
// adjoint holds the weights fixed: since h w(p, q) is symmetric in p and q, the transpose of a
// level is the same stencil applied to g / k. Every launch covers a stack of images of one size.
#include "render.h"

namespace {

__constant__ float kB3[5] = {1.0f / 16.0f, 4.0f / 16.0f, 6.0f / 16.0f, 4.0f / 16.0f, 1.0f / 16.0f};

// The level kernels read packed float4 images (colour / normal / position in .xyz): one
// 16-byte load per buffer and tap instead of three scalar loads.
__global__ void __launch_bounds__(256) k_eawt_pack(const float* __restrict__ a, float4* __restrict__ out, int64_t npx)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npx; p += (int64_t)gridDim.x * blockDim.x)
        out[p] = make_float4(__ldg(a + 3 * p), __ldg(a + 3 * p + 1), __ldg(a + 3 * p + 2), 0.0f);
}

__device__ __forceinline__ float d2(float4 a, float4 b)
{
    const float x = a.x - b.x, y = a.y - b.y, z = a.z - b.z;
    return x * x + y * y + z * z;
}

__device__ __forceinline__ void store(float4* o4, float* o3, int64_t p, float x, float y, float z)
{
    if (o3) {
        o3[3 * p] = x;
        o3[3 * p + 1] = y;
        o3[3 * p + 2] = z;
    } else {
        o4[p] = make_float4(x, y, z, 0.0f);
    }
}

// The level kernels run over a stack of N images of W x H. A thread takes a strip of EAWT_R
// output pixels of one column spaced `step` rows apart (rows y0 + j step): their 5 x 5 footprints
// overlap in all but the first and last rows, so the strip reads its (EAWT_R + 4) x 5 taps once
// each and applies every tap to the outputs it falls on -- (EAWT_R + 4) 5 / EAWT_R tap reads per
// output instead of 25 (15 for strips of two). Consecutive threads take consecutive columns of the same rows (coalesced
// tap rows). Each output still sums its taps row by row, column by column.
// Measured on 20 views of config 3 (forward + adjoint, 3 levels): strips of 2 at 64 registers
// (4 blocks per SM) 5.29 ms; 4 at 80 (3 blocks, spilling) 5.61; 4 at 128 (2 blocks) 5.59;
// 2 at 2 blocks 6.18; 8 at 1 block 8.97.
#ifndef MR_EAWT_R
#define MR_EAWT_R 2  // outputs per strip
#endif
#ifndef MR_EAWT_MINB
#define MR_EAWT_MINB 4  // resident 256-thread blocks per SM the register cap aims at
#endif
constexpr int EAWT_R = MR_EAWT_R;

struct Strip {
    int img, x, y0;
};

// strip t of the stack: image, column, first row (row block B of EAWT_R step rows, residue ry)
__device__ __forceinline__ Strip strip_of(int64_t t, int W, int step, int64_t per_img)
{
    Strip s;
    s.img = (int)(t / per_img);
    const int64_t r = t - (int64_t)s.img * per_img;
    s.x = (int)(r % W);
    const int64_t sr = r / W;
    s.y0 = (int)(sr / step) * (EAWT_R * step) + (int)(sr % step);
    return s;
}

__device__ __forceinline__ int64_t strips_per_image(int W, int H, int step)
{
    return (int64_t)((H + EAWT_R * step - 1) / (EAWT_R * step)) * step * W;
}

// forward level: cin -> cout (packed, or [N][H][W][3] when out3 is given), and 1 / k
__global__ void __launch_bounds__(256, MR_EAWT_MINB) k_eawt_level(const float4* __restrict__ cin, const float4* __restrict__ nrm,
                                                    const float4* __restrict__ pos, int N, int W, int H, int step,
                                                    float inv_rt2, float inv_n2, float inv_x2, float4* __restrict__ cout,
                                                    float* __restrict__ out3, float* __restrict__ ikout)
{
    const int64_t npx = (int64_t)W * H, per_img = strips_per_image(W, H, step), total = per_img * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const Strip sp = strip_of(t, W, step, per_img);
        if (sp.y0 >= H) continue;
        const int64_t base = (int64_t)sp.img * npx;
        float4 cp[EAWT_R], np_[EAWT_R], xp[EAWT_R];
        float ax[EAWT_R], ay[EAWT_R], az[EAWT_R], k[EAWT_R];
#pragma unroll
        for (int j = 0; j < EAWT_R; ++j) {
            const int y = sp.y0 + j * step;
            const int64_t p = base + (int64_t)min(y, H - 1) * W + sp.x;
            cp[j] = __ldg(cin + p);
            np_[j] = __ldg(nrm + p);
            xp[j] = __ldg(pos + p);
            ax[j] = ay[j] = az[j] = k[j] = 0.f;
        }
#pragma unroll
        for (int m = 0; m < EAWT_R + 4; ++m) {
            const int qy = sp.y0 + (m - 2) * step;
            if (qy < 0 || qy >= H) continue;
#pragma unroll
            for (int b = 0; b < 5; ++b) {
                const int qx = sp.x + (b - 2) * step;
                if (qx < 0 || qx >= W) continue;
                const int64_t q = base + (int64_t)qy * W + qx;
                const float4 cq = __ldg(cin + q), nq = __ldg(nrm + q), xq = __ldg(pos + q);
#pragma unroll
                for (int j = 0; j < EAWT_R; ++j) {
                    const int a = m - j;  // the tap's row in output j's footprint
                    if (a < 0 || a > 4) continue;
                    const float e = d2(cp[j], cq) * inv_rt2 + d2(np_[j], nq) * inv_n2 + d2(xp[j], xq) * inv_x2;
                    const float w = kB3[a] * kB3[b] * __expf(-e);
                    ax[j] += w * cq.x;
                    ay[j] += w * cq.y;
                    az[j] += w * cq.z;
                    k[j] += w;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < EAWT_R; ++j) {
            const int y = sp.y0 + j * step;
            if (y >= H) break;
            const int64_t p = base + (int64_t)y * W + sp.x;
            const float ik = 1.0f / k[j];  // k >= (6/16)^2: the centre tap has weight 1
            store(cout, out3, p, ax[j] * ik, ay[j] * ik, az[j] * ik);
            ikout[p] = ik;
        }
    }
}

// adjoint level: gout(q) = sum over taps of h w(q, q + tap) gin(q + tap) / k(q + tap), the
// weights recomputed from the level's recorded input c, 1 / k read from the record
__global__ void __launch_bounds__(256, MR_EAWT_MINB) k_eawt_level_adjoint(const float4* __restrict__ gin, const float4* __restrict__ c,
                                                            const float* __restrict__ ikin, const float4* __restrict__ nrm,
                                                            const float4* __restrict__ pos, int N, int W, int H, int step,
                                                            float inv_rt2, float inv_n2, float inv_x2,
                                                            float4* __restrict__ gout, float* __restrict__ out3)
{
    const int64_t npx = (int64_t)W * H, per_img = strips_per_image(W, H, step), total = per_img * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const Strip sp = strip_of(t, W, step, per_img);
        if (sp.y0 >= H) continue;
        const int64_t base = (int64_t)sp.img * npx;
        float4 cp[EAWT_R], np_[EAWT_R], xp[EAWT_R];
        float ax[EAWT_R], ay[EAWT_R], az[EAWT_R];
#pragma unroll
        for (int j = 0; j < EAWT_R; ++j) {
            const int y = sp.y0 + j * step;
            const int64_t p = base + (int64_t)min(y, H - 1) * W + sp.x;
            cp[j] = __ldg(c + p);
            np_[j] = __ldg(nrm + p);
            xp[j] = __ldg(pos + p);
            ax[j] = ay[j] = az[j] = 0.f;
        }
#pragma unroll
        for (int m = 0; m < EAWT_R + 4; ++m) {
            const int qy = sp.y0 + (m - 2) * step;
            if (qy < 0 || qy >= H) continue;
#pragma unroll
            for (int b = 0; b < 5; ++b) {
                const int qx = sp.x + (b - 2) * step;
                if (qx < 0 || qx >= W) continue;
                const int64_t q = base + (int64_t)qy * W + qx;
                const float4 cq = __ldg(c + q), nq = __ldg(nrm + q), xq = __ldg(pos + q), g = __ldg(gin + q);
                const float ik = __ldg(ikin + q);
#pragma unroll
                for (int j = 0; j < EAWT_R; ++j) {
                    const int a = m - j;
                    if (a < 0 || a > 4) continue;
                    const float e = d2(cp[j], cq) * inv_rt2 + d2(np_[j], nq) * inv_n2 + d2(xp[j], xq) * inv_x2;
                    const float w = kB3[a] * kB3[b] * __expf(-e) * ik;
                    ax[j] += w * g.x;
                    ay[j] += w * g.y;
                    az[j] += w * g.z;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < EAWT_R; ++j) {
            const int y = sp.y0 + j * step;
            if (y >= H) break;
            store(gout, out3, base + (int64_t)y * W + sp.x, ax[j], ay[j], az[j]);
        }
    }
}

// G-buffer: the primary hit through each pixel centre, face normal turned towards the camera
// and hit position; 0 for both where the ray escapes
__global__ void __launch_bounds__(256) k_gbuffer(SceneDev s, ViewDev v, float* __restrict__ nrm, float* __restrict__ pos)
{
    extern __shared__ __align__(16) uint32_t sstk[];
    const int64_t npx = (int64_t)v.width * v.height;
    const float3 o = f3(v.c2w[3], v.c2w[7], v.c2w[11]);
    const float tmin = *s.tmin_dev;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npx; p += (int64_t)gridDim.x * blockDim.x) {
        const int px = (int)(p % v.width), py = (int)(p / v.width);
        const float3 d = camera_dir(v, px, py, 0.5f, 0.5f);
        Hit h;
        trace<false>(s, o, d, -1, tmin, __int_as_float(0x7f800000), h, sstk + threadIdx.x);
        float3 n = f3(0.f, 0.f, 0.f), x = n;
        if (h.tri >= 0) {
            float3 v0, e1, e2;
            int tchk;
            load_tri(s, __ldg(s.leaf_of + h.tri), v0, e1, e2, tchk);
            n = normalize(cross(e1, e2));
            if (dot(n, d) > 0.0f) n = f3(-n.x, -n.y, -n.z);
            x = f3(o.x + h.t * d.x, o.y + h.t * d.y, o.z + h.t * d.z);
        }
        nrm[3 * p] = n.x;
        nrm[3 * p + 1] = n.y;
        nrm[3 * p + 2] = n.z;
        pos[3 * p] = x.x;
        pos[3 * p + 1] = x.y;
        pos[3 * p + 2] = x.z;
    }
}

unsigned grid_for_pixels(int64_t n, int sms)
{
    const int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

void mr_launch_eawt_pack(const float* a, float4* out, int64_t npx, int sms, cudaStream_t st)
{
    k_eawt_pack<<<grid_for_pixels(npx, sms), 256, 0, st>>>(a, out, npx);
}

static int64_t level_strips(int N, int W, int H, int step)
{
    return (int64_t)N * ((H + EAWT_R * step - 1) / (EAWT_R * step)) * step * W;
}

void mr_launch_eawt_level(const float4* cin, const float4* nrm, const float4* pos, int N, int W, int H, int step,
                          float inv_rt2, float inv_n2, float inv_x2, float4* cout, float* out3, float* ikout, int sms,
                          cudaStream_t st)
{
    k_eawt_level<<<grid_for_pixels(level_strips(N, W, H, step), sms), 256, 0, st>>>(
        cin, nrm, pos, N, W, H, step, inv_rt2, inv_n2, inv_x2, cout, out3, ikout);
}

void mr_launch_eawt_level_adjoint(const float4* gin, const float4* c, const float* ikin, const float4* nrm,
                                  const float4* pos, int N, int W, int H, int step, float inv_rt2, float inv_n2,
                                  float inv_x2, float4* gout, float* out3, int sms, cudaStream_t st)
{
    k_eawt_level_adjoint<<<grid_for_pixels(level_strips(N, W, H, step), sms), 256, 0, st>>>(
        gin, c, ikin, nrm, pos, N, W, H, step, inv_rt2, inv_n2, inv_x2, gout, out3);
}

void mr_launch_gbuffer(const SceneDev& s, const ViewDev& v, float* nrm, float* pos, int sms, cudaStream_t st)
{
    k_gbuffer<<<grid_for_pixels((int64_t)v.width * v.height, sms), 256, sizeof(uint32_t) * MR_SSTACK * 256, st>>>(
        s, v, nrm, pos);
}
