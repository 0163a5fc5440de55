// denoise.cu -- the edge-avoiding a-trous wavelet denoiser between the rendered image and the
// loss (Appendix A, "Denoiser"), its adjoint, and the G-buffer it stops at.
//
// Level i smooths c_i into c_{i+1}(p) = sum_q h(q - p) w(p, q) c_i(q) / k(p) over the 5 x 5
// B3-spline taps (1, 4, 6, 4, 1) / 16 placed 2^i pixels apart, with
// w(p, q) = exp(-|c_i(p) - c_i(q)|^2 / sigma_rt_i^2 - |n_p - n_q|^2 / sigma_n^2 - |x_p - x_q|^2 / sigma_x^2),
// sigma_rt_i = sigma_rt / 2^i and k(p) = sum_q h w; taps outside the image are left out. The
// adjoint holds the weights fixed: since h w(p, q) is symmetric in p and q, the transpose of a
// level is the same stencil applied to g / k. One thread per pixel; the taps are L1/L2 hits.
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

// forward level: cin -> cout (packed, or [H][W][3] when out3 is given), and the normaliser k
__global__ void __launch_bounds__(256) k_eawt_level(const float4* __restrict__ cin, const float4* __restrict__ nrm,
                                                    const float4* __restrict__ pos, int W, int H, int step,
                                                    float inv_rt2, float inv_n2, float inv_x2, float4* __restrict__ cout,
                                                    float* __restrict__ out3, float* __restrict__ kout)
{
    const int64_t npx = (int64_t)W * H;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npx; p += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(p / W), x = (int)(p % W);
        const float4 cp = __ldg(cin + p), np_ = __ldg(nrm + p), xp = __ldg(pos + p);
        float ax = 0.f, ay = 0.f, az = 0.f, k = 0.f;
        for (int a = 0; a < 5; ++a) {
            const int qy = y + (a - 2) * step;
            if (qy < 0 || qy >= H) continue;
#pragma unroll
            for (int b = 0; b < 5; ++b) {
                const int qx = x + (b - 2) * step;
                if (qx < 0 || qx >= W) continue;
                const int64_t q = (int64_t)qy * W + qx;
                const float4 cq = __ldg(cin + q);
                const float e = d2(cp, cq) * inv_rt2 + d2(np_, __ldg(nrm + q)) * inv_n2 + d2(xp, __ldg(pos + q)) * inv_x2;
                const float w = kB3[a] * kB3[b] * __expf(-e);
                ax += w * cq.x;
                ay += w * cq.y;
                az += w * cq.z;
                k += w;
            }
        }
        const float ik = 1.0f / k;  // k >= (6/16)^2: the centre tap has weight 1
        store(cout, out3, p, ax * ik, ay * ik, az * ik);
        kout[p] = k;
    }
}

// adjoint level: gout(q) = sum over taps of h w(q, q + tap) gin(q + tap) / k(q + tap), the
// weights recomputed from the level's recorded input c
__global__ void __launch_bounds__(256) k_eawt_level_adjoint(const float4* __restrict__ gin, const float4* __restrict__ c,
                                                            const float* __restrict__ kin, const float4* __restrict__ nrm,
                                                            const float4* __restrict__ pos, int W, int H, int step,
                                                            float inv_rt2, float inv_n2, float inv_x2,
                                                            float4* __restrict__ gout, float* __restrict__ out3)
{
    const int64_t npx = (int64_t)W * H;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npx; p += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(p / W), x = (int)(p % W);
        const float4 cp = __ldg(c + p), np_ = __ldg(nrm + p), xp = __ldg(pos + p);
        float ax = 0.f, ay = 0.f, az = 0.f;
        for (int a = 0; a < 5; ++a) {
            const int qy = y + (a - 2) * step;
            if (qy < 0 || qy >= H) continue;
#pragma unroll
            for (int b = 0; b < 5; ++b) {
                const int qx = x + (b - 2) * step;
                if (qx < 0 || qx >= W) continue;
                const int64_t q = (int64_t)qy * W + qx;
                const float e = d2(cp, __ldg(c + q)) * inv_rt2 + d2(np_, __ldg(nrm + q)) * inv_n2 + d2(xp, __ldg(pos + q)) * inv_x2;
                const float w = kB3[a] * kB3[b] * __expf(-e) / __ldg(kin + q);
                const float4 g = __ldg(gin + q);
                ax += w * g.x;
                ay += w * g.y;
                az += w * g.z;
            }
        }
        store(gout, out3, p, ax, ay, az);
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

void mr_launch_eawt_level(const float4* cin, const float4* nrm, const float4* pos, int W, int H, int step, float inv_rt2,
                          float inv_n2, float inv_x2, float4* cout, float* out3, float* kout, int sms, cudaStream_t st)
{
    k_eawt_level<<<grid_for_pixels((int64_t)W * H, sms), 256, 0, st>>>(cin, nrm, pos, W, H, step, inv_rt2, inv_n2,
                                                                      inv_x2, cout, out3, kout);
}

void mr_launch_eawt_level_adjoint(const float4* gin, const float4* c, const float* kin, const float4* nrm,
                                  const float4* pos, int W, int H, int step, float inv_rt2, float inv_n2, float inv_x2,
                                  float4* gout, float* out3, int sms, cudaStream_t st)
{
    k_eawt_level_adjoint<<<grid_for_pixels((int64_t)W * H, sms), 256, 0, st>>>(gin, c, kin, nrm, pos, W, H, step,
                                                                              inv_rt2, inv_n2, inv_x2, gout, out3);
}

void mr_launch_gbuffer(const SceneDev& s, const ViewDev& v, float* nrm, float* pos, int sms, cudaStream_t st)
{
    k_gbuffer<<<grid_for_pixels((int64_t)v.width * v.height, sms), 256, sizeof(uint32_t) * MR_SSTACK * 256, st>>>(
        s, v, nrm, pos);
}
