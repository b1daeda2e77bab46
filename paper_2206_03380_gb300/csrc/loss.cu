// Image-space loss of the optimisation step, fused with the composite and its
// adjoint (App. A "Image Loss" and "Regularizers"; Sec. 4.2 composite):
//   c       = k_d,out * D(c_d) + D(c_s)
//   T(x)    = Gamma(log(max(x, 0) + 1)), Gamma the sRGB transfer function
//   L_image = mean over pixels and channels of |T(c) - T(ref)|
//   L_light = mean over pixels of |Y(T(D(c_d) + D(c_s))) - V(T(ref))|,
//             Y = channel mean, V = channel max
//   L       = L_image + lambda_light * L_light
// One pass over the pixels writes the three input gradients (overwritten) and
// per-block FP64 partial sums; a one-block pass adds the partials in a fixed
// order, so the loss is bitwise repeatable.
#include "internal.h"

namespace mcdi {
namespace {

constexpr int kLossThreads = 256;
constexpr int kLossMaxBlocks = 1024;

// T(x) and dT/dx (0 below zero, where the clamp holds the value); one power serves both:
// Gamma'(y) = (1.055 / 2.4) y^(1/2.4) / y on the power branch
__device__ __forceinline__ float tonemap(float x, float* slope) {
    const float xc = fmaxf(x, 0.0f);
    const float y = log1pf(xc);
    float t, dg;
    if (y <= 0.0031308f) {
        t = 12.92f * y;
        dg = 12.92f;
    } else {
        const float p = powf(y, 1.0f / 2.4f);
        t = 1.055f * p - 0.055f;
        dg = (1.055f / 2.4f) * (p / y);
    }
    *slope = x >= 0.0f ? dg / (xc + 1.0f) : 0.0f;
    return t;
}

__device__ __forceinline__ float sgn(float d) { return d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f); }

__global__ void __launch_bounds__(kLossThreads) image_loss_kernel(
    const float4* __restrict__ kd, const float4* __restrict__ dd, const float4* __restrict__ ds,
    const float4* __restrict__ ref, long long n, float inv_img, float lam_inv_pix, float4* __restrict__ c_out,
    float4* __restrict__ g_kd, float4* __restrict__ g_dd, float4* __restrict__ g_ds, double* __restrict__ partials) {
    pdl_prologue();
    float s_img = 0.0f, s_light = 0.0f;  // a few pixels per thread; blocks reduce in FP64
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float4 k4 = kd[i], a4 = dd[i], b4 = ds[i], r4 = ref[i];
        const float k[3] = {k4.x, k4.y, k4.z}, a[3] = {a4.x, a4.y, a4.z}, b[3] = {b4.x, b4.y, b4.z};
        const float r[3] = {r4.x, r4.y, r4.z};
        float c[3], gc[3], gs[3], tr[3], ts[3], sl_s[3];
        float img = 0.0f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            c[ch] = k[ch] * a[ch] + b[ch];
            float sl_c, sl_r;
            const float tc = tonemap(c[ch], &sl_c);
            tr[ch] = tonemap(r[ch], &sl_r);
            img += fabsf(tc - tr[ch]);
            gc[ch] = sgn(tc - tr[ch]) * sl_c * inv_img;
            ts[ch] = tonemap(a[ch] + b[ch], &sl_s[ch]);
        }
        const float y = (ts[0] + ts[1] + ts[2]) * (1.0f / 3.0f);
        const float v = fmaxf(fmaxf(tr[0], tr[1]), tr[2]);
        const float gy = sgn(y - v) * lam_inv_pix * (1.0f / 3.0f);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) gs[ch] = gy * sl_s[ch];
        s_img += img;
        s_light += fabsf(y - v);
        if (c_out) c_out[i] = make_float4(c[0], c[1], c[2], 0.0f);
        g_kd[i] = make_float4(gc[0] * a[0], gc[1] * a[1], gc[2] * a[2], 0.0f);
        g_dd[i] = make_float4(gc[0] * k[0] + gs[0], gc[1] * k[1] + gs[1], gc[2] * k[2] + gs[2], 0.0f);
        g_ds[i] = make_float4(gc[0] + gs[0], gc[1] + gs[1], gc[2] + gs[2], 0.0f);
    }
    // fixed-order block reduction in FP64
    __shared__ double red[2][kLossThreads];
    red[0][threadIdx.x] = (double)s_img;
    red[1][threadIdx.x] = (double)s_light;
    __syncthreads();
    for (int h = kLossThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            red[0][threadIdx.x] += red[0][threadIdx.x + h];
            red[1][threadIdx.x] += red[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = red[0][0];
        partials[2 * blockIdx.x + 1] = red[1][0];
    }
}

// one block: thread t adds partials t, t + 256, ... in order, then a fixed tree
__global__ void __launch_bounds__(kLossThreads) loss_finish_kernel(const double* __restrict__ partials, int n_blocks,
                                                                   long long n, double lam,
                                                                   double* __restrict__ loss) {
    pdl_prologue();
    __shared__ double red[2][kLossThreads];
    double img = 0.0, light = 0.0;
    for (int b = threadIdx.x; b < n_blocks; b += kLossThreads) {
        img += partials[2 * b];
        light += partials[2 * b + 1];
    }
    red[0][threadIdx.x] = img;
    red[1][threadIdx.x] = light;
    __syncthreads();
    for (int h = kLossThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            red[0][threadIdx.x] += red[0][threadIdx.x + h];
            red[1][threadIdx.x] += red[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double li = red[0][0] / (3.0 * (double)n), ll = red[1][0] / (double)n;
        loss[0] = li + lam * ll;
        loss[1] = li;
        loss[2] = ll;
    }
}

int loss_blocks(long long n) {
    const long long b = (n + kLossThreads - 1) / kLossThreads;
    return (int)(b < kLossMaxBlocks ? b : kLossMaxBlocks);
}

}  // namespace

size_t image_loss_workspace_bytes(long long n) { return (size_t)loss_blocks(n) * 2 * sizeof(double); }

cudaError_t launch_image_loss(const float* kd, const float* dd, const float* ds, const float* ref, long long n,
                              float lambda_light, float* c, double* loss, float* g_kd, float* g_dd, float* g_ds,
                              void* workspace, cudaStream_t s) {
    const int blocks = loss_blocks(n);
    double* partials = static_cast<double*>(workspace);
    launch_k(image_loss_kernel, blocks, kLossThreads, 0, s, reinterpret_cast<const float4*>(kd),
             reinterpret_cast<const float4*>(dd), reinterpret_cast<const float4*>(ds),
             reinterpret_cast<const float4*>(ref), n, (float)(1.0 / (3.0 * (double)n)),
             (float)((double)lambda_light / (double)n), reinterpret_cast<float4*>(c), reinterpret_cast<float4*>(g_kd),
             reinterpret_cast<float4*>(g_dd), reinterpret_cast<float4*>(g_ds), partials);
    launch_k(loss_finish_kernel, 1, kLossThreads, 0, s, partials, blocks, n, (double)lambda_light, loss);
    return cudaGetLastError();
}

}  // namespace mcdi
