// Cross-bilateral denoiser (App. B "Bilateral Denoiser": the spatial part of
// SVGF, evaluated densely over the footprint, gradients to the colours only):
//   c_hat(p) = sum_q c(q) w(p, q) / W(p),   W(p) = sum_q w(p, q)
//   w(p, q)  = exp(-|p - q|^2 / (2 sigma^2))
//            * exp(-|z(p) - z(q)| / (sigma_z |grad z(p) . (p - q)| + 1e-3 z(p)))
//            * max(0, n(p) . n(q))^128,  sigma_z = 1
// z is camera-space depth, grad z the central difference over covered
// neighbours (one-sided at borders and coverage edges), n the normalised
// G-buffer normal; uncovered pixels pass through and are never neighbours.
// Forward: one CTA per 16 x 16 tile of one view; depth, normal and the colours
// of all images of that view over the tile plus its halo are staged in shared
// memory, and one pass over the footprint accumulates every image with the
// same weights.  Backward: the transpose as a gather, g(q) = sum_p g(p) w(p, q)
// / W(p) over the footprint of q, with W saved by the forward (no atomics, so
// the gradient is deterministic).
#include "internal.h"

namespace mcdi {
namespace {

constexpr int kTile = 16;
constexpr int kMaxImgPerView = 4;
constexpr float kSigmaZ = 1.0f;
constexpr float kEpsRel = 1e-3f;

struct Guide {  // one staged pixel
    float z;    // camera-space depth, < 0: uncovered or outside the image
    float nx, ny, nz;
};

__device__ __forceinline__ Guide load_guide(const float4* pos, const float4* nrm, const mcdi_camera& C, int H, int W,
                                            size_t base, int x, int y) {
    Guide g{-1.0f, 0.0f, 0.0f, 0.0f};
    if (x < 0 || y < 0 || x >= W || y >= H) return g;
    const float4 p = pos[base + (size_t)y * W + x];
    if (!(p.w > 0.0f)) return g;
    const float4 n = nrm[base + (size_t)y * W + x];
    const float l = sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
    const float inv = l > 0.0f ? 1.0f / l : 0.0f;
    g.z = (p.x - C.origin[0]) * C.forward[0] + (p.y - C.origin[1]) * C.forward[1] + (p.z - C.origin[2]) * C.forward[2];
    g.nx = n.x * inv;
    g.ny = n.y * inv;
    g.nz = n.z * inv;
    return g;
}

// central difference over covered neighbours, one-sided where one is missing
__device__ __forceinline__ float depth_slope(float zm, float z0, float zp) {
    const bool cm = zm >= 0.0f, cp = zp >= 0.0f;
    return cm && cp ? 0.5f * (zp - zm) : (cp ? zp - z0 : (cm ? z0 - zm : 0.0f));
}

__device__ __forceinline__ float pow128(float d) {
    float v = fmaxf(d, 0.0f);
#pragma unroll
    for (int i = 0; i < 7; ++i) v *= v;
    return v;
}

struct Center {  // the pixel p of a weight w(p, q)
    float z, gx, gy, eps, nx, ny, nz;
};

__device__ __forceinline__ float bilateral_weight(const Center& p, const Guide& q, int dx, int dy, float inv2s2) {
    const float ws = expf(-(float)(dx * dx + dy * dy) * inv2s2);
    const float pred = fabsf(p.gx * (float)dx + p.gy * (float)dy);
    const float wz = expf(-fabsf(p.z - q.z) / (kSigmaZ * pred + p.eps));
    const float wn = pow128(p.nx * q.nx + p.ny * q.ny + p.nz * q.nz);
    return ws * wz * wn;
}

__device__ __forceinline__ Center center_of(const Guide* s, int sw, int sx, int sy) {
    const Guide g = s[sy * sw + sx];
    Center c;
    c.z = g.z;
    c.gx = depth_slope(s[sy * sw + sx - 1].z, g.z, s[sy * sw + sx + 1].z);
    c.gy = depth_slope(s[(sy - 1) * sw + sx].z, g.z, s[(sy + 1) * sw + sx].z);
    c.eps = kEpsRel * fabsf(g.z);
    c.nx = g.nx;
    c.ny = g.ny;
    c.nz = g.nz;
    return c;
}

// Forward.  Shared memory: guides over tile + halo R + 1 (the slopes of the
// tile's pixels need one more ring), colours over tile + halo R.
__global__ void __launch_bounds__(kTile* kTile) bilateral_fwd_kernel(const float4* __restrict__ pos,
                                                                     const float4* __restrict__ nrm,
                                                                     const mcdi_camera* __restrict__ cams, int N, int H,
                                                                     int W, int K, const float4* __restrict__ c_in,
                                                                     float inv2s2, int R, float4* __restrict__ c_out,
                                                                     float* __restrict__ wsum) {
    pdl_prologue();
    extern __shared__ float4 smem[];
    const int view = blockIdx.z;
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const int gw = kTile + 2 * (R + 1), cw = kTile + 2 * R;
    Guide* sg = reinterpret_cast<Guide*>(smem);
    float4* sc = smem + gw * gw;  // K planes of cw * cw colours
    const mcdi_camera C = cams[view];
    const size_t plane = (size_t)H * W;
    const size_t gbase = (size_t)view * plane;
    for (int i = threadIdx.x; i < gw * gw; i += blockDim.x) {
        const int sx = i % gw, sy = i / gw;
        sg[i] = load_guide(pos, nrm, C, H, W, gbase, x0 + sx - (R + 1), y0 + sy - (R + 1));
    }
    for (int k = 0; k < K; ++k) {
        const size_t cbase = (size_t)(view + k * N) * plane;
        for (int i = threadIdx.x; i < cw * cw; i += blockDim.x) {
            const int x = x0 + i % cw - R, y = y0 + i / cw - R;
            sc[k * cw * cw + i] =
                (x >= 0 && y >= 0 && x < W && y < H) ? c_in[cbase + (size_t)y * W + x] : make_float4(0, 0, 0, 0);
        }
    }
    __syncthreads();
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= W || y >= H) return;
    const size_t pix = (size_t)y * W + x;
    const Center p = center_of(sg, gw, tx + R + 1, ty + R + 1);
    if (p.z < 0.0f) {  // uncovered: pass through
        for (int k = 0; k < K; ++k) {
            const float4 c = sc[k * cw * cw + (ty + R) * cw + tx + R];
            c_out[(size_t)(view + k * N) * plane + pix] = make_float4(c.x, c.y, c.z, 0.0f);
        }
        wsum[gbase + pix] = 0.0f;
        return;
    }
    float acc[kMaxImgPerView][3] = {};
    float wt = 0.0f;
    for (int dy = -R; dy <= R; ++dy) {
        for (int dx = -R; dx <= R; ++dx) {
            const Guide q = sg[(ty + R + 1 + dy) * gw + tx + R + 1 + dx];
            if (q.z < 0.0f) continue;
            const float w = bilateral_weight(p, q, dx, dy, inv2s2);
            wt += w;
            const int ci = (ty + R + dy) * cw + tx + R + dx;
#pragma unroll
            for (int k = 0; k < kMaxImgPerView; ++k) {
                if (k >= K) break;
                const float4 c = sc[k * cw * cw + ci];
                acc[k][0] += w * c.x;
                acc[k][1] += w * c.y;
                acc[k][2] += w * c.z;
            }
        }
    }
    const float inv = 1.0f / wt;
    for (int k = 0; k < K; ++k)
        c_out[(size_t)(view + k * N) * plane + pix] = make_float4(acc[k][0] * inv, acc[k][1] * inv, acc[k][2] * inv, 0.0f);
    wsum[gbase + pix] = wt;
}

// Backward (gather).  Shared memory: guides over tile + halo R + 1, the
// upstream gradients divided by W(p) over tile + halo R.
__global__ void __launch_bounds__(kTile* kTile) bilateral_bwd_kernel(const float4* __restrict__ pos,
                                                                     const float4* __restrict__ nrm,
                                                                     const mcdi_camera* __restrict__ cams, int N, int H,
                                                                     int W, int K, const float* __restrict__ wsum,
                                                                     const float4* __restrict__ g_out, float inv2s2,
                                                                     int R, float4* __restrict__ g_in) {
    pdl_prologue();
    extern __shared__ float4 smem[];
    const int view = blockIdx.z;
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const int gw = kTile + 2 * (R + 1), cw = kTile + 2 * R;
    Guide* sg = reinterpret_cast<Guide*>(smem);
    float4* sgw = smem + gw * gw;  // K planes of g / W over cw * cw
    const mcdi_camera C = cams[view];
    const size_t plane = (size_t)H * W;
    const size_t gbase = (size_t)view * plane;
    for (int i = threadIdx.x; i < gw * gw; i += blockDim.x) {
        const int sx = i % gw, sy = i / gw;
        sg[i] = load_guide(pos, nrm, C, H, W, gbase, x0 + sx - (R + 1), y0 + sy - (R + 1));
    }
    for (int k = 0; k < K; ++k) {
        const size_t cbase = (size_t)(view + k * N) * plane;
        for (int i = threadIdx.x; i < cw * cw; i += blockDim.x) {
            const int x = x0 + i % cw - R, y = y0 + i / cw - R;
            float4 v = make_float4(0, 0, 0, 0);
            if (x >= 0 && y >= 0 && x < W && y < H) {
                const float w = wsum[gbase + (size_t)y * W + x];
                if (w > 0.0f) {
                    const float4 g = g_out[cbase + (size_t)y * W + x];
                    const float iw = 1.0f / w;
                    v = make_float4(g.x * iw, g.y * iw, g.z * iw, 0.0f);
                }
            }
            sgw[k * cw * cw + i] = v;
        }
    }
    __syncthreads();
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= W || y >= H) return;
    const size_t pix = (size_t)y * W + x;
    const Guide q = sg[(ty + R + 1) * gw + tx + R + 1];
    if (q.z < 0.0f) {  // uncovered: pass through
        for (int k = 0; k < K; ++k) {
            const size_t i = (size_t)(view + k * N) * plane + pix;
            const float4 g = g_out[i];
            g_in[i] = make_float4(g.x, g.y, g.z, 0.0f);
        }
        return;
    }
    float acc[kMaxImgPerView][3] = {};
    // p = q + (ox, oy); the offset of q seen from p is (-ox, -oy)
    for (int oy = -R; oy <= R; ++oy) {
        for (int ox = -R; ox <= R; ++ox) {
            const int sx = tx + R + 1 + ox, sy = ty + R + 1 + oy;
            if (sg[sy * gw + sx].z < 0.0f) continue;
            const Center p = center_of(sg, gw, sx, sy);
            const float w = bilateral_weight(p, q, -ox, -oy, inv2s2);
            const int ci = (ty + R + oy) * cw + tx + R + ox;
#pragma unroll
            for (int k = 0; k < kMaxImgPerView; ++k) {
                if (k >= K) break;
                const float4 g = sgw[k * cw * cw + ci];
                acc[k][0] += w * g.x;
                acc[k][1] += w * g.y;
                acc[k][2] += w * g.z;
            }
        }
    }
    for (int k = 0; k < K; ++k)
        g_in[(size_t)(view + k * N) * plane + pix] = make_float4(acc[k][0], acc[k][1], acc[k][2], 0.0f);
}

size_t bilateral_smem(int R, int K) {
    const int gw = kTile + 2 * (R + 1), cw = kTile + 2 * R;
    return (size_t)gw * gw * sizeof(Guide) + (size_t)K * cw * cw * sizeof(float4);
}

}  // namespace

int bilateral_max_images_per_view() { return kMaxImgPerView; }

cudaError_t launch_bilateral(bool backward, const float* gb_pos, const float* gb_nrm, const mcdi_camera* cams, int N,
                             int H, int W, int n_img, const float* in, float sigma, int R, const float* wsum_in,
                             float* out, float* wsum_out, cudaStream_t s) {
    const int K = n_img / N;
    const size_t smem = bilateral_smem(R, K);
    const dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile, N);
    const float inv2s2 = 1.0f / (2.0f * sigma * sigma);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(backward ? (const void*)bilateral_bwd_kernel : (const void*)bilateral_fwd_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (backward)
        launch_k(bilateral_bwd_kernel, grid, kTile * kTile, smem, s, reinterpret_cast<const float4*>(gb_pos),
                 reinterpret_cast<const float4*>(gb_nrm), cams, N, H, W, K, wsum_in,
                 reinterpret_cast<const float4*>(in), inv2s2, R, reinterpret_cast<float4*>(out));
    else
        launch_k(bilateral_fwd_kernel, grid, kTile * kTile, smem, s, reinterpret_cast<const float4*>(gb_pos),
                 reinterpret_cast<const float4*>(gb_nrm), cams, N, H, W, K, reinterpret_cast<const float4*>(in), inv2s2,
                 R, reinterpret_cast<float4*>(out), wsum_out);
    return cudaGetLastError();
}

}  // namespace mcdi
