// G-buffer by rasterisation (the paper rasterises primary visibility with
// nvdiffrast, Sec. 3.1): every triangle is scan-converted over the pixels of
// its screen bounding box, and each candidate pixel is decided by the same
// FP32 ray/triangle test the ray-cast G-buffer uses (the camera ray through
// the pixel centre against v0, e1 = v1 - v0, e2 = v2 - v0, the values of the
// BVH's triangle records), so it covers the pixels the ray cast covers, with
// the same triangles.
// The nearest hit per pixel wins through a 64-bit atomicMin of (t bits,
// triangle index): depth first, then the lowest triangle index on an exact tie.
// A resolve pass then writes the G-buffer entries from the winning triangle as
// the ray cast does.  The mesh alone is read, not the BVH, so the pass can run
// concurrently with the BVH build.
#include "common.cuh"
#include "internal.h"
#include "shading.cuh"

namespace mcdi {
namespace {

constexpr int kRasterThreads = 128;
constexpr int kBigArea = 64;          // pixels: larger boxes are walked by the whole warp
constexpr float kNearPlane = 1e-6f;   // the part of a triangle closer to the eye plane than this is ignored
constexpr float kBoxSlack = 1.0f / 64.0f;  // pixels of slack around the projected box
constexpr unsigned long long kEmpty = ~0ull;

__global__ void __launch_bounds__(kRasterThreads) zclear_kernel(unsigned long long* z, long long n) {
    pdl_prologue();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) z[i] = kEmpty;
}

// pixel coordinates (continuous, pixel centres at integers) of a camera-space point
__device__ __forceinline__ float2 project(const mcdi_camera& C, f3 q, float zc, int W, int H) {
    const float xc = q.x * C.right[0] + q.y * C.right[1] + q.z * C.right[2];
    const float yc = q.x * C.up[0] + q.y * C.up[1] + q.z * C.up[2];
    const float sx = xc / (zc * C.tan_half_fovy * C.aspect), sy = yc / (zc * C.tan_half_fovy);
    return make_float2((sx + 1.0f) * 0.5f * (float)W - 0.5f, (1.0f - sy) * 0.5f * (float)H - 0.5f);
}

// Screen box of a triangle, clipped at the near plane: the pixels whose
// centres lie within kBoxSlack of the projected box (the projection's
// rounding, about 1e-6 of the coordinates, is far below it, so no pixel the
// exact test covers is dropped); false when the triangle lies behind the near
// plane or covers no pixel centre.
__device__ __forceinline__ bool screen_box(const mcdi_camera& C, const f3 p[3], int W, int H, int4* box) {
    const f3 o = mk(C.origin[0], C.origin[1], C.origin[2]);
    const f3 fw = mk(C.forward[0], C.forward[1], C.forward[2]);
    f3 q[3];
    float z[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        q[i] = p[i] - o;
        z[i] = dot(q[i], fw);
    }
    float x0 = FLT_MAX, y0 = FLT_MAX, x1 = -FLT_MAX, y1 = -FLT_MAX;
    bool any = false;
    auto add = [&](f3 qq, float zz) {
        const float2 s = project(C, qq, zz, W, H);
        x0 = fminf(x0, s.x);
        x1 = fmaxf(x1, s.x);
        y0 = fminf(y0, s.y);
        y1 = fmaxf(y1, s.y);
        any = true;
    };
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3;
        if (z[i] > kNearPlane) add(q[i], z[i]);
        if ((z[i] > kNearPlane) != (z[j] > kNearPlane)) {  // the edge crosses the near plane
            const float a = (kNearPlane - z[i]) / (z[j] - z[i]);
            add(q[i] + (q[j] - q[i]) * a, kNearPlane);
        }
    }
    if (!any) return false;
    // clamp in float before converting, so that far-off projections cannot overflow
    const float bx0 = fmaxf(ceilf(x0 - kBoxSlack), 0.0f), by0 = fmaxf(ceilf(y0 - kBoxSlack), 0.0f);
    const float bx1 = fminf(floorf(x1 + kBoxSlack), (float)(W - 1)), by1 = fminf(floorf(y1 + kBoxSlack), (float)(H - 1));
    if (!(bx0 <= bx1) || !(by0 <= by1)) return false;
    *box = make_int4((int)bx0, (int)by0, (int)bx1, (int)by1);
    return true;
}

__device__ __forceinline__ void raster_pixel(const mcdi_camera& C, f3 v0, f3 e1, f3 e2, int k, int x, int y, int W,
                                             int H, unsigned long long* zview) {
    const f3 o = mk(C.origin[0], C.origin[1], C.origin[2]);
    const float t = tri_hit_v(make_ray(o, camera_dir(C, x, y, W, H)), v0, e1, e2, nullptr, nullptr);
    if (t < FLT_MAX) {
        const unsigned long long key = ((unsigned long long)__float_as_uint(t) << 32) | (unsigned)k;
        atomicMin(zview + (size_t)y * W + x, key);
    }
}

// one thread per (view, triangle)
__global__ void __launch_bounds__(kRasterThreads) raster_kernel(const float* __restrict__ verts, int n_verts,
                                                                const int* __restrict__ tri_idx, int n_tris,
                                                                const mcdi_camera* __restrict__ cams, int N, int H,
                                                                int W, unsigned long long* z) {
    pdl_prologue();
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in_range = tid < (long long)N * n_tris;
    const int view = in_range ? (int)(tid / n_tris) : 0;
    const int k = in_range ? (int)(tid - (long long)view * n_tris) : 0;
    const mcdi_camera& C = cams[view];
    unsigned long long* zview = z + (size_t)view * H * W;
    int4 box = make_int4(0, 0, -1, -1);
    f3 a{}, e1{}, e2{};
    bool ok = false;
    if (in_range) {
        f3 b, c;
        load_tri(verts, n_verts, tri_idx, k, a, b, c);
        e1 = b - a;
        e2 = c - a;
        const f3 p[3] = {a, a + e1, a + e2};
        ok = screen_box(C, p, W, H, &box);
    }
    const int bw = box.z - box.x + 1, bh = box.w - box.y + 1;
    const bool big = ok && bw * bh > kBigArea;
    if (ok && !big)
        for (int y = box.y; y <= box.w; ++y)
            for (int x = box.x; x <= box.z; ++x) raster_pixel(C, a, e1, e2, k, x, y, W, H, zview);
    // large boxes: the whole warp walks each one's pixels
    const int lane = threadIdx.x & 31;
    for (unsigned todo = __ballot_sync(0xffffffffu, big); todo; todo &= todo - 1u) {
        const int src = __ffs(todo) - 1;
        const int sv = __shfl_sync(0xffffffffu, view, src), sk = __shfl_sync(0xffffffffu, k, src);
        const f3 sa = mk(__shfl_sync(0xffffffffu, a.x, src), __shfl_sync(0xffffffffu, a.y, src),
                         __shfl_sync(0xffffffffu, a.z, src));
        const f3 s1 = mk(__shfl_sync(0xffffffffu, e1.x, src), __shfl_sync(0xffffffffu, e1.y, src),
                         __shfl_sync(0xffffffffu, e1.z, src));
        const f3 s2 = mk(__shfl_sync(0xffffffffu, e2.x, src), __shfl_sync(0xffffffffu, e2.y, src),
                         __shfl_sync(0xffffffffu, e2.z, src));
        const int x0 = __shfl_sync(0xffffffffu, box.x, src), y0 = __shfl_sync(0xffffffffu, box.y, src);
        const int w = __shfl_sync(0xffffffffu, bw, src), n = w * __shfl_sync(0xffffffffu, bh, src);
        const mcdi_camera& SC = cams[sv];
        unsigned long long* sz = z + (size_t)sv * H * W;
        for (int i = lane; i < n; i += 32) raster_pixel(SC, sa, s1, s2, sk, x0 + i % w, y0 + i / w, W, H, sz);
    }
}

// the G-buffer entries of every pixel from its winning triangle
template <int kCh>
__global__ void __launch_bounds__(kRasterThreads) resolve_kernel(
    const unsigned long long* __restrict__ z, const float* __restrict__ verts, const float* __restrict__ vnrm,
    const int* __restrict__ tri_idx, int n_verts, int n_tris, const mcdi_camera* __restrict__ cams, int N, int H, int W,
    const float* __restrict__ tex_kd, const float* __restrict__ tex_korm, int S, float uv_ox, float uv_oz,
    float uv_s, float4* __restrict__ gb_pos, float4* __restrict__ gb_nrm, float4* __restrict__ gb_kd,
    float4* __restrict__ gb_korm) {
    pdl_prologue();
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * H * W) return;
    float4 P = make_float4(0.f, 0.f, 0.f, 0.f), Nn = P, KD = P, KORM = P;
    const unsigned long long key = z[idx];
    const int k = (int)(unsigned)(key & 0xffffffffull);
    if (key != kEmpty && (unsigned)k < (unsigned)n_tris) {
        const int view = (int)(idx / ((long long)H * W));
        const int pix = (int)(idx - (long long)view * H * W);
        const mcdi_camera& C = cams[view];
        f3 a, b, c;
        load_tri(verts, n_verts, tri_idx, k, a, b, c);
        float u = 0.f, v = 0.f;
        const float t = tri_hit_v(make_ray(mk(C.origin[0], C.origin[1], C.origin[2]), camera_dir(C, pix % W, pix / W, W, H)),
                                  a, b - a, c - a, &u, &v);
        if (t < FLT_MAX)
            gbuffer_hit<kCh>(k, u, v, verts, vnrm, tri_idx, n_verts, tex_kd, tex_korm, S, uv_ox, uv_oz, uv_s, &P, &Nn,
                             &KD, &KORM);
    }
    gb_pos[idx] = P;
    gb_nrm[idx] = Nn;
    gb_kd[idx] = KD;
    gb_korm[idx] = KORM;
}

inline int blocks_for(long long n) { return (int)((n + kRasterThreads - 1) / kRasterThreads); }

}  // namespace

size_t raster_workspace_bytes(long long pixels) {
    return align256((size_t)(pixels > 0 ? pixels : 1) * sizeof(unsigned long long));
}

cudaError_t launch_raster_gbuffer(const float* verts, const float* vnrm, const int* tri_idx, int n_verts, int n_tris,
                                  const mcdi_camera* cams, int N, int H, int W, const float* tex_kd,
                                  const float* tex_korm, int tex_size, float uv_ox, float uv_oz, float uv_s,
                                  float* gb_pos, float* gb_nrm, float* gb_kd, float* gb_korm, void* workspace,
                                  cudaStream_t stream, int parts, int tex_channels) {
    const long long P = (long long)N * H * W;
    auto* z = static_cast<unsigned long long*>(workspace);
    if (parts & 1) {  // depth pass: the mesh and the cameras only
        launch_k(zclear_kernel, blocks_for(P) < 4096 ? blocks_for(P) : 4096, kRasterThreads, 0, stream, z, P);
        if (n_tris > 0)
            launch_k(raster_kernel, blocks_for((long long)N * n_tris), kRasterThreads, 0, stream, verts, n_verts,
                     tri_idx, n_tris, cams, N, H, W, z);
    }
    if (!(parts & 2)) return cudaGetLastError();
    auto* rk = tex_channels == 3 ? resolve_kernel<3> : resolve_kernel<4>;
    launch_k(rk, blocks_for(P), kRasterThreads, 0, stream, (const unsigned long long*)z, verts, vnrm, tri_idx, n_verts,
             n_tris, cams, N, H, W, tex_kd, tex_korm, tex_size, uv_ox, uv_oz, uv_s, reinterpret_cast<float4*>(gb_pos),
             reinterpret_cast<float4*>(gb_nrm), reinterpret_cast<float4*>(gb_kd), reinterpret_cast<float4*>(gb_korm));
    return cudaGetLastError();
}

}  // namespace mcdi
