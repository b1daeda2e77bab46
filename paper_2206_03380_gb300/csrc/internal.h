// Host-side declarations shared between the C-ABI layer and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/mcdi.h"
#include "common.cuh"

namespace mcdi {

// ---- BVH build scratch layout (offsets in bytes, 256-byte aligned) ----
struct BvhScratch {
    size_t bounds, keys0, keys1, vals0, vals1, hist, digit_tot, parent_int, parent_leaf, flags, box_int, box_leaf;
    size_t total;
    int nblocks;  // radix-sort tiles
};
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortDigitBits = 10;  // 30-bit Morton keys: three passes
constexpr int kSortPasses = 3;
static_assert(kSortDigitBits * kSortPasses >= 30, "the passes must cover the 30 key bits");
// the same sort in one kernel per pass for meshes of up to kTileSortMax triangles: tiles of kTileKeys
// sorted positions, each pass's digit counts per tile made by the kernel before it
// (each tile reads every tile's counts: the cost grows with the square of the tile count)
constexpr int kTileThreads = 256;
constexpr int kTileItems = 8;
constexpr int kTileKeys = kTileThreads * kTileItems;  // 2,048
constexpr int kTileSortMax = 128 * kTileKeys;         // 262,144 triangles (at most 128 tiles)
inline constexpr bool bvh_tile_sort(int n) { return n >= 1 && n <= kTileSortMax; }

__host__ __device__ constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr BvhScratch bvh_scratch_layout(int n) {
    BvhScratch s{};
    const size_t un = (size_t)(n > 0 ? n : 1);
    const size_t ni = un > 1 ? un - 1 : 1;
    s.nblocks = (int)((un + kSortTile - 1) / kSortTile);
    size_t o = 0;
    s.bounds = o; o = align256(o + 8 * sizeof(uint32_t));
    s.keys0 = o; o = align256(o + un * sizeof(uint32_t));
    s.keys1 = o; o = align256(o + un * sizeof(uint32_t));
    s.vals0 = o; o = align256(o + un * sizeof(uint32_t));
    s.vals1 = o; o = align256(o + un * sizeof(uint32_t));
    const size_t tiles = (un + kTileKeys - 1) / kTileKeys;
    const size_t hist_rows = (size_t)s.nblocks > kSortPasses * tiles ? (size_t)s.nblocks : kSortPasses * tiles;
    s.hist = o; o = align256(o + ((size_t)1 << kSortDigitBits) * hist_rows * sizeof(uint32_t));
    s.digit_tot = o; o = align256(o + ((size_t)1 << kSortDigitBits) * sizeof(uint32_t));
    s.parent_int = o; o = align256(o + ni * sizeof(int));
    s.parent_leaf = o; o = align256(o + un * sizeof(int));
    s.flags = o; o = align256(o + ni * sizeof(uint32_t));
    s.box_int = o; o = align256(o + ni * 2 * sizeof(float4));
    s.box_leaf = o; o = align256(o + un * 2 * sizeof(float4));
    s.total = o;
    return s;
}

// two-child nodes (64 B each), then the depth-first copy with escape links
// (2 n - 1 nodes of 32 B) and the four-wide nodes (one 64-byte slot per
// two-child node), each at a 256-byte aligned offset
inline size_t bvh_node_bytes(int n) { return wide_offset(n) + (size_t)(n > 1 ? n - 1 : 1) * sizeof(WideNode); }
inline size_t bvh_tri_bytes(int n) { return (size_t)(n > 0 ? n : 1) * 48; }

// Record the reason returned by mcdi_last_error() on this thread ("" clears it).
void set_last_error(const char* msg);

// ---- launchers (each enqueues kernels on `stream`, returns cudaGetLastError) ----
cudaError_t launch_envmap_cdf(const float* env, int W, int H, float* cond, float* marg, double* row_sum,
                              double* total, cudaStream_t stream);

cudaError_t launch_build_bvh(const float* verts, int n_verts, const int* tris, int n_tris, void* nodes,
                             void* tri_records, void* scratch, const BvhScratch& layout, cudaStream_t stream);
cudaError_t launch_refit_bvh(const float* verts, int n_verts, const int* tris, int n_tris, void* nodes,
                             void* tri_records, void* scratch, const BvhScratch& layout, cudaStream_t stream);

struct ShadeArgs {
    const void* nodes;
    const void* tris;
    int n_tris;
    const float4* env;
    int Wp, Hp;
    const float* cond;
    const float* marg;
    const double* total;
    const float4* gb_pos;
    const float4* gb_nrm;
    const float4* gb_kd;
    const float4* gb_korm;
    const mcdi_camera* cams;
    int N, H, W;
    int n_light, n_cos, n_ggx;
    unsigned long long seed;
    float tau, ray_eps;
    uint32_t stream_word;
};

cudaError_t launch_primary_cast(const void* nodes, const void* tris, int n_tris, const float* verts,
                                const float* vnrm, const int* tri_idx, int n_verts, const mcdi_camera* cams, int N,
                                int H, int W, const float* tex_kd, const float* tex_korm, int tex_size, float uv_ox,
                                float uv_oz, float uv_s, float* gb_pos, float* gb_nrm, float* gb_kd, float* gb_korm,
                                cudaStream_t stream);

size_t raster_workspace_bytes(long long pixels);
cudaError_t launch_raster_gbuffer(const float* verts, const float* vnrm, const int* tri_idx, int n_verts, int n_tris,
                                  const mcdi_camera* cams, int N, int H, int W, const float* tex_kd,
                                  const float* tex_korm, int tex_size, float uv_ox, float uv_oz, float uv_s,
                                  float* gb_pos, float* gb_nrm, float* gb_kd, float* gb_korm, void* workspace,
                                  cudaStream_t stream, int parts = 3, int tex_channels = 4);

cudaError_t launch_shade_fwd(const ShadeArgs& a, float4* c_d, float4* kd_out, float4* c_s, uint32_t* vis_mask,
                             cudaStream_t stream);

size_t shade_workspace_bytes(long long pixels, int spp);
cudaError_t launch_shade_fwd_wave(const ShadeArgs& a, float4* c_d, float4* kd_out, float4* c_s, uint32_t* vis_mask,
                                  void* ws, cudaStream_t stream,
                                  int parts = 3);
cudaError_t launch_shadow_ray_stats(const ShadeArgs& a, const void* ws, unsigned long long* stats,
                                    cudaStream_t stream);
cudaError_t launch_shadow_ray_retrace(const ShadeArgs& a, void* ws, cudaStream_t stream);

// ---- shadow-visibility gradients by edge sampling (shadow_grad.cu)
struct EdgeScratch {
    size_t keys, first, second, slot_of, tile_count, tile_off, err, total;
    size_t cap;   // hash-table slots (a power of two >= 2 x the half-edges)
    int n_tiles;  // compaction tiles of half-edges
};
EdgeScratch edge_scratch_layout(int n_tris);
cudaError_t launch_build_edge_table(const int* tris, int n_tris, int4* edges, int* n_edges, void* scratch,
                                    const EdgeScratch& layout, cudaStream_t stream);
cudaError_t launch_shadow_edge_grad(const ShadeArgs& a, const float* verts, int n_verts, const int4* edges,
                                    const int* n_edges, int max_edges, int n_samples, float eta, const float4* g_cd,
                                    const float4* g_cs, float* g_verts, float* sample_w, cudaStream_t stream);

// ---- measurement aid (measure.cu): L2-resident read sweep
cudaError_t launch_read_sweep(const void* buf, size_t bytes, int passes, unsigned* sink, cudaStream_t stream);

cudaError_t launch_shade_bwd(const ShadeArgs& a, const float4* g_cd, const float4* g_kdout, const float4* g_cs,
                             const uint32_t* vis_mask, float4* g_kd, float4* g_korm, float4* g_nrm, float4* g_env,
                             cudaStream_t stream, long long first = 0, long long count = -1);

// ---- denoiser (U-Net of 15 3x3 convolutions; denoise.cu)
constexpr int kUnetConvs = 15;
struct UnetWeightLayout {
    size_t wk[kUnetConvs], wf[kUnetConvs], bias[kUnetConvs];
    size_t wk8[kUnetConvs], wf8[kUnetConvs], amax;  // E4M3 forms and per-convolution weight amax
    size_t total;
    size_t n_params;  // fp32 parameters in the plan's order (W[co][ci][3][3], then b[co], per conv)
};
UnetWeightLayout unet_weight_layout();
size_t unet_act_bytes(int n, int H, int W, int precision);
size_t unet_grad_bytes(int n, int H, int W, int precision);
cudaError_t launch_unet_pack_weights(const float* params, void* weights, cudaStream_t s);
cudaError_t launch_unet_fwd(const void* weights, int precision, int n, int H, int W, const float* term,
                            const float* kd, const float* nrm, int n_aux, float* y, void* acts, unsigned* err,
                            cudaStream_t s, const char** why);
cudaError_t launch_unet_bwd(const void* weights, int precision, int n, int H, int W, const void* acts,
                            const float* gy, float* gx_term, void* grad_ws, unsigned* err, cudaStream_t s,
                            const char** why);
size_t unet_wgrad_bytes(int n, int H, int W);
cudaError_t launch_unet_wgrad(const void* acts, const void* grad_ws, int n, int H, int W, float* gw, void* scratch,
                              unsigned* err, cudaStream_t s, const char** why);
// one convolution's weight and bias gradient (wgrad.cu): x [n][x_ctot / 8][H][W][8] and g [n][g_ctot / 8][H][W][8]
// BF16 planes -> gw = dW[co][ci][3][3] then db[co] (FP32)
size_t wgrad_scratch_bytes(int x_ctot, int g_ctot, int n_img, int H, int W);
cudaError_t launch_wgrad(const void* x, int x_ctot, const void* g, int g_ctot, int n_img, int H, int W, int ci,
                         int co, void* scratch, float* gw, unsigned* err, cudaStream_t s, const char** why);
constexpr int kPlanRecordInts = 8;
void set_plan_recorder(int* rec, int cap, int* count);  // nullptr rec: stop recording
cudaError_t launch_conv3x3(const void* x, int n, int H, int W, int cin_pad, const void* w, const float* bias,
                           int cout_pad, int relu, void* y, unsigned* err, cudaStream_t s, const char** why);
cudaError_t launch_conv3x3_e4m3(const void* x, int n, int H, int W, int cin_pad, const void* w, const float* x_amax,
                                const float* w_amax, const float* bias, int cout_pad, int relu, void* y, unsigned* err,
                                cudaStream_t s, const char** why);

int bilateral_max_images_per_view();
cudaError_t launch_bilateral(bool backward, const float* gb_pos, const float* gb_nrm, const mcdi_camera* cams, int N,
                             int H, int W, int n_img, const float* in, float sigma, int R, const float* wsum_in,
                             float* out, float* wsum_out, cudaStream_t s);

size_t image_loss_workspace_bytes(long long n);
cudaError_t launch_image_loss(const float* kd, const float* dd, const float* ds, const float* ref, long long n,
                              float lambda_light, float* c, double* loss, float* g_kd, float* g_dd, float* g_ds,
                              void* workspace, cudaStream_t s);

cudaError_t launch_composite(const float* kd, const float* dd, const float* ds, long long n, float* c,
                             cudaStream_t s);

}  // namespace mcdi
