// C-ABI entry points of libmcdi: argument checks, then kernel launches on the
// caller's stream.  No entry point allocates device memory or synchronises.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "internal.h"

namespace {

thread_local char g_err[512] = "";

mcdi_status fail(mcdi_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

mcdi_status ok() {
    g_err[0] = '\0';
    return MCDI_OK;
}

mcdi_status launched(cudaError_t e, const char* what) {
    if (e != cudaSuccess) return fail(MCDI_DEVICE_ERROR, "%s: %s", what, cudaGetErrorString(e));
    return ok();
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

#define REQUIRE(cond, ...)                                  \
    do {                                                    \
        if (!(cond)) return fail(MCDI_INVALID_ARG, __VA_ARGS__); \
    } while (0)

#define REQUIRE_BUF16(p) REQUIRE((p) != nullptr && aligned16(p), "%s must be a non-NULL 16-byte aligned device pointer", #p)
// BVH node arrays are read with 32-byte vector loads
#define REQUIRE_NODES(p) \
    REQUIRE((p) != nullptr && ((uintptr_t)(p) & 255u) == 0, "%s must be a non-NULL 256-byte aligned device pointer", #p)

mcdi_status check_params(const mcdi_shade_params* prm) {
    REQUIRE(prm != nullptr, "params is NULL");
    REQUIRE(prm->n_light >= 0 && prm->n_cos >= 0 && prm->n_ggx >= 0, "sample counts must be >= 0");
    const long long spp = (long long)prm->n_light + prm->n_cos + prm->n_ggx;
    REQUIRE(spp >= 1 && spp <= 1024, "spp = n_light + n_cos + n_ggx must be in [1, 1024], got %lld", spp);
    REQUIRE(prm->tau >= 0.0f && prm->tau <= 1.0f, "tau must be in [0, 1]");
    REQUIRE(prm->ray_eps >= 0.0f && prm->ray_eps < 1e30f, "ray_eps must be finite and >= 0");
    return MCDI_OK;
}

mcdi_status shade_common(const mcdi_bvh_view* bvh, const float* env, int Wp, int Hp, const float* cond,
                         const float* marg, const double* total, const float* gb_pos, const float* gb_nrm,
                         const float* gb_kd, const float* gb_korm, const mcdi_camera* cams, int N, int H, int W,
                         const mcdi_shade_params* prm, mcdi::ShadeArgs* a) {
    REQUIRE(bvh != nullptr, "bvh is NULL");
    REQUIRE(bvh->n_tris >= 0, "bvh->n_tris must be >= 0");
    if (bvh->n_tris > 0) {
        REQUIRE_NODES(bvh->nodes);
        REQUIRE_BUF16(bvh->tri_records);
    }
    REQUIRE_BUF16(env);
    REQUIRE(Wp >= 1 && Wp <= 8192 && Hp >= 1 && Hp <= 4096, "probe size %dx%d out of range", Wp, Hp);
    REQUIRE(cond != nullptr && marg != nullptr && total != nullptr, "CDF tables must be non-NULL");
    REQUIRE_BUF16(gb_pos);
    REQUIRE_BUF16(gb_nrm);
    REQUIRE_BUF16(gb_kd);
    REQUIRE_BUF16(gb_korm);
    REQUIRE(cams != nullptr && ((uintptr_t)cams & 3u) == 0, "cams must be a non-NULL 4-byte aligned device pointer");
    REQUIRE(N >= 1 && H >= 1 && W >= 1, "image shape must be positive");
    REQUIRE((long long)N * H * W <= (1LL << 31) - 1, "too many pixels");
    REQUIRE((long long)H * W <= 0xffffffffLL, "too many pixels per view");
    mcdi_status s = check_params(prm);
    if (s != MCDI_OK) return s;
    a->nodes = bvh->nodes;
    a->tris = bvh->tri_records;
    a->n_tris = bvh->n_tris;
    a->env = reinterpret_cast<const float4*>(env);
    a->Wp = Wp;
    a->Hp = Hp;
    a->cond = cond;
    a->marg = marg;
    a->total = total;
    a->gb_pos = reinterpret_cast<const float4*>(gb_pos);
    a->gb_nrm = reinterpret_cast<const float4*>(gb_nrm);
    a->gb_kd = reinterpret_cast<const float4*>(gb_kd);
    a->gb_korm = reinterpret_cast<const float4*>(gb_korm);
    a->cams = cams;
    a->N = N;
    a->H = H;
    a->W = W;
    a->n_light = prm->n_light;
    a->n_cos = prm->n_cos;
    a->n_ggx = prm->n_ggx;
    a->seed = prm->seed;
    a->tau = prm->tau;
    a->ray_eps = prm->ray_eps;
    a->stream_word = 0;
    return MCDI_OK;
}

}  // namespace

namespace mcdi {
void set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace mcdi

extern "C" {

const char* mcdi_last_error(void) { return g_err; }

int mcdi_version(void) { return 100; }

mcdi_status mcdi_build_envmap_cdf(const float* env, int W, int H, float* cond_cdf, float* marg_cdf, double* row_sum,
                                  double* total, void* stream) {
    REQUIRE_BUF16(env);
    REQUIRE(W >= 1 && W <= 8192 && H >= 1 && H <= 4096, "probe size %dx%d out of range", W, H);
    REQUIRE(cond_cdf != nullptr && marg_cdf != nullptr, "CDF outputs must be non-NULL");
    REQUIRE(row_sum != nullptr && total != nullptr && ((uintptr_t)row_sum & 7u) == 0 && ((uintptr_t)total & 7u) == 0,
            "row_sum / total must be non-NULL 8-byte aligned");
    return launched(mcdi::launch_envmap_cdf(env, W, H, cond_cdf, marg_cdf, row_sum, total,
                                            static_cast<cudaStream_t>(stream)),
                    "build_envmap_cdf");
}

mcdi_status mcdi_bvh_sizes(int n_tris, size_t* node_bytes, size_t* tri_bytes, size_t* scratch_bytes) {
    REQUIRE(n_tris >= 1 && n_tris <= (1 << 27), "n_tris must be in [1, 2^27], got %d", n_tris);
    REQUIRE(node_bytes && tri_bytes && scratch_bytes, "size outputs must be non-NULL");
    *node_bytes = mcdi::bvh_node_bytes(n_tris);
    *tri_bytes = mcdi::bvh_tri_bytes(n_tris);
    *scratch_bytes = mcdi::bvh_scratch_layout(n_tris).total;
    return ok();
}

mcdi_status mcdi_build_bvh(const float* verts, int n_verts, const int* tris, int n_tris, void* nodes,
                           void* tri_records, void* scratch, size_t scratch_bytes, void* stream) {
    REQUIRE(n_tris >= 1 && n_tris <= (1 << 27), "n_tris must be in [1, 2^27], got %d", n_tris);
    REQUIRE(n_verts >= 1, "n_verts must be >= 1");
    REQUIRE(verts != nullptr && tris != nullptr, "verts / tris must be non-NULL");
    REQUIRE(((uintptr_t)verts & 3u) == 0 && ((uintptr_t)tris & 3u) == 0, "verts / tris must be 4-byte aligned");
    REQUIRE_NODES(nodes);
    REQUIRE_BUF16(tri_records);
    REQUIRE(scratch != nullptr && ((uintptr_t)scratch & 255u) == 0, "scratch must be non-NULL 256-byte aligned");
    const mcdi::BvhScratch L = mcdi::bvh_scratch_layout(n_tris);
    REQUIRE(scratch_bytes >= L.total, "scratch too small: %zu < %zu bytes", scratch_bytes, L.total);
    return launched(mcdi::launch_build_bvh(verts, n_verts, tris, n_tris, nodes, tri_records, scratch, L,
                                           static_cast<cudaStream_t>(stream)),
                    "build_bvh");
}

mcdi_status mcdi_bvh_build_launches(int n_tris, int* launches) {
    REQUIRE(n_tris >= 1 && n_tris <= (1 << 27), "n_tris must be in [1, 2^27], got %d", n_tris);
    REQUIRE(launches != nullptr, "launches is NULL");
    // bounds (2), Morton codes, the sort, leaf records with the hierarchy, boxes, depth-first copy (a single
    // triangle: leaf record, root)
    *launches = 3 + (mcdi::bvh_tile_sort(n_tris) ? 1 : 3) * mcdi::kSortPasses + 2 + 1;
    return ok();
}

mcdi_status mcdi_refit_bvh(const float* verts, int n_verts, const int* tris, int n_tris, void* nodes,
                           void* tri_records, void* scratch, size_t scratch_bytes, void* stream) {
    REQUIRE(n_tris >= 1 && n_tris <= (1 << 27), "n_tris must be in [1, 2^27], got %d", n_tris);
    REQUIRE(n_verts >= 1, "n_verts must be >= 1");
    REQUIRE(verts != nullptr && tris != nullptr, "verts / tris must be non-NULL");
    REQUIRE(((uintptr_t)verts & 3u) == 0 && ((uintptr_t)tris & 3u) == 0, "verts / tris must be 4-byte aligned");
    REQUIRE_NODES(nodes);
    REQUIRE_BUF16(tri_records);
    REQUIRE(scratch != nullptr && ((uintptr_t)scratch & 255u) == 0, "scratch must be non-NULL 256-byte aligned");
    const mcdi::BvhScratch L = mcdi::bvh_scratch_layout(n_tris);
    REQUIRE(scratch_bytes >= L.total, "scratch too small: %zu < %zu bytes", scratch_bytes, L.total);
    return launched(mcdi::launch_refit_bvh(verts, n_verts, tris, n_tris, nodes, tri_records, scratch, L,
                                           static_cast<cudaStream_t>(stream)),
                    "refit_bvh");
}

mcdi_status mcdi_primary_cast(const mcdi_bvh_view* bvh, const float* verts, const float* vnrm, const int* tris,
                              int n_verts, const mcdi_camera* cams, int N, int H, int W, const float* tex_kd,
                              const float* tex_korm, int tex_size, const float* uvmap, float* gb_pos, float* gb_nrm,
                              float* gb_kd, float* gb_korm, void* stream) {
    REQUIRE(bvh != nullptr && bvh->n_tris >= 0, "bvh is NULL or invalid");
    if (bvh->n_tris > 0) {
        REQUIRE_NODES(bvh->nodes);
        REQUIRE_BUF16(bvh->tri_records);
    }
    REQUIRE(verts && vnrm && tris && n_verts >= 1, "mesh arrays must be non-NULL");
    REQUIRE(cams != nullptr, "cams is NULL");
    REQUIRE(N >= 1 && H >= 1 && W >= 1 && (long long)N * H * W <= (1LL << 31) - 1, "bad image shape");
    REQUIRE(tex_size >= 1 && tex_size <= 16384, "tex_size out of range");
    REQUIRE_BUF16(tex_kd);
    REQUIRE_BUF16(tex_korm);
    REQUIRE(uvmap != nullptr, "uvmap (host, 3 floats) is NULL");
    REQUIRE_BUF16(gb_pos);
    REQUIRE_BUF16(gb_nrm);
    REQUIRE_BUF16(gb_kd);
    REQUIRE_BUF16(gb_korm);
    return launched(mcdi::launch_primary_cast(bvh->nodes, bvh->tri_records, bvh->n_tris, verts, vnrm, tris, n_verts,
                                              cams, N, H, W, tex_kd, tex_korm, tex_size, uvmap[0], uvmap[1],
                                              uvmap[2], gb_pos, gb_nrm, gb_kd, gb_korm,
                                              static_cast<cudaStream_t>(stream)),
                    "primary_cast");
}

mcdi_status mcdi_raster_workspace_size(int N, int H, int W, size_t* bytes) {
    REQUIRE(N >= 1 && H >= 1 && W >= 1 && (long long)N * H * W <= (1LL << 31) - 1, "bad image shape");
    REQUIRE(bytes != nullptr, "bytes is NULL");
    *bytes = mcdi::raster_workspace_bytes((long long)N * H * W);
    return ok();
}

static mcdi_status raster_gbuffer(const float* verts, const float* vnrm, const int* tris, int n_verts, int n_tris,
                                  const mcdi_camera* cams, int N, int H, int W, const float* tex_kd,
                                  const float* tex_korm, int tex_size, int tex_channels, const float* uvmap,
                                  float* gb_pos, float* gb_nrm, float* gb_kd, float* gb_korm, void* workspace,
                                  size_t workspace_bytes, void* stream, int parts) {
    REQUIRE(verts && vnrm && n_verts >= 1, "verts / vnrm must be non-NULL and n_verts >= 1");
    REQUIRE(n_tris >= 0 && (n_tris == 0 || tris != nullptr), "tris must be non-NULL when n_tris > 0");
    REQUIRE(((uintptr_t)verts & 3u) == 0 && ((uintptr_t)vnrm & 3u) == 0 && ((uintptr_t)tris & 3u) == 0,
            "verts / vnrm / tris must be 4-byte aligned");
    REQUIRE(cams != nullptr && ((uintptr_t)cams & 3u) == 0, "cams must be a non-NULL 4-byte aligned device pointer");
    REQUIRE(N >= 1 && H >= 1 && W >= 1 && (long long)N * H * W <= (1LL << 31) - 1, "bad image shape");
    REQUIRE((long long)N * n_tris <= (1LL << 31) - 1, "N*n_tris too large");
    REQUIRE(tex_size >= 1 && tex_size <= 16384, "tex_size out of range");
    REQUIRE(tex_channels == 3 || tex_channels == 4, "tex_channels must be 3 or 4, got %d", tex_channels);
    if (tex_channels == 4) {
        REQUIRE_BUF16(tex_kd);
        REQUIRE_BUF16(tex_korm);
    } else {
        REQUIRE(tex_kd != nullptr && tex_korm != nullptr && ((uintptr_t)tex_kd & 3u) == 0 &&
                    ((uintptr_t)tex_korm & 3u) == 0,
                "tex_kd / tex_korm must be non-NULL 4-byte aligned device pointers");
    }
    REQUIRE(uvmap != nullptr, "uvmap (host, 3 floats) is NULL");
    REQUIRE_BUF16(gb_pos);
    REQUIRE_BUF16(gb_nrm);
    REQUIRE_BUF16(gb_kd);
    REQUIRE_BUF16(gb_korm);
    REQUIRE(workspace != nullptr && ((uintptr_t)workspace & 255u) == 0,
            "workspace must be a non-NULL 256-byte aligned device pointer");
    const size_t need = mcdi::raster_workspace_bytes((long long)N * H * W);
    REQUIRE(workspace_bytes >= need, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
    return launched(mcdi::launch_raster_gbuffer(verts, vnrm, tris, n_verts, n_tris, cams, N, H, W, tex_kd, tex_korm,
                                                tex_size, uvmap[0], uvmap[1], uvmap[2], gb_pos, gb_nrm, gb_kd, gb_korm,
                                                workspace, static_cast<cudaStream_t>(stream), parts, tex_channels),
                    "raster_gbuffer");
}

mcdi_status mcdi_raster_gbuffer(const float* verts, const float* vnrm, const int* tris, int n_verts, int n_tris,
                                const mcdi_camera* cams, int N, int H, int W, const float* tex_kd,
                                const float* tex_korm, int tex_size, const float* uvmap, float* gb_pos, float* gb_nrm,
                                float* gb_kd, float* gb_korm, void* workspace, size_t workspace_bytes, void* stream) {
    return raster_gbuffer(verts, vnrm, tris, n_verts, n_tris, cams, N, H, W, tex_kd, tex_korm, tex_size, 4, uvmap,
                          gb_pos, gb_nrm, gb_kd, gb_korm, workspace, workspace_bytes, stream, 3);
}

mcdi_status mcdi_raster_gbuffer_part(const float* verts, const float* vnrm, const int* tris, int n_verts, int n_tris,
                                     const mcdi_camera* cams, int N, int H, int W, const float* tex_kd,
                                     const float* tex_korm, int tex_size, int tex_channels, const float* uvmap,
                                     float* gb_pos, float* gb_nrm, float* gb_kd, float* gb_korm, void* workspace,
                                     size_t workspace_bytes, int part, void* stream) {
    REQUIRE(part == 1 || part == 2, "part must be 1 (depth) or 2 (resolve), got %d", part);
    return raster_gbuffer(verts, vnrm, tris, n_verts, n_tris, cams, N, H, W, tex_kd, tex_korm, tex_size,
                          tex_channels, uvmap, gb_pos, gb_nrm, gb_kd, gb_korm, workspace, workspace_bytes, stream,
                          part);
}

mcdi_status mcdi_shade_workspace_size(int N, int H, int W, const mcdi_shade_params* params, size_t* bytes) {
    REQUIRE(N >= 1 && H >= 1 && W >= 1, "image shape must be positive");
    REQUIRE(bytes != nullptr, "bytes is NULL");
    mcdi_status s = check_params(params);
    if (s != MCDI_OK) return s;
    const long long spp = (long long)params->n_light + params->n_cos + params->n_ggx;
    REQUIRE((long long)N * H * W * spp <= (1LL << 31) - 1, "N*H*W*spp too large for the wavefront path");
    *bytes = mcdi::shade_workspace_bytes((long long)N * H * W, (int)spp);
    return ok();
}

mcdi_status mcdi_shade_mc_fwd(const mcdi_bvh_view* bvh, const float* env, int Wp, int Hp, const float* cond_cdf,
                              const float* marg_cdf, const double* total, const float* gb_pos, const float* gb_nrm,
                              const float* gb_kd, const float* gb_korm, const mcdi_camera* cams, int N, int H, int W,
                              const mcdi_shade_params* params, float* c_d, float* kd_out, float* c_s,
                              uint32_t* vis_mask, void* workspace, size_t workspace_bytes, void* stream) {
    mcdi::ShadeArgs a;
    mcdi_status s = shade_common(bvh, env, Wp, Hp, cond_cdf, marg_cdf, total, gb_pos, gb_nrm, gb_kd, gb_korm, cams, N,
                                 H, W, params, &a);
    if (s != MCDI_OK) return s;
    REQUIRE_BUF16(c_d);
    REQUIRE_BUF16(kd_out);
    REQUIRE_BUF16(c_s);
    REQUIRE(vis_mask == nullptr || ((uintptr_t)vis_mask & 3u) == 0, "vis_mask must be 4-byte aligned");
    if (workspace != nullptr) {
        size_t need = 0;
        s = mcdi_shade_workspace_size(N, H, W, params, &need);
        if (s != MCDI_OK) return s;
        REQUIRE(((uintptr_t)workspace & 255u) == 0, "workspace must be 256-byte aligned");
        REQUIRE(workspace_bytes >= need, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
        return launched(mcdi::launch_shade_fwd_wave(a, reinterpret_cast<float4*>(c_d),
                                                    reinterpret_cast<float4*>(kd_out), reinterpret_cast<float4*>(c_s),
                                                    vis_mask, workspace, static_cast<cudaStream_t>(stream)),
                        "shade_mc_fwd");
    }
    return launched(mcdi::launch_shade_fwd(a, reinterpret_cast<float4*>(c_d), reinterpret_cast<float4*>(kd_out),
                                           reinterpret_cast<float4*>(c_s), vis_mask,
                                           static_cast<cudaStream_t>(stream)),
                    "shade_mc_fwd");
}

mcdi_status mcdi_shade_mc_fwd_part(const mcdi_bvh_view* bvh, const float* env, int Wp, int Hp, const float* cond_cdf,
                                   const float* marg_cdf, const double* total, const float* gb_pos,
                                   const float* gb_nrm, const float* gb_kd, const float* gb_korm,
                                   const mcdi_camera* cams, int N, int H, int W, const mcdi_shade_params* params,
                                   float* c_d, float* kd_out, float* c_s, uint32_t* vis_mask, void* workspace,
                                   size_t workspace_bytes, int part, void* stream) {
    REQUIRE(part == 1 || part == 2, "part must be 1 (sample generation) or 2 (shadow rays and accumulation)");
    mcdi::ShadeArgs a;
    mcdi_status s = shade_common(bvh, env, Wp, Hp, cond_cdf, marg_cdf, total, gb_pos, gb_nrm, gb_kd, gb_korm, cams, N,
                                 H, W, params, &a);
    if (s != MCDI_OK) return s;
    REQUIRE_BUF16(c_d);
    REQUIRE_BUF16(kd_out);
    REQUIRE_BUF16(c_s);
    REQUIRE(vis_mask == nullptr || ((uintptr_t)vis_mask & 3u) == 0, "vis_mask must be 4-byte aligned");
    size_t need = 0;
    s = mcdi_shade_workspace_size(N, H, W, params, &need);
    if (s != MCDI_OK) return s;
    REQUIRE(workspace != nullptr && ((uintptr_t)workspace & 255u) == 0, "workspace must be non-NULL, 256-byte aligned");
    REQUIRE(workspace_bytes >= need, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
    return launched(mcdi::launch_shade_fwd_wave(a, reinterpret_cast<float4*>(c_d), reinterpret_cast<float4*>(kd_out),
                                                reinterpret_cast<float4*>(c_s), vis_mask, workspace,
                                                static_cast<cudaStream_t>(stream), part),
                    "shade_mc_fwd_part");
}

}  // extern "C"

namespace {

// the BVH, image shape and sample counts of a forward pass whose workspace is
// reused by the traversal-statistics calls
mcdi_status wave_common(const mcdi_bvh_view* bvh, int N, int H, int W, const mcdi_shade_params* prm,
                        const void* workspace, size_t workspace_bytes, mcdi::ShadeArgs* a) {
    REQUIRE(bvh != nullptr, "bvh is NULL");
    REQUIRE(bvh->n_tris >= 0, "bvh->n_tris must be >= 0");
    if (bvh->n_tris > 0) {
        REQUIRE_NODES(bvh->nodes);
        REQUIRE_BUF16(bvh->tri_records);
    }
    size_t need = 0;
    mcdi_status s = mcdi_shade_workspace_size(N, H, W, prm, &need);
    if (s != MCDI_OK) return s;
    REQUIRE(workspace != nullptr && ((uintptr_t)workspace & 255u) == 0,
            "workspace must be a non-NULL 256-byte aligned device pointer");
    REQUIRE(workspace_bytes >= need, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
    *a = mcdi::ShadeArgs{};
    a->nodes = bvh->nodes;
    a->tris = bvh->tri_records;
    a->n_tris = bvh->n_tris;
    a->N = N;
    a->H = H;
    a->W = W;
    a->n_light = prm->n_light;
    a->n_cos = prm->n_cos;
    a->n_ggx = prm->n_ggx;
    return MCDI_OK;
}

}  // namespace

extern "C" {

mcdi_status mcdi_shadow_ray_stats(const mcdi_bvh_view* bvh, int N, int H, int W, const mcdi_shade_params* params,
                                  const void* workspace, size_t workspace_bytes, unsigned long long* stats,
                                  void* stream) {
    mcdi::ShadeArgs a;
    mcdi_status s = wave_common(bvh, N, H, W, params, workspace, workspace_bytes, &a);
    if (s != MCDI_OK) return s;
    REQUIRE(stats != nullptr && ((uintptr_t)stats & 7u) == 0, "stats must be a non-NULL 8-byte aligned device pointer");
    return launched(mcdi::launch_shadow_ray_stats(a, workspace, stats, static_cast<cudaStream_t>(stream)),
                    "shadow_ray_stats");
}

mcdi_status mcdi_shadow_ray_retrace(const mcdi_bvh_view* bvh, int N, int H, int W, const mcdi_shade_params* params,
                                    void* workspace, size_t workspace_bytes, void* stream) {
    mcdi::ShadeArgs a;
    mcdi_status s = wave_common(bvh, N, H, W, params, workspace, workspace_bytes, &a);
    if (s != MCDI_OK) return s;
    return launched(mcdi::launch_shadow_ray_retrace(a, workspace, static_cast<cudaStream_t>(stream)),
                    "shadow_ray_retrace");
}

mcdi_status mcdi_edge_table_workspace_size(int n_tris, size_t* bytes) {
    REQUIRE(n_tris >= 1 && n_tris <= (1 << 27), "n_tris must be in [1, 2^27], got %d", n_tris);
    REQUIRE(bytes != nullptr, "bytes is NULL");
    *bytes = mcdi::edge_scratch_layout(n_tris).total;
    return ok();
}

mcdi_status mcdi_build_edge_table(const int* tris, int n_tris, int* edges, int* n_edges, void* workspace,
                                  size_t workspace_bytes, void* stream) {
    REQUIRE(n_tris >= 1 && n_tris <= (1 << 27), "n_tris must be in [1, 2^27], got %d", n_tris);
    REQUIRE(tris != nullptr && ((uintptr_t)tris & 3u) == 0, "tris must be a non-NULL 4-byte aligned device pointer");
    REQUIRE_BUF16(edges);
    REQUIRE(n_edges != nullptr && ((uintptr_t)n_edges & 3u) == 0,
            "n_edges must be a non-NULL 4-byte aligned device pointer");
    REQUIRE(workspace != nullptr && ((uintptr_t)workspace & 255u) == 0,
            "workspace must be a non-NULL 256-byte aligned device pointer");
    const mcdi::EdgeScratch L = mcdi::edge_scratch_layout(n_tris);
    REQUIRE(workspace_bytes >= L.total, "workspace too small: %zu < %zu bytes", workspace_bytes, L.total);
    return launched(mcdi::launch_build_edge_table(tris, n_tris, reinterpret_cast<int4*>(edges), n_edges, workspace,
                                                  L, static_cast<cudaStream_t>(stream)),
                    "build_edge_table");
}

mcdi_status mcdi_shadow_edge_grad(const mcdi_bvh_view* bvh, const float* verts, int n_verts, const int* edges,
                                  const int* n_edges, int max_edges, const float* env, int Wp, int Hp,
                                  const float* gb_pos, const float* gb_nrm, const float* gb_kd, const float* gb_korm,
                                  const mcdi_camera* cams, int N, int H, int W, const mcdi_shade_params* params,
                                  int n_edge_samples, float eta, const float* g_cd, const float* g_cs,
                                  float* g_verts, float* sample_w, void* stream) {
    REQUIRE(bvh != nullptr && bvh->n_tris >= 0, "bvh is NULL or invalid");
    if (bvh->n_tris > 0) {
        REQUIRE_NODES(bvh->nodes);
        REQUIRE_BUF16(bvh->tri_records);
    }
    REQUIRE(n_verts >= 1, "n_verts must be >= 1");
    REQUIRE(verts != nullptr && ((uintptr_t)verts & 3u) == 0, "verts must be a non-NULL 4-byte aligned device pointer");
    REQUIRE_BUF16(edges);
    REQUIRE(n_edges != nullptr && ((uintptr_t)n_edges & 3u) == 0,
            "n_edges must be a non-NULL 4-byte aligned device pointer");
    REQUIRE(max_edges >= 0, "max_edges must be >= 0");
    REQUIRE_BUF16(env);
    REQUIRE(Wp >= 1 && Wp <= 8192 && Hp >= 1 && Hp <= 4096, "probe size %dx%d out of range", Wp, Hp);
    REQUIRE_BUF16(gb_pos);
    REQUIRE_BUF16(gb_nrm);
    REQUIRE_BUF16(gb_kd);
    REQUIRE_BUF16(gb_korm);
    REQUIRE(cams != nullptr && ((uintptr_t)cams & 3u) == 0, "cams must be a non-NULL 4-byte aligned device pointer");
    REQUIRE(N >= 1 && H >= 1 && W >= 1, "image shape must be positive");
    REQUIRE((long long)H * W <= 0xffffffffLL, "too many pixels per view");
    REQUIRE(n_edge_samples >= 0 && n_edge_samples <= 4096, "n_edge_samples must be in [0, 4096]");
    REQUIRE((long long)N * H * W * n_edge_samples <= (1LL << 37), "N*H*W*n_edge_samples too large");
    REQUIRE(eta > 0.0f && eta <= 0.1f, "eta must be in (0, 0.1]");
    REQUIRE(params != nullptr, "params is NULL");
    REQUIRE(params->tau >= 0.0f && params->tau <= 1.0f, "tau must be in [0, 1]");
    REQUIRE(params->ray_eps >= 0.0f && params->ray_eps < 1e30f, "ray_eps must be finite and >= 0");
    REQUIRE_BUF16(g_cd);
    REQUIRE_BUF16(g_cs);
    REQUIRE(g_verts != nullptr && ((uintptr_t)g_verts & 3u) == 0,
            "g_verts must be a non-NULL 4-byte aligned device pointer");
    REQUIRE(sample_w == nullptr || ((uintptr_t)sample_w & 3u) == 0, "sample_w must be 4-byte aligned");
    mcdi::ShadeArgs a{};
    a.nodes = bvh->nodes;
    a.tris = bvh->tri_records;
    a.n_tris = bvh->n_tris;
    a.env = reinterpret_cast<const float4*>(env);
    a.Wp = Wp;
    a.Hp = Hp;
    a.gb_pos = reinterpret_cast<const float4*>(gb_pos);
    a.gb_nrm = reinterpret_cast<const float4*>(gb_nrm);
    a.gb_kd = reinterpret_cast<const float4*>(gb_kd);
    a.gb_korm = reinterpret_cast<const float4*>(gb_korm);
    a.cams = cams;
    a.N = N;
    a.H = H;
    a.W = W;
    a.seed = params->seed;
    a.tau = params->tau;
    a.ray_eps = params->ray_eps;
    a.stream_word = 2;
    return launched(mcdi::launch_shadow_edge_grad(a, verts, n_verts, reinterpret_cast<const int4*>(edges), n_edges,
                                                  max_edges, n_edge_samples, eta, reinterpret_cast<const float4*>(g_cd),
                                                  reinterpret_cast<const float4*>(g_cs), g_verts, sample_w,
                                                  static_cast<cudaStream_t>(stream)),
                    "shadow_edge_grad");
}

mcdi_status mcdi_read_sweep(const void* buf, size_t bytes, int passes, unsigned* sink, void* stream) {
    REQUIRE(buf != nullptr && aligned16(buf), "buf must be a non-NULL 16-byte aligned device pointer");
    REQUIRE(bytes >= 16 && bytes % 16 == 0, "bytes must be a positive multiple of 16");
    REQUIRE(passes >= 1, "passes must be >= 1");
    REQUIRE(sink != nullptr && ((uintptr_t)sink & 3u) == 0, "sink must be a non-NULL 4-byte aligned device pointer");
    return launched(mcdi::launch_read_sweep(buf, bytes, passes, sink, static_cast<cudaStream_t>(stream)),
                    "read_sweep");
}

static mcdi_status shade_bwd(const mcdi_bvh_view* bvh, const float* env, int Wp, int Hp, const float* cond_cdf,
                             const float* marg_cdf, const double* total, const float* gb_pos, const float* gb_nrm,
                             const float* gb_kd, const float* gb_korm, const mcdi_camera* cams, int N, int H, int W,
                             const mcdi_shade_params* params, const float* g_cd, const float* g_kdout,
                             const float* g_cs, const uint32_t* vis_mask, float* g_kd, float* g_korm, float* g_nrm,
                             float* g_env, long long first, long long count, void* stream) {
    mcdi::ShadeArgs a;
    mcdi_status s = shade_common(bvh, env, Wp, Hp, cond_cdf, marg_cdf, total, gb_pos, gb_nrm, gb_kd, gb_korm, cams, N,
                                 H, W, params, &a);
    if (s != MCDI_OK) return s;
    const long long P = (long long)N * H * W;
    if (count < 0) count = P;
    REQUIRE(first >= 0 && first <= P && count <= P - first,
            "pixel span [%lld, %lld + %lld) outside the %lld pixels of [N][H][W]", first, first, count, P);
    REQUIRE_BUF16(g_cd);
    REQUIRE_BUF16(g_kdout);
    REQUIRE_BUF16(g_cs);
    REQUIRE_BUF16(g_kd);
    REQUIRE_BUF16(g_korm);
    REQUIRE_BUF16(g_nrm);
    REQUIRE_BUF16(g_env);
    REQUIRE(vis_mask == nullptr || ((uintptr_t)vis_mask & 3u) == 0, "vis_mask must be 4-byte aligned");
    const uint32_t* mask = vis_mask;
    if (params->decorrelate_bwd) {
        a.stream_word = 1;  // fresh samples: the forward's visibility does not apply
        mask = nullptr;
    }
    return launched(mcdi::launch_shade_bwd(a, reinterpret_cast<const float4*>(g_cd),
                                           reinterpret_cast<const float4*>(g_kdout),
                                           reinterpret_cast<const float4*>(g_cs), mask,
                                           reinterpret_cast<float4*>(g_kd), reinterpret_cast<float4*>(g_korm),
                                           reinterpret_cast<float4*>(g_nrm), reinterpret_cast<float4*>(g_env),
                                           static_cast<cudaStream_t>(stream), first, count),
                    "shade_mc_bwd");
}

mcdi_status mcdi_shade_mc_bwd(const mcdi_bvh_view* bvh, const float* env, int Wp, int Hp, const float* cond_cdf,
                              const float* marg_cdf, const double* total, const float* gb_pos, const float* gb_nrm,
                              const float* gb_kd, const float* gb_korm, const mcdi_camera* cams, int N, int H, int W,
                              const mcdi_shade_params* params, const float* g_cd, const float* g_kdout,
                              const float* g_cs, const uint32_t* vis_mask, float* g_kd, float* g_korm, float* g_nrm,
                              float* g_env, void* stream) {
    return shade_bwd(bvh, env, Wp, Hp, cond_cdf, marg_cdf, total, gb_pos, gb_nrm, gb_kd, gb_korm, cams, N, H, W,
                     params, g_cd, g_kdout, g_cs, vis_mask, g_kd, g_korm, g_nrm, g_env, 0, -1, stream);
}

mcdi_status mcdi_shade_mc_bwd_span(const mcdi_bvh_view* bvh, const float* env, int Wp, int Hp,
                                   const float* cond_cdf, const float* marg_cdf, const double* total,
                                   const float* gb_pos, const float* gb_nrm, const float* gb_kd, const float* gb_korm,
                                   const mcdi_camera* cams, int N, int H, int W, const mcdi_shade_params* params,
                                   const float* g_cd, const float* g_kdout, const float* g_cs,
                                   const uint32_t* vis_mask, float* g_kd, float* g_korm, float* g_nrm, float* g_env,
                                   long long first, long long count, void* stream) {
    REQUIRE(count >= 0, "count must be >= 0, got %lld", count);
    return shade_bwd(bvh, env, Wp, Hp, cond_cdf, marg_cdf, total, gb_pos, gb_nrm, gb_kd, gb_korm, cams, N, H, W,
                     params, g_cd, g_kdout, g_cs, vis_mask, g_kd, g_korm, g_nrm, g_env, first, count, stream);
}

mcdi_status mcdi_denoise_sizes(int n_img, int H, int W, int precision, size_t* weight_bytes, size_t* act_bytes,
                               size_t* grad_bytes, size_t* n_params) {
    REQUIRE(precision == MCDI_DENOISE_BF16 || precision == MCDI_DENOISE_E4M3,
            "precision must be MCDI_DENOISE_BF16 or MCDI_DENOISE_E4M3 (got %d)", precision);
    REQUIRE(n_img >= 1 && H >= 8 && W >= 8 && H % 8 == 0 && W % 8 == 0,
            "denoiser needs n_img >= 1 and H, W positive multiples of 8 (got %d x %d)", H, W);
    REQUIRE((long long)n_img * H * W <= (1LL << 28), "denoiser image batch too large");
    const mcdi::UnetWeightLayout L = mcdi::unet_weight_layout();
    if (weight_bytes) *weight_bytes = L.total;
    if (act_bytes) *act_bytes = mcdi::unet_act_bytes(n_img, H, W, precision);
    if (grad_bytes) *grad_bytes = mcdi::unet_grad_bytes(n_img, H, W, precision);
    if (n_params) *n_params = L.n_params;
    return ok();
}

mcdi_status mcdi_denoise_pack_weights(const float* params, void* weights, void* stream) {
    REQUIRE(params != nullptr && ((uintptr_t)params & 3u) == 0, "params must be a non-NULL device pointer");
    REQUIRE(weights != nullptr && ((uintptr_t)weights & 255u) == 0, "weights must be 256-byte aligned");
    return launched(mcdi::launch_unet_pack_weights(params, weights, static_cast<cudaStream_t>(stream)),
                    "denoise_pack_weights");
}

mcdi_status mcdi_denoise_fwd(const void* weights, int precision, int n_img, int H, int W, const float* term,
                             const float* kd, const float* nrm, int n_aux, float* y, void* acts, size_t act_bytes,
                             unsigned* err, void* stream) {
    size_t need = 0;
    mcdi_status s = mcdi_denoise_sizes(n_img, H, W, precision, nullptr, &need, nullptr, nullptr);
    if (s != MCDI_OK) return s;
    REQUIRE(weights != nullptr && ((uintptr_t)weights & 255u) == 0, "weights must be 256-byte aligned");
    REQUIRE_BUF16(term);
    REQUIRE_BUF16(kd);
    REQUIRE_BUF16(nrm);
    REQUIRE_BUF16(y);
    REQUIRE(n_aux >= 1 && n_aux <= n_img, "n_aux must be in [1, n_img]");
    REQUIRE(acts != nullptr && ((uintptr_t)acts & 255u) == 0, "acts must be 256-byte aligned");
    REQUIRE(act_bytes >= need, "acts too small: %zu < %zu bytes", act_bytes, need);
    REQUIRE(err != nullptr && ((uintptr_t)err & 3u) == 0, "err must be a device uint32");
    const char* why = "";
    cudaError_t e = mcdi::launch_unet_fwd(weights, precision, n_img, H, W, term, kd, nrm, n_aux, y, acts, err,
                                          static_cast<cudaStream_t>(stream), &why);
    if (e == cudaErrorInvalidValue && why[0]) return fail(MCDI_DEVICE_ERROR, "denoise_fwd: %s", why);
    return launched(e, "denoise_fwd");
}

mcdi_status mcdi_denoise_bwd(const void* weights, int precision, int n_img, int H, int W, const void* acts,
                             size_t act_bytes, const float* gy, float* gx, void* grad_ws, size_t grad_bytes,
                             unsigned* err, void* stream) {
    size_t need_a = 0, need_g = 0;
    mcdi_status s = mcdi_denoise_sizes(n_img, H, W, precision, nullptr, &need_a, &need_g, nullptr);
    if (s != MCDI_OK) return s;
    REQUIRE(weights != nullptr && ((uintptr_t)weights & 255u) == 0, "weights must be 256-byte aligned");
    REQUIRE(acts != nullptr && act_bytes >= need_a, "acts too small");
    REQUIRE_BUF16(gy);
    REQUIRE_BUF16(gx);
    REQUIRE(grad_ws != nullptr && ((uintptr_t)grad_ws & 255u) == 0, "grad_ws must be 256-byte aligned");
    REQUIRE(grad_bytes >= need_g, "grad_ws too small: %zu < %zu bytes", grad_bytes, need_g);
    REQUIRE(err != nullptr && ((uintptr_t)err & 3u) == 0, "err must be a device uint32");
    const char* why = "";
    cudaError_t e = mcdi::launch_unet_bwd(weights, precision, n_img, H, W, acts, gy, gx, grad_ws, err,
                                          static_cast<cudaStream_t>(stream), &why);
    if (e == cudaErrorInvalidValue && why[0]) return fail(MCDI_DEVICE_ERROR, "denoise_bwd: %s", why);
    return launched(e, "denoise_bwd");
}

mcdi_status mcdi_denoise_wgrad_bytes(int n_img, int H, int W, size_t* scratch_bytes) {
    mcdi_status s = mcdi_denoise_sizes(n_img, H, W, MCDI_DENOISE_BF16, nullptr, nullptr, nullptr, nullptr);
    if (s != MCDI_OK) return s;
    REQUIRE(scratch_bytes != nullptr, "scratch_bytes must be non-NULL");
    *scratch_bytes = mcdi::unet_wgrad_bytes(n_img, H, W);
    return ok();
}

mcdi_status mcdi_denoise_wgrad(int precision, int n_img, int H, int W, const void* acts, size_t act_bytes,
                               const void* grad_ws, size_t grad_bytes, float* gw, void* scratch, size_t scratch_bytes,
                               unsigned* err, void* stream) {
    size_t need_a = 0, need_g = 0;
    mcdi_status s = mcdi_denoise_sizes(n_img, H, W, precision, nullptr, &need_a, &need_g, nullptr);
    if (s != MCDI_OK) return s;
    REQUIRE(acts != nullptr && ((uintptr_t)acts & 255u) == 0 && act_bytes >= need_a,
            "acts must be 256-byte aligned and hold %zu bytes", need_a);
    REQUIRE(grad_ws != nullptr && ((uintptr_t)grad_ws & 255u) == 0 && grad_bytes >= need_g,
            "grad_ws must be 256-byte aligned and hold %zu bytes", need_g);
    REQUIRE(gw != nullptr && ((uintptr_t)gw & 3u) == 0, "gw must be a non-NULL device float pointer");
    const size_t need_s = mcdi::unet_wgrad_bytes(n_img, H, W);
    REQUIRE(scratch != nullptr && ((uintptr_t)scratch & 255u) == 0, "scratch must be 256-byte aligned");
    REQUIRE(scratch_bytes >= need_s, "scratch too small: %zu < %zu bytes", scratch_bytes, need_s);
    REQUIRE(err != nullptr && ((uintptr_t)err & 3u) == 0, "err must be a device uint32");
    const char* why = "";
    const cudaError_t e =
        mcdi::launch_unet_wgrad(acts, grad_ws, n_img, H, W, gw, scratch, err, static_cast<cudaStream_t>(stream), &why);
    if (e == cudaErrorInvalidValue && why[0]) return fail(MCDI_DEVICE_ERROR, "denoise_wgrad: %s", why);
    return launched(e, "denoise_wgrad");
}

mcdi_status mcdi_denoise_record_plan(int* rec, int cap, int* count) {
    if (rec == nullptr) {
        mcdi::set_plan_recorder(nullptr, 0, nullptr);
        return MCDI_OK;
    }
    REQUIRE(cap >= 1 && count != nullptr, "cap must be >= 1 and count non-NULL when recording");
    mcdi::set_plan_recorder(rec, cap, count);
    return MCDI_OK;
}

mcdi_status mcdi_composite(const float* kd_out, const float* den_cd, const float* den_cs, long long n, float* c,
                           void* stream) {
    REQUIRE(n >= 1, "n must be >= 1");
    REQUIRE_BUF16(kd_out);
    REQUIRE_BUF16(den_cd);
    REQUIRE_BUF16(den_cs);
    REQUIRE_BUF16(c);
    return launched(mcdi::launch_composite(kd_out, den_cd, den_cs, n, c, static_cast<cudaStream_t>(stream)),
                    "composite");
}

static mcdi_status bilateral_call(bool backward, const float* gb_pos, const float* gb_nrm, const mcdi_camera* cams,
                                  int N, int H, int W, int n_img, const float* in, float sigma, int radius,
                                  const float* wsum_in, float* out, float* wsum_out, void* stream, const char* name) {
    REQUIRE(N >= 1 && H >= 1 && W >= 1 && (long long)N * H * W <= (1LL << 30), "%s: bad image shape", name);
    REQUIRE(n_img >= N && n_img % N == 0 && n_img / N <= mcdi::bilateral_max_images_per_view(),
            "%s: n_img must be K * N with 1 <= K <= %d", name, mcdi::bilateral_max_images_per_view());
    REQUIRE(sigma > 0.0f && sigma <= 8.0f, "%s: sigma must be in (0, 8]", name);
    const int R = radius < 0 ? (int)ceilf(2.0f * sigma) : radius;
    REQUIRE(R >= 0 && R <= 8, "%s: radius must be in [0, 8]", name);
    REQUIRE_BUF16(gb_pos);
    REQUIRE_BUF16(gb_nrm);
    REQUIRE(cams != nullptr, "%s: cams is NULL", name);
    REQUIRE_BUF16(in);
    REQUIRE_BUF16(out);
    REQUIRE((backward ? wsum_in : wsum_out) != nullptr, "%s: wsum is NULL", name);
    return launched(mcdi::launch_bilateral(backward, gb_pos, gb_nrm, cams, N, H, W, n_img, in, sigma, R, wsum_in, out,
                                           wsum_out, static_cast<cudaStream_t>(stream)),
                    name);
}

mcdi_status mcdi_bilateral_fwd(const float* gb_pos, const float* gb_nrm, const mcdi_camera* cams, int N, int H, int W,
                               int n_img, const float* c_in, float sigma, int radius, float* c_out, float* wsum,
                               void* stream) {
    return bilateral_call(false, gb_pos, gb_nrm, cams, N, H, W, n_img, c_in, sigma, radius, nullptr, c_out, wsum,
                          stream, "bilateral_fwd");
}

mcdi_status mcdi_bilateral_bwd(const float* gb_pos, const float* gb_nrm, const mcdi_camera* cams, int N, int H, int W,
                               int n_img, const float* wsum, const float* g_out, float sigma, int radius, float* g_in,
                               void* stream) {
    return bilateral_call(true, gb_pos, gb_nrm, cams, N, H, W, n_img, g_out, sigma, radius, wsum, g_in, nullptr,
                          stream, "bilateral_bwd");
}

mcdi_status mcdi_image_loss_workspace_size(long long n, size_t* bytes) {
    REQUIRE(n >= 1 && n <= (1LL << 31), "n must be in [1, 2^31]");
    REQUIRE(bytes != nullptr, "bytes must be non-NULL");
    *bytes = mcdi::image_loss_workspace_bytes(n);
    return ok();
}

mcdi_status mcdi_image_loss(const float* kd_out, const float* den_cd, const float* den_cs, const float* ref,
                            long long n, float lambda_light, float* c, double* loss, float* g_kdout, float* g_dcd,
                            float* g_dcs, void* workspace, size_t workspace_bytes, void* stream) {
    size_t need = 0;
    mcdi_status s = mcdi_image_loss_workspace_size(n, &need);
    if (s != MCDI_OK) return s;
    REQUIRE_BUF16(kd_out);
    REQUIRE_BUF16(den_cd);
    REQUIRE_BUF16(den_cs);
    REQUIRE_BUF16(ref);
    REQUIRE_BUF16(g_kdout);
    REQUIRE_BUF16(g_dcd);
    REQUIRE_BUF16(g_dcs);
    REQUIRE(c == nullptr || ((uintptr_t)c & 15u) == 0, "c must be 16-byte aligned");
    REQUIRE(loss != nullptr && ((uintptr_t)loss & 7u) == 0, "loss must be 3 device doubles");
    REQUIRE(lambda_light >= 0.0f, "lambda_light must be >= 0");
    REQUIRE(workspace != nullptr && ((uintptr_t)workspace & 7u) == 0 && workspace_bytes >= need,
            "workspace too small: %zu < %zu bytes", workspace_bytes, need);
    return launched(mcdi::launch_image_loss(kd_out, den_cd, den_cs, ref, n, lambda_light, c, loss, g_kdout, g_dcd,
                                            g_dcs, workspace, static_cast<cudaStream_t>(stream)),
                    "image_loss");
}

mcdi_status mcdi_conv3x3_bf16(const void* x, int n_img, int H, int W, int cin_pad, const void* w, const float* bias,
                              int cout_pad, int relu, void* y, unsigned* err, void* stream) {
    REQUIRE(n_img >= 1 && H >= 1 && W >= 1 && (long long)n_img * H * W <= (1LL << 28), "bad image shape");
    REQUIRE(cin_pad >= 16 && cin_pad % 16 == 0 && cin_pad <= 1024, "cin_pad must be a multiple of 16 in [16, 1024]");
    REQUIRE(cout_pad >= 16 && cout_pad % 16 == 0 && cout_pad <= 256, "cout_pad must be a multiple of 16 in [16, 256]");
    REQUIRE(x != nullptr && ((uintptr_t)x & 15u) == 0, "x must be 16-byte aligned");
    REQUIRE(w != nullptr && ((uintptr_t)w & 15u) == 0, "w must be 16-byte aligned");
    REQUIRE(y != nullptr && ((uintptr_t)y & 15u) == 0, "y must be 16-byte aligned");
    REQUIRE(bias == nullptr || ((uintptr_t)bias & 3u) == 0, "bias must be 4-byte aligned");
    REQUIRE(err != nullptr && ((uintptr_t)err & 3u) == 0, "err must be a device uint32");
    const char* why = "";
    cudaError_t e = mcdi::launch_conv3x3(x, n_img, H, W, cin_pad, w, bias, cout_pad, relu, y, err,
                                         static_cast<cudaStream_t>(stream), &why);
    if (e == cudaErrorInvalidValue && why[0]) return fail(MCDI_DEVICE_ERROR, "conv3x3_bf16: %s", why);
    return launched(e, "conv3x3_bf16");
}

static mcdi_status wgrad_shape_ok(int n_img, int H, int W, int cin_pad, int cout_pad) {
    REQUIRE(n_img >= 1 && H >= 1 && W >= 1 && (long long)n_img * H * W <= (1LL << 28), "bad image shape");
    REQUIRE(cin_pad >= 8 && cin_pad % 8 == 0 && cin_pad <= 1024, "cin_pad must be a multiple of 8 in [8, 1024]");
    REQUIRE(cout_pad >= 16 && cout_pad % 16 == 0 && cout_pad <= 96,
            "cout_pad must be a multiple of 16 in [16, 96]");
    return ok();
}

mcdi_status mcdi_conv3x3_wgrad_bytes(int n_img, int H, int W, int cin_pad, int cout_pad, size_t* bytes) {
    mcdi_status s = wgrad_shape_ok(n_img, H, W, cin_pad, cout_pad);
    if (s != MCDI_OK) return s;
    REQUIRE(bytes != nullptr, "bytes must be non-NULL");
    *bytes = mcdi::wgrad_scratch_bytes(cin_pad, cout_pad, n_img, H, W);
    return ok();
}

mcdi_status mcdi_conv3x3_wgrad(const void* x, const void* g, int n_img, int H, int W, int cin_pad, int cout_pad,
                               int cin, int cout, float* gw, void* scratch, size_t scratch_bytes, unsigned* err,
                               void* stream) {
    mcdi_status s = wgrad_shape_ok(n_img, H, W, cin_pad, cout_pad);
    if (s != MCDI_OK) return s;
    REQUIRE(cin >= 1 && cin <= cin_pad && cout >= 1 && cout <= cout_pad, "need 1 <= cin <= cin_pad, 1 <= cout <= cout_pad");
    REQUIRE(x != nullptr && ((uintptr_t)x & 15u) == 0, "x must be 16-byte aligned");
    REQUIRE(g != nullptr && ((uintptr_t)g & 15u) == 0, "g must be 16-byte aligned");
    REQUIRE(gw != nullptr && ((uintptr_t)gw & 3u) == 0, "gw must be a device float pointer");
    const size_t need = mcdi::wgrad_scratch_bytes(cin_pad, cout_pad, n_img, H, W);
    REQUIRE(scratch != nullptr && ((uintptr_t)scratch & 255u) == 0, "scratch must be 256-byte aligned");
    REQUIRE(scratch_bytes >= need, "scratch too small: %zu < %zu bytes", scratch_bytes, need);
    REQUIRE(err != nullptr && ((uintptr_t)err & 3u) == 0, "err must be a device uint32");
    const char* why = "";
    const cudaError_t e = mcdi::launch_wgrad(x, cin_pad, g, cout_pad, n_img, H, W, cin, cout, scratch, gw, err,
                                             static_cast<cudaStream_t>(stream), &why);
    if (e == cudaErrorInvalidValue && why[0]) return fail(MCDI_DEVICE_ERROR, "conv3x3_wgrad: %s", why);
    return launched(e, "conv3x3_wgrad");
}

mcdi_status mcdi_conv3x3_e4m3(const void* x, int n_img, int H, int W, int cin_pad, const void* w, const float* x_amax,
                              const float* w_amax, const float* bias, int cout_pad, int relu, void* y, unsigned* err,
                              void* stream) {
    REQUIRE(n_img >= 1 && H >= 1 && W >= 1 && (long long)n_img * H * W <= (1LL << 28), "bad image shape");
    REQUIRE(cin_pad >= 32 && cin_pad % 32 == 0 && cin_pad <= 2048, "cin_pad must be a multiple of 32 in [32, 2048]");
    REQUIRE(cout_pad >= 16 && cout_pad % 16 == 0 && cout_pad <= 256, "cout_pad must be a multiple of 16 in [16, 256]");
    REQUIRE(x != nullptr && ((uintptr_t)x & 15u) == 0, "x must be 16-byte aligned");
    REQUIRE(w != nullptr && ((uintptr_t)w & 15u) == 0, "w must be 16-byte aligned");
    REQUIRE(y != nullptr && ((uintptr_t)y & 15u) == 0, "y must be 16-byte aligned");
    REQUIRE(x_amax != nullptr && w_amax != nullptr, "x_amax and w_amax must be device floats");
    REQUIRE(bias == nullptr || ((uintptr_t)bias & 3u) == 0, "bias must be 4-byte aligned");
    REQUIRE(err != nullptr && ((uintptr_t)err & 3u) == 0, "err must be a device uint32");
    const char* why = "";
    cudaError_t e = mcdi::launch_conv3x3_e4m3(x, n_img, H, W, cin_pad, w, x_amax, w_amax, bias, cout_pad, relu, y, err,
                                              static_cast<cudaStream_t>(stream), &why);
    if (e == cudaErrorInvalidValue && why[0]) return fail(MCDI_DEVICE_ERROR, "conv3x3_e4m3: %s", why);
    return launched(e, "conv3x3_e4m3");
}

}  // extern "C"

namespace mcdi {
thread_local bool t_graph_dependent_launch = true;
}

mcdi_status mcdi_set_graph_dependent_launch(int enable) {
    mcdi::t_graph_dependent_launch = enable != 0;
    return ok();
}

// ---- CUDA graphs with per-node priorities
mcdi_status mcdi_graph_instantiate(void* graph, void** graph_exec) {
    REQUIRE(graph != nullptr && graph_exec != nullptr, "graph / graph_exec must be non-NULL");
    *graph_exec = nullptr;
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiateWithFlags(&exec, static_cast<cudaGraph_t>(graph),
                                                        cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) return launched(e, "graph_instantiate");
    *graph_exec = exec;
    return ok();
}

mcdi_status mcdi_graph_launch(void* graph_exec, void* stream) {
    REQUIRE(graph_exec != nullptr, "graph_exec must be non-NULL");
    return launched(cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec), static_cast<cudaStream_t>(stream)),
                    "graph_launch");
}

mcdi_status mcdi_graph_destroy(void* graph_exec) {
    if (graph_exec == nullptr) return ok();
    return launched(cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec)), "graph_destroy");
}

