/*
 * mcdi.h -- C ABI of the GB300 (sm_103a) differentiable Monte Carlo
 * direct-illumination library: the shading hot path of Hasselgren, Hofmann and
 * Munkberg, "Shape, Light, and Material Decomposition from Images using Monte
 * Carlo Rendering and Denoising" (NeurIPS 2022).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an mcdi_status and never aborts, traps or prints.
 *   On failure mcdi_last_error() (per calling thread) holds a one-line reason.
 * - Every pointer argument named as a buffer is a DEVICE pointer on the
 *   current CUDA device, owned by the caller; the library keeps no reference
 *   after the call returns.  Host-side arguments are marked "host".
 * - Work is enqueued asynchronously on the caller's stream (a cudaStream_t
 *   passed as void*; NULL = the legacy default stream).  No entry point
 *   synchronises the device or allocates device memory; scratch is passed in
 *   by the caller, sized by the matching *_sizes query.
 * - float4 / int arrays are 16-byte aligned (checked: MCDI_INVALID_ARG).
 * - Images are N views x H rows x W columns, row-major, one float4 per pixel.
 * - Bad shapes, NULL buffers, misalignment or an invalid sample split give
 *   MCDI_INVALID_ARG before anything is enqueued; a failed launch gives
 *   MCDI_DEVICE_ERROR.
 */
#ifndef MCDI_H
#define MCDI_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MCDI_API __attribute__((visibility("default")))
#else
#define MCDI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MCDI_OK = 0,
    MCDI_INVALID_ARG = 1,
    MCDI_UNSUPPORTED = 2,
    MCDI_OOM = 3,
    MCDI_TIMEOUT = 4,
    MCDI_DEVICE_ERROR = 5
} mcdi_status;

/* Reason for the last failure on the calling thread ("" if none). */
MCDI_API const char* mcdi_last_error(void);

/* Library ABI version (major * 100 + minor). */
MCDI_API int mcdi_version(void);

/* ------------------------------------------------------------------------
 * Light probe sampling distribution.
 * Sec. 4.1: light importance sampling with a piecewise-constant 2D
 * distribution over the HDR probe, recomputed whenever the probe changes.
 *
 * env      [H][W] float4 lat-long probe (y up; row j spans polar angle
 *          [pi j/H, pi (j+1)/H), column i azimuth [2 pi i/W, 2 pi (i+1)/W);
 *          rgb radiance, w ignored).  1 <= W <= 8192, 1 <= H <= 4096.
 * Texel weight w_ij = max((r+g+b)/3, 0) * sin(pi (j+0.5)/H); sums in FP64.
 * cond_cdf [H][W+1] float out: cond[j][k] = sum_{i<k} w_ij / R_j, cond[j][W] = 1
 *          (uniform k/W for a black row).
 * marg_cdf [H+1]    float out: marg[k] = sum_{j<k} R_j / T, marg[H] = 1
 *          (uniform k/H for a black probe).
 * row_sum  [H]      double out: R_j.   total [1] double out: T.
 * ------------------------------------------------------------------------ */
MCDI_API mcdi_status mcdi_build_envmap_cdf(const float* env, int W, int H, float* cond_cdf, float* marg_cdf,
                                  double* row_sum, double* total, void* stream);

/* ------------------------------------------------------------------------
 * Shadow-ray acceleration structure: a linear BVH over the triangle mesh
 * extracted in each iteration (Sec. 3; the paper traces shadow rays with
 * hardware ray tracing, Sec. 6 "Compute resources").
 *
 * mcdi_bvh_sizes (host): bytes of the node array, the triangle-record array
 * and the build scratch for n_tris triangles (1 <= n_tris <= 2^27).
 * mcdi_build_bvh: verts [n_verts][3] float, tris [n_tris][3] int32 (vertex
 * indices, checked in range on the device: a bad index yields a degenerate
 * triangle, never an out-of-bounds read).  Writes `nodes` (256-byte aligned)
 * and `tri_records` (16-byte aligned), opaque layouts valid until the caller
 * frees them; `scratch` is
 * overwritten.  Build = Morton codes -> LSD radix sort -> Karras hierarchy ->
 * bottom-up bounds -> a depth-first copy with escape links, which shadow rays
 * traverse without a stack.  Deterministic for a given input.
 * ------------------------------------------------------------------------ */
MCDI_API mcdi_status mcdi_bvh_sizes(int n_tris, size_t* node_bytes, size_t* tri_bytes, size_t* scratch_bytes);
MCDI_API mcdi_status mcdi_build_bvh(const float* verts, int n_verts, const int* tris, int n_tris, void* nodes,
                           void* tri_records, void* scratch, size_t scratch_bytes, void* stream);

/* Number of kernels mcdi_build_bvh launches for n_tris triangles (the Morton
 * keys of a mesh of up to 262,144 triangles are sorted by one kernel per radix
 * pass, of larger meshes by three).  For launch accounting; no device work. */
MCDI_API mcdi_status mcdi_bvh_build_launches(int n_tris, int* launches);

/* ------------------------------------------------------------------------
 * mcdi_refit_bvh: bounds-only update for a mesh whose vertices moved but
 * whose triangles (the tris array and n_tris) are those of the last
 * mcdi_build_bvh into the same nodes, tri_records and scratch (for example
 * the fixed-topology stage of a reconstruction, where each iteration moves
 * vertices only).  The leaf order and hierarchy of that build are kept; the
 * triangle records, every box and the depth-first copy are recomputed from
 * `verts`, so traversal results are exact for the new positions, while the
 * tree's quality degrades as vertices move away from where it was built.
 * `scratch` must hold what that build left there (do not reuse it in
 * between; mcdi_build_bvh_noalloc leaves nothing to refit).  Arguments and
 * errors as mcdi_build_bvh.
 * ------------------------------------------------------------------------ */
MCDI_API mcdi_status mcdi_refit_bvh(const float* verts, int n_verts, const int* tris, int n_tris, void* nodes,
                           void* tri_records, void* scratch, size_t scratch_bytes, void* stream);

/* ------------------------------------------------------------------------
 * mcdi_build_bvh_noalloc: the same build as mcdi_build_bvh (identical nodes
 * and triangle records for the same mesh) with no scratch argument.  The
 * paper has no counterpart; this entry point exists for callers that cannot
 * allocate device memory themselves, for example a plugin running inside a
 * host application that owns every device allocation, or a request loop
 * whose memory budget is fixed at start-up and may not grow (cudaMalloc can
 * also block on the device, which such loops cannot afford).
 * Scratch lives in one fixed device array inside the library (7 MB,
 * held on every GPU that loads the library until the process exits); the
 * first call on a device looks up its address on that device, so make that
 * first call before any stream capture.  The call allocates and frees
 * nothing.  n_tris is limited to MCDI_NOALLOC_MAX_TRIS (larger meshes give
 * MCDI_INVALID_ARG: use mcdi_build_bvh).  All calls share the array: calls
 * whose work overlaps on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  Other arguments as mcdi_build_bvh.
 * ------------------------------------------------------------------------ */
#define MCDI_NOALLOC_MAX_TRIS 65536
MCDI_API mcdi_status mcdi_build_bvh_noalloc(const float* verts, int n_verts, const int* tris, int n_tris,
                                            void* nodes, void* tri_records, void* stream);

/* A built BVH as the shading kernels read it (host struct, device pointers). */
typedef struct {
    const void* nodes;
    const void* tri_records;
    int n_tris;
} mcdi_bvh_view;

/* Pinhole camera (14 floats): origin, right, up, forward (orthonormal),
 * tan(fovy/2), aspect = W/H.  Pixel (x, y), y down, looks along
 * normalize(forward + sx right + sy up), sx = (2(x+.5)/W - 1) tan aspect,
 * sy = (1 - 2(y+.5)/H) tan. */
typedef struct {
    float origin[3], right[3], up[3], forward[3];
    float tan_half_fovy, aspect;
} mcdi_camera;

/* ------------------------------------------------------------------------
 * Primary visibility -> G-buffer.  The paper rasterises it (nvdiffrast,
 * Sec. 3.1); this closest-hit ray cast on the same BVH stands in.
 * cams [N] mcdi_camera (device).  Hit: position and normal are barycentric
 * interpolations of verts / vnrm ([n_verts][3] float); k_d and k_orm are
 * bilinear, clamp-to-edge lookups of tex_kd / tex_korm ([S][S] float4) at the
 * planar coordinate ((x - uvmap[0]) uvmap[2], (z - uvmap[1]) uvmap[2])
 * (uvmap: host, 3 floats).  Outputs [N][H][W] float4:
 *   gb_pos (x, y, z, coverage), gb_nrm (N, 0), gb_kd (r, g, b, 0),
 *   gb_korm (o, r, m, 0); a miss writes zeros.
 * ------------------------------------------------------------------------ */
MCDI_API mcdi_status mcdi_primary_cast(const mcdi_bvh_view* bvh, const float* verts, const float* vnrm, const int* tris,
                              int n_verts, const mcdi_camera* cams, int N, int H, int W, const float* tex_kd,
                              const float* tex_korm, int tex_size, const float* uvmap, float* gb_pos,
                              float* gb_nrm, float* gb_kd, float* gb_korm, void* stream);

/* ------------------------------------------------------------------------
 * The same G-buffer by rasterisation, as the paper produces it (nvdiffrast,
 * Sec. 3.1), from the mesh alone (verts [n_verts][3], tris [n_tris][3]; no
 * BVH, so it can run concurrently with mcdi_build_bvh).  Every triangle is
 * scan-converted over its screen box, clipped at a near plane 1e-6 in front
 * of the eye; each pixel of the box is decided by the ray cast's own FP32 test
 * of the camera ray through the pixel centre against v0, v1 - v0, v2 - v0, so
 * it covers the pixels the ray cast covers with the same triangles; the
 * attributes agree with the ray cast's to FP32 rounding.  The nearest hit
 * wins (ties: the lowest triangle index); its entries are written as by
 * mcdi_primary_cast.  workspace: mcdi_raster_workspace_size(N, H, W) bytes,
 * 256-byte aligned (a 64-bit depth buffer), overwritten.
 * ------------------------------------------------------------------------ */
MCDI_API mcdi_status mcdi_raster_workspace_size(int N, int H, int W, size_t* bytes);
MCDI_API mcdi_status mcdi_raster_gbuffer(const float* verts, const float* vnrm, const int* tris, int n_verts,
                                         int n_tris, const mcdi_camera* cams, int N, int H, int W,
                                         const float* tex_kd, const float* tex_korm, int tex_size, const float* uvmap,
                                         float* gb_pos, float* gb_nrm, float* gb_kd, float* gb_korm, void* workspace,
                                         size_t workspace_bytes, void* stream);

/* mcdi_raster_gbuffer in two calls on the same workspace, so that the depth
 * pass can run before the material textures are in device memory (for
 * example while they are still being copied from the host): part 1 (depth)
 * scan-converts the mesh into the workspace's depth buffer and reads only
 * verts, tris and cams; part 2 (resolve), on a stream ordered after part 1,
 * interpolates the winning triangle's attributes, looks up tex_kd / tex_korm
 * and writes the four G-buffer planes.  tex_channels: 4 = [S][S] float4 (the
 * 4th channel unused; 16-byte aligned), as mcdi_raster_gbuffer; 3 = packed
 * [S][S][3] float (k_d RGB, k_orm = occlusion, roughness, metallic; 4-byte
 * aligned), a quarter fewer bytes to copy from the host; both give the same
 * G-buffer bit for bit.  Other arguments as mcdi_raster_gbuffer; both parts
 * must receive the same ones.  Any other part or tex_channels:
 * MCDI_INVALID_ARG. */
MCDI_API mcdi_status mcdi_raster_gbuffer_part(const float* verts, const float* vnrm, const int* tris, int n_verts,
                                              int n_tris, const mcdi_camera* cams, int N, int H, int W,
                                              const float* tex_kd, const float* tex_korm, int tex_size,
                                              int tex_channels, const float* uvmap, float* gb_pos, float* gb_nrm,
                                              float* gb_kd, float* gb_korm, void* workspace, size_t workspace_bytes,
                                              int part, void* stream);

/* Sampling and shading parameters (host struct). */
typedef struct {
    int n_light;              /* samples of the probe distribution            */
    int n_cos;                /* cosine-weighted samples (diffuse lobe)       */
    int n_ggx;                /* GGX visible-normal samples (specular lobe)   */
    int decorrelate_bwd;      /* 1: backward draws its own samples (App. D)   */
    unsigned long long seed;  /* Philox4x32-10 key                            */
    float tau;                /* shadow leakage, H = 1 - tau on a hit (App. A) */
    float ray_eps;            /* shadow-ray origin offset along the normal    */
} mcdi_shade_params;

/* ------------------------------------------------------------------------
 * Forward Monte Carlo direct illumination (Sec. 3.1 estimator, Sec. 4.1 MIS
 * with the balance heuristic, Sec. 4.2 light separation).
 *
 * Per covered pixel, spp = n_light + n_cos + n_ggx samples (1 <= spp <= 1024;
 * sample j < n_light is a probe sample, then n_cos cosine, then n_ggx GGX).
 * Sample j draws two 24-bit uniforms from Philox4x32-10 with key = seed and
 * counter = (pixel index y*W + x, view, j, 0).  Each sample contributes
 *   g(w) / sum_k n_k p_k(w),   g = L(w) H(w) f(w, wo) (n.w)^+,
 * split into c_d (L H (n.w)/pi, demodulated diffuse) and c_s (specular GGX,
 * alpha = max(r^2, 1e-4), Smith height-correlated masking, Schlick Fresnel
 * with F0 = 0.04 (1 - m) + k_d m); kd_out = k_d (1 - m).  Shadow rays start
 * at p + ray_eps n and test every triangle (two-sided, t > 0); the probe is
 * looked up at the nearest texel.
 *
 * Inputs: G-buffer planes [N][H][W] float4 as written by mcdi_primary_cast;
 * env [Hp][Wp] float4; the three tables of mcdi_build_envmap_cdf (total is
 * read on the device); cams [N] (origins give the view vectors).
 * Outputs [N][H][W] float4 (w = 0): c_d, kd_out, c_s.
 * vis_mask (nullable) [N][H][W][ceil(spp/32)] uint32: bit j = sample j's
 * shadow ray was blocked; the backward pass can reuse it.
 * workspace (nullable): scratch of mcdi_shade_workspace_size bytes (256-byte
 * aligned, overwritten).  With it the forward runs as three kernels (sample
 * generation, a persistent shadow-ray tracer, accumulation; N*H*W*spp must
 * stay below 2^31); with NULL it runs as one fused kernel.  Both give the same
 * samples and visibility; sums agree to FP32 rounding.
 * ------------------------------------------------------------------------ */
MCDI_API mcdi_status mcdi_shade_workspace_size(int N, int H, int W, const mcdi_shade_params* params,
                                               size_t* bytes);
MCDI_API mcdi_status mcdi_shade_mc_fwd(const mcdi_bvh_view* bvh, const float* env, int Wp, int Hp,
                                       const float* cond_cdf, const float* marg_cdf, const double* total,
                                       const float* gb_pos, const float* gb_nrm, const float* gb_kd,
                                       const float* gb_korm, const mcdi_camera* cams, int N, int H, int W,
                                       const mcdi_shade_params* params, float* c_d, float* kd_out, float* c_s,
                                       uint32_t* vis_mask, void* workspace, size_t workspace_bytes, void* stream);

/* mcdi_shade_mc_fwd in two calls on the same workspace (required), so that
 * the sample generation, which reads no BVH, can run while the BVH is still
 * being built: part 1 draws every sample (Sec. 3.1 estimator, Sec. 4.1 MIS)
 * and writes kd_out, the shadow rays and the unshadowed contributions to
 * `workspace` (bvh may be the view of a BVH not built yet: its buffers are
 * not read); part 2, on a stream ordered after part 1 and after the BVH
 * build, traces the shadow rays and writes c_d, c_s and vis_mask.  Arguments
 * as mcdi_shade_mc_fwd; both parts must receive the same ones. */
MCDI_API mcdi_status mcdi_shade_mc_fwd_part(const mcdi_bvh_view* bvh, const float* env, int Wp, int Hp,
                                            const float* cond_cdf, const float* marg_cdf, const double* total,
                                            const float* gb_pos, const float* gb_nrm, const float* gb_kd,
                                            const float* gb_korm, const mcdi_camera* cams, int N, int H, int W,
                                            const mcdi_shade_params* params, float* c_d, float* kd_out, float* c_s,
                                            uint32_t* vis_mask, void* workspace, size_t workspace_bytes, int part,
                                            void* stream);

/* ------------------------------------------------------------------------
 * Hand-written adjoint of mcdi_shade_mc_fwd (Sec. 4.1: detached importance
 * sampling, the forward seed reused in the backward pass; Sec. 3.1: shadow
 * visibility detached).  Samples are regenerated from the same Philox
 * counters (stream word 1 instead of 0 when decorrelate_bwd is set), sample
 * directions, MIS denominators and visibility are held constant, and the
 * gradient of  sum <g_cd, c_d> + <g_kdout, kd_out> + <g_cs, c_s>  is taken
 * with respect to the G-buffer normal (before normalisation), k_d, k_orm and
 * the probe texels.
 *
 * Same scene / G-buffer / table / camera inputs and params as the forward.
 * g_cd, g_kdout, g_cs: [N][H][W] float4 upstream gradients.
 * vis_mask: the forward's mask (reused when not decorrelating), or NULL to
 *           re-trace the shadow rays.
 * Outputs (overwritten) [N][H][W] float4: g_kd (rgb), g_korm (o = 0, r, m),
 * g_nrm (xyz).  g_env [Hp][Wp] float4 is ACCUMULATED (rgb; zero it first).
 * ------------------------------------------------------------------------ */
MCDI_API mcdi_status mcdi_shade_mc_bwd(const mcdi_bvh_view* bvh, const float* env, int Wp, int Hp, const float* cond_cdf,
                              const float* marg_cdf, const double* total, const float* gb_pos,
                              const float* gb_nrm, const float* gb_kd, const float* gb_korm,
                              const mcdi_camera* cams, int N, int H, int W, const mcdi_shade_params* params,
                              const float* g_cd, const float* g_kdout, const float* g_cs,
                              const uint32_t* vis_mask, float* g_kd, float* g_korm, float* g_nrm, float* g_env,
                              void* stream);

/* mcdi_shade_mc_bwd restricted to the pixels [first, first + count) of the
 * flattened [N][H][W] image (index (view H + y) W + x): writes g_kd, g_korm
 * and g_nrm of those pixels only and accumulates their probe-texel gradients
 * into g_env.  Every pixel's gradient is computed alone, so calls over
 * disjoint spans that cover the image write the per-pixel outputs of one
 * mcdi_shade_mc_bwd bit for bit (g_env: the same sum in another atomic
 * order); a caller can then read back each span's outputs while the next span
 * runs.  count = 0 launches nothing.  A span outside the image or count < 0:
 * MCDI_INVALID_ARG.  Other arguments as mcdi_shade_mc_bwd. */
MCDI_API mcdi_status mcdi_shade_mc_bwd_span(const mcdi_bvh_view* bvh, const float* env, int Wp, int Hp,
                                            const float* cond_cdf, const float* marg_cdf, const double* total,
                                            const float* gb_pos, const float* gb_nrm, const float* gb_kd,
                                            const float* gb_korm, const mcdi_camera* cams, int N, int H, int W,
                                            const mcdi_shade_params* params, const float* g_cd,
                                            const float* g_kdout, const float* g_cs, const uint32_t* vis_mask,
                                            float* g_kd, float* g_korm, float* g_nrm, float* g_env, long long first,
                                            long long count, void* stream);

/* ------------------------------------------------------------------------
 * Shadow-visibility gradients (the ablation of the paper's appendix
 * "Visibility gradients from shadows"; off in the paper's main results, where
 * visibility is detached, Sec. 3.1 "Shadow gradients").  The gradient of
 *   sum <g_cd, c_d> + <g_cs, c_s>
 * with respect to the mesh's vertex positions through the shadow rays'
 * blocked set: with H = 1 - tau B, the boundary term
 *   -tau sum over silhouette edges (seen from o = p + ray_eps n) of
 *    int_0^1 g(w) V+ n_out . ((1 - s) da + s db) |w x (b - a)| / r^2 ds,
 * x = a + s (b - a), r = |x - o|, w = (x - o) / r, n_out the unit normal of
 * the plane (o, a, b) away from the edge's faces, V+ = 1 when the ray along
 * normalize(w + eta n_out) reaches the probe, and g the forward integrand
 * L(w) (n.w) [g_cd / pi + g_cs f_s(w)] (specular only where the lobe is on).
 * An edge is on the silhouette when its two faces lie strictly on one side of
 * that plane, or when it has one face.  Estimated by edge sampling: each pixel
 * draws n_edge_samples edges uniformly, edge e = floor(u0 E) computed as
 * ((x0 >> 8) * E) >> 24 from the Philox output x0 of counter (pixel, view, j,
 * 2) (the forward uses stream word 0, a decorrelated adjoint 1), s = u1, and
 * weighs each by E / n_edge_samples.
 *
 * mcdi_edge_table_workspace_size (host): scratch bytes for n_tris triangles.
 * mcdi_build_edge_table: tris [n_tris][3] int32 (indices in [0, n_verts)) ->
 *   edges [3 n_tris][4] int32 (capacity for every half-edge; 16-byte
 *   aligned): one record (a, b, c1, c2) per undirected edge in the order of
 *   its first half-edge 3 t + i (a = v_i, b = v_(i+1), c1 = v_(i+2) of that
 *   face, c2 the opposite vertex of the next face on the edge or -1 on a
 *   boundary; further faces of a non-manifold edge are ignored), and
 *   *n_edges (device int) the number of records, or -1 if the hash table
 *   overflowed (it cannot with the scratch size given above).  Deterministic.
 * mcdi_shadow_edge_grad: bvh and verts [n_verts][3] float (4-byte aligned) of
 *   the same mesh, the edge table (edges, n_edges on the device, max_edges its
 *   capacity in records), the probe and the G-buffer / cameras of the
 *   forward, params (seed, tau and ray_eps are used), n_edge_samples >= 0,
 *   0 < eta <= 0.1, g_cd and g_cs [N][H][W] float4.  g_verts [n_verts][3]
 *   float is ACCUMULATED (zero it first).  sample_w (nullable) [N][H][W]
 *   [n_edge_samples] float receives each sample's weight
 *   -tau g J E / n_edge_samples (0 when the sample does not contribute).
 *   Edge records whose indices are out of range are skipped.
 * ------------------------------------------------------------------------ */
MCDI_API mcdi_status mcdi_edge_table_workspace_size(int n_tris, size_t* bytes);
MCDI_API mcdi_status mcdi_build_edge_table(const int* tris, int n_tris, int* edges, int* n_edges, void* workspace,
                                           size_t workspace_bytes, void* stream);
MCDI_API mcdi_status mcdi_shadow_edge_grad(const mcdi_bvh_view* bvh, const float* verts, int n_verts,
                                           const int* edges, const int* n_edges, int max_edges, const float* env,
                                           int Wp, int Hp, const float* gb_pos, const float* gb_nrm,
                                           const float* gb_kd, const float* gb_korm, const mcdi_camera* cams, int N,
                                           int H, int W, const mcdi_shade_params* params, int n_edge_samples,
                                           float eta, const float* g_cd, const float* g_cs, float* g_verts,
                                           float* sample_w, void* stream);

/* ------------------------------------------------------------------------
 * Measurement aids for the shadow-ray traversal (the visibility term of the
 * Sec. 3.1 estimator, traced as in App. A), not part of the hot path.  Both
 * take the BVH, image shape and params of a preceding mcdi_shade_mc_fwd that
 * ran with `workspace` (its compacted shadow rays are still there) and launch
 * on `stream` after it.
 *
 * mcdi_shadow_ray_stats re-traces those rays one per thread with counters and
 * OVERWRITES stats[5] (device, 8-byte aligned): [0] rays, [1] node visits
 * (one 32-byte node fetch and one slab test each), [2] triangle tests (48-byte
 * triangle record fetch each), [3] rays blocked, [4] rays whose result differs
 * from the forward pass's (0 when the two traversals agree).
 *
 * mcdi_shadow_ray_retrace runs the forward pass's tracer kernel again over
 * the same rays (it sets the same hit flags, so the forward's outputs and the
 * workspace stay valid): the tracer timed on its own.
 *
 * mcdi_read_sweep reads `bytes` (a multiple of 16, buf 16-byte aligned) of
 * device memory `passes` times with L2-cached, L1-bypassing 16-byte loads;
 * *sink (device) is written only in a case that does not occur for real data.
 * Timed over a buffer that fits in L2 it measures the L2 read bandwidth.
 * ------------------------------------------------------------------------ */
MCDI_API mcdi_status mcdi_shadow_ray_stats(const mcdi_bvh_view* bvh, int N, int H, int W,
                                           const mcdi_shade_params* params, const void* workspace,
                                           size_t workspace_bytes, unsigned long long* stats, void* stream);
MCDI_API mcdi_status mcdi_shadow_ray_retrace(const mcdi_bvh_view* bvh, int N, int H, int W,
                                             const mcdi_shade_params* params, void* workspace,
                                             size_t workspace_bytes, void* stream);
MCDI_API mcdi_status mcdi_read_sweep(const void* buf, size_t bytes, int passes, unsigned* sink, void* stream);

/* ------------------------------------------------------------------------
 * Differentiable denoiser (Sec. 4.2 "Neural denoisers": a U-Net applied to
 * the demodulated diffuse and the specular terms separately; App. B).
 * The network: widths 32/48/64/96 over four levels, two 3x3 zero-padded
 * convolutions with ReLU per level, 2x2 max-pool down, nearest 2x upsample
 * and [upsampled, skip] concatenation up, a final linear 3x3 convolution to
 * 3 channels.  Input per image: 9 channels = term rgb, k_d rgb, normal xyz.
 * Convolutions run on the tcgen05 tensor cores with FP32 accumulation and
 * operands of the chosen precision: MCDI_DENOISE_BF16, or MCDI_DENOISE_E4M3
 * (FP8 E4M3 with per-tensor scaling: each convolution's input and weights are
 * quantised as round-to-nearest-even, saturating, of v * 448 / amax, and the
 * accumulator is rescaled by (amax_x / 448) (amax_w / 448)).  Activations
 * and gradients are stored as BF16 in both modes.
 *
 * mcdi_denoise_sizes (host): bytes of the packed weights (both precisions),
 * of the forward's saved activations and of the backward's gradient scratch
 * for n_img images of H x W (H, W multiples of 8) in `precision`, and the
 * number of FP32 parameters.
 * mcdi_denoise_pack_weights: params (device, FP32, for each of the 15
 * convolutions in order enc1a enc1b enc2a enc2b enc3a enc3b bot_a bot_b dec3a
 * dec3b dec2a dec2b dec1a dec1b out: W[co][ci][3][3] then b[co]) -> weights.
 * mcdi_denoise_fwd: term [n_img][H][W] float4, kd and nrm [n_aux][H][W]
 * float4 (image i uses guide i % n_aux) -> y [n_img][H][W] float4 (rgb, w=0);
 * acts (act_bytes) receives the activations the backward needs.
 * mcdi_denoise_bwd: gy [n_img][H][W] float4 -> gx [n_img][H][W] float4, the
 * gradient with respect to the term channels; acts from a forward of the
 * same precision.  grad_ws keeps every intermediate gradient for
 * mcdi_denoise_wgrad.  err: device uint32 the kernels set to 1 if a pipeline
 * wait timed out (zero it before the call; outputs are then invalid).
 *
 * Weight gradient (the live-trained denoiser of App. B; the main results of
 * Sec. 4.2 lock the weights and need none):
 * mcdi_denoise_wgrad_bytes (host): scratch bytes mcdi_denoise_wgrad needs for
 * n_img images of H x W.
 * mcdi_denoise_wgrad: after mcdi_denoise_fwd (acts) and mcdi_denoise_bwd
 * (grad_ws) of the same images, precision and sizes, writes gw (device FP32,
 * n_params values in the order of mcdi_denoise_pack_weights' params:
 * dL/dW[co][ci][3][3] then dL/db[co] per convolution) for the loss whose
 * gradient gy mcdi_denoise_bwd received.  Every entry is overwritten (no
 * accumulation into gw).  Computed on the tensor cores from the BF16-stored
 * activations and gradients with FP32 accumulation; with E4M3 operands the
 * stored BF16 tensors are used (the quantisers pass gradients straight
 * through).  Results are bitwise repeatable for a given GPU.  scratch:
 * device, 256-byte aligned, scratch_bytes from mcdi_denoise_wgrad_bytes; acts
 * and grad_ws are only read.  err as for mcdi_denoise_bwd.
 * ------------------------------------------------------------------------ */
#define MCDI_DENOISE_BF16 0
#define MCDI_DENOISE_E4M3 1
MCDI_API mcdi_status mcdi_denoise_sizes(int n_img, int H, int W, int precision, size_t* weight_bytes,
                                        size_t* act_bytes, size_t* grad_bytes, size_t* n_params);
MCDI_API mcdi_status mcdi_denoise_pack_weights(const float* params, void* weights, void* stream);
MCDI_API mcdi_status mcdi_denoise_fwd(const void* weights, int precision, int n_img, int H, int W, const float* term,
                                      const float* kd, const float* nrm, int n_aux, float* y, void* acts,
                                      size_t act_bytes, unsigned* err, void* stream);
MCDI_API mcdi_status mcdi_denoise_bwd(const void* weights, int precision, int n_img, int H, int W, const void* acts,
                                      size_t act_bytes, const float* gy, float* gx, void* grad_ws,
                                      size_t grad_bytes, unsigned* err, void* stream);

MCDI_API mcdi_status mcdi_denoise_wgrad_bytes(int n_img, int H, int W, size_t* scratch_bytes);
MCDI_API mcdi_status mcdi_denoise_wgrad(int precision, int n_img, int H, int W, const void* acts, size_t act_bytes,
                                        const void* grad_ws, size_t grad_bytes, float* gw, void* scratch,
                                        size_t scratch_bytes, unsigned* err, void* stream);

/* mcdi_denoise_record_plan (host; a measurement and test aid, not on the
 * hot path): while rec is non-NULL, each convolution that mcdi_denoise_fwd /
 * mcdi_denoise_bwd launch from the calling host thread appends one record of
 * 8 ints to rec (host memory, room for cap records; later ones are dropped):
 *   {pass (0 forward, 1 input gradient), convolution index 0..14 (the order of
 *    mcdi_denoise_pack_weights), level (0 = full resolution), row-tile form
 *    (1) or one CTA per 128-pixel tile (0), output rows per row tile R (0 in
 *    the tile form), ReLU-mask prefetching variant (0/1), 2x2 max-pool written
 *    from the epilogue (0/1), E4M3 operands (0/1)};
 * *count (host) is reset to 0 by this call and counts the records written.
 * mcdi_denoise_record_plan(NULL, 0, NULL) stops recording.  The records say
 * which kernel variants a launch configuration runs. */
MCDI_API mcdi_status mcdi_denoise_record_plan(int* rec, int cap, int* count);

/* Final colour (Sec. 4.2): c = kd_out * D(c_d) + D(c_s), n pixels of float4
 * planes (w of c = 0). */
MCDI_API mcdi_status mcdi_composite(const float* kd_out, const float* den_cd, const float* den_cs, long long n,
                                    float* c, void* stream);

/* ------------------------------------------------------------------------
 * Cross-bilateral denoiser (App. B "Bilateral Denoiser": the spatial part of
 * SVGF, evaluated densely over the footprint; gradients to the colours only):
 *   c_hat(p) = sum_q c(q) w(p, q) / W(p),  W(p) = sum_q w(p, q)
 *   w(p, q)  = exp(-|p - q|^2 / (2 sigma^2))
 *            * exp(-|z(p) - z(q)| / (|grad z(p) . (p - q)| + 1e-3 z(p)))
 *            * max(0, n(p) . n(q))^128
 * (sigma_z = 1, sigma_n = 128 as in the paper), q over the square of radius
 * `radius` (< 0: ceil(2 sigma); at most 8) inside the image.  z = (pos - eye)
 * . forward of the view's camera, grad z the central difference over covered
 * neighbours (one-sided at borders and coverage edges), n the normalised
 * G-buffer normal.  Uncovered pixels (gb_pos.w = 0) pass through and are
 * never neighbours.
 * gb_pos, gb_nrm [N][H][W] float4 and cams [N] (device): the guides of N
 * views; the batch c_in / c_out [n_img][H][W] float4 (rgb; w written 0)
 * holds n_img = K N images, image i filtered with the guides of view i % N,
 * 1 <= K <= 4.  wsum [N][H][W] float: W(p) written by the forward, read by
 * the backward.  mcdi_bilateral_bwd: g_in = dL/dc_in from g_out = dL/dc_hat
 * (overwritten; deterministic, no atomics).  sigma in (0, 8].
 * ------------------------------------------------------------------------ */
MCDI_API mcdi_status mcdi_bilateral_fwd(const float* gb_pos, const float* gb_nrm, const mcdi_camera* cams, int N,
                                        int H, int W, int n_img, const float* c_in, float sigma, int radius,
                                        float* c_out, float* wsum, void* stream);
MCDI_API mcdi_status mcdi_bilateral_bwd(const float* gb_pos, const float* gb_nrm, const mcdi_camera* cams, int N,
                                        int H, int W, int n_img, const float* wsum, const float* g_out, float sigma,
                                        int radius, float* g_in, void* stream);

/* ------------------------------------------------------------------------
 * Image loss of the optimisation step, fused with the composite and its
 * adjoint (App. A "Image Loss", "Regularizers"; Sec. 4.2 composite):
 *   c       = kd_out * den_cd + den_cs
 *   T(x)    = sRGB(log(max(x, 0) + 1))   (negative radiance clamps to 0)
 *   L_image = mean over the n pixels and 3 channels of |T(c) - T(ref)|
 *   L_light = mean over the n pixels of |Y(T(den_cd + den_cs)) - V(T(ref))|,
 *             Y = (r + g + b) / 3, V = max(r, g, b)
 *   L       = L_image + lambda_light * L_light      (the paper uses 0.15)
 * kd_out, den_cd, den_cs, ref: n pixels of float4 (rgb, w ignored).
 * Outputs: c (nullable) the composite; loss (device, 3 doubles) = (L,
 * L_image, L_light); g_kdout, g_dcd, g_dcs (overwritten, w = 0) = dL/d of
 * the three inputs (|0| has zero gradient).  Deterministic: FP64 partial
 * sums per block in `workspace` (mcdi_image_loss_workspace_size bytes),
 * added in a fixed order.
 * ------------------------------------------------------------------------ */
MCDI_API mcdi_status mcdi_image_loss_workspace_size(long long n, size_t* bytes);
MCDI_API mcdi_status mcdi_image_loss(const float* kd_out, const float* den_cd, const float* den_cs, const float* ref,
                                     long long n, float lambda_light, float* c, double* loss, float* g_kdout,
                                     float* g_dcd, float* g_dcs, void* workspace, size_t workspace_bytes,
                                     void* stream);

/* One 3x3 convolution layer of the denoiser on its own (same kernels):
 * activations are BF16 in 8-channel planes, the layout the denoiser keeps
 * them in: channel c of pixel (x, y) of image i is element
 * (((i * C/8 + c/8) * H + y) * W + x) * 8 + c % 8 of a C-channel tensor.
 * x: cin_pad channels, w [cout_pad][9][cin_pad] BF16 (tap = 3 ky + kx,
 * cross-correlation, zero padding 1), bias [cout_pad] FP32 (nullable),
 * y: cout_pad channels = act(conv + bias), act = ReLU if relu else identity.
 * cin_pad, cout_pad multiples of 16, cout_pad <= 256. */
MCDI_API mcdi_status mcdi_conv3x3_bf16(const void* x, int n_img, int H, int W, int cin_pad, const void* w,
                                       const float* bias, int cout_pad, int relu, void* y, unsigned* err,
                                       void* stream);

/* Weight gradient of one such layer (the kernels of mcdi_denoise_wgrad):
 * x: cin_pad channels, g: cout_pad channels (the gradient at the layer's
 * pre-activation output), both BF16 8-channel planes as above; gw (device
 * FP32) receives dW[co][ci][ky][kx] = sum over images and pixels p of
 * g[co](p) x[ci](p + (ky - 1, kx - 1)) (x zero outside the image) for
 * co < cout, ci < cin, then db[co] = sum over images and pixels of g[co]:
 * cout * cin * 9 + cout floats, every one overwritten.  cin <= cin_pad (a
 * multiple of 8, <= 1024), cout <= cout_pad (a multiple of 16, <= 96).
 * scratch: device, 256-byte aligned, mcdi_conv3x3_wgrad_bytes bytes. */
MCDI_API mcdi_status mcdi_conv3x3_wgrad_bytes(int n_img, int H, int W, int cin_pad, int cout_pad, size_t* bytes);
MCDI_API mcdi_status mcdi_conv3x3_wgrad(const void* x, const void* g, int n_img, int H, int W, int cin_pad,
                                        int cout_pad, int cin, int cout, float* gw, void* scratch,
                                        size_t scratch_bytes, unsigned* err, void* stream);

/* The same layer with E4M3 operands (the denoiser's FP8 path): x holds E4M3
 * codes in 16-channel planes (element (((i * C/16 + c/16) * H + y) * W + x)
 * * 16 + c % 16, one byte each), w [cout_pad][9][cin_pad] E4M3 codes;
 * x_amax, w_amax (device float) give the scales: y = act(conv(x) *
 * (x_amax / 448) * (w_amax / 448) + bias) as BF16 8-channel planes.
 * cin_pad a multiple of 32, cout_pad a multiple of 16, <= 256. */
MCDI_API mcdi_status mcdi_conv3x3_e4m3(const void* x, int n_img, int H, int W, int cin_pad, const void* w,
                                       const float* x_amax, const float* w_amax, const float* bias, int cout_pad,
                                       int relu, void* y, unsigned* err, void* stream);

/* ------------------------------------------------------------------------
 * CUDA graphs whose nodes run at their own priorities (runtime support, no
 * counterpart in the paper).  A graph captured from streams of different
 * priorities records each kernel node's priority (the library's kernels carry
 * their stream's priority as a launch attribute); a graph instantiated
 * without cudaGraphInstantiateFlagUseNodePriority runs every node at the
 * priority of the stream it is launched into, so the block scheduler cannot
 * favour, for example, the BVH build's chain of small kernels over the
 * sample generation beside it.
 * mcdi_graph_instantiate: graph = a cudaGraph_t (for instance a kept graph of
 *   torch.cuda.CUDAGraph(keep_graph=True)); the caller keeps it alive (and
 *   every buffer its nodes use) while the instance exists.  *graph_exec
 *   receives a cudaGraphExec_t instantiated with node priorities (NULL on
 *   error).  Instantiation failure: MCDI_DEVICE_ERROR.
 * mcdi_graph_launch: launches the instance into `stream` (cudaGraphLaunch).
 * mcdi_graph_destroy: frees the instance (NULL is a no-op).
 * ------------------------------------------------------------------------ */
MCDI_API mcdi_status mcdi_graph_instantiate(void* graph, void** graph_exec);
MCDI_API mcdi_status mcdi_graph_launch(void* graph_exec, void* stream);
MCDI_API mcdi_status mcdi_graph_destroy(void* graph_exec);

/* Whether the denoiser's convolutions launched by the calling thread into a
 * stream that is being captured keep their programmatic dependence on the
 * kernel before them (enable != 0, the default: their tensor-memory
 * allocation and weight load then overlap that kernel's tail in the replay)
 * or are captured like every other kernel (0).  Graphs replayed concurrently
 * with other work (several requests on several streams) can run better
 * without it, since a dependent launch's blocks hold SM slots while they wait.
 * Applies to launches made after the call, on this thread only; launches
 * outside capture are unaffected.  Always MCDI_OK. */
MCDI_API mcdi_status mcdi_set_graph_dependent_launch(int enable);

#ifdef __cplusplus
}
#endif

#endif /* MCDI_H */
