// Shading kernels: the G-buffer ray cast, the forward MIS estimator and its
// hand-written adjoint (Sec. 3.1, Sec. 4.1, Sec. 4.2).  One thread shades one
// pixel with all of its samples; G-buffer planes are read and outputs written
// as coalesced float4.
#include "common.cuh"
#include "internal.h"
#include "shading.cuh"

namespace mcdi {
namespace {

constexpr int kShadeThreads = 128;

__device__ __forceinline__ Probe make_probe(const ShadeArgs& a) {
    Probe P;
    P.env = a.env;
    P.cond = a.cond;
    P.marg = a.marg;
    P.W = a.Wp;
    P.H = a.Hp;
    P.on = *a.total > 0.0;
    return P;
}

__device__ __forceinline__ f3 cam_origin(const mcdi_camera* cams, int view) {
    return mk(cams[view].origin[0], cams[view].origin[1], cams[view].origin[2]);
}

// ---------------------------------------------------------------- G-buffer
__global__ void __launch_bounds__(kShadeThreads) primary_cast_kernel(
    const BvhNode* __restrict__ nodes, const TriRecord* __restrict__ tris, int n_tris, const float* __restrict__ verts,
    const float* __restrict__ vnrm, const int* __restrict__ tri_idx, int n_verts, const mcdi_camera* __restrict__ cams,
    int N, int H, int W, const float4* __restrict__ tex_kd, const float4* __restrict__ tex_korm, int S, float uv_ox,
    float uv_oz, float uv_s, float4* __restrict__ gb_pos, float4* __restrict__ gb_nrm, float4* __restrict__ gb_kd,
    float4* __restrict__ gb_korm) {
    pdl_prologue();
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * H * W) return;
    const int view = (int)(idx / ((long long)H * W));
    const int pix = (int)(idx - (long long)view * H * W);
    const int x = pix % W, y = pix / W;
    const mcdi_camera& C = cams[view];
    const f3 o = mk(C.origin[0], C.origin[1], C.origin[2]);
    const f3 d = camera_dir(C, x, y, W, H);
    float t, u = 0.f, v = 0.f;
    const int leaf = closest_hit(nodes, tris, n_tris, make_ray(o, d), &t, &u, &v);
    float4 P = make_float4(0.f, 0.f, 0.f, 0.f), Nn = P, KD = P, KORM = P;
    if (leaf >= 0)
        gbuffer_hit(__float_as_int(__ldg(&tris[leaf].v0.w)), u, v, verts, vnrm, tri_idx, n_verts,
                    reinterpret_cast<const float*>(tex_kd), reinterpret_cast<const float*>(tex_korm), S, uv_ox, uv_oz,
                    uv_s, &P, &Nn, &KD, &KORM);
    gb_pos[idx] = P;
    gb_nrm[idx] = Nn;
    gb_kd[idx] = KD;
    gb_korm[idx] = KORM;
}

// ---------------------------------------------------------------- forward
__global__ void __launch_bounds__(kShadeThreads) shade_fwd_kernel(ShadeArgs a, float4* __restrict__ c_d,
                                                                  float4* __restrict__ kd_out,
                                                                  float4* __restrict__ c_s,
                                                                  uint32_t* __restrict__ vis_mask) {
    pdl_prologue();
    extern __shared__ float s_marg[];
    Probe Pr = make_probe(a);
    stage_marginal(Pr, s_marg);
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long P = (long long)a.N * a.H * a.W;
    if (idx >= P) return;
    const int view = (int)(idx / ((long long)a.H * a.W));
    const uint32_t pix = (uint32_t)(idx - (long long)view * a.H * a.W);
    const int spp = a.n_light + a.n_cos + a.n_ggx;
    const int nwords = (spp + 31) >> 5;
    Pixel px;
    const bool covered = load_pixel(a.gb_pos[idx], a.gb_nrm[idx], a.gb_kd[idx], a.gb_korm[idx],
                                    cam_origin(a.cams, view), &px);
    f3 cd = mk(0.f, 0.f, 0.f), cs = cd;
    const BvhNode* nodes = static_cast<const BvhNode*>(a.nodes);
    const TriRecord* tris = static_cast<const TriRecord*>(a.tris);
    uint32_t word = 0;
    for (int j = 0; j < spp; ++j) {
        if (covered) {
            f3 wi;
            int t;
            float ci, inv_denom;
            const float2 u = sample_uniforms(a.seed, pix, (uint32_t)view, (uint32_t)j, a.stream_word);
            if (draw_sample(Pr, px, a.n_light, a.n_cos, a.n_ggx, j, u, &wi, &t, &ci, &inv_denom)) {
                const bool hit = any_hit(nodes, tris, a.n_tris, make_ray(px.p + px.n * a.ray_eps, wi));
                const float Hv = hit ? 1.0f - a.tau : 1.0f;
                if (hit) word |= 1u << (j & 31);
                const float4 L = __ldg(Pr.env + t);
                const float wd = Hv * ci * MCDI_INV_PI * inv_denom;
                cd = cd + mk(L.x, L.y, L.z) * wd;
                if (px.spec_on) {
                    const f3 h = normalize(wi + px.wo);
                    const float D = ggx_D(dot(px.n, h), sin2_between(px.n, h), px.a2);
                    const float G2 = 1.0f / (1.0f + ggx_lambda(ci, px.a2) + ggx_lambda(px.co, px.a2));
                    const float q = schlick_weight(dot(px.wo, h));
                    const float ws = Hv * D * G2 / (4.0f * px.co) * inv_denom;
                    cs = cs + spec_colour(L, px.F0, q, ws);
                }
            }
        }
        if (vis_mask && ((j & 31) == 31 || j == spp - 1)) {
            vis_mask[(size_t)idx * nwords + (j >> 5)] = word;
            word = 0;
        }
    }
    c_d[idx] = make_float4(cd.x, cd.y, cd.z, 0.f);
    c_s[idx] = make_float4(cs.x, cs.y, cs.z, 0.f);
    kd_out[idx] = covered ? make_float4(px.kd.x * (1.f - px.m), px.kd.y * (1.f - px.m), px.kd.z * (1.f - px.m), 0.f)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------- adjoint
// A CTA covers 32 consecutive pixels with kBwdQuarters warps; warp q handles
// the samples j = q, q + 4, ... of its lane's pixel (in increasing j) and the
// per-pixel partial sums of the four warps are added in order q = 0..3, so
// every pixel's gradient has one fixed summation order.
constexpr int kBwdQuarters = kShadeThreads / 32;
constexpr int kBwdPartials = 8;  // g_n (3), g_F0 (3), g_co, g_alpha

__global__ void __launch_bounds__(kShadeThreads, 6) shade_bwd_kernel(ShadeArgs a, const float4* __restrict__ g_cd,
                                                                  const float4* __restrict__ g_kdout,
                                                                  const float4* __restrict__ g_cs,
                                                                  const uint32_t* __restrict__ vis_mask,
                                                                  float4* __restrict__ g_kd,
                                                                  float4* __restrict__ g_korm,
                                                                  float4* __restrict__ g_nrm,
                                                                  float4* __restrict__ g_env, long long first,
                                                                  long long end) {
    pdl_prologue();
    extern __shared__ float s_marg[];  // marginal CDF, then [kBwdQuarters][kBwdPartials][32] partial sums
    Probe Pr = make_probe(a);
    stage_marginal(Pr, s_marg);
    float* s_part = s_marg + ((a.Hp + 1 + 3) & ~3);
    const int lane = threadIdx.x & 31, quarter = threadIdx.x >> 5;
    const long long idx = first + (long long)blockIdx.x * 32 + lane;  // pixels [first, end) of [N][H][W]
    const bool in_range = idx < end;
    const int view = in_range ? (int)(idx / ((long long)a.H * a.W)) : 0;
    const uint32_t pix = (uint32_t)(idx - (long long)view * a.H * a.W);
    const int spp = a.n_light + a.n_cos + a.n_ggx;
    const int nwords = (spp + 31) >> 5;
    Pixel px{};
    const bool covered = in_range && load_pixel(a.gb_pos[idx], a.gb_nrm[idx], a.gb_kd[idx], a.gb_korm[idx],
                                                cam_origin(a.cams, view), &px);
    f3 gn = mk(0.f, 0.f, 0.f), gF0 = gn;
    float g_co = 0.f, g_alpha = 0.f;
    f3 gd = gn, gk = gn, gs = gn;
    if (covered) {
        gd = xyz(g_cd[idx]);
        gk = xyz(g_kdout[idx]);
        gs = xyz(g_cs[idx]);
    }
    const BvhNode* nodes = static_cast<const BvhNode*>(a.nodes);
    const TriRecord* tris = static_cast<const TriRecord*>(a.tris);
    const float a2 = px.a2;
    for (int j = covered ? quarter : spp; j < spp; j += kBwdQuarters) {
        const uint32_t word = vis_mask ? vis_mask[(size_t)idx * nwords + (j >> 5)] : 0u;
        f3 wi;
        int t;
        float ci, inv_denom;
        const float2 u = sample_uniforms(a.seed, pix, (uint32_t)view, (uint32_t)j, a.stream_word);
        if (!draw_sample(Pr, px, a.n_light, a.n_cos, a.n_ggx, j, u, &wi, &t, &ci, &inv_denom)) continue;
        bool hit;
        if (vis_mask) hit = (word >> (j & 31)) & 1u;
        else hit = any_hit_threaded(nodes, tris, a.n_tris, make_ray(px.p + px.n * a.ray_eps, wi));  // no stack
        const float A = (hit ? 1.0f - a.tau : 1.0f) * inv_denom;
        const float4 L4 = __ldg(Pr.env + t);
        const f3 L = xyz(L4);
        // diffuse: c_d = A L ci / pi
        f3 ge = gd * (A * ci * MCDI_INV_PI);
        float g_ci = A * dot(gd, L) * MCDI_INV_PI;
        if (px.spec_on) {
            const f3 h = normalize(wi + px.wo);
            const float nh = dot(px.n, h), vh = dot(px.wo, h);
            const float s2 = sin2_between(px.n, h);
            const float D = ggx_D(nh, s2, a2);
            const float li = ggx_lambda(ci, a2), lo = ggx_lambda(px.co, a2);
            const float G2 = 1.0f / (1.0f + li + lo);
            const float S = D * G2 / (4.0f * px.co);
            const float q = schlick_weight(vh);
            const f3 F = mk(px.F0.x + (1.f - px.F0.x) * q, px.F0.y + (1.f - px.F0.y) * q,
                            px.F0.z + (1.f - px.F0.z) * q);
            ge = ge + mk(gs.x * F.x, gs.y * F.y, gs.z * F.z) * (A * S);
            const float gS = A * (gs.x * L.x * F.x + gs.y * L.y * F.y + gs.z * L.z * F.z);
            gF0 = gF0 + mk(gs.x * L.x, gs.y * L.y, gs.z * L.z) * (A * S * (1.0f - q));
            float dD_dnh = 0.f, dD_dalpha = 0.f;
            if (nh > 0.0f) {
                const float dd = ggx_D_denom(nh, s2, a2);
                dD_dnh = -4.0f * D * nh * (a2 - 1.0f) / dd;
                dD_dalpha = D * (2.0f / px.alpha - 4.0f * px.alpha * nh * nh / dd);
            }
            const float ici2 = 1.0f / (ci * ci), ico2 = 1.0f / (px.co * px.co);
            const float si = sqrtf(1.0f + a2 * (ici2 - 1.0f)), so = sqrtf(1.0f + a2 * (ico2 - 1.0f));
            const float dli_dci = (-2.0f * a2 * ici2 / ci) / (4.0f * si);
            const float dlo_dco = (-2.0f * a2 * ico2 / px.co) / (4.0f * so);
            const float dli_da = 2.0f * px.alpha * (ici2 - 1.0f) / (4.0f * si);
            const float dlo_da = 2.0f * px.alpha * (ico2 - 1.0f) / (4.0f * so);
            const float dS_dD = G2 / (4.0f * px.co);
            const float dS_dLam = -D * G2 * G2 / (4.0f * px.co);
            const float g_nh = gS * dS_dD * dD_dnh;
            g_alpha += gS * (dS_dD * dD_dalpha + dS_dLam * (dli_da + dlo_da));
            g_ci += gS * dS_dLam * dli_dci;
            g_co += gS * (dS_dLam * dlo_dco - S / px.co);
            gn = gn + h * g_nh;
        }
        gn = gn + wi * g_ci;
        // Warp-aggregated scatter: lanes whose samples landed on the same texel
        // (light samples crowd onto the bright lobes) sum their contributions
        // in lane order and the lowest lane issues one atomic for the group.
        const unsigned peers = __match_any_sync(__activemask(), t);
        if (__popc(peers) > 1) {
            f3 sum = mk(0.f, 0.f, 0.f);
            for (unsigned rest = peers; rest; rest &= rest - 1u) {
                const int q = __ffs(rest) - 1;
                sum = sum + mk(__shfl_sync(peers, ge.x, q), __shfl_sync(peers, ge.y, q), __shfl_sync(peers, ge.z, q));
            }
            ge = sum;
        }
        if (lane == __ffs(peers) - 1) atomicAdd(g_env + t, make_float4(ge.x, ge.y, ge.z, 0.f));
    }
    // the four warps' partial sums of each pixel, added in warp order by warp 0
    const float part[kBwdPartials] = {gn.x, gn.y, gn.z, gF0.x, gF0.y, gF0.z, g_co, g_alpha};
#pragma unroll
    for (int k = 0; k < kBwdPartials; ++k) s_part[(quarter * kBwdPartials + k) * 32 + lane] = part[k];
    __syncthreads();
    if (quarter != 0 || !in_range) return;
    if (!covered) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        g_kd[idx] = z;
        g_korm[idx] = z;
        g_nrm[idx] = z;
        return;
    }
    float sum[kBwdPartials];
#pragma unroll
    for (int k = 0; k < kBwdPartials; ++k) {
        sum[k] = s_part[k * 32 + lane];
        for (int q = 1; q < kBwdQuarters; ++q) sum[k] += s_part[(q * kBwdPartials + k) * 32 + lane];
    }
    gn = mk(sum[0], sum[1], sum[2]);
    gF0 = mk(sum[3], sum[4], sum[5]);
    g_co = sum[6];
    g_alpha = sum[7];
    gn = gn + px.wo * g_co;
    const float ng = dot(px.n, gn);
    const f3 gN = (gn - px.n * ng) * (1.0f / px.lN);
    const float om = 1.0f - px.m;
    g_kd[idx] = make_float4(gk.x * om + gF0.x * px.m, gk.y * om + gF0.y * px.m, gk.z * om + gF0.z * px.m, 0.f);
    const float g_m = -(gk.x * px.kd.x + gk.y * px.kd.y + gk.z * px.kd.z) + gF0.x * (px.kd.x - 0.04f) +
                      gF0.y * (px.kd.y - 0.04f) + gF0.z * (px.kd.z - 0.04f);
    const float g_r = (px.r * px.r > 1e-4f) ? g_alpha * 2.0f * px.r : 0.0f;
    g_korm[idx] = make_float4(0.f, g_r, g_m, 0.f);
    g_nrm[idx] = make_float4(gN.x, gN.y, gN.z, 0.f);
}

inline int grid_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_primary_cast(const void* nodes, const void* tris, int n_tris, const float* verts,
                                const float* vnrm, const int* tri_idx, int n_verts, const mcdi_camera* cams, int N,
                                int H, int W, const float* tex_kd, const float* tex_korm, int tex_size, float uv_ox,
                                float uv_oz, float uv_s, float* gb_pos, float* gb_nrm, float* gb_kd, float* gb_korm,
                                cudaStream_t stream) {
    const long long P = (long long)N * H * W;
    launch_k(primary_cast_kernel, grid_for(P, kShadeThreads), kShadeThreads, 0, stream,
             static_cast<const BvhNode*>(nodes), static_cast<const TriRecord*>(tris), n_tris, verts, vnrm, tri_idx,
             n_verts, cams, N, H, W, reinterpret_cast<const float4*>(tex_kd), reinterpret_cast<const float4*>(tex_korm),
             tex_size, uv_ox, uv_oz, uv_s, reinterpret_cast<float4*>(gb_pos), reinterpret_cast<float4*>(gb_nrm),
             reinterpret_cast<float4*>(gb_kd), reinterpret_cast<float4*>(gb_korm));
    return cudaGetLastError();
}

cudaError_t launch_shade_fwd(const ShadeArgs& a, float4* c_d, float4* kd_out, float4* c_s, uint32_t* vis_mask,
                             cudaStream_t stream) {
    const long long P = (long long)a.N * a.H * a.W;
    const size_t smem = (size_t)(a.Hp + 1) * sizeof(float);
    launch_k(shade_fwd_kernel, grid_for(P, kShadeThreads), kShadeThreads, smem, stream, a, c_d, kd_out, c_s, vis_mask);
    return cudaGetLastError();
}

cudaError_t launch_shade_bwd(const ShadeArgs& a, const float4* g_cd, const float4* g_kdout, const float4* g_cs,
                             const uint32_t* vis_mask, float4* g_kd, float4* g_korm, float4* g_nrm, float4* g_env,
                             cudaStream_t stream, long long first, long long count) {
    const long long P = (long long)a.N * a.H * a.W;
    if (count < 0) count = P - first;
    if (count <= 0) return cudaSuccess;
    const size_t smem = (size_t)(((a.Hp + 1 + 3) & ~3) + kBwdQuarters * kBwdPartials * 32) * sizeof(float);
    launch_k(shade_bwd_kernel, grid_for(count, 32), kShadeThreads, smem, stream, a, g_cd, g_kdout, g_cs, vis_mask,
             g_kd, g_korm, g_nrm, g_env, first, first + count);
    return cudaGetLastError();
}

}  // namespace mcdi
