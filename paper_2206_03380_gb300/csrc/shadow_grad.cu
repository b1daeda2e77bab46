// Shadow-visibility gradients (the ablation of the paper's appendix
// "Visibility gradients from shadows"; Sec. 3.1 "Shadow gradients"): the
// boundary term of the blocked set of each pixel's shadow rays, estimated by
// edge sampling, scattered to the mesh's vertex positions.
//
// With H = 1 - tau B (B: the shadow ray from o = p + eps n is blocked), the
// pixel's integral of g(w) H(w) moves with the mesh only through the boundary
// of the blocked set, made of silhouette edges seen from o.  For an edge (a, b)
// and x(s) = a + s (b - a), w = (x - o) / r:
//   d/d(a, b) = -tau int_0^1 g(w) V+(s) n_out ((1 - s), s) |w x (b - a)| / r^2 ds,
// n_out the unit normal of the plane (o, a, b) away from the edge's faces and
// V+ whether the ray just outside the edge (w + eta n_out) reaches the probe.
// g is the forward integrand weighted by the upstream gradients of c_d, c_s.
// Each pixel draws M edges uniformly (e = floor(u0 E) in integer arithmetic)
// and s = u1; a sample weighs E / M.
//
// The edge table lists each undirected edge once, in the order of its first
// half-edge h = 3 t + i, as (a, b, c1, c2): the owner half-edge's endpoints,
// the opposite vertex of its face and that of the next face on the edge (-1
// on a boundary).  It is built with a hash table (first and second half-edge
// of each key by atomicMin), then an ordered compaction.
#include <limits.h>

#include "common.cuh"
#include "internal.h"
#include "shading.cuh"

namespace mcdi {
namespace {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kEdgeThreads = 256;
constexpr int kEdgeItems = 8;  // half-edges per thread in the ordered compaction
constexpr int kEdgeTile = kEdgeThreads * kEdgeItems;
constexpr int kGradThreads = 128;

__device__ __forceinline__ unsigned long long edge_key(int a, int b) {
    const unsigned lo = (unsigned)min(a, b), hi = (unsigned)max(a, b);
    return ((unsigned long long)lo << 32) | hi;
}

// 64-bit finaliser of MurmurHash3 (Appleby), spreading keys over the table
__device__ __forceinline__ unsigned long long mix64(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

__device__ __forceinline__ int tri_vertex(const int* __restrict__ tris, int h, int step) {
    const int t = h / 3, i = h - 3 * t;
    return __ldg(tris + 3 * t + (i + step) % 3);
}

__global__ void __launch_bounds__(kEdgeThreads) edge_clear_kernel(unsigned long long* keys, int* first, int* second,
                                                                  long long cap) {
    pdl_prologue();
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < cap; k += (long long)gridDim.x * blockDim.x) {
        keys[k] = kEmptyKey;
        first[k] = INT_MAX;
        second[k] = INT_MAX;
    }
}

// insert every half-edge's key (linear probing, at most `cap` probes) and keep
// the smallest half-edge index per key
__global__ void __launch_bounds__(kEdgeThreads) edge_insert_kernel(const int* __restrict__ tris, int n_half,
                                                                   unsigned long long* keys, int* first, int* slot_of,
                                                                   long long cap, unsigned* err) {
    pdl_prologue();
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= n_half) return;
    const unsigned long long key = edge_key(tri_vertex(tris, h, 0), tri_vertex(tris, h, 1));
    long long slot = (long long)(mix64(key) & (unsigned long long)(cap - 1));
    for (long long probe = 0; probe < cap; ++probe) {
        const unsigned long long old = atomicCAS(keys + slot, kEmptyKey, key);
        if (old == kEmptyKey || old == key) {
            atomicMin(first + slot, h);
            slot_of[h] = (int)slot;
            return;
        }
        slot = (slot + 1) & (cap - 1);
    }
    slot_of[h] = -1;
    atomicOr(err, 1u);
}

// the smallest half-edge index after the first, per key
__global__ void __launch_bounds__(kEdgeThreads) edge_second_kernel(int n_half, const int* __restrict__ slot_of,
                                                                   const int* __restrict__ first, int* second) {
    pdl_prologue();
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= n_half) return;
    const int s = slot_of[h];
    if (s >= 0 && first[s] != h) atomicMin(second + s, h);
}

__device__ __forceinline__ bool owns_edge(const int* __restrict__ slot_of, const int* __restrict__ first, int h) {
    const int s = slot_of[h];
    return s >= 0 && first[s] == h;
}

// edges owned by each tile of kEdgeTile half-edges
__global__ void __launch_bounds__(kEdgeThreads) edge_count_kernel(int n_half, const int* __restrict__ slot_of,
                                                                  const int* __restrict__ first, int* tile_count) {
    pdl_prologue();
    __shared__ int s_warp[kEdgeThreads / 32];
    const int base = blockIdx.x * kEdgeTile + threadIdx.x * kEdgeItems;
    int c = 0;
#pragma unroll
    for (int k = 0; k < kEdgeItems; ++k) c += (base + k < n_half && owns_edge(slot_of, first, base + k)) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kEdgeThreads / 32; ++w) t += s_warp[w];
        tile_count[blockIdx.x] = t;
    }
}

// exclusive scan of the tile counts (one block); the total is the edge count,
// or -1 if a key found no slot
__global__ void __launch_bounds__(1024) edge_offsets_kernel(int n_tiles, const int* __restrict__ tile_count,
                                                            int* tile_off, int* n_edges, const unsigned* err) {
    pdl_prologue();
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < n_tiles; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < n_tiles ? tile_count[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const int incl = x + (warp > 0 ? s_warp[warp - 1] : 0);
        if (i < n_tiles) tile_off[i] = s_carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_edges = *err ? -1 : s_carry;
}

// write each owned edge at its rank in half-edge order
__global__ void __launch_bounds__(kEdgeThreads) edge_write_kernel(const int* __restrict__ tris, int n_half,
                                                                  const int* __restrict__ slot_of,
                                                                  const int* __restrict__ first,
                                                                  const int* __restrict__ second,
                                                                  const int* __restrict__ tile_off, int4* edges) {
    pdl_prologue();
    __shared__ int s_warp[kEdgeThreads / 32];
    const int base = blockIdx.x * kEdgeTile + threadIdx.x * kEdgeItems;
    unsigned own = 0;
#pragma unroll
    for (int k = 0; k < kEdgeItems; ++k)
        if (base + k < n_half && owns_edge(slot_of, first, base + k)) own |= 1u << k;
    const int c = __popc(own), lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    int rank = tile_off[blockIdx.x] + before + x - c;
    for (; own; own &= own - 1u) {
        const int h = base + __ffs(own) - 1;
        const int s2 = second[slot_of[h]];
        edges[rank++] = make_int4(tri_vertex(tris, h, 0), tri_vertex(tris, h, 1), tri_vertex(tris, h, 2),
                                  s2 == INT_MAX ? -1 : tri_vertex(tris, s2, 2));
    }
}

__device__ __forceinline__ f3 load_vert(const float* __restrict__ v, int i) {
    return mk(__ldg(v + 3 * (size_t)i), __ldg(v + 3 * (size_t)i + 1), __ldg(v + 3 * (size_t)i + 2));
}

__device__ __forceinline__ void scatter3(float* g, int i, f3 d) {
    atomicAdd(g + 3 * (size_t)i, d.x);
    atomicAdd(g + 3 * (size_t)i + 1, d.y);
    atomicAdd(g + 3 * (size_t)i + 2, d.z);
}

// Any hit for one ray with the whole warp: lane k walks the k-th of 32 equal
// segments of the depth-first node array along the escape links.  A lane that
// starts inside a subtree skips the box tests of its ancestors outside the
// segment, which only adds box tests: a triangle the ray hits has every
// ancestor box hit (boxes are conservative), so some lane reaches its leaf,
// and the result equals the one-lane traversal's.  All lanes call this with
// the same ray; the loop runs uniformly and ends when a lane finds a hit or
// every lane has left its segment (each step moves strictly forward).
__device__ __forceinline__ bool warp_any_hit(const void* nodes, const TriRecord* __restrict__ tris, int n_tris,
                                             const RayInv& r, int lane) {
    if (n_tris <= 0) return false;
    const ThreadedNode* tn = threaded_nodes(nodes, n_tris);
    const int m = 2 * n_tris - 1, seg = (m + 31) / 32;
    int i = lane * seg;
    const int hi = min(m, i + seg);
    bool found = false;
    for (;;) {
        const bool active = i < hi;
        if (!__any_sync(0xffffffffu, active)) return false;
        if (active) {
            i = threaded_step(tn, tris, r, i);
            if (i < 0) {
                found = true;
                i = hi;
            }
        }
        if (__any_sync(0xffffffffu, found)) return true;
    }
}

// One thread per (pixel, edge sample).  The rare samples that reach the outer
// ray (silhouette, above the horizon) are traced one after another by the
// whole warp, so that each grazing ray's long chain of dependent node fetches
// is split 32 ways.
__global__ void __launch_bounds__(kGradThreads) shadow_edge_grad_kernel(
    ShadeArgs a, const float* __restrict__ verts, int n_verts, const int4* __restrict__ edges,
    const int* __restrict__ n_edges_dev, int max_edges, int M, float eta, const float4* __restrict__ g_cd,
    const float4* __restrict__ g_cs, float* g_verts, float* sample_w) {
    pdl_prologue();
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long P = (long long)a.N * a.H * a.W;
    const bool in_range = tid < P * M;
    const long long idx = in_range ? tid / M : 0;
    const int j = (int)(tid - idx * M);
    const int lane = threadIdx.x & 31;
    const int E = min(max(*n_edges_dev, 0), max_edges);
    const int view = (int)(idx / ((long long)a.H * a.W));
    const uint32_t pix = (uint32_t)(idx - (long long)view * a.H * a.W);
    // position and normal only (the shading setup waits for the few samples that reach the outer ray);
    // n is formed exactly as load_pixel forms it
    const float4 pos = in_range ? a.gb_pos[idx] : make_float4(0.f, 0.f, 0.f, 0.f);
    const f3 N = in_range ? xyz(a.gb_nrm[idx]) : mk(0.f, 0.f, 0.f);
    const float l2 = dot(N, N);
    bool cand = false;
    f3 o{}, w{}, nout{}, ab{};
    float s = 0.f, r2 = 1.f, ci = 0.f;
    int4 ed{};
    do {
        if (!(pos.w > 0.0f) || !(l2 > 0.0f) || E <= 0) break;
        const f3 nrm = N * (1.0f / sqrtf(l2));
        const uint4 x = philox4x32_10(make_uint4(pix, (uint32_t)view, (uint32_t)j, a.stream_word),
                                      make_uint2((uint32_t)(a.seed & 0xffffffffull), (uint32_t)(a.seed >> 32)));
        const int e = (int)(((unsigned long long)(x.x >> 8) * (unsigned)E) >> 24);
        s = (float)(x.y >> 8) * 5.9604644775390625e-8f;
        ed = __ldg(edges + e);
        if ((unsigned)ed.x >= (unsigned)n_verts || (unsigned)ed.y >= (unsigned)n_verts ||
            (unsigned)ed.z >= (unsigned)n_verts || ed.w >= n_verts)
            break;
        o = xyz(pos) + nrm * a.ray_eps;
        const f3 va = load_vert(verts, ed.x), vb = load_vert(verts, ed.y);
        const f3 m = cross(va - o, vb - o);
        const float lm = sqrtf(dot(m, m));
        if (!(lm > 0.0f)) break;
        const float s1 = dot(m, load_vert(verts, ed.z) - o);
        const float s2 = ed.w >= 0 ? dot(m, load_vert(verts, ed.w) - o) : s1;
        if (!(s1 * s2 > 0.0f)) break;  // both faces on one side of the plane (o, a, b): silhouette
        ab = vb - va;
        const f3 d = va + ab * s - o;
        r2 = dot(d, d);
        w = d * (1.0f / sqrtf(r2));
        ci = dot(nrm, w);
        if (!(ci > 0.0f)) break;
        nout = m * ((s1 > 0.0f ? -1.0f : 1.0f) / lm);
        cand = true;
    } while (false);
    // the outer rays of this warp's candidates, each traced by all 32 lanes
    bool open = false;
    const f3 dir = normalize(w + nout * eta);
    for (unsigned todo = __ballot_sync(0xffffffffu, cand); todo; todo &= todo - 1u) {
        const int src = __ffs(todo) - 1;
        const f3 ro = mk(__shfl_sync(0xffffffffu, o.x, src), __shfl_sync(0xffffffffu, o.y, src),
                         __shfl_sync(0xffffffffu, o.z, src));
        const f3 rd = mk(__shfl_sync(0xffffffffu, dir.x, src), __shfl_sync(0xffffffffu, dir.y, src),
                         __shfl_sync(0xffffffffu, dir.z, src));
        const bool hit = warp_any_hit(a.nodes, static_cast<const TriRecord*>(a.tris), a.n_tris, make_ray(ro, rd), lane);
        if (lane == src) open = !hit;
    }
    float wt = 0.0f;
    if (open) {
        Pixel px{};
        load_pixel(pos, a.gb_nrm[idx], a.gb_kd[idx], a.gb_korm[idx],
                   mk(a.cams[view].origin[0], a.cams[view].origin[1], a.cams[view].origin[2]), &px);
        Probe Pr;
        Pr.W = a.Wp;
        Pr.H = a.Hp;
        float st;
        const int t = texel_of_dir(Pr, w, &st);
        const f3 L = xyz(__ldg(a.env + t));
        const f3 gd = xyz(g_cd[idx]);
        float gw = (L.x * gd.x + L.y * gd.y + L.z * gd.z) * ci * MCDI_INV_PI;
        if (px.spec_on) {
            const f3 gs = xyz(g_cs[idx]);
            const f3 h = normalize(w + px.wo);
            const float nh = dot(px.n, h), vh = dot(px.wo, h);
            const float D = ggx_D(nh, sin2_between(px.n, h), px.a2);
            const float G2 = 1.0f / (1.0f + ggx_lambda(ci, px.a2) + ggx_lambda(px.co, px.a2));
            const float q = schlick_weight(vh);
            const f3 F = mk(px.F0.x + (1.f - px.F0.x) * q, px.F0.y + (1.f - px.F0.y) * q,
                            px.F0.z + (1.f - px.F0.z) * q);
            gw += (L.x * gs.x * F.x + L.y * gs.y * F.y + L.z * gs.z * F.z) * D * G2 / (4.0f * px.co);
        }
        const f3 c = cross(w, ab);
        const float J = sqrtf(dot(c, c)) / r2;
        wt = -a.tau * gw * J * ((float)E / (float)M);
        if (wt != 0.0f) {
            scatter3(g_verts, ed.x, nout * (wt * (1.0f - s)));
            scatter3(g_verts, ed.y, nout * (wt * s));
        }
    }
    if (sample_w && in_range) sample_w[tid] = wt;
}

inline size_t edge_table_cap(int n_tris) {
    size_t cap = 1;
    while (cap < (size_t)6 * (size_t)(n_tris > 0 ? n_tris : 1)) cap <<= 1;  // >= 2 x the half-edges
    return cap;
}

}  // namespace

EdgeScratch edge_scratch_layout(int n_tris) {
    EdgeScratch L{};
    const size_t nh = (size_t)3 * (n_tris > 0 ? n_tris : 1);
    L.cap = edge_table_cap(n_tris);
    L.n_tiles = (int)((nh + kEdgeTile - 1) / kEdgeTile);
    size_t o = 0;
    L.keys = o; o = align256(o + L.cap * sizeof(unsigned long long));
    L.first = o; o = align256(o + L.cap * sizeof(int));
    L.second = o; o = align256(o + L.cap * sizeof(int));
    L.slot_of = o; o = align256(o + nh * sizeof(int));
    L.tile_count = o; o = align256(o + (size_t)L.n_tiles * sizeof(int));
    L.tile_off = o; o = align256(o + (size_t)L.n_tiles * sizeof(int));
    L.err = o; o = align256(o + sizeof(unsigned));
    L.total = o;
    return L;
}

cudaError_t launch_build_edge_table(const int* tris, int n_tris, int4* edges, int* n_edges, void* scratch,
                                    const EdgeScratch& L, cudaStream_t stream) {
    char* ws = static_cast<char*>(scratch);
    auto* keys = reinterpret_cast<unsigned long long*>(ws + L.keys);
    int* first = reinterpret_cast<int*>(ws + L.first);
    int* second = reinterpret_cast<int*>(ws + L.second);
    int* slot_of = reinterpret_cast<int*>(ws + L.slot_of);
    int* tile_count = reinterpret_cast<int*>(ws + L.tile_count);
    int* tile_off = reinterpret_cast<int*>(ws + L.tile_off);
    unsigned* err = reinterpret_cast<unsigned*>(ws + L.err);
    const int n_half = 3 * n_tris;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    const long long cap = (long long)L.cap;
    const int clear_blocks = (int)((cap + kEdgeThreads - 1) / kEdgeThreads < 4096 ? (cap + kEdgeThreads - 1) / kEdgeThreads
                                                                                   : 4096);
    launch_k(edge_clear_kernel, clear_blocks, kEdgeThreads, 0, stream, keys, first, second, cap);
    const int hb = (n_half + kEdgeThreads - 1) / kEdgeThreads;
    launch_k(edge_insert_kernel, hb, kEdgeThreads, 0, stream, tris, n_half, keys, first, slot_of, cap, err);
    launch_k(edge_second_kernel, hb, kEdgeThreads, 0, stream, n_half, (const int*)slot_of, (const int*)first, second);
    launch_k(edge_count_kernel, L.n_tiles, kEdgeThreads, 0, stream, n_half, (const int*)slot_of, (const int*)first,
             tile_count);
    launch_k(edge_offsets_kernel, 1, 1024, 0, stream, L.n_tiles, (const int*)tile_count, tile_off, n_edges,
             (const unsigned*)err);
    launch_k(edge_write_kernel, L.n_tiles, kEdgeThreads, 0, stream, tris, n_half, (const int*)slot_of,
             (const int*)first, (const int*)second, (const int*)tile_off, edges);
    return cudaGetLastError();
}

cudaError_t launch_shadow_edge_grad(const ShadeArgs& a, const float* verts, int n_verts, const int4* edges,
                                    const int* n_edges, int max_edges, int n_samples, float eta, const float4* g_cd,
                                    const float4* g_cs, float* g_verts, float* sample_w, cudaStream_t stream) {
    const long long n = (long long)a.N * a.H * a.W * n_samples;
    if (n <= 0) return cudaGetLastError();
    launch_k(shadow_edge_grad_kernel, (int)((n + kGradThreads - 1) / kGradThreads), kGradThreads, 0, stream, a, verts,
             n_verts, edges, n_edges, max_edges, n_samples, eta, g_cd, g_cs, g_verts, sample_w);
    return cudaGetLastError();
}

}  // namespace mcdi
