// Linear BVH over the triangle mesh extracted each iteration (the paper traces
// shadow rays with hardware ray tracing, Sec. 3 and Sec. 6; GB300 has no RT
// cores, so the acceleration structure is built and traversed in software).
//
// Build (Karras 2012, "Maximizing parallelism in the construction of BVHs,
// octrees, and k-d trees"):
//   1. centroid bounds (block min/max + one atomic per block and axis);
//   2. 30-bit Morton code of each centroid;
//   3. stable LSD radix sort, 3 passes of 10 bits (histogram / per-digit scan
//      across tiles / scatter with warp match_any ranking; up to 262,144
//      triangles one kernel per pass: each pass's digit counts per tile come
//      from the kernel before it, the Morton kernel for the first);
//   4. one thread per internal node finds its key range and split from the
//      common-prefix lengths of the sorted keys (ties broken by position);
//   5. bottom-up bounds: each leaf walks to the root, the second thread to
//      reach a node (atomic arrival counter) writes its two child boxes;
//   6. one thread per node: the depth-first copy with escape links and, for
//      internal nodes at even depth, the four-wide node with 8-bit child boxes
//      that shadow rays traverse.
// Output: 64-byte two-child nodes (root = node 0), the depth-first copy, the
// four-wide nodes and 48-byte triangle records in leaf (Morton) order.
#include <float.h>
#include <algorithm>
#include <limits.h>

#include "common.cuh"
#include "internal.h"

namespace mcdi {
namespace {

__device__ __forceinline__ uint32_t f2ord(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// bounds to the empty box; the tile-sort digit counts (n_vec4 vectors) to zero
__global__ void init_bounds_kernel(uint32_t* bounds, uint4* hist, int n_vec4) {
    pdl_prologue();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 3) bounds[i] = f2ord(FLT_MAX);
    else if (i < 6) bounds[i] = f2ord(-FLT_MAX);
    for (int k = i; k < n_vec4; k += gridDim.x * blockDim.x) hist[k] = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void __launch_bounds__(256) centroid_bounds_kernel(const float* __restrict__ verts, int n_verts,
                                                              const int* __restrict__ tris, int n,
                                                              uint32_t* __restrict__ bounds) {
    pdl_prologue();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    if (k < n) {
        f3 a, b, c;
        load_tri(verts, n_verts, tris, k, a, b, c);
        const f3 m = (a + b + c) * (1.0f / 3.0f);
        lo[0] = hi[0] = m.x;
        lo[1] = hi[1] = m.y;
        lo[2] = hi[2] = m.z;
    }
    __shared__ float red[6][8];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            lo[ax] = fminf(lo[ax], __shfl_xor_sync(0xffffffffu, lo[ax], off));
            hi[ax] = fmaxf(hi[ax], __shfl_xor_sync(0xffffffffu, hi[ax], off));
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        for (int ax = 0; ax < 3; ++ax) {
            red[ax][warp] = lo[ax];
            red[3 + ax][warp] = hi[ax];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int r = threadIdx.x;
        float v = red[r][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = r < 3 ? fminf(v, red[r][w]) : fmaxf(v, red[r][w]);
        if (r < 3) atomicMin(bounds + r, f2ord(v));
        else atomicMax(bounds + r, f2ord(v));
    }
}

constexpr int kDigits = 1 << kSortDigitBits;

// spread the low 10 bits of v so that bit i lands at bit 3i
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// (tile_hist non-null: also counts each key's first digit in its tile of kTileKeys keys,
// one atomic per distinct (tile, digit) of a warp)
__global__ void __launch_bounds__(256) morton_kernel(const float* __restrict__ verts, int n_verts,
                                                     const int* __restrict__ tris, int n,
                                                     const uint32_t* __restrict__ bounds, uint32_t* __restrict__ keys,
                                                     uint32_t* __restrict__ vals, uint32_t* __restrict__ tile_hist) {
    pdl_prologue();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = k < n;
    uint32_t code = 0;
    if (valid) {
        f3 a, b, c;
        load_tri(verts, n_verts, tris, k, a, b, c);
        const f3 m = (a + b + c) * (1.0f / 3.0f);
        const float lo[3] = {ord2f(bounds[0]), ord2f(bounds[1]), ord2f(bounds[2])};
        const float hi[3] = {ord2f(bounds[3]), ord2f(bounds[4]), ord2f(bounds[5])};
        const float p[3] = {m.x, m.y, m.z};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const float ext = hi[ax] - lo[ax];
            float t = ext > 0.f ? (p[ax] - lo[ax]) / ext : 0.5f;
            t = fminf(fmaxf(t, 0.f), 1.f);
            const uint32_t q = min(1023u, (uint32_t)(t * 1024.f));
            code |= spread3(q) << (2 - ax);
        }
        keys[k] = code;
        vals[k] = (uint32_t)k;
    }
    if (tile_hist) {  // every lane of the warp takes part (blocks are whole warps)
        const int lane = threadIdx.x & 31;
        const uint32_t slot = valid ? (uint32_t)(k / kTileKeys) * kDigits + (code & (kDigits - 1)) : 0x80000000u | lane;
        const unsigned peers = __match_any_sync(0xffffffffu, slot);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(tile_hist + slot, (uint32_t)__popc(peers));
    }
}

// ---- radix sort: 30-bit Morton keys in three passes of one 10-bit digit ----
// (LSD and stable, so equal keys keep their triangle order)
constexpr int kDigitsPerThread = kDigits / kSortThreads;

__global__ void __launch_bounds__(kSortThreads) digit_hist_kernel(const uint32_t* __restrict__ keys, int n, int shift,
                                                                  int nblocks, uint32_t* __restrict__ hist) {
    pdl_prologue();
    __shared__ uint32_t h[kDigits];
#pragma unroll
    for (int q = 0; q < kDigitsPerThread; ++q) h[q * kSortThreads + threadIdx.x] = 0;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const size_t i = base + (size_t)it * kSortThreads + threadIdx.x;
        if (i < (size_t)n) atomicAdd(&h[(keys[i] >> shift) & (kDigits - 1)], 1u);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kDigitsPerThread; ++q) {
        const int d = q * kSortThreads + threadIdx.x;
        hist[(size_t)d * nblocks + blockIdx.x] = h[d];
    }
}

// one block per digit: exclusive scan of that digit's counts across tiles
__global__ void __launch_bounds__(256) digit_scan_kernel(uint32_t* __restrict__ hist, int nblocks,
                                                         uint32_t* __restrict__ digit_tot) {
    pdl_prologue();
    uint32_t* row = hist + (size_t)blockIdx.x * nblocks;
    __shared__ uint32_t warp_tot[8];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nblocks; base += 256) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nblocks ? row[i] : 0u;
        uint32_t inc = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += t;
        }
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        uint32_t woff = 0, all = 0;
        for (int w = 0; w < 8; ++w) {
            if (w < warp) woff += warp_tot[w];
            all += warp_tot[w];
        }
        if (i < nblocks) row[i] = carry + woff + inc - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) digit_tot[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kSortThreads) digit_scatter_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, int n, int shift, int nblocks,
    const uint32_t* __restrict__ hist, const uint32_t* __restrict__ digit_tot, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out) {
    pdl_prologue();
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t wc[kWarps][kDigits];  // per-warp digit counters, then per-warp offsets
    __shared__ uint32_t dbase[kDigits];       // global start of each digit in this tile
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int w = 0; w < kWarps; ++w)
#pragma unroll
        for (int q = 0; q < kDigitsPerThread; ++q) wc[w][q * kSortThreads + threadIdx.x] = 0;
    {  // exclusive scan of the digit totals: thread t owns digits [t * kDigitsPerThread, +kDigitsPerThread)
        __shared__ uint32_t wt[kWarps];
        uint32_t v[kDigitsPerThread], sum = 0;
#pragma unroll
        for (int q = 0; q < kDigitsPerThread; ++q) {
            v[q] = digit_tot[threadIdx.x * kDigitsPerThread + q];
            sum += v[q];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += t;
        }
        if (lane == 31) wt[warp] = inc;
        __syncthreads();
        uint32_t run = inc - sum;
        for (int w = 0; w < warp; ++w) run += wt[w];
#pragma unroll
        for (int q = 0; q < kDigitsPerThread; ++q) {
            const int d = threadIdx.x * kDigitsPerThread + q;
            dbase[d] = run + hist[(size_t)d * nblocks + blockIdx.x];
            run += v[q];
        }
    }
    __syncthreads();
    // warp w ranks elements [base + w*256, base + (w+1)*256) in order, 32 at a time
    const size_t base = (size_t)blockIdx.x * kSortTile + (size_t)warp * (32 * kSortItems);
    uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const size_t i = base + (size_t)it * 32 + lane;
        const bool valid = i < (size_t)n;
        key[it] = valid ? keys_in[i] : 0u;
        val[it] = valid ? vals_in[i] : 0u;
        const uint32_t d = valid ? ((key[it] >> shift) & (kDigits - 1)) : ((uint32_t)kDigits + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0;
        if (valid) before = wc[warp][d];
        __syncwarp();
        if (valid && (peers & lt) == 0) wc[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[it] = before + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: exclusive scan over warps (warp order = element order)
#pragma unroll
    for (int q = 0; q < kDigitsPerThread; ++q) {
        const int d = q * kSortThreads + threadIdx.x;
        uint32_t run = 0;
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = wc[w][d];
            wc[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const size_t i = base + (size_t)it * 32 + lane;
        if (i < (size_t)n) {
            const uint32_t d = (key[it] >> shift) & (kDigits - 1);
            const uint32_t pos = dbase[d] + wc[warp][d] + rank[it];
            keys_out[pos] = key[it];
            vals_out[pos] = val[it];
        }
    }
}

// One radix pass over tiles of kTileKeys sorted positions, without a separate
// count or scan launch: tile t's count of each digit in every tile comes from
// `hist` (row t' = tile t'; made by the kernel before), so the tile finds its
// start in each digit (the digit's keys in all tiles, digits before it, plus
// those in tiles before it) itself; ranks within the tile as in
// digit_scatter_kernel.  With hist_next it also counts, for the next pass, the
// next digit of each key in the tile of its new position.
constexpr int kTileValBits = 19;  // key index bits (n <= kTileSortMax); a warp-local rank above them
static_assert(kTileSortMax <= (1 << kTileValBits), "key indices must fit below the rank bits");

template <int kThreads, int kItems>
__global__ void __launch_bounds__(kThreads, 1) tile_scatter_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, int n, int shift, int n_tiles,
    const uint32_t* __restrict__ hist, uint32_t* __restrict__ hist_next, int next_shift,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
    constexpr int kWarps = kThreads / 32, kKeys = kThreads * kItems, kDp = kDigits / kThreads;
    static_assert(32 * kItems <= (1 << (32 - kTileValBits)), "a warp-local rank must fit above the index bits");
    static_assert(kDp == 2 || kDp == 4, "each thread owns two or four digits");
    pdl_prologue();
    __shared__ uint16_t wc[kWarps][kDigits];  // per-warp digit counters, then per-warp offsets
    __shared__ uint32_t dbase[kDigits];       // this tile's first position in each digit
    __shared__ uint32_t wsum[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int t = blockIdx.x;
    const int base = t * kKeys;
    const int cnt = min(kKeys, n - base);
    const uint32_t vmask = (1u << kTileValBits) - 1u;
    for (int i = tid; i < kWarps * kDigits / 2; i += kThreads) reinterpret_cast<uint32_t*>(&wc[0][0])[i] = 0u;
    // element (warp, item, lane) is tile position warp * 32 kItems + item * 32 + lane
    uint32_t key[kItems], v[kItems];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int lp = warp * (32 * kItems) + it * 32 + lane;
        key[it] = lp < cnt ? keys_in[base + lp] : 0u;
        v[it] = lp < cnt ? vals_in[base + lp] : 0u;
    }
    // digits kDp tid ... kDp tid + kDp - 1: their keys in the tiles before this one and in all tiles
    const int d0 = kDp * tid;
    uint32_t pre[kDp], tot[kDp];
#pragma unroll
    for (int q = 0; q < kDp; ++q) pre[q] = tot[q] = 0u;
#pragma unroll 8
    for (int r = 0; r < n_tiles; ++r) {
        uint32_t h[kDp];
        if constexpr (kDp == 2) {
            const uint2 x = __ldcg(reinterpret_cast<const uint2*>(hist + (size_t)r * kDigits + d0));
            h[0] = x.x, h[1] = x.y;
        } else {
            const uint4 x = __ldcg(reinterpret_cast<const uint4*>(hist + (size_t)r * kDigits + d0));
            h[0] = x.x, h[1] = x.y, h[2] = x.z, h[3] = x.w;
        }
#pragma unroll
        for (int q = 0; q < kDp; ++q) {
            if (r < t) pre[q] += h[q];
            tot[q] += h[q];
        }
    }
    __syncthreads();
    uint16_t* mywc = wc[warp];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const bool valid = warp * (32 * kItems) + it * 32 + lane < cnt;
        const uint32_t d = valid ? ((key[it] >> shift) & (kDigits - 1)) : ((uint32_t)kDigits + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0;
        if (valid) before = mywc[d];
        __syncwarp();
        if (valid && (peers & lt) == 0) mywc[d] = (uint16_t)(before + __popc(peers));
        __syncwarp();
        v[it] = (v[it] & vmask) | ((before + __popc(peers & lt)) << kTileValBits);
    }
    // exclusive scan of the digit totals over the digits
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < kDp; ++q) sum += tot[q];
    uint32_t inc = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += x;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();  // also: every warp's counters are complete
    uint32_t g = inc - sum;
    for (int w = 0; w < warp; ++w) g += wsum[w];
#pragma unroll
    for (int q = 0; q < kDp; ++q) {
        dbase[d0 + q] = g + pre[q];
        g += tot[q];
    }
#pragma unroll
    for (int q = 0; q < kDp; ++q) {  // per digit: exclusive scan over the warps (warp order = element order)
        uint32_t run = 0;
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = wc[w][d0 + q];
            wc[w][d0 + q] = (uint16_t)run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const bool valid = warp * (32 * kItems) + it * 32 + lane < cnt;
        uint32_t slot = 0x80000000u | lane;  // invalid lanes: a value no valid lane has
        if (valid) {
            const uint32_t d = (key[it] >> shift) & (kDigits - 1);
            const uint32_t pos = dbase[d] + wc[warp][d] + (v[it] >> kTileValBits);  // < n
            keys_out[pos] = key[it];
            vals_out[pos] = v[it] & vmask;
            slot = (pos / (uint32_t)kKeys) * kDigits + ((key[it] >> next_shift) & (kDigits - 1));
        }
        if (hist_next) {
            const unsigned peers = __match_any_sync(0xffffffffu, slot);
            if (valid && lane == __ffs(peers) - 1) atomicAdd(hist_next + slot, (uint32_t)__popc(peers));
        }
    }
}

// ---- hierarchy ----
__device__ __forceinline__ int common_prefix(const uint32_t* __restrict__ keys, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const uint32_t a = keys[i], b = keys[j];
    if (a == b) return 32 + __clz((uint32_t)(i ^ j));
    return __clz(a ^ b);
}

// internal node i (0 <= i < n - 1) of the hierarchy over the sorted keys
__device__ __forceinline__ void karras_node(const uint32_t* __restrict__ keys, int n, int i,
                                            BvhNode* __restrict__ nodes, int* __restrict__ parent_int,
                                            int* __restrict__ parent_leaf) {
    const int d = (common_prefix(keys, n, i, i + 1) - common_prefix(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = common_prefix(keys, n, i, i - d);
    int lmax = 2;
    while (common_prefix(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (common_prefix(keys, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = common_prefix(keys, n, i, j);
    int s = 0;
    for (int div = 2;; div <<= 1) {
        const int t = (l + div - 1) / div;
        if (common_prefix(keys, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
    }
    const int g = i + s * d + min(d, 0);
    const int left = (min(i, j) == g) ? ~g : g;
    const int right = (max(i, j) == g + 1) ? ~(g + 1) : g + 1;
    nodes[i].d = make_int4(left, right, min(i, j), max(i, j));  // links, leaf range [first, last]
    if (left < 0) parent_leaf[g] = i;
    else parent_int[g] = i;
    if (right < 0) parent_leaf[g + 1] = i;
    else parent_int[g + 1] = i;
    if (i == 0) parent_int[0] = -1;
}

// triangle record, leaf box and cleared arrival counter of leaf position p (0 <= p < n)
__device__ __forceinline__ void leaf_record(const float* __restrict__ verts, int n_verts,
                                            const int* __restrict__ tris, int n, int p,
                                            const uint32_t* __restrict__ order, TriRecord* __restrict__ recs,
                                            float4* __restrict__ box_leaf, uint32_t* __restrict__ flags) {
    if (p < n - 1) flags[p] = 0u;
    const int k = (int)order[p];
    f3 a, b, c;
    load_tri(verts, n_verts, tris, k, a, b, c);
    TriRecord r;
    r.v0 = make_float4(a.x, a.y, a.z, __int_as_float(k));
    r.e1 = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, 0.f);
    r.e2 = make_float4(c.x - a.x, c.y - a.y, c.z - a.z, 0.f);
    recs[p] = r;
    // box of the triangle, widened by a few ulps so that it also holds the
    // triangle v0 + u e1 + v e2 the intersection test actually sees
    float lo[3] = {fminf(a.x, fminf(b.x, c.x)), fminf(a.y, fminf(b.y, c.y)), fminf(a.z, fminf(b.z, c.z))};
    float hi[3] = {fmaxf(a.x, fmaxf(b.x, c.x)), fmaxf(a.y, fmaxf(b.y, c.y)), fmaxf(a.z, fmaxf(b.z, c.z))};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float pad = 4.0f * FLT_EPSILON * fmaxf(fabsf(lo[ax]), fabsf(hi[ax])) + 1e-30f;
        lo[ax] -= pad;
        hi[ax] += pad;
    }
    box_leaf[2 * (size_t)p] = make_float4(lo[0], lo[1], lo[2], 0.f);
    box_leaf[2 * (size_t)p + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
}

// triangle records in leaf order + leaf boxes + cleared arrival counters
__global__ void __launch_bounds__(256) leaf_kernel(const float* __restrict__ verts, int n_verts,
                                                   const int* __restrict__ tris, int n,
                                                   const uint32_t* __restrict__ order, TriRecord* __restrict__ recs,
                                                   float4* __restrict__ box_leaf, uint32_t* __restrict__ flags) {
    pdl_prologue();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) leaf_record(verts, n_verts, tris, n, p, order, recs, box_leaf, flags);
}

// the leaf records and the hierarchy in one launch (they read different outputs of the sort)
__global__ void __launch_bounds__(256) leaf_karras_kernel(const float* __restrict__ verts, int n_verts,
                                                          const int* __restrict__ tris, int n,
                                                          const uint32_t* __restrict__ keys,
                                                          const uint32_t* __restrict__ order,
                                                          TriRecord* __restrict__ recs, float4* __restrict__ box_leaf,
                                                          uint32_t* __restrict__ flags, BvhNode* __restrict__ nodes,
                                                          int* __restrict__ parent_int, int* __restrict__ parent_leaf) {
    pdl_prologue();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n - 1) karras_node(keys, n, p, nodes, parent_int, parent_leaf);
    if (p < n) leaf_record(verts, n_verts, tris, n, p, order, recs, box_leaf, flags);
}

__device__ __forceinline__ void child_box(int link, const float4* box_int, const float4* box_leaf, float4& lo,
                                          float4& hi) {
    const float4* b = link < 0 ? box_leaf + 2 * (size_t)(~link) : box_int + 2 * (size_t)link;
    lo = __ldcg(b);
    hi = __ldcg(b + 1);
}

// Bottom-up boxes: one thread per leaf climbs while it is the second to
// arrive at a node.  It carries its subtree's box in registers, so at a node
// it needs only the sibling's box; the node's links and parent (written by the
// hierarchy kernel) are loaded before its arrival counter, which leaves one
// dependent load per level after the atomic.
__global__ void __launch_bounds__(256) refit_kernel(int n, BvhNode* __restrict__ nodes,
                                                    const int* __restrict__ parent_int,
                                                    const int* __restrict__ parent_leaf, uint32_t* __restrict__ flags,
                                                    float4* __restrict__ box_int,
                                                    const float4* __restrict__ box_leaf) {
    pdl_prologue();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int me = ~p;  // link of the subtree this thread carries (leaf p)
    float4 lo = box_leaf[2 * (size_t)p], hi = box_leaf[2 * (size_t)p + 1];
    int node = parent_leaf[p];
    // at most n - 1 steps: each internal node is completed by exactly one thread
    for (int steps = 0; node >= 0 && steps < n; ++steps) {
        const int4 d = __ldcg(&nodes[node].d);
        const int up = __ldcg(parent_int + node);
        __threadfence();
        if (atomicAdd(flags + node, 1u) == 0u) return;  // first arrival: the sibling finishes this node
        const bool left = d.x == me;
        float4 sl, sh;
        child_box(left ? d.y : d.x, box_int, box_leaf, sl, sh);
        const float4 l0 = left ? lo : sl, h0 = left ? hi : sh, l1 = left ? sl : lo, h1 = left ? sh : hi;
        nodes[node].a = make_float4(l0.x, h0.x, l0.y, h0.y);
        nodes[node].b = make_float4(l1.x, h1.x, l1.y, h1.y);
        nodes[node].c = make_float4(l0.z, h0.z, l1.z, h1.z);
        lo = make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.f);
        hi = make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.f);
        box_int[2 * (size_t)node] = lo;
        box_int[2 * (size_t)node + 1] = hi;
        me = node;
        node = up;
    }
}

// one triangle: a root whose two links both point at leaf 0
__global__ void single_leaf_root_kernel(BvhNode* nodes, const float4* box_leaf) {
    pdl_prologue();
    const float4 lo = box_leaf[0], hi = box_leaf[1];
    nodes[0].a = make_float4(lo.x, hi.x, lo.y, hi.y);
    nodes[0].b = nodes[0].a;
    nodes[0].c = make_float4(lo.z, hi.z, lo.z, hi.z);
    nodes[0].d = make_int4(~0, ~0, 0, 0);
}

// ---- four-wide nodes for shadow rays
// One axis of a four-wide node: step s = the smallest power of two with
// extent / s <= 250 and s >= s_min, origin one step below the union's minimum
// (rounded down); child boxes quantised outwards (differences rounded away
// from the box, scaled exactly by 1 / s) and widened by one more step.  All in
// FP32 with directed rounding: the decoded box o + q s always holds the child's
// box with at least one step to spare on each side.
struct WideAxis {
    float o, s, inv_s;
};

// smallest power of two >= x (x a positive normal float)
__device__ __forceinline__ float pow2_ceil(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xffu;
    return __uint_as_float(((b & 0x7fffffu) ? e + 1u : e) << 23);
}

__device__ __forceinline__ WideAxis wide_axis(float lo, float hi, float s_min) {
    float x = __fmul_ru(__fsub_ru(hi, lo), 1.0f / 250.0f) * 1.0000002f;
    if (!(x >= s_min)) x = s_min;  // also catches a NaN extent
    const float s = pow2_ceil(fminf(x, 1e30f));
    return {__fsub_rd(lo, s), s, 1.0f / s};
}

__device__ __forceinline__ uint32_t wide_q(float v, const WideAxis& ax, bool upper) {
    const float t = upper ? __fsub_ru(v, ax.o) * ax.inv_s : __fsub_rd(v, ax.o) * ax.inv_s;
    float q = upper ? ceilf(t) + 1.0f : floorf(t) - 1.0f;
    q = fminf(fmaxf(q, 0.0f), 255.0f);  // NaN -> 0 (fmaxf returns the non-NaN operand)
    return (uint32_t)q;
}

__device__ __forceinline__ void write_wide_node(int k, const BvhNode* __restrict__ nodes,
                                                const float4* __restrict__ box_int,
                                                const float4* __restrict__ box_leaf, float s_min,
                                                WideNode* __restrict__ out) {
    int links[4];
    int nl = 0;
    const int4 d = nodes[k].d;
    const int c2[2] = {d.x, d.y};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (c2[h] < 0) {
            links[nl++] = c2[h];
        } else {
            const int4 e = nodes[c2[h]].d;
            links[nl++] = e.x;
            links[nl++] = e.y;
        }
    }
    float4 lo[4], hi[4];
    float ulo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, uhi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int q = 0; q < nl; ++q) {
        child_box(links[q], box_int, box_leaf, lo[q], hi[q]);
        ulo[0] = fminf(ulo[0], lo[q].x), ulo[1] = fminf(ulo[1], lo[q].y), ulo[2] = fminf(ulo[2], lo[q].z);
        uhi[0] = fmaxf(uhi[0], hi[q].x), uhi[1] = fmaxf(uhi[1], hi[q].y), uhi[2] = fmaxf(uhi[2], hi[q].z);
    }
    WideAxis ax[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ax[a] = wide_axis(ulo[a], uhi[a], s_min);
    uint32_t qlo[3] = {0, 0, 0}, qhi[3] = {0, 0, 0};
    int lk[4];
    for (int q = 0; q < 4; ++q) {
        uint32_t l3[3], h3[3];
        if (q < nl) {
            const float cl[3] = {lo[q].x, lo[q].y, lo[q].z}, ch[3] = {hi[q].x, hi[q].y, hi[q].z};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                l3[a] = wide_q(cl[a], ax[a], false);
                h3[a] = wide_q(ch[a], ax[a], true);
            }
            lk[q] = links[q];
        } else {  // empty slot: an inverted box on every axis
            l3[0] = l3[1] = l3[2] = 255u;
            h3[0] = h3[1] = h3[2] = 0u;
            lk[q] = INT_MIN;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            qlo[a] |= l3[a] << (8 * q);
            qhi[a] |= h3[a] << (8 * q);
        }
    }
    WideNode w;
    w.a = make_float4(ax[0].o, ax[1].o, ax[2].o, ax[0].s);
    w.b = make_float4(ax[1].s, ax[2].s, __uint_as_float(qlo[0]), __uint_as_float(qlo[1]));
    w.c = make_float4(__uint_as_float(qlo[2]), __uint_as_float(qhi[0]), __uint_as_float(qhi[1]),
                      __uint_as_float(qhi[2]));
    w.d = make_int4(lk[0], lk[1], lk[2], lk[3]);
    out[k] = w;
}

// Smallest quantisation step: 2^-17 of the largest coordinate magnitude of the
// root box, far above the FP32 rounding of slab distances for ray origins
// inside the scene's bounds (about 4 u |o - origin| per axis).
__device__ __forceinline__ float wide_min_step(const float4* box_int, const float4* box_leaf, int n) {
    const float4 lo = n > 1 ? box_int[0] : box_leaf[0], hi = n > 1 ? box_int[1] : box_leaf[1];
    const float m = fmaxf(fmaxf(fmaxf(fabsf(lo.x), fabsf(lo.y)), fmaxf(fabsf(lo.z), fabsf(hi.x))),
                          fmaxf(fabsf(hi.y), fabsf(hi.z)));
    return fmaxf(m * 7.62939453125e-6f, 1e-30f);
}

// Depth-first (pre-order) copy of the tree with escape links.  For a node
// whose subtree holds leaves [f, l], the nodes before it in pre-order are its
// ancestors plus the subtrees hanging to the left of its root path, which
// hold exactly the leaves [0, f): 2 f minus one per right turn of the path.
// Hence dfs = 2 f + (left turns on the path from the root), and the subtree
// of 2 (l - f) + 1 nodes ends just before skip = dfs + 2 (l - f) + 1.
// The same walk gives each internal node's depth: nodes at even depth also
// write their four-wide node, the others zero their slot.  A leaf's path is
// its parent's plus one step, so each internal node also writes the entries
// of its leaf children (one walk per internal node, none per leaf).
__global__ void __launch_bounds__(256) threaded_kernel(int n, const BvhNode* __restrict__ nodes,
                                                       const int* __restrict__ parent_int,
                                                       const int* __restrict__ parent_leaf,
                                                       const float4* __restrict__ box_int,
                                                       const float4* __restrict__ box_leaf, float4* gap,
                                                       int gap_vec4, ThreadedNode* __restrict__ out, float4* wgap,
                                                       int wgap_vec4, WideNode* __restrict__ wide) {
    pdl_prologue();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    // zero the alignment gaps before the arrays, so that equal meshes give equal bytes
    if (v < gap_vec4) gap[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v < wgap_vec4) wgap[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n == 1) {  // one triangle: a single leaf, and a four-wide root with that one leaf child
        if (v != 0) return;
        const float4 lo = box_leaf[0], hi = box_leaf[1];
        WideNode w;
        const float s_min = wide_min_step(box_int, box_leaf, 1);
        WideAxis ax[3] = {wide_axis(lo.x, hi.x, s_min), wide_axis(lo.y, hi.y, s_min), wide_axis(lo.z, hi.z, s_min)};
        const float cl[3] = {lo.x, lo.y, lo.z}, ch[3] = {hi.x, hi.y, hi.z};
        uint32_t ql[3], qh[3];
        for (int a = 0; a < 3; ++a) {
            ql[a] = 0xffffff00u | wide_q(cl[a], ax[a], false);
            qh[a] = wide_q(ch[a], ax[a], true);
        }
        w.a = make_float4(ax[0].o, ax[1].o, ax[2].o, ax[0].s);
        w.b = make_float4(ax[1].s, ax[2].s, __uint_as_float(ql[0]), __uint_as_float(ql[1]));
        w.c = make_float4(__uint_as_float(ql[2]), __uint_as_float(qh[0]), __uint_as_float(qh[1]),
                          __uint_as_float(qh[2]));
        w.d = make_int4(~0, INT_MIN, INT_MIN, INT_MIN);
        wide[0] = w;
        out[0].lo = make_float4(lo.x, lo.y, lo.z, __int_as_float(1));
        out[0].hi = make_float4(hi.x, hi.y, hi.z, __int_as_float(0));
        return;
    }
    // One thread per internal node: its path to the root gives its depth and left turns; a leaf child's
    // path is the node's plus one step (a left turn for the first child), so the node writes those too.
    if (v >= n - 1) return;
    const int k = v;
    const int4 d = nodes[k].d;
    const int f = d.z, l = d.w;
    int link = k, par = parent_int[k];
    int lefts = 0, depth = 0;
    for (int steps = 0; par >= 0 && steps < n; ++steps) {  // the path to the root is shorter than n
        if (nodes[par].d.x == link) ++lefts;
        ++depth;
        link = par;
        par = parent_int[par];
    }
    if ((depth & 1) == 0) write_wide_node(k, nodes, box_int, box_leaf, wide_min_step(box_int, box_leaf, n), wide);
    else wide[k] = WideNode{make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f),
                            make_float4(0.f, 0.f, 0.f, 0.f), make_int4(0, 0, 0, 0)};
    const int dfs = 2 * f + lefts;
    const int skip = dfs + 2 * (l - f) + 1;
    if (dfs >= 0 && dfs < 2 * n - 1) {  // always, for a well-formed tree
        const float4 lo = box_int[2 * (size_t)k], hi = box_int[2 * (size_t)k + 1];
        out[dfs].lo = make_float4(lo.x, lo.y, lo.z, __int_as_float(skip));
        out[dfs].hi = make_float4(hi.x, hi.y, hi.z, __int_as_float(-1));
    }
    const int kids[2] = {d.x, d.y};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (kids[h] >= 0) continue;
        const int q = ~kids[h];  // leaf position: range [q, q]
        const int dl = 2 * q + lefts + (h == 0 ? 1 : 0);
        if (dl < 0 || dl >= 2 * n - 1) continue;
        const float4 lo = box_leaf[2 * (size_t)q], hi = box_leaf[2 * (size_t)q + 1];
        out[dl].lo = make_float4(lo.x, lo.y, lo.z, __int_as_float(dl + 1));
        out[dl].hi = make_float4(hi.x, hi.y, hi.z, __int_as_float(q));
    }
}

}  // namespace

// depth-first copy and four-wide nodes (one launch; zeroes the alignment gaps)
static cudaError_t launch_threaded(int n, void* nodes_v, const BvhNode* nodes, const int* parent_int,
                                   const int* parent_leaf, const float4* box_int, const float4* box_leaf,
                                   cudaStream_t stream) {
    char* nb = static_cast<char*>(nodes_v);
    ThreadedNode* tn = reinterpret_cast<ThreadedNode*>(nb + threaded_offset(n));
    const size_t two_child = (size_t)(n > 1 ? n - 1 : 1) * sizeof(BvhNode);
    const int gap_vec4 = (int)((threaded_offset(n) - two_child) / 16);
    const size_t threaded_end = threaded_offset(n) + (size_t)(2 * n - 1) * sizeof(ThreadedNode);
    const int wgap_vec4 = (int)((wide_offset(n) - threaded_end) / 16);
    WideNode* wide = reinterpret_cast<WideNode*>(nb + wide_offset(n));
    // one thread per internal node (at least 32: the alignment gaps are zeroed by the first threads)
    launch_k(threaded_kernel, (std::max(n - 1, 32) + 255) / 256, 256, 0, stream, n, nodes, parent_int, parent_leaf,
             box_int, box_leaf, reinterpret_cast<float4*>(nb + two_child), gap_vec4, tn,
             reinterpret_cast<float4*>(nb + threaded_end), wgap_vec4, wide);
    return cudaGetLastError();
}

cudaError_t launch_build_bvh(const float* verts, int n_verts, const int* tris, int n, void* nodes_v, void* recs_v,
                             void* scratch, const BvhScratch& L, cudaStream_t stream) {
    char* s = static_cast<char*>(scratch);
    uint32_t* bounds = reinterpret_cast<uint32_t*>(s + L.bounds);
    uint32_t* keys[2] = {reinterpret_cast<uint32_t*>(s + L.keys0), reinterpret_cast<uint32_t*>(s + L.keys1)};
    uint32_t* vals[2] = {reinterpret_cast<uint32_t*>(s + L.vals0), reinterpret_cast<uint32_t*>(s + L.vals1)};
    uint32_t* hist = reinterpret_cast<uint32_t*>(s + L.hist);
    uint32_t* dtot = reinterpret_cast<uint32_t*>(s + L.digit_tot);
    int* parent_int = reinterpret_cast<int*>(s + L.parent_int);
    int* parent_leaf = reinterpret_cast<int*>(s + L.parent_leaf);
    uint32_t* flags = reinterpret_cast<uint32_t*>(s + L.flags);
    float4* box_int = reinterpret_cast<float4*>(s + L.box_int);
    float4* box_leaf = reinterpret_cast<float4*>(s + L.box_leaf);
    BvhNode* nodes = static_cast<BvhNode*>(nodes_v);
    TriRecord* recs = static_cast<TriRecord*>(recs_v);

    const int g256 = (n + 255) / 256;
    const bool tiled = bvh_tile_sort(n);
    const int n_tiles = (n + kTileKeys - 1) / kTileKeys;
    const int hist_vec4 = tiled ? kSortPasses * n_tiles * kDigits / 4 : 0;  // one row of counts per tile and pass
    launch_k(init_bounds_kernel, tiled ? std::min(64, (hist_vec4 + 255) / 256) : 1, tiled ? 256 : 32, 0, stream,
             bounds, reinterpret_cast<uint4*>(hist), hist_vec4);
    launch_k(centroid_bounds_kernel, g256, 256, 0, stream, verts, n_verts, tris, n, bounds);
    launch_k(morton_kernel, g256, 256, 0, stream, verts, n_verts, tris, n, bounds, keys[0], vals[0],
             tiled ? hist : nullptr);
    int cur = 0;
    for (int pass = 0; pass < kSortPasses; ++pass) {
        const int shift = pass * kSortDigitBits;
        if (tiled) {
            uint32_t* h = hist + (size_t)pass * n_tiles * kDigits;
            uint32_t* h_next = pass + 1 < kSortPasses ? h + (size_t)n_tiles * kDigits : nullptr;
            launch_k(tile_scatter_kernel<kTileThreads, kTileItems>, n_tiles, kTileThreads, 0, stream, keys[cur],
                     vals[cur], n, shift, n_tiles, h, h_next, shift + kSortDigitBits, keys[cur ^ 1], vals[cur ^ 1]);
        } else {
            launch_k(digit_hist_kernel, L.nblocks, kSortThreads, 0, stream, keys[cur], n, shift, L.nblocks, hist);
            launch_k(digit_scan_kernel, kDigits, 256, 0, stream, hist, L.nblocks, dtot);
            launch_k(digit_scatter_kernel, L.nblocks, kSortThreads, 0, stream, keys[cur], vals[cur], n, shift,
                     L.nblocks, hist, dtot, keys[cur ^ 1], vals[cur ^ 1]);
        }
        cur ^= 1;
    }
    if (n == 1) {
        launch_k(leaf_kernel, g256, 256, 0, stream, verts, n_verts, tris, n, vals[cur], recs, box_leaf, flags);
        launch_k(single_leaf_root_kernel, 1, 1, 0, stream, nodes, box_leaf);
    } else {
        launch_k(leaf_karras_kernel, g256, 256, 0, stream, verts, n_verts, tris, n, keys[cur], vals[cur], recs,
                 box_leaf, flags, nodes, parent_int, parent_leaf);
        launch_k(refit_kernel, g256, 256, 0, stream, n, nodes, parent_int, parent_leaf, flags, box_int, box_leaf);
    }
    return launch_threaded(n, nodes_v, nodes, parent_int, parent_leaf, box_int, box_leaf, stream);
}

// New vertex positions, same triangles: the leaf order (the final sort pass's
// values), the hierarchy links and the parent arrays from the last build stay;
// triangle records, leaf boxes, internal boxes and the depth-first copy are
// recomputed (3 launches instead of 16).
cudaError_t launch_refit_bvh(const float* verts, int n_verts, const int* tris, int n, void* nodes_v, void* recs_v,
                             void* scratch, const BvhScratch& L, cudaStream_t stream) {
    char* s = static_cast<char*>(scratch);
    // the sort's passes alternate between the two key/value buffers
    const uint32_t* order = reinterpret_cast<const uint32_t*>(s + (kSortPasses % 2 ? L.vals1 : L.vals0));
    int* parent_int = reinterpret_cast<int*>(s + L.parent_int);
    int* parent_leaf = reinterpret_cast<int*>(s + L.parent_leaf);
    uint32_t* flags = reinterpret_cast<uint32_t*>(s + L.flags);
    float4* box_int = reinterpret_cast<float4*>(s + L.box_int);
    float4* box_leaf = reinterpret_cast<float4*>(s + L.box_leaf);
    BvhNode* nodes = static_cast<BvhNode*>(nodes_v);
    TriRecord* recs = static_cast<TriRecord*>(recs_v);
    const int g256 = (n + 255) / 256;
    launch_k(leaf_kernel, g256, 256, 0, stream, verts, n_verts, tris, n, order, recs, box_leaf, flags);
    if (n == 1) launch_k(single_leaf_root_kernel, 1, 1, 0, stream, nodes, box_leaf);
    else launch_k(refit_kernel, g256, 256, 0, stream, n, nodes, parent_int, parent_leaf, flags, box_int, box_leaf);
    return launch_threaded(n, nodes_v, nodes, parent_int, parent_leaf, box_int, box_leaf, stream);
}

}  // namespace mcdi
