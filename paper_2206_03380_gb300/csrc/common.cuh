// Device-side building blocks shared by the mcdi kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pdl.cuh"

#define MCDI_PI 3.14159265358979323846f
#define MCDI_INV_PI 0.318309886183790671538f

namespace mcdi {

// ---------------------------------------------------------------- float3 math
struct f3 {
    float x, y, z;
};
__device__ __forceinline__ f3 mk(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator*(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ f3 operator*(float s, f3 a) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ f3 normalize(f3 a) { return a * rsqrtf(dot(a, a)); }
__device__ __forceinline__ f3 xyz(float4 v) { return {v.x, v.y, v.z}; }

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC 2011).  Ten rounds of the 4x32 S-box with multipliers 0xD2511F53 and
// 0xCD9E8D57 and the Weyl key schedule 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo_a = 0xD2511F53u * c.x, hi_a = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo_b = 0xCD9E8D57u * c.z, hi_b = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi_b ^ c.y ^ k.x, lo_b, hi_a ^ c.w ^ k.y, lo_a);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// The two uniforms of sample `j` of `pixel` in `view`: 24-bit fractions
// (x >> 8) * 2^-24, exact in float.
__device__ __forceinline__ float2 sample_uniforms(unsigned long long seed, uint32_t pixel, uint32_t view, uint32_t j,
                                                  uint32_t stream) {
    const uint4 x = philox4x32_10(make_uint4(pixel, view, j, stream),
                                  make_uint2((uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32)));
    return make_float2((float)(x.x >> 8) * 5.9604644775390625e-8f, (float)(x.y >> 8) * 5.9604644775390625e-8f);
}

// ---------------------------------------------------------------- mesh
// triangle k's corners; a bad vertex index gives a degenerate triangle at the
// origin, which no ray hits
__device__ __forceinline__ void load_tri(const float* __restrict__ verts, int n_verts, const int* __restrict__ tris,
                                         int k, f3& a, f3& b, f3& c) {
    const int i0 = tris[3 * (size_t)k], i1 = tris[3 * (size_t)k + 1], i2 = tris[3 * (size_t)k + 2];
    if ((unsigned)i0 >= (unsigned)n_verts || (unsigned)i1 >= (unsigned)n_verts || (unsigned)i2 >= (unsigned)n_verts) {
        a = b = c = mk(0.f, 0.f, 0.f);  // bad index: degenerate triangle, never hit
        return;
    }
    a = mk(verts[3 * (size_t)i0], verts[3 * (size_t)i0 + 1], verts[3 * (size_t)i0 + 2]);
    b = mk(verts[3 * (size_t)i1], verts[3 * (size_t)i1 + 1], verts[3 * (size_t)i1 + 2]);
    c = mk(verts[3 * (size_t)i2], verts[3 * (size_t)i2 + 1], verts[3 * (size_t)i2 + 2]);
}

// ---------------------------------------------------------------- BVH layout
// Internal node of a binary BVH, 64 bytes: the bounds of both children (so one
// node fetch tests two boxes) and the two child links.  link >= 0: internal
// node index; link < 0: leaf, ~link = index into the triangle records.
struct __align__(16) BvhNode {
    float4 a;  // child0 lo.x, hi.x, lo.y, hi.y
    float4 b;  // child1 lo.x, hi.x, lo.y, hi.y
    float4 c;  // child0 lo.z, hi.z, child1 lo.z, hi.z
    int4 d;    // child0 link, child1 link, -, -
};

// Triangle in leaf order, 48 bytes: v0 (w = original triangle index as int
// bits), e1 = v1 - v0, e2 = v2 - v0.
struct __align__(16) TriRecord {
    float4 v0;
    float4 e1;
    float4 e2;
};

// Node of the same tree in depth-first (pre-order) layout with escape links,
// 32 bytes, for stackless traversal: the first child of an internal node is
// the next node; `skip` is the node that follows the subtree (the escape link
// taken when the box is missed or a leaf is done).  The array follows the
// two-child nodes in the same allocation.
struct __align__(32) ThreadedNode {
    float4 lo;  // xyz: box minimum, w: skip index (int bits)
    float4 hi;  // xyz: box maximum, w: triangle-record index (int bits) of a leaf, -1 for an internal node
};

__host__ __device__ inline size_t threaded_offset(int n_tris) {
    const size_t n_int = (size_t)(n_tris > 1 ? n_tris - 1 : 1);
    return (n_int * sizeof(BvhNode) + 255) & ~(size_t)255;
}

__host__ __device__ inline const ThreadedNode* threaded_nodes(const void* nodes, int n_tris) {
    return reinterpret_cast<const ThreadedNode*>(static_cast<const char*>(nodes) + threaded_offset(n_tris));
}

// Four-wide node with compressed child boxes, 64 bytes, for shadow rays.  It
// stands for a two-child node at even depth of the same tree together with its
// children: its children are that node's grandchildren (or its children where
// those are leaves), so one fetch tests up to four boxes.  Child k's box on
// axis x is [o.x + qlo_x[k] s.x, o.x + qhi_x[k] s.x] with 8-bit q and a power
// of two s, rounded outwards by at least one step s, which is what keeps the
// slab test conservative in FP32 (the rounding of the slab distances stays
// below one step for ray origins inside the scene's bounds).  An empty slot
// has qlo = 255 and qhi = 0 on every axis, a box no ray hits.  Links: >= 0
// index of a four-wide node (the node array is indexed like the two-child
// nodes; odd-depth slots are unused and zero), < 0 leaf, ~link = index into
// the triangle records.
struct __align__(64) WideNode {
    float4 a;  // o.x, o.y, o.z, s.x
    float4 b;  // s.y, s.z, qlo_x[0..3] (bytes), qlo_y[0..3]
    float4 c;  // qlo_z[0..3], qhi_x[0..3], qhi_y[0..3], qhi_z[0..3]
    int4 d;    // links of children 0..3
};

__host__ __device__ inline size_t wide_offset(int n_tris) {
    const size_t n = (size_t)(n_tris > 0 ? n_tris : 1);
    return (threaded_offset(n_tris) + (2 * n - 1) * sizeof(ThreadedNode) + 255) & ~(size_t)255;
}

__host__ __device__ inline const WideNode* wide_nodes(const void* nodes, int n_tris) {
    return reinterpret_cast<const WideNode*>(static_cast<const char*>(nodes) + wide_offset(n_tris));
}

constexpr int kTraversalStack = 64;  // >= depth of a tree over 62-bit unique keys

}  // namespace mcdi
