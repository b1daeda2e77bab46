// Device functions of the Monte Carlo direct-illumination estimator (Sec. 3.1,
// Sec. 4.1): BVH traversal, probe / cosine / GGX sampling and densities, the
// GGX lobe, and the per-sample MIS weight.  Everything is FP32.
#pragma once

#include <float.h>

#include "common.cuh"

namespace mcdi {

// ---------------------------------------------------------------- traversal
struct RayInv {
    f3 o, d, inv;
};

__device__ __forceinline__ RayInv make_ray(f3 o, f3 d) {
    // direction components are kept away from zero so that slab distances stay finite
    auto safe = [](float x) { return fabsf(x) < 1e-20f ? copysignf(1e-20f, x) : x; };
    RayInv r;
    r.o = o;
    r.d = d;
    r.inv = mk(1.0f / safe(d.x), 1.0f / safe(d.y), 1.0f / safe(d.z));
    return r;
}

// slab test of one box given as (lo.x, hi.x, lo.y, hi.y) + (lo.z, hi.z);
// returns the entry distance or +inf on a miss.  The exit distance is scaled by
// 1 + 2 gamma_3 so that rounding never drops a box the ray touches (Ize 2013).
__device__ __forceinline__ float slab(const RayInv& r, float4 xy, float2 z, float tmax) {
    const float tx0 = (xy.x - r.o.x) * r.inv.x, tx1 = (xy.y - r.o.x) * r.inv.x;
    const float ty0 = (xy.z - r.o.y) * r.inv.y, ty1 = (xy.w - r.o.y) * r.inv.y;
    const float tz0 = (z.x - r.o.z) * r.inv.z, tz1 = (z.y - r.o.z) * r.inv.z;
    const float t0 = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
    const float t1 = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax)) * 1.00000036f;
    return t0 <= t1 ? t0 : FLT_MAX;
}

// Moller-Trumbore, two-sided, edges inclusive, for the triangle v0 + u e1 + v e2;
// returns t (> 0) or +inf
__device__ __forceinline__ float tri_hit_v(const RayInv& r, f3 v0, f3 e1, f3 e2, float* bu, float* bv) {
    const f3 p = cross(r.d, e2);
    const float det = dot(e1, p);
    if (det == 0.0f) return FLT_MAX;
    const float inv = 1.0f / det;
    const f3 s = r.o - v0;
    const float u = dot(s, p) * inv;
    if (u < 0.0f || u > 1.0f) return FLT_MAX;
    const f3 q = cross(s, e1);
    const float v = dot(r.d, q) * inv;
    if (v < 0.0f || u + v > 1.0f) return FLT_MAX;
    const float t = dot(e2, q) * inv;
    if (!(t > 0.0f)) return FLT_MAX;
    if (bu) {
        *bu = u;
        *bv = v;
    }
    return t;
}

// the same test against triangle record k
__device__ __forceinline__ float tri_hit(const RayInv& r, const TriRecord* __restrict__ tris, int k, float* bu,
                                         float* bv) {
    const float4 v0 = __ldg(&tris[k].v0), e1 = __ldg(&tris[k].e1), e2 = __ldg(&tris[k].e2);
    return tri_hit_v(r, xyz(v0), xyz(e1), xyz(e2), bu, bv);
}

// slab test of a box given by its corners (xyz of lo and hi); same rounding
// rule as slab()
__device__ __forceinline__ bool slab_hit(const RayInv& r, float4 lo, float4 hi) {
    const float tx0 = (lo.x - r.o.x) * r.inv.x, tx1 = (hi.x - r.o.x) * r.inv.x;
    const float ty0 = (lo.y - r.o.y) * r.inv.y, ty1 = (hi.y - r.o.y) * r.inv.y;
    const float tz0 = (lo.z - r.o.z) * r.inv.z, tz1 = (hi.z - r.o.z) * r.inv.z;
    const float t0 = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
    const float t1 = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1)) * 1.00000036f;
    return t0 <= t1;
}

// One step of stackless any-hit traversal at node i of the depth-first
// layout: returns the next node index (> i), or -1 when the ray is blocked.
// kCount adds the triangle tests made to *tri_tests (traversal statistics).
template <bool kCount = false>
__device__ __forceinline__ int threaded_step(const ThreadedNode* __restrict__ tn, const TriRecord* __restrict__ tris,
                                             const RayInv& r, int i, unsigned* tri_tests = nullptr) {
    float4 lo, hi;  // one 32-byte load (the node array is 256-byte aligned, nodes 32 bytes)
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
        : "l"(tn + i));
    const int skip = __float_as_int(lo.w), tri = __float_as_int(hi.w);
    int next = skip;
    if (slab_hit(r, lo, hi)) {
        if (tri < 0) {
            next = i + 1;
        } else {
            if (kCount) ++*tri_tests;
            if (tri_hit(r, tris, tri, nullptr, nullptr) < FLT_MAX) return -1;
        }
    }
    return next > i ? next : i + 1;  // strictly increasing: at most 2 n - 1 steps
}

// any hit with t > 0 (shadow ray, no far limit): stackless traversal of the
// depth-first layout, no ordering needed since any blocker ends the ray
__device__ __forceinline__ bool any_hit_threaded(const void* nodes, const TriRecord* __restrict__ tris, int n_tris,
                                                 const RayInv& r) {
    if (n_tris <= 0) return false;
    const ThreadedNode* tn = threaded_nodes(nodes, n_tris);
    const int end = 2 * n_tris - 1;
    for (int i = 0; i < end;) {
        i = threaded_step(tn, tris, r, i);
        if (i < 0) return true;
    }
    return false;
}

// ---------------------------------------------------------------- four-wide traversal
constexpr int kWideStack = 24;          // pending nodes per ray; a deeper need falls back to the stackless walk
constexpr int kWideBlocked = -1;        // wide_step: a triangle blocks the ray
constexpr int kWideDone = -2;           // wide_step: nothing left to visit

// three-operand minimum / maximum (one instruction on sm_100 and later)
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// byte k of w in the low mantissa bits of 2^23: the float 2^23 + q, exact
__device__ __forceinline__ float qbyte(uint32_t w, int k) {
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u + (uint32_t)k));
}

// Slab tests of the four child boxes of a four-wide node; bit k of the result
// is set when the ray (t >= 0, no far limit) meets child k's box.  Per axis
// the near plane is the low one for a non-negative direction, the high one
// otherwise, so the plane at q needs no min / max:
//   t = (o + q s - origin) / d = (2^23 + q) A + B',  A = s / d,  B' = (o - origin) / d - 2^23 A,
// one fused multiply-add per plane (2^23 + q is the byte placed in a float's
// mantissa).  Rounding B' costs at most half a step of t, the other roundings
// far less for origins inside the scene's bounds; the boxes are widened by a
// whole step on every side, so a ray that meets a child's box passes its test.
__device__ __forceinline__ unsigned wide_child_hits(const RayInv& r, float4 a, float4 b, float4 c) {
    const uint32_t lox = __float_as_uint(b.z), loy = __float_as_uint(b.w), loz = __float_as_uint(c.x);
    const uint32_t hix = __float_as_uint(c.y), hiy = __float_as_uint(c.z), hiz = __float_as_uint(c.w);
    const bool px = r.inv.x >= 0.0f, py = r.inv.y >= 0.0f, pz = r.inv.z >= 0.0f;
    const uint32_t nx = px ? lox : hix, fx = px ? hix : lox;
    const uint32_t ny = py ? loy : hiy, fy = py ? hiy : loy;
    const uint32_t nz = pz ? loz : hiz, fz = pz ? hiz : loz;
    const float ax = a.w * r.inv.x, ay = b.x * r.inv.y, az = b.y * r.inv.z;
    const float bx = fmaf(-8388608.0f, ax, (a.x - r.o.x) * r.inv.x);
    const float by = fmaf(-8388608.0f, ay, (a.y - r.o.y) * r.inv.y);
    const float bz = fmaf(-8388608.0f, az, (a.z - r.o.z) * r.inv.z);
    unsigned m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float t0 = fmax3(fmaf(qbyte(nx, k), ax, bx), fmaf(qbyte(ny, k), ay, by),
                               fmaxf(fmaf(qbyte(nz, k), az, bz), 0.0f));
        const float t1 = fmin3(fmaf(qbyte(fx, k), ax, bx), fmaf(qbyte(fy, k), ay, by), fmaf(qbyte(fz, k), az, bz));
        m |= (t0 <= t1 ? 1u : 0u) << k;
    }
    return m;
}

// One node of the four-wide any-hit traversal: tests the node's children,
// tests the triangles of hit leaf children at once, continues with the first
// hit inner child and pushes the others.  Returns the next node, kWideBlocked
// or kWideDone.  Stack entry i lives at stack[i * kStride] (a thread's column
// of a shared-memory array, or a local array); a push beyond kWideStack sets
// *overflow instead (the caller then decides the ray by the stackless walk);
// kCount adds the triangle tests made to *tri_tests.
template <int kStride = 1, bool kCount = false>
__device__ __forceinline__ int wide_step(const WideNode* __restrict__ wn, const TriRecord* __restrict__ tris,
                                         const RayInv& r, int node, int* stack, int& sp, bool& overflow,
                                         unsigned* tri_tests = nullptr) {
    float4 a, b, c;
    int4 d;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(wn + node));
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(c.x), "=f"(c.y), "=f"(c.z), "=f"(c.w), "=r"(d.x), "=r"(d.y), "=r"(d.z), "=r"(d.w)
        : "l"(reinterpret_cast<const char*>(wn + node) + 32));
    const unsigned m = wide_child_hits(r, a, b, c);
    unsigned leaves = 0;
    int next = kWideDone;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int l = k == 0 ? d.x : k == 1 ? d.y : k == 2 ? d.z : d.w;
        if (!((m >> k) & 1u)) continue;
        if (l < 0) {
            leaves |= 1u << k;
        } else if (next == kWideDone) {
            next = l;
        } else if (sp < kWideStack) {
            stack[kStride * sp++] = l;
        } else {
            overflow = true;
        }
    }
    while (leaves) {
        const int k = __ffs(leaves) - 1;
        leaves &= leaves - 1;
        const int l = k == 0 ? d.x : k == 1 ? d.y : k == 2 ? d.z : d.w;
        if (kCount) ++*tri_tests;
        if (tri_hit(r, tris, ~l, nullptr, nullptr) < FLT_MAX) return kWideBlocked;
    }
    if (next == kWideDone && sp > 0) next = stack[kStride * --sp];
    return next;
}

// The node part of wide_step for a traversal that postpones its triangle
// tests: hit leaf children are appended to the lane's leaf queue
// (leafq[i * kStride], lq entries; the caller keeps room for four) instead of
// being tested.  Returns the next node or kWideDone.
template <int kStride>
__device__ __forceinline__ int wide_visit(const WideNode* __restrict__ wn, const RayInv& r, int node, int* stack,
                                          int& sp, bool& overflow, int* leafq, int& lq) {
    float4 a, b, c;
    int4 d;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(wn + node));
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(c.x), "=f"(c.y), "=f"(c.z), "=f"(c.w), "=r"(d.x), "=r"(d.y), "=r"(d.z), "=r"(d.w)
        : "l"(reinterpret_cast<const char*>(wn + node) + 32));
    const unsigned m = wide_child_hits(r, a, b, c);
    int next = kWideDone;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int l = k == 0 ? d.x : k == 1 ? d.y : k == 2 ? d.z : d.w;
        if (!((m >> k) & 1u)) continue;
        if (l < 0) {
            leafq[kStride * lq++] = l;
        } else if (next == kWideDone) {
            next = l;
        } else if (sp < kWideStack) {
            stack[kStride * sp++] = l;
        } else {
            overflow = true;
        }
    }
    if (next == kWideDone && sp > 0) next = stack[kStride * --sp];
    return next;
}

// any hit with t > 0 (shadow ray, no far limit) over the four-wide nodes
// (at most 2 n - 1 node visits: each node is pushed at most once)
__device__ __forceinline__ bool any_hit(const void* nodes, const TriRecord* __restrict__ tris, int n_tris,
                                        const RayInv& r) {
    if (n_tris <= 0) return false;
    const WideNode* wn = wide_nodes(nodes, n_tris);
    int stack[kWideStack];
    int sp = 0, node = 0;
    bool overflow = false, done = false;
    for (int it = 0; it < 2 * n_tris; ++it) {
        node = wide_step(wn, tris, r, node, stack, sp, overflow);
        if (node == kWideBlocked) return true;
        if (node == kWideDone) {
            done = true;
            break;
        }
    }
    return (overflow || !done) ? any_hit_threaded(nodes, tris, n_tris, r) : false;
}

// closest hit; returns the leaf (triangle record) index or -1
__device__ __forceinline__ int closest_hit(const BvhNode* __restrict__ nodes, const TriRecord* __restrict__ tris,
                                           int n_tris, const RayInv& r, float* t_out, float* bu, float* bv) {
    int best = -1;
    float tbest = FLT_MAX;
    if (n_tris <= 0) return -1;
    int stack[kTraversalStack];
    int sp = 0;
    int node = 0;
    for (int iter = 0; iter < n_tris + 1; ++iter) {
        float4 a, b, c;  // the 64-byte node as two 32-byte loads (node arrays are 256-byte aligned)
        int4 d;
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
            : "l"(nodes + node));
        asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(c.x), "=f"(c.y), "=f"(c.z), "=f"(c.w), "=r"(d.x), "=r"(d.y), "=r"(d.z), "=r"(d.w)
            : "l"(reinterpret_cast<const char*>(nodes + node) + 32));
        float t0 = slab(r, a, make_float2(c.x, c.y), tbest);
        float t1 = slab(r, b, make_float2(c.z, c.w), tbest);
        if (t0 < FLT_MAX && d.x < 0) {
            float u, v;
            const float t = tri_hit(r, tris, ~d.x, &u, &v);
            if (t < tbest) tbest = t, best = ~d.x, *bu = u, *bv = v;
            t0 = FLT_MAX;
        }
        if (t1 < FLT_MAX && d.y < 0) {
            float u, v;
            const float t = tri_hit(r, tris, ~d.y, &u, &v);
            if (t < tbest) tbest = t, best = ~d.y, *bu = u, *bv = v;
            t1 = FLT_MAX;
        }
        if (t0 < FLT_MAX && t1 < FLT_MAX) {
            const bool first0 = t0 <= t1;
            if (sp < kTraversalStack) stack[sp++] = first0 ? d.y : d.x;
            node = first0 ? d.x : d.y;
        } else if (t0 < FLT_MAX) {
            node = d.x;
        } else if (t1 < FLT_MAX) {
            node = d.y;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    *t_out = tbest;
    return best;
}

// ---------------------------------------------------------------- probe
// largest k in [0, n-1] with cdf[k] <= u
__device__ __forceinline__ int upper_index(const float* __restrict__ cdf, int n, float u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(cdf + mid) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// the same search with generic loads (the marginal lives in shared memory)
__device__ __forceinline__ int upper_index_generic(const float* cdf, int n, float u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cdf[mid] <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// (u, v) -> direction: phi = 2 pi u, theta = pi v, y up
__device__ __forceinline__ f3 dir_from_uv(float u, float v, float* sin_theta) {
    float sp, cp, st, ct;
    sincospif(2.0f * u, &sp, &cp);
    sincospif(v, &st, &ct);
    *sin_theta = st;
    return mk(st * cp, ct, st * sp);
}

struct Probe {
    const float4* env;
    const float* cond;
    const float* marg;  // read with generic loads: the kernels stage it in shared memory
    int W, H;
    bool on;  // total > 0
};

// the marginal CDF (H + 1 floats) copied into the block's shared memory; every
// thread of the block must call this before any of them returns
__device__ __forceinline__ void stage_marginal(Probe& P, float* s_marg) {
    for (int i = threadIdx.x; i <= P.H; i += blockDim.x) s_marg[i] = __ldg(P.marg + i);
    __syncthreads();
    P.marg = s_marg;
}

// probe texel of a direction and sin(theta) (accurate near the poles)
__device__ __forceinline__ int texel_of_dir(const Probe& P, f3 d, float* sin_theta) {
    const float st = sqrtf(d.x * d.x + d.z * d.z);
    float u = atan2f(d.z, d.x) * (0.5f * MCDI_INV_PI);
    if (u < 0.0f) u += 1.0f;
    const float v = atan2f(st, d.y) * MCDI_INV_PI;
    const int i = min(P.W - 1, (int)(u * (float)P.W));
    const int j = min(P.H - 1, (int)(v * (float)P.H));
    *sin_theta = st;
    return j * P.W + i;
}

// density of the probe technique at texel t for a direction with sin(theta) st
__device__ __forceinline__ float pdf_light_texel(const Probe& P, int t, float st) {
    if (!P.on || !(st > 0.0f)) return 0.0f;
    const int j = t / P.W, i = t - j * P.W;
    const float* c = P.cond + (size_t)j * (P.W + 1);
    const float wr = P.marg[j + 1] - P.marg[j];
    const float wc = __ldg(c + i + 1) - __ldg(c + i);
    return ((float)P.W * (float)P.H * wr * wc) / (2.0f * MCDI_PI * MCDI_PI * st);
}

// probe sample; returns false if the technique is off
__device__ __forceinline__ bool sample_light(const Probe& P, float u0, float u1, f3* d, int* texel, float* pdf) {
    if (!P.on) return false;
    const int j = upper_index_generic(P.marg, P.H, u0);
    const float m0 = P.marg[j], m1 = P.marg[j + 1];
    const float* c = P.cond + (size_t)j * (P.W + 1);
    const int i = upper_index(c, P.W, u1);
    const float c0 = __ldg(c + i), c1 = __ldg(c + i + 1);
    const float dv = fminf((u0 - m0) / (m1 - m0), 0.99999994f);
    const float du = fminf((u1 - c0) / (c1 - c0), 0.99999994f);
    float st;
    *d = dir_from_uv(((float)i + du) / (float)P.W, ((float)j + dv) / (float)P.H, &st);
    *texel = j * P.W + i;
    *pdf = st > 0.0f ? ((float)P.W * (float)P.H * (m1 - m0) * (c1 - c0)) / (2.0f * MCDI_PI * MCDI_PI * st) : 0.0f;
    return true;
}

// ---------------------------------------------------------------- frame + lobes
// orthonormal basis of Duff et al. 2017 (sign(0) = +1)
__device__ __forceinline__ void frame(f3 n, f3* b1, f3* b2) {
    const float s = n.z >= 0.0f ? 1.0f : -1.0f;
    const float a = -1.0f / (s + n.z);
    const float b = n.x * n.y * a;
    *b1 = mk(1.0f + s * n.x * n.x * a, s * b, -s * n.x);
    *b2 = mk(b, s + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ f3 sample_cosine(f3 n, f3 b1, f3 b2, float u0, float u1) {
    float sp, cp;
    sincospif(2.0f * u1, &sp, &cp);
    const float r = sqrtf(u0);
    const float z = sqrtf(1.0f - u0);
    return b1 * (r * cp) + b2 * (r * sp) + n * z;
}

// GGX normal distribution with the denominator term nh^2 (a2 - 1) + 1 written as
// sin^2 + nh^2 a2 (s2 = |n x h|^2): free of the cancellation of 1 - nh^2 near the
// lobe peak, which in FP32 would cost ~1e-3 relative accuracy at alpha ~ 0.006.
__device__ __forceinline__ float ggx_D_denom(float nh, float s2, float a2) { return s2 + nh * nh * a2; }
__device__ __forceinline__ float ggx_D(float nh, float s2, float a2) {
    if (!(nh > 0.0f)) return 0.0f;
    const float d = ggx_D_denom(nh, s2, a2);
    return a2 / (MCDI_PI * d * d);
}
__device__ __forceinline__ float sin2_between(f3 n, f3 h) {
    const f3 c = cross(n, h);
    return dot(c, c);
}

__device__ __forceinline__ float ggx_lambda(float c, float a2) {
    const float z = a2 * (1.0f / (c * c) - 1.0f);
    return 0.5f * (sqrtf(1.0f + z) - 1.0f);
}

// Heitz 2018 visible-normal sample, returns the reflected light direction
__device__ __forceinline__ f3 sample_ggx(f3 n, f3 b1, f3 b2, f3 wo, float alpha, float u0, float u1) {
    const f3 lo = mk(dot(wo, b1), dot(wo, b2), dot(wo, n));
    const f3 vh = normalize(mk(alpha * lo.x, alpha * lo.y, lo.z));
    const float lensq = vh.x * vh.x + vh.y * vh.y;
    f3 t1v = lensq > 0.0f ? mk(-vh.y, vh.x, 0.0f) * rsqrtf(lensq) : mk(1.0f, 0.0f, 0.0f);
    const f3 t2v = cross(vh, t1v);
    float sp, cp;
    sincospif(2.0f * u1, &sp, &cp);
    const float r = sqrtf(u0);
    const float t1 = r * cp;
    float t2 = r * sp;
    const float s = 0.5f * (1.0f + vh.z);
    t2 = (1.0f - s) * sqrtf(1.0f - t1 * t1) + s * t2;
    const float tz = sqrtf(fmaxf(0.0f, 1.0f - t1 * t1 - t2 * t2));
    const f3 nh = t1v * t1 + t2v * t2 + vh * tz;
    const f3 hl = normalize(mk(alpha * nh.x, alpha * nh.y, fmaxf(nh.z, 0.0f)));
    const f3 h = b1 * hl.x + b2 * hl.y + n * hl.z;
    const float voh = dot(wo, h);
    return h * (2.0f * voh) - wo;
}

__device__ __forceinline__ float pdf_ggx(f3 n, f3 wo, float co, float a2, float g1o, f3 wi) {
    f3 h = wi + wo;
    const float l2 = dot(h, h);
    if (!(l2 > 0.0f)) return 0.0f;
    h = h * rsqrtf(l2);
    if (!(dot(wo, h) > 0.0f)) return 0.0f;
    return g1o * ggx_D(dot(n, h), sin2_between(n, h), a2) / (4.0f * co);
}

__device__ __forceinline__ float schlick_weight(float vh) {
    const float x = 1.0f - fminf(fmaxf(vh, 0.0f), 1.0f);
    const float x2 = x * x;
    return x2 * x2 * x;
}

// ---------------------------------------------------------------- G-buffer
// direction of the camera ray through the centre of pixel (x, y), y down
__device__ __forceinline__ f3 camera_dir(const mcdi_camera& C, int x, int y, int W, int H) {
    const float sx = (2.0f * ((float)x + 0.5f) / (float)W - 1.0f) * C.tan_half_fovy * C.aspect;
    const float sy = (1.0f - 2.0f * ((float)y + 0.5f) / (float)H) * C.tan_half_fovy;
    return normalize(mk(C.forward[0] + sx * C.right[0] + sy * C.up[0], C.forward[1] + sx * C.right[1] + sy * C.up[1],
                        C.forward[2] + sx * C.right[2] + sy * C.up[2]));
}

// texel i of a texture stored with kCh floats per texel (4: float4, the 4th
// channel unused; 3: packed RGB), as a float4 with w = 0 for kCh = 3
template <int kCh>
__device__ __forceinline__ float4 texel(const float* __restrict__ tex, size_t i) {
    if constexpr (kCh == 4) {
        return __ldg(reinterpret_cast<const float4*>(tex) + i);
    } else {
        return make_float4(__ldg(tex + 3 * i), __ldg(tex + 3 * i + 1), __ldg(tex + 3 * i + 2), 0.0f);
    }
}

template <int kCh = 4>
__device__ __forceinline__ float4 bilinear(const float* __restrict__ tex, int S, float u, float v) {
    const float x = u * (float)S - 0.5f, y = v * (float)S - 0.5f;
    const float x0 = floorf(x), y0 = floorf(y);
    const float fx = x - x0, fy = y - y0;
    const int xi0 = min(max((int)x0, 0), S - 1), xi1 = min(max((int)x0 + 1, 0), S - 1);
    const int yi0 = min(max((int)y0, 0), S - 1), yi1 = min(max((int)y0 + 1, 0), S - 1);
    const float4 t00 = texel<kCh>(tex, (size_t)yi0 * S + xi0), t10 = texel<kCh>(tex, (size_t)yi0 * S + xi1);
    const float4 t01 = texel<kCh>(tex, (size_t)yi1 * S + xi0), t11 = texel<kCh>(tex, (size_t)yi1 * S + xi1);
    auto lerp = [](float a, float b, float t) { return a + (b - a) * t; };
    return make_float4(lerp(lerp(t00.x, t10.x, fx), lerp(t01.x, t11.x, fx), fy),
                       lerp(lerp(t00.y, t10.y, fx), lerp(t01.y, t11.y, fx), fy),
                       lerp(lerp(t00.z, t10.z, fx), lerp(t01.z, t11.z, fx), fy),
                       lerp(lerp(t00.w, t10.w, fx), lerp(t01.w, t11.w, fx), fy));
}

// The G-buffer entries of a primary hit on triangle k (original index) at
// barycentrics (u, v): interpolated position and normal, and the textures at
// the planar coordinate of the position (textures of kCh floats per texel);
// left as they are for bad vertex indices.
template <int kCh = 4>
__device__ __forceinline__ void gbuffer_hit(int k, float u, float v, const float* __restrict__ verts,
                                            const float* __restrict__ vnrm,
                                            const int* __restrict__ tri_idx, int n_verts,
                                            const float* __restrict__ tex_kd, const float* __restrict__ tex_korm,
                                            int S, float uv_ox, float uv_oz, float uv_s, float4* P, float4* Nn,
                                            float4* KD, float4* KORM) {
    const int i0 = tri_idx[3 * (size_t)k], i1 = tri_idx[3 * (size_t)k + 1], i2 = tri_idx[3 * (size_t)k + 2];
    if ((unsigned)i0 >= (unsigned)n_verts || (unsigned)i1 >= (unsigned)n_verts || (unsigned)i2 >= (unsigned)n_verts)
        return;
    const float w = 1.0f - u - v;
    float pp[3], nn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        pp[c] = w * verts[3 * (size_t)i0 + c] + u * verts[3 * (size_t)i1 + c] + v * verts[3 * (size_t)i2 + c];
        nn[c] = w * vnrm[3 * (size_t)i0 + c] + u * vnrm[3 * (size_t)i1 + c] + v * vnrm[3 * (size_t)i2 + c];
    }
    *P = make_float4(pp[0], pp[1], pp[2], 1.0f);
    *Nn = make_float4(nn[0], nn[1], nn[2], 0.0f);
    const float tu = (pp[0] - uv_ox) * uv_s, tv = (pp[2] - uv_oz) * uv_s;
    *KD = bilinear<kCh>(tex_kd, S, tu, tv);
    *KORM = bilinear<kCh>(tex_korm, S, tu, tv);
    KD->w = 0.f;
    KORM->w = 0.f;
}

// ---------------------------------------------------------------- per pixel
// Schlick's normal-incidence reflectance of the metallic blend (reading c1)
__device__ __forceinline__ f3 fresnel0(f3 kd, float m) {
    return mk(0.04f * (1.0f - m) + kd.x * m, 0.04f * (1.0f - m) + kd.y * m, 0.04f * (1.0f - m) + kd.z * m);
}

// the specular integrand's colour for probe radiance L: L (F0 + (1 - F0) q) ws, q the Schlick weight and ws
// the scalar rest of the term (D G2 / (4 cos_o) over the MIS denominator)
__device__ __forceinline__ f3 spec_colour(float4 L, f3 F0, float q, float ws) {
    return mk(L.x * (F0.x + (1.0f - F0.x) * q), L.y * (F0.y + (1.0f - F0.y) * q), L.z * (F0.z + (1.0f - F0.z) * q)) *
           ws;
}

struct Pixel {
    f3 p, n, wo, b1, b2;
    float lN, co, alpha, a2, g1o, r, m;
    f3 kd, F0;
    bool spec_on;
};

__device__ __forceinline__ bool load_pixel(float4 pos, float4 nrm, float4 kd, float4 korm, f3 cam, Pixel* px) {
    const f3 N = xyz(nrm);
    const float l2 = dot(N, N);
    if (!(pos.w > 0.0f) || !(l2 > 0.0f)) return false;
    px->lN = sqrtf(l2);
    px->n = N * (1.0f / px->lN);
    px->p = xyz(pos);
    px->wo = normalize(cam - px->p);
    px->co = dot(px->n, px->wo);
    px->spec_on = px->co >= 1e-4f;
    px->r = korm.y;
    px->m = korm.z;
    px->alpha = fmaxf(px->r * px->r, 1e-4f);
    px->a2 = px->alpha * px->alpha;
    px->g1o = px->spec_on ? 1.0f / (1.0f + ggx_lambda(px->co, px->a2)) : 0.0f;
    px->kd = xyz(kd);
    px->F0 = fresnel0(px->kd, px->m);
    frame(px->n, &px->b1, &px->b2);
    return true;
}

// One sample of the MIS estimator: direction, texel and 1/denominator.
// Returns false when the sample does not contribute (technique off, below the
// horizon, zero density).
__device__ __forceinline__ bool draw_sample(const Probe& P, const Pixel& px, int n_light, int n_cos, int n_ggx,
                                            int j, float2 u, f3* wi, int* texel, float* ci, float* inv_denom) {
    float pl = 0.0f, st = 0.0f;
    int t = -1;
    if (j < n_light) {
        if (!sample_light(P, u.x, u.y, wi, &t, &pl)) return false;
    } else if (j < n_light + n_cos) {
        *wi = sample_cosine(px.n, px.b1, px.b2, u.x, u.y);
    } else {
        if (!px.spec_on) return false;
        *wi = sample_ggx(px.n, px.b1, px.b2, px.wo, px.alpha, u.x, u.y);
    }
    const float c = dot(px.n, *wi);
    if (!(c > 0.0f)) return false;
    if (t < 0) {
        t = texel_of_dir(P, *wi, &st);
        pl = pdf_light_texel(P, t, st);
    }
    float denom = (float)n_light * pl + (float)n_cos * (c * MCDI_INV_PI);
    if (px.spec_on && n_ggx > 0) denom += (float)n_ggx * pdf_ggx(px.n, px.wo, px.co, px.a2, px.g1o, *wi);
    if (!(denom > 0.0f)) return false;
    *texel = t;
    *ci = c;
    *inv_denom = 1.0f / denom;
    return true;
}

}  // namespace mcdi
