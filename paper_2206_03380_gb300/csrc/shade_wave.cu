// Wavefront form of the forward estimator (Sec. 3.1, 4.1, 4.2): the same
// samples, weights and shadow rays as shade_fwd_kernel, split so that the
// incoherent shadow-ray traversal runs in a lean kernel of its own.
//
//   gen    one thread per pixel: draws every sample; for a sample with a shadow
//          ray it writes the scalars of its unshadowed contribution (probe texel,
//          diffuse and specular weights, 16 bytes) to slot j*P + pixel and
//          appends the ray to a dense ray list (a warp's rays for one sample
//          index stay together: neighbouring pixels, same technique, nearby
//          origins and similar directions); a sample without one (it
//          contributes nothing) only marks its slot;
//   trace  persistent warps pull rays from a global counter; a lane whose ray
//          has finished takes the next ray at the next refill, so lanes do not
//          wait for the warp's longest ray;
//   accum  one thread per pixel: rebuilds each marked-active sample's c_d and c_s
//          parts from its scalars (the same arithmetic as gen), sums
//          contribution_j x H_j in sample order j = 0..S-1 (bitwise repeatable)
//          and packs the visibility mask.
#include "common.cuh"
#include "internal.h"
#include "shading.cuh"

namespace mcdi {
namespace {

constexpr int kGenThreads = 128;
constexpr int kTraceThreads = 128;
constexpr int kTraceBlocksPerSM = 8;
constexpr int kTraceStepsPerRefill = 8;
constexpr int kLeafQueue = 8;   // postponed triangle tests per lane
constexpr int kLeafBatch = 16;  // lanes holding one that start a triangle round

struct WaveBuffers {
    float4* ray;        // [rays] direction, w = slot index (int bits) of the sample
    float4* origin;     // [P] shadow-ray origin of each covered pixel (p + ray_eps n)
    float4* rec;        // [slots] active samples: probe texel (int bits), diffuse weight, Schlick weight,
                        // specular weight (c_d = L sd, c_s = spec_colour(L, F0, q, ws), L the texel's radiance)
    uint8_t* hit;       // [slots] 0 shadow ray clear, 1 blocked, 2 no shadow ray (the sample contributes nothing)
    unsigned* counter;  // [0] rays appended by gen, [1] trace work queue head
};

// byte offsets of the arrays (P pixels, slots = P spp), 256-byte aligned
__host__ __device__ __forceinline__ size_t wave_origin_offset(long long slots) { return align256((size_t)slots * 16); }
__host__ __device__ __forceinline__ size_t wave_contrib_offset(long long P, long long slots) {
    return wave_origin_offset(slots) + align256((size_t)P * 16);
}
__host__ __device__ __forceinline__ size_t wave_hit_offset(long long P, long long slots) {
    return wave_contrib_offset(P, slots) + align256((size_t)slots * 16);
}
__host__ __device__ __forceinline__ size_t wave_counter_offset(long long P, long long slots) {
    return wave_hit_offset(P, slots) + align256((size_t)slots);
}

__device__ __forceinline__ WaveBuffers wave_buffers(void* ws, long long P, long long slots) {
    char* p = static_cast<char*>(ws);
    WaveBuffers b;
    b.ray = reinterpret_cast<float4*>(p);
    b.origin = reinterpret_cast<float4*>(p + wave_origin_offset(slots));
    b.rec = reinterpret_cast<float4*>(p + wave_contrib_offset(P, slots));
    b.hit = reinterpret_cast<uint8_t*>(p + wave_hit_offset(P, slots));
    b.counter = reinterpret_cast<unsigned*>(p + wave_counter_offset(P, slots));
    return b;
}

__device__ __forceinline__ Probe wave_probe(const ShadeArgs& a) {
    Probe P;
    P.env = a.env;
    P.cond = a.cond;
    P.marg = a.marg;
    P.W = a.Wp;
    P.H = a.Hp;
    P.on = *a.total > 0.0;
    return P;
}

__global__ void wave_reset_kernel(void* ws, long long P, long long slots) {
    pdl_prologue();
    WaveBuffers B = wave_buffers(ws, P, slots);
    B.counter[0] = 0u;
    B.counter[1] = 0u;
}

// A CTA covers 32 consecutive pixels with kGenQuarters warps; warp q draws the
// samples j = q, q + 4, q + 8, ... of its lane's pixel (strided, so every warp
// gets a mix of the three techniques), which keeps four times as many
// independent sample chains in flight as one thread per pixel would.
// Active shadow rays are appended densely (one atomic per warp and sample):
// a warp's rays for sample j stay together (32 neighbouring pixels, one
// technique), so the tracer sees coherent batches and no empty slots.  What
// a sample writes goes to its own slot j * P + pixel, so the results do not
// depend on which warp drew it.
constexpr int kGenQuarters = kGenThreads / 32;

__global__ void __launch_bounds__(kGenThreads) wave_gen_kernel(ShadeArgs a, void* ws, float4* __restrict__ kd_out) {
    pdl_prologue();
    extern __shared__ float s_marg[];
    const int lane = threadIdx.x & 31, quarter = threadIdx.x >> 5;
    const long long idx0 = (long long)blockIdx.x * 32 + lane;
    const long long P = (long long)a.N * a.H * a.W;
    const int spp = a.n_light + a.n_cos + a.n_ggx;
    const long long slots = P * spp;
    WaveBuffers B = wave_buffers(ws, P, slots);
    const bool in_range = idx0 < P;
    const long long idx = in_range ? idx0 : P - 1;  // out-of-range lanes idle but join the warp votes
    const int view = (int)(idx / ((long long)a.H * a.W));
    const uint32_t pix = (uint32_t)(idx - (long long)view * a.H * a.W);
    Pixel px;
    const mcdi_camera& C = a.cams[view];
    const bool covered = in_range && load_pixel(a.gb_pos[idx], a.gb_nrm[idx], a.gb_kd[idx], a.gb_korm[idx],
                                                mk(C.origin[0], C.origin[1], C.origin[2]), &px);
    if (in_range && quarter == 0)
        kd_out[idx] = covered ? make_float4(px.kd.x * (1.f - px.m), px.kd.y * (1.f - px.m),
                                            px.kd.z * (1.f - px.m), 0.f)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
    Probe Pr = wave_probe(a);
    stage_marginal(Pr, s_marg);
    const f3 origin = covered ? px.p + px.n * a.ray_eps : mk(0.f, 0.f, 0.f);
    if (covered && quarter == 0) B.origin[idx] = make_float4(origin.x, origin.y, origin.z, 0.0f);
    for (int j = quarter; j < spp; j += kGenQuarters) {
        const long long s = (long long)j * P + idx;
        f3 wi = mk(0.f, 0.f, 0.f);
        float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
        bool active = false;
        if (covered) {
            int t;
            float ci, inv_denom;
            const float2 u = sample_uniforms(a.seed, pix, (uint32_t)view, (uint32_t)j, a.stream_word);
            if (draw_sample(Pr, px, a.n_light, a.n_cos, a.n_ggx, j, u, &wi, &t, &ci, &inv_denom)) {
                active = true;
                rec.x = __int_as_float(t);
                rec.y = ci * MCDI_INV_PI * inv_denom;  // c_d = L rec.y
                if (px.spec_on) {
                    const f3 h = normalize(wi + px.wo);
                    const float D = ggx_D(dot(px.n, h), sin2_between(px.n, h), px.a2);
                    const float G2 = 1.0f / (1.0f + ggx_lambda(ci, px.a2) + ggx_lambda(px.co, px.a2));
                    rec.z = schlick_weight(dot(px.wo, h));
                    rec.w = D * G2 / (4.0f * px.co) * inv_denom;  // c_s = spec_colour(L, F0, rec.z, rec.w)
                }
            }
        }
        const unsigned act = __ballot_sync(0xffffffffu, active);
        if (act) {
            const int leader = __ffs(act) - 1;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(B.counter, (unsigned)__popc(act));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (active) {
                const unsigned r = base + __popc(act & ((1u << lane) - 1u));
                B.ray[r] = make_float4(wi.x, wi.y, wi.z, __int_as_float((int)s));
            }
        }
        if (!in_range) continue;
        B.hit[s] = active ? 0 : 2;  // every slot, so that the accumulation needs no coverage test
        if (active) B.rec[s] = rec;
    }
}

// Persistent any-hit tracer with per-lane refill.  A lane holds one ray, the
// four-wide node it visits next, a short stack of pending nodes and a queue of
// leaf triangles whose boxes the ray hit (columns of shared-memory arrays);
// every kTraceStepsPerRefill steps the warp refills the lanes that are idle
// from the global slot counter.  A step visits one node per lane; triangle
// tests are postponed and run as warp-wide rounds, one triangle per lane with
// a non-empty queue, once kLeafBatch lanes hold one or a lane must drain its
// queue (its nodes are done, or the queue cannot take another node's four
// leaves), so most rounds run with many lanes converged instead of a few
// lanes testing while the rest wait.  A ray whose pending nodes outgrow the
// stack is decided by the stackless walk of the depth-first copy instead.
__global__ void __launch_bounds__(kTraceThreads, kTraceBlocksPerSM) wave_trace_kernel(
    const void* __restrict__ nodes, const TriRecord* __restrict__ tris, int n_tris, void* ws, long long P,
    long long slots) {
    pdl_prologue();
    WaveBuffers B = wave_buffers(ws, P, slots);
    const long long n_rays = (long long)*((volatile unsigned*)B.counter);
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    long long ray = -1;  // -1 idle, -2 no work left, >= 0 tracing
    int slot = 0;
    RayInv r;
    int node = 0, sp = 0, lq = 0;
    bool overflow = false;
    // one column per thread, so a warp's accesses fall in 32 different banks
    __shared__ int s_stack[kWideStack * kTraceThreads];
    __shared__ int s_leaf[kLeafQueue * kTraceThreads];
    int* stack = s_stack + threadIdx.x;
    int* leafq = s_leaf + threadIdx.x;
    if (n_tris <= 0) return;  // nothing can block a ray; gen already wrote misses
    const WideNode* wn = wide_nodes(nodes, n_tris);
    while (true) {
        const unsigned need = __ballot_sync(full, ray == -1);
        if (need) {
            const int leader = __ffs(need) - 1;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(B.counter + 1, (unsigned)__popc(need));
            base = __shfl_sync(full, base, leader);
            if (ray == -1) {
                const long long my = (long long)base + __popc(need & lt);
                if (my >= n_rays) {
                    ray = -2;
                } else {
                    const float4 d = __ldg(B.ray + my);
                    slot = __float_as_int(d.w);
                    const float4 o = __ldg(B.origin + (uint32_t)slot % (uint32_t)P);  // slots < 2^31
                    r = make_ray(mk(o.x, o.y, o.z), mk(d.x, d.y, d.z));
                    node = 0;
                    sp = 0;
                    lq = 0;
                    overflow = false;
                    ray = my;
                }
            }
        }
        if (__all_sync(full, ray == -2)) break;
        // kTraceStepsPerRefill steps; every node is visited at most once, so a ray
        // ends within n - 1 node visits and as many triangle rounds
        for (int step = 0; step < kTraceStepsPerRefill; ++step) {
            const bool act = ray >= 0;
            // a visit appends at most four leaves: a fuller queue waits for the rounds it forces
            if (act && node >= 0 && lq <= kLeafQueue - 4)
                node = wide_visit<kTraceThreads>(wn, r, node, stack, sp, overflow, leafq, lq);
            const bool pend = act && lq > 0;
            const bool must = pend && (node == kWideDone || lq > kLeafQueue - 4);
            const unsigned vote = __ballot_sync(full, pend);
            if (__popc(vote) >= kLeafBatch || __any_sync(full, must)) {
                if (pend) {
                    const int l = leafq[kTraceThreads * --lq];
                    if (tri_hit(r, tris, ~l, nullptr, nullptr) < FLT_MAX) {
                        B.hit[slot] = 1;
                        ray = -1;
                    }
                }
            }
            if (ray >= 0 && node == kWideDone && lq == 0) {  // nodes done and no triangle left: a miss
                if (overflow && any_hit_threaded(nodes, tris, n_tris, r)) B.hit[slot] = 1;
                ray = -1;
            }
        }
    }
}

__global__ void __launch_bounds__(kGenThreads) wave_accum_kernel(ShadeArgs a, const void* ws,
                                                                 float4* __restrict__ c_d, float4* __restrict__ c_s,
                                                                 uint32_t* __restrict__ vis_mask) {
    pdl_prologue();
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long P = (long long)a.N * a.H * a.W;
    if (idx >= P) return;
    const int spp = a.n_light + a.n_cos + a.n_ggx;
    const int nwords = (spp + 31) >> 5;
    const long long slots = P * spp;
    WaveBuffers B = wave_buffers(const_cast<void*>(ws), P, slots);
    // every slot is marked (uncovered pixels' slots as without a shadow ray), so an uncovered pixel
    // sums nothing and its outputs come out zero
    const float hv = 1.0f - a.tau;
    f3 F0 = mk(0.f, 0.f, 0.f);  // formed as load_pixel forms it in gen, at the first active sample
    bool have_f0 = false;
    f3 cd = mk(0.f, 0.f, 0.f), cs = cd;
    uint32_t word = 0;
    for (int j = 0; j < spp; ++j) {
        const long long s = (long long)j * P + idx;
        const uint8_t h = B.hit[s];
        if (h == 1) word |= 1u << (j & 31);
        if (h != 2) {  // a sample without a shadow ray contributes nothing
            if (!have_f0) {
                F0 = fresnel0(xyz(a.gb_kd[idx]), a.gb_korm[idx].z);
                have_f0 = true;
            }
            const float Hv = h ? hv : 1.0f;
            const float4 rec = B.rec[s];
            const float4 L = __ldg(a.env + __float_as_int(rec.x));
            cd = cd + mk(L.x, L.y, L.z) * rec.y * Hv;
            cs = cs + spec_colour(L, F0, rec.z, rec.w) * Hv;
        }
        if (vis_mask && ((j & 31) == 31 || j == spp - 1)) {
            vis_mask[(size_t)idx * nwords + (j >> 5)] = word;
            word = 0;
        }
    }
    c_d[idx] = make_float4(cd.x, cd.y, cd.z, 0.f);
    c_s[idx] = make_float4(cs.x, cs.y, cs.z, 0.f);
}

// Traversal statistics: the rays of the last forward pass re-traced one per
// thread, with counters (stats[0] rays, [1] node visits = 64-byte four-wide
// node fetches, [2] triangle tests, [3] rays blocked, [4] rays whose result
// differs from the forward's hit flag).  Warp sums, one 64-bit atomic each.
__global__ void __launch_bounds__(kTraceThreads) wave_stats_kernel(const void* __restrict__ nodes,
                                                                   const TriRecord* __restrict__ tris, int n_tris,
                                                                   const void* ws, long long P, long long slots,
                                                                   unsigned long long* __restrict__ stats) {
    pdl_prologue();
    WaveBuffers B = wave_buffers(const_cast<void*>(ws), P, slots);
    const long long n_rays = (long long)B.counter[0];
    unsigned long long c[5] = {0, 0, 0, 0, 0};
    const WideNode* wn = wide_nodes(nodes, n_tris > 0 ? n_tris : 1);
    int stack[kWideStack];
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_rays;
         k += (long long)gridDim.x * blockDim.x) {
        const float4 d = B.ray[k];
        const int slot = __float_as_int(d.w);
        const float4 o = B.origin[(uint32_t)slot % (uint32_t)P];
        const RayInv r = make_ray(mk(o.x, o.y, o.z), mk(d.x, d.y, d.z));
        bool blocked = false, overflow = false;
        unsigned tests = 0;
        int node = 0, sp = 0;
        for (int it = 0; it < 2 * n_tris && node >= 0; ++it) {
            ++c[1];
            node = wide_step<1, true>(wn, tris, r, node, stack, sp, overflow, &tests);
        }
        blocked = node == kWideBlocked || (node >= 0 || overflow ? any_hit_threaded(nodes, tris, n_tris, r) : false);
        c[0] += 1;
        c[2] += tests;
        c[3] += blocked;
        c[4] += blocked != (B.hit[slot] != 0);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        unsigned long long v = c[q];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(stats + q, v);
    }
}

}  // namespace

cudaError_t launch_shadow_ray_stats(const ShadeArgs& a, const void* ws, unsigned long long* stats,
                                    cudaStream_t stream) {
    const long long P = (long long)a.N * a.H * a.W, slots = P * (a.n_light + a.n_cos + a.n_ggx);
    cudaError_t e = cudaMemsetAsync(stats, 0, 5 * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    launch_k(wave_stats_kernel, sms * 8, kTraceThreads, 0, stream, a.nodes, static_cast<const TriRecord*>(a.tris),
             a.n_tris, ws, P, slots, stats);
    return cudaGetLastError();
}

cudaError_t launch_shadow_ray_retrace(const ShadeArgs& a, void* ws, cudaStream_t stream) {
    const long long P = (long long)a.N * a.H * a.W, slots = P * (a.n_light + a.n_cos + a.n_ggx);
    // rewind the work queue head; the rays, and the hit flags they set again, stay as they are
    cudaError_t e = cudaMemsetAsync(static_cast<char*>(ws) + wave_counter_offset(P, slots) + sizeof(unsigned), 0,
                                    sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152, per_sm = 8;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wave_trace_kernel, kTraceThreads, 0);
    if (per_sm < 1) per_sm = 1;
    launch_k(wave_trace_kernel, sms * per_sm, kTraceThreads, 0, stream, a.nodes, static_cast<const TriRecord*>(a.tris),
             a.n_tris, ws, P, slots);
    return cudaGetLastError();
}

size_t shade_workspace_bytes(long long P, int spp) {
    return wave_counter_offset(P, P * spp) + 256;
}

cudaError_t launch_shade_fwd_wave(const ShadeArgs& a, float4* c_d, float4* kd_out, float4* c_s, uint32_t* vis_mask,
                                  void* ws, cudaStream_t stream, int parts) {
    const long long P = (long long)a.N * a.H * a.W;
    const int spp = a.n_light + a.n_cos + a.n_ggx;
    const int gblocks = (int)((P + kGenThreads - 1) / kGenThreads);
    if (parts & 1) {
        launch_k(wave_reset_kernel, 1, 1, 0, stream, ws, P, P * spp);
        launch_k(wave_gen_kernel, (int)((P + 31) / 32), kGenThreads, (size_t)(a.Hp + 1) * sizeof(float), stream, a,
                 ws, kd_out);
    }
    if (!(parts & 2)) return cudaGetLastError();
    int dev = 0, sms = 152, per_sm = 8;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wave_trace_kernel, kTraceThreads, 0);
    if (per_sm < 1) per_sm = 1;
    launch_k(wave_trace_kernel, sms * per_sm, kTraceThreads, 0, stream, a.nodes, static_cast<const TriRecord*>(a.tris),
             a.n_tris, ws, P, P * spp);
    launch_k(wave_accum_kernel, gblocks, kGenThreads, 0, stream, a, ws, c_d, c_s, vis_mask);
    return cudaGetLastError();
}

}  // namespace mcdi
