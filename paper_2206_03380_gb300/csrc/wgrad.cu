// Weight gradients of the denoiser's 3x3 convolutions on the tcgen05 tensor
// cores (the live-trained variant of the denoiser, App. B; Sec. 4.2 locks the
// weights for the main results, where this is not run).
//
// For a convolution with input X (ci channels) and G, the gradient of the
// loss with respect to its pre-activation output (co channels):
//   dW[co][ci][dy][dx] = sum over images and pixels p of G[co](p) X[ci](p + (dy - 1, dx - 1)),
//   db[co]             = sum over images and pixels of G[co](p),
// X and G zero outside the image.  Substituting q = p + dx - 1 for the input
// column, per output row y and input-column segment [q0, q0 + seg):
//   D[(dy, ci)][(dx, co)]  +=  sum over k < seg of  X[ci](y + dy - 1, q0 + k) G[co](y, q0 + k - dx + 1),
// one chain of MMAs over the segment (K = 16 columns each) with A = the three
// input rows of up to 5 8-channel planes stacked on M (15 slots of 8
// channels, an M group of 128) and B = three copies of the G row, shifted by
// dx, stacked on N (N = 3 co, split in two chains when above 256).  Segments
// partition the input columns, so every (input, gradient) pair is counted
// once; the shifts read zeros past the image edge.  Both operands are
// MN-major straight from the planar BF16 layout [img][C / 8][H][W][8] (a core
// matrix is 8 pixels x 8 channels of one plane), loaded by tiled TMA: one box
// of [planes][3 rows][seg px] for A and three boxes of [planes][1 row][seg px]
// for B per item, zeros outside the tensor.  Slot 15 of the first M group
// holds ones in channel 0, so its accumulator row at dx = 1 is the bias
// gradient.
//
// A CTA owns a run of image rows (of all images in order) and one M group
// (3 co <= 512 tensor-memory columns); two CTAs share an SM, so that their
// MMA streams interleave (measured: 7% faster than one CTA with twice the
// stages).  Warp 0 lane 0 keeps a ring of as many stages as half the shared
// memory holds (2 to 6) filled; warp 1 lane 0 issues the
// MMAs from per-stage base descriptors plus constant offsets.  At the end all
// four warps read the accumulators back and store this CTA's partial sums
// ([dx][co][row], one 128-byte line per warp store), and a second kernel adds
// the partials of each weight in a fixed order, so results are bitwise
// repeatable.  Every wait is bounded (2 s of %globaltimer): on a timeout the
// kernel sets *err, drains its own copies and frees its tensor memory.
#include <cuda_bf16.h>

#include "internal.h"
#include "pdl.cuh"
#include "tc_conv.cuh"
#include "tcgen05.cuh"

namespace mcdi {
namespace {

constexpr int kWgThreads = 128;
constexpr int kWgMaxStages = 6;
constexpr int kGroupSlots = 16;     // 8-channel slots of an M group of 128
constexpr int kGroupPlanes = 5;     // input planes per M group: 15 slots of (plane, dy)
constexpr int kOnesSlot = 15;       // the bias gradient's ones row (first group)
constexpr int kMaxGPlanes = 12;     // co <= 96
constexpr size_t kWgSmemMax = 112 * 1024;  // two CTAs per SM (their MMA streams interleave)

struct WgradArgs {
    int xp, gp;               // 8-channel planes of X and G (N = 8 gp)
    int n_img, H, W;
    int seg;                  // input columns per item: 32, 64 or 128
    int n_groups;             // M groups (CTAs across the input planes per row block)
    int rows_per_cta, n_rows;
    int stages;
    uint32_t tmem_cols, slot_bytes, stage_bytes;
    uint32_t x_bytes_full, x_bytes_last, g_bytes;  // bytes of the TMA boxes
    float* partial;           // [grid][3][N][128]
    unsigned* err;
};

__device__ __forceinline__ int group_planes(const WgradArgs& a, int g) {
    return g == a.n_groups - 1 ? a.xp - kGroupPlanes * (a.n_groups - 1) : kGroupPlanes;
}

// coordinates (2 x, y, plane) of a plane-row map (8-byte elements, two per pixel)
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mma_mn(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

// tmap_xf / tmap_xl: input boxes of 5 planes (all groups but the last) and of the last group's planes;
// tmap_g: gradient boxes of all gp planes, one row.
__global__ void __launch_bounds__(kWgThreads, 2) wgrad_kernel(const __grid_constant__ CUtensorMap tmap_xf,
                                                              const __grid_constant__ CUtensorMap tmap_xl,
                                                              const __grid_constant__ CUtensorMap tmap_g,
                                                              const WgradArgs a) {
    pdl_prologue();
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kWgMaxStages], empty_bar[kWgMaxStages], acc_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    uint8_t* const base_ptr = smem_raw + (base - smem_u32(smem_raw));
    const int bid = blockIdx.x;
    const int grp = bid % a.n_groups, rb = bid / a.n_groups;
    const int P = group_planes(a, grp);
    const int x_slots = 3 * P;  // slots (plane, dy) filled by TMA
    const int N = 8 * a.gp;
    const int r0 = rb * a.rows_per_cta;
    const int r1 = min(r0 + a.rows_per_cta, a.n_rows);
    const int n_seg = (a.W + a.seg - 1) / a.seg;
    const int n_items = (r1 > r0 ? r1 - r0 : 0) * n_seg;
    const uint32_t x_region = kGroupSlots * a.slot_bytes;

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&acc_bar), 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // slots past the TMA box are never loaded: set them once per stage, to zero, except channel 0 of the
    // ones slot in the first group
    {
        const int px = (int)(a.slot_bytes / 16);
        const int n_pad = (kGroupSlots - x_slots) * px;
        for (int s = 0; s < a.stages; ++s) {
            uint4* pad = reinterpret_cast<uint4*>(base_ptr + (size_t)s * a.stage_bytes + (size_t)x_slots * a.slot_bytes);
            for (int i = threadIdx.x; i < n_pad; i += blockDim.x) {
                const bool one = grp == 0 && x_slots + i / px == kOnesSlot;
                pad[i] = make_uint4(one ? 0x3F80u : 0u, 0u, 0u, 0u);  // BF16 1.0 in channel 0
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    int issued = 0;

    if (warp == 0) {
        if (lane == 0) {
            // ---- loader: per item one input box (3 rows of this group's planes) and three G boxes (dx = 0, 1, 2)
            const CUtensorMap* xmap = grp == a.n_groups - 1 ? &tmap_xl : &tmap_xf;
            const uint32_t tx = (grp == a.n_groups - 1 ? a.x_bytes_last : a.x_bytes_full) + 3u * a.g_bytes;
            const uint32_t g_copy = (uint32_t)a.gp * a.slot_bytes;  // bytes of one shifted G copy in shared memory
            int img = r0 / a.H, y = r0 - img * a.H, q0 = 0, s = 0;
            uint32_t phase = 0;
            for (int it = 0; it < n_items; ++it) {
                if (!mbar_wait(smem_u32(&empty_bar[s]), phase ^ 1u)) {
                    failed = 1;
                    break;
                }
                const uint32_t st = base + (uint32_t)s * a.stage_bytes, fb = smem_u32(&full_bar[s]);
                mbar_expect_tx(fb, tx);
                tma_load_3d(st, xmap, 2 * q0, y - 1, img * a.xp + grp * kGroupPlanes, fb);
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
                    tma_load_3d(st + x_region + (uint32_t)dx * g_copy, &tmap_g, 2 * (q0 + 1 - dx), y, img * a.gp, fb);
                issued = it + 1;
                q0 += a.seg;  // next item: segment, then row, then image
                if (q0 >= a.W) {
                    q0 = 0;
                    if (++y == a.H) {
                        y = 0;
                        ++img;
                    }
                }
                if (++s == a.stages) {
                    s = 0;
                    phase ^= 1u;
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: per item, seg / 16 K-steps of one or two chains (dx ranges with N <= 256);
            // descriptors are the stage's base descriptors plus constant offsets (16-byte units)
            const int dx_split = 3 * N <= 256 ? 3 : 2;  // first chain: dx < dx_split
            const uint32_t idesc0 = bf16_idesc_mn(128, dx_split * N), idesc1 = bf16_idesc_mn(128, (3 - dx_split) * N);
            const uint64_t a_desc0 = mn_desc(base, 128u, a.slot_bytes);
            const uint64_t b_desc0 = mn_desc(base + x_region, 128u, a.slot_bytes);
            const uint64_t b_chain1 = (uint64_t)(((uint32_t)dx_split * (uint32_t)a.gp * a.slot_bytes) >> 4);
            const int k_steps = a.seg / 16;
            int it = 0, s = 0;
            uint32_t phase = 0;
            for (; it < n_items; ++it) {
                if (!mbar_wait(smem_u32(&full_bar[s]), phase)) {
                    failed = 1;
                    break;
                }
                tc_fence_after();
                const uint64_t so = (uint64_t)((uint32_t)s * (a.stage_bytes >> 4));
                for (int ks = 0; ks < k_steps; ++ks) {
                    const uint64_t ad = a_desc0 + so + (uint64_t)(ks * 16), bd = b_desc0 + so + (uint64_t)(ks * 16);
                    const uint32_t acc = (it > 0 || ks > 0) ? 1u : 0u;
                    mma_mn(tmem, ad, bd, idesc0, acc);
                    if (dx_split < 3) mma_mn(tmem + (uint32_t)(dx_split * N), ad, bd + b_chain1, idesc1, acc);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&empty_bar[s]))
                             : "memory");
                if (++s == a.stages) {
                    s = 0;
                    phase ^= 1u;
                }
            }
            if (it == n_items && n_items > 0)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&acc_bar))
                             : "memory");
        }
        __syncwarp();
    }

    // ---- epilogue: lane m of warp w reads accumulator row 32 w + m (slot m / 8); stored as partial[bid][dx][n][m]
    bool ok = true;
    if (n_items > 0) {
        ok = mbar_wait(smem_u32(&acc_bar), 0u);
        ok = __all_sync(0xffffffffu, ok) && !failed;
    }
    if (!ok) failed = 1;
    tc_fence_after();
    const int last = grp == 0 ? kOnesSlot : x_slots - 1;  // the last slot whose rows are stored
    if (ok && warp * 4 <= last) {
        const int m = warp * 32 + lane;
        const bool row_ok = m / 8 < x_slots || (grp == 0 && m / 8 == kOnesSlot && (m & 7) == 0);
        float* out = a.partial + (size_t)bid * 3 * N * 128 + m;
        for (int c0 = 0; c0 < 3 * N; c0 += 16) {
            uint32_t v[16];
            tmem_ld16_async(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            tmem_wait_ld();
            if (!row_ok) continue;
#pragma unroll
            for (int k = 0; k < 16; ++k) out[(size_t)(c0 + k) * 128] = n_items > 0 ? __uint_as_float(v[k]) : 0.0f;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (failed) {
        if (threadIdx.x == 0) atomicExch(a.err, 1u);
        if (warp == 0 && lane == 0)  // let this CTA's copies in flight land before it exits
            for (int it = 0; it < issued; ++it)
                if (!mbar_wait(smem_u32(&full_bar[it % a.stages]), (uint32_t)(it / a.stages) & 1u)) break;
        __syncthreads();
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}

// The sum over row blocks of the CTAs' partials, in a fixed order, stored at each element's weight
// gw[co][ci][dy][dx] (n = co; slot m / 8 = 3 plane + dy within the group) or, for the ones row (first
// group, slot 15, channel 0) at dx = 1, at the bias gradient db[co].  Elements r = (dx, n, m) of a group run
// with m fastest (coalesced).  kSplit: a block of 8 warps owns 32 consecutive elements, warp w adds the
// partials of row blocks w, w + 8, ... and warp 0 adds the 8 warp sums in order (many row blocks); else one
// thread per element adds all row blocks in order (few row blocks).
constexpr int kReduceWarps = 8;
template <bool kSplit>
__global__ void __launch_bounds__(32 * kReduceWarps) wgrad_reduce_kernel(const WgradArgs a, int ci, int co, int n_rb,
                                                                        float* __restrict__ gw) {
    pdl_prologue();
    __shared__ float red[kReduceWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = 8 * a.gp;
    const int per_group = 3 * N * 128;
    const int elems_per_block = kSplit ? 32 : 32 * kReduceWarps;
    const int blocks_per_group = per_group / elems_per_block;
    const int grp = blockIdx.x / blocks_per_group;
    const int r = (blockIdx.x - grp * blocks_per_group) * elems_per_block + (kSplit ? lane : (int)threadIdx.x);
    const int m = r & 127, n = (r >> 7) % N, dx = (r >> 7) / N;
    const int slot = m / 8, pl = slot / 3, dy = slot - 3 * pl;
    const int c_in = (grp * kGroupPlanes + pl) * 8 + (m & 7);
    const bool bias = grp == 0 && slot == kOnesSlot && (m & 7) == 0 && dx == 1;
    const bool valid = n < co && ((slot < 3 * group_planes(a, grp) && c_in < ci) || bias);
    const int b0 = kSplit ? warp : 0, db = kSplit ? kReduceWarps : 1;
    float s = 0.0f;
    if (valid) {
        const float* p = a.partial + (size_t)grp * per_group + r;
        const size_t stride = (size_t)a.n_groups * per_group;
        int b = b0;
        for (; b + 3 * db < n_rb; b += 4 * db) {
            const float v0 = p[(size_t)b * stride], v1 = p[(size_t)(b + db) * stride];
            const float v2 = p[(size_t)(b + 2 * db) * stride], v3 = p[(size_t)(b + 3 * db) * stride];
            s += v0;
            s += v1;
            s += v2;
            s += v3;
        }
        for (; b < n_rb; b += db) s += p[(size_t)b * stride];
    }
    if (kSplit) {
        red[warp][lane] = s;
        __syncthreads();
        if (warp != 0) return;
#pragma unroll
        for (int w = 1; w < kReduceWarps; ++w) s += red[w][lane];
    }
    if (valid) gw[bias ? (size_t)co * ci * 9 + n : (((size_t)n * ci + c_in) * 3 + dy) * 3 + dx] = s;
}

struct WgradPlan {
    WgradArgs a;
    int grid, n_rb;
    size_t smem, partial_bytes;
};

WgradPlan wgrad_plan(int xp, int gp, int n_img, int H, int W, int sms) {
    WgradPlan P{};
    WgradArgs& a = P.a;
    a.xp = xp;
    a.gp = gp;
    a.n_img = n_img;
    a.H = H;
    a.W = W;
    const int N = 8 * gp;
    a.n_groups = (xp + kGroupPlanes - 1) / kGroupPlanes;
    a.tmem_cols = 32;
    while (a.tmem_cols < (uint32_t)(3 * N)) a.tmem_cols <<= 1;
    // segment width: the widest of 128, 64, 32 columns that the row does not leave mostly empty and that
    // leaves room for two stages
    auto stage_of = [&](int seg) { return ((uint32_t)(kGroupSlots + 3 * gp) * (uint32_t)seg * 16u + 1023u) & ~1023u; };
    a.seg = 128;
    while (a.seg > 32 && (a.seg / 2 >= W || 2 * (size_t)stage_of(a.seg) + 1024 > kWgSmemMax)) a.seg /= 2;
    a.slot_bytes = (uint32_t)a.seg * 16u;
    a.stage_bytes = stage_of(a.seg);
    a.stages = (int)((kWgSmemMax - 1024) / a.stage_bytes);
    if (a.stages > kWgMaxStages) a.stages = kWgMaxStages;
    if (a.stages < 2) a.stages = 2;
    const int p_full = xp < kGroupPlanes ? xp : kGroupPlanes, p_last = xp - kGroupPlanes * (a.n_groups - 1);
    a.x_bytes_full = (uint32_t)(3 * p_full) * a.slot_bytes;
    a.x_bytes_last = (uint32_t)(3 * p_last) * a.slot_bytes;
    a.g_bytes = (uint32_t)gp * a.slot_bytes;
    a.n_rows = n_img * H;
    // row blocks: two CTAs per SM, but at least 8 items per CTA (each CTA stores a whole accumulator of
    // partial sums, 3 N x 128 floats, which outweighs the work of a few items at the small levels)
    int n_rb = (2 * sms + a.n_groups - 1) / a.n_groups;
    const int n_seg = (W + a.seg - 1) / a.seg;
    const long long by_items = (long long)a.n_rows * n_seg / 8;
    if (n_rb > by_items) n_rb = (int)by_items;
    if (n_rb > a.n_rows) n_rb = a.n_rows;
    if (n_rb < 1) n_rb = 1;
    a.rows_per_cta = (a.n_rows + n_rb - 1) / n_rb;
    P.n_rb = (a.n_rows + a.rows_per_cta - 1) / a.rows_per_cta;
    P.grid = P.n_rb * a.n_groups;
    P.smem = (size_t)a.stages * a.stage_bytes + 1024;
    P.partial_bytes = (size_t)P.grid * 3 * N * 128 * sizeof(float);
    return P;
}

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 152;
    return sms;
}

}  // namespace

size_t wgrad_scratch_bytes(int x_ctot, int g_ctot, int n_img, int H, int W) {
    const WgradPlan P = wgrad_plan(x_ctot / 8, g_ctot / 8, n_img, H, W, device_sms());
    return align256(P.partial_bytes);
}

cudaError_t launch_wgrad(const void* x, int x_ctot, const void* g, int g_ctot, int n_img, int H, int W, int ci,
                         int co, void* scratch, float* gw, unsigned* err, cudaStream_t s, const char** why) {
    WgradPlan P = wgrad_plan(x_ctot / 8, g_ctot / 8, n_img, H, W, device_sms());
    if (P.smem > kWgSmemMax || x_ctot % 8 || g_ctot % 16 || ci > x_ctot || co > g_ctot ||
        g_ctot / 8 > kMaxGPlanes) {
        *why = "weight-gradient shape outside the supported range";
        return cudaErrorInvalidValue;
    }
    const int xp = x_ctot / 8, p_full = xp < kGroupPlanes ? xp : kGroupPlanes;
    const int p_last = xp - kGroupPlanes * (P.a.n_groups - 1);
    CUtensorMap mxf, mxl, mg;
    if (!encode_plane_rows_map(&mxf, x, W, H, (long long)n_img * xp, P.a.seg, 3, p_full, why) ||
        !encode_plane_rows_map(&mxl, x, W, H, (long long)n_img * xp, P.a.seg, 3, p_last, why) ||
        !encode_plane_rows_map(&mg, g, W, H, (long long)n_img * (g_ctot / 8), P.a.seg, 1, g_ctot / 8, why))
        return cudaErrorInvalidValue;
    P.a.partial = static_cast<float*>(scratch);
    P.a.err = err;
    cudaError_t e = cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem);
    if (e != cudaSuccess) return e;
    e = launch_k(wgrad_kernel, P.grid, kWgThreads, P.smem, s, mxf, mxl, mg, P.a);
    if (e != cudaSuccess) return e;
    // one thread per element while the row blocks are few; else 8 warps per 32 elements
    const int per_group = 3 * g_ctot * 128;
    if (P.n_rb <= 24)
        return launch_k(wgrad_reduce_kernel<false>, per_group / (32 * kReduceWarps) * P.a.n_groups, 32 * kReduceWarps, 0,
                        s, P.a, ci, co, P.n_rb, gw);
    return launch_k(wgrad_reduce_kernel<true>, per_group / 32 * P.a.n_groups, 32 * kReduceWarps, 0, s, P.a, ci, co,
                    P.n_rb, gw);
}

}  // namespace mcdi
