// tcgen05 implicit-GEMM 3x3 convolution (see tc_conv.cuh).
//
// One CTA computes a tile of 128 output pixels (tw x th) for all output
// channels: D[128 x cout_pad] (FP32, in tensor memory) = sum over the 9 taps
// and over input-channel chunks of 16 of
//   A[128 pixels x 16 ch] (the input shifted by the tap, zero outside the
//   image: TMA out-of-bounds fill) x B[cout_pad x 16 ch]^T (weights).
// Every chunk is one tcgen05.mma (M = 128, N = cout_pad, K = 16, BF16 inputs,
// FP32 accumulation).  Operands are staged by TMA through a ring of kStages
// shared-memory buffers guarded by mbarriers: the A tile as two 8-channel
// planes of 16-byte rows (no swizzle; activations live in 8-channel planes in
// global memory, so each plane's box is a run of contiguous rows), the weight
// slice with the 32-byte swizzle:
//   warp 0 lane 0  issues the TMA loads      (waits "empty", arms "full"),
//   warp 1 lane 0  issues the MMAs           (waits "full", commits to "empty"),
//   all 4 warps    run the epilogue: tcgen05.ld of their 32 TMEM lanes, bias,
//                  ReLU / gradient mask, BF16 (or FP32) stores.
// Every wait is bounded (2 s of %globaltimer); on a timeout the kernel sets
// *err, stops issuing work, drains its own copies in flight and frees TMEM.
#include <stdio.h>

#include <mutex>

#include <cudaTypedefs.h>

#include "tc_conv.cuh"
#include "tcgen05.cuh"

namespace mcdi {
namespace {

constexpr int kStages = 6;
constexpr int kConvThreads = 128;

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand whose rows are 32 bytes
// (16 BF16 channels) with the 32-byte swizzle: 8-row atoms of 256 bytes
// stacked along M/N (stride 256 B); the K extent of one MMA is one row.
__device__ __forceinline__ uint64_t sw32_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);     // start address
    d |= (uint64_t)(16u >> 4) << 16;              // leading byte offset (unused with a one-row K extent)
    d |= (uint64_t)(256u >> 4) << 32;             // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                       // descriptor version
    d |= (uint64_t)6 << 61;                       // swizzle: 32 bytes
    return d;
}

// K-major operand without swizzle: core matrices of 8 rows x 16 bytes with
// rows 16 bytes apart, 8-row groups 128 bytes apart (stride byte offset) and
// the second 8-channel half of K one plane further (leading byte offset).
__device__ __forceinline__ uint64_t noswz_desc(uint32_t saddr, uint32_t lbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)(128u >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version; swizzle mode 0 (none)
    return d;
}

// Instruction descriptor of kind::f8f6f4 with E4M3 A and B (format code 0),
// K-major, FP32 D, M x N.
__host__ __device__ constexpr uint32_t e4m3_idesc(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// A-operand collector use: kAPlain reads A from shared memory for this MMA
// only; kAFill also keeps it in the collector buffer, kAUse takes it from
// there (same A descriptor), kALast takes it and releases the buffer.
enum ACollector { kAPlain, kAFill, kAUse, kALast };

#define MCDI_MMA(KIND, COLL)                                                                       \
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"                             \
                 "tcgen05.mma.cta_group::1.kind::" KIND COLL " [%0], %1, %2, %3, p;\n\t}" ::"r"(d), \
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)                                    \
                 : "memory")

template <bool FP8, int COLL = kAPlain>
__device__ __forceinline__ void mma_issue(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
    if constexpr (FP8) {
        if constexpr (COLL == kAFill) MCDI_MMA("f8f6f4", ".collector::a::fill");
        else if constexpr (COLL == kAUse) MCDI_MMA("f8f6f4", ".collector::a::use");
        else if constexpr (COLL == kALast) MCDI_MMA("f8f6f4", ".collector::a::lastuse");
        else MCDI_MMA("f8f6f4", "");
    } else {
        if constexpr (COLL == kAFill) MCDI_MMA("f16", ".collector::a::fill");
        else if constexpr (COLL == kAUse) MCDI_MMA("f16", ".collector::a::use");
        else if constexpr (COLL == kALast) MCDI_MMA("f16", ".collector::a::lastuse");
        else MCDI_MMA("f16", "");
    }
}
#undef MCDI_MMA




__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void store8_bf16(__nv_bfloat16* dst, const float* f) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// Element offset of pixel (x, y) of image img in 8-channel group g of a
// tensor with G groups at H x W (layout [img][g][y][x][8]).
__device__ __forceinline__ size_t plane_off(int img, int G, int g, int H, int W, int y, int x) {
    return ((((size_t)img * G + g) * H + y) * W + x) * 8;
}

// the ReLU mask words of 16 channels (two 8-channel groups) of one pixel
__device__ __forceinline__ void load_mask16(const ConvParams& p, int c0, int img, int x, int y, uint4* m) {
    const __nv_bfloat16* mk = p.mask + plane_off(img, p.mask_ctotal >> 3, (p.mask_coff + c0) >> 3, p.H, p.W, y, x);
    m[0] = __ldg(reinterpret_cast<const uint4*>(mk));
    m[1] = __ldg(reinterpret_cast<const uint4*>(mk + (size_t)p.H * p.W * 8));
}

// bias / activation / mask and store of 16 output channels (two 8-channel
// groups) of one pixel; pre: the pixel's mask words are already in (ma, mb)
template <bool kPoolBwd>
__device__ __forceinline__ void epilogue16(const ConvParams& p, const uint32_t* v, int c0, int img, int x, int y,
                                           const float* bias16, float dq, float* amax, bool pre = false,
                                           uint4 ma = uint4{}, uint4 mb = uint4{}, uint32_t* keep = nullptr) {
    float f[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i] = __uint_as_float(v[i]) * dq;
    const size_t hw = (size_t)p.H * p.W;
    if constexpr (kPoolBwd) {  // the instantiation for kDgradPoolBwd (its loads would crowd the others' registers)
        // (y, x) is a pooled pixel: its window is (2y + dy, 2x + dx) at twice the size
        const int H2 = 2 * p.H, W2 = 2 * p.W;
        auto bf = [](uint32_t w, int hi) {  // BF16 half of a packed pair as float
            return __uint_as_float(hi ? (w & 0xffff0000u) : (w << 16));
        };
#pragma unroll
        for (int gg = 0; gg < 2; ++gg) {
            const size_t e0 =
                plane_off(img, p.mask_ctotal >> 3, ((p.mask_coff + c0) >> 3) + gg, H2, W2, 2 * y, 2 * x);
            uint32_t we[4][4];  // the window's E values, packed BF16 pairs
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint4 t = __ldg(reinterpret_cast<const uint4*>(p.mask + e0 + ((size_t)(k >> 1) * W2 + (k & 1)) * 8));
                we[k][0] = t.x, we[k][1] = t.y, we[k][2] = t.z, we[k][3] = t.w;
            }
            int arg[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {  // the window's first maximum, in window order
                arg[c] = 0;
                float best = bf(we[0][c >> 1], c & 1);
#pragma unroll
                for (int k = 1; k < 4; ++k) {
                    const float e = bf(we[k][c >> 1], c & 1);
                    if (e > best) best = e, arg[c] = k;
                }
            }
            const size_t o0 = plane_off(img, p.out_ctotal >> 3, ((p.out_coff + c0) >> 3) + gg, H2, W2, 2 * y, 2 * x);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const size_t off = ((size_t)(k >> 1) * W2 + (k & 1)) * 8;
                const uint4 t = __ldg(reinterpret_cast<const uint4*>(p.gskip + e0 + off));
                const uint32_t wg[4] = {t.x, t.y, t.z, t.w};
                float o[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float gp = __bfloat162float(__float2bfloat16_rn(f[8 * gg + c]));  // as stored unfused
                    const float v = bf(wg[c >> 1], c & 1) + (arg[c] == k ? gp : 0.0f);
                    o[c] = bf(we[k][c >> 1], c & 1) > 0.0f ? v : 0.0f;
                    *amax = fmaxf(*amax, fabsf(o[c]));
                }
                store8_bf16(p.out + o0 + off, o);
            }
        }
        return;
    } else {
    if (p.mode == kDgradMask || p.mode == kDgradPlain) {
        if (p.mode == kDgradMask) {
            uint4 mm[2] = {ma, mb};
            if (!pre) load_mask16(p, c0, img, x, y, mm);
            const uint4 m0 = mm[0], m1 = mm[1];
            const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&mw[i]);
                if (!(__bfloat162float(h.x) > 0.0f)) f[2 * i] = 0.0f;
                if (!(__bfloat162float(h.y) > 0.0f)) f[2 * i + 1] = 0.0f;
            }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) *amax = fmaxf(*amax, fabsf(f[i]));
        __nv_bfloat16* o = p.out + plane_off(img, p.out_ctotal >> 3, (p.out_coff + c0) >> 3, p.H, p.W, y, x);
        store8_bf16(o, f);
        store8_bf16(o + hw * 8, f + 8);
        return;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        f[i] += bias16 ? bias16[i] : 0.0f;
        if (p.relu) f[i] = fmaxf(f[i], 0.0f);
        *amax = fmaxf(*amax, fabsf(f[i]));
    }
    if (keep) {  // the 16 stored values as packed BF16 pairs
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
            keep[i] = *reinterpret_cast<uint32_t*>(&h);
        }
    }
    if (p.mode == kStoreF32) {
        p.out_f32[((size_t)img * p.H + y) * p.W + x] = make_float4(f[0], f[1], f[2], 0.0f);
    } else if (p.mode == kStoreUp2) {
        const int W2 = 2 * p.W, H2 = 2 * p.H;
        __nv_bfloat16* o = p.out + plane_off(img, p.out_ctotal >> 3, (p.out_coff + c0) >> 3, H2, W2, 2 * y, 2 * x);
        const size_t hw2 = (size_t)H2 * W2 * 8;
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                __nv_bfloat16* q = o + ((size_t)j * W2 + i) * 8;
                store8_bf16(q, f);
                store8_bf16(q + hw2, f + 8);
            }
    } else {
        __nv_bfloat16* o = p.out + plane_off(img, p.out_ctotal >> 3, (p.out_coff + c0) >> 3, p.H, p.W, y, x);
        store8_bf16(o, f);
        store8_bf16(o + hw * 8, f + 8);
    }
    }
}

// Publish a thread's running max |value| of the stored output: rounded to BF16
// like the stored values (rounding is monotonic, so this is the max over the
// stored tensor), reduced over the warp, one atomic per warp.
__device__ __forceinline__ void publish_amax(unsigned* out_amax, float m, unsigned mask) {
    if (out_amax == nullptr) return;
    const unsigned b = __float_as_uint(__bfloat162float(__float2bfloat16_rn(m)));
    const unsigned w = __reduce_max_sync(mask, b);
    if ((threadIdx.x & 31) == __ffs(mask) - 1 && w) atomicMax(out_amax, w);
}

// accumulator scale: 1 for BF16; (amax_x / 448) (amax_w / 448) for E4M3
// operands quantised as round(v 448 / amax)
__device__ __forceinline__ float dequant_factor(const ConvParams& p) {
    if (!p.fp8) return 1.0f;
    return (__ldg(p.x_amax) * (1.0f / 448.0f)) * (__ldg(p.w_amax) * (1.0f / 448.0f));
}

template <bool FP8, bool PB>
__global__ void __launch_bounds__(kConvThreads) conv_tc_kernel(const __grid_constant__ CUtensorMap tmap_x,
                                                               const __grid_constant__ CUtensorMap tmap_w,
                                                               const ConvParams p) {
    pdl_prologue();
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], acc_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // 1024-byte aligned staging ring
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t a_bytes = 128u * 32u, b_bytes = (uint32_t)p.cout_pad * 32u;
    const uint32_t stage_bytes = (a_bytes + b_bytes + 1023u) & ~1023u;
    const uint32_t ncols = p.cout_pad <= 32 ? 32u : (p.cout_pad <= 64 ? 64u : (p.cout_pad <= 128 ? 128u : 256u));

    int tile = blockIdx.x;
    const int tx = tile % p.tiles_x;
    tile /= p.tiles_x;
    const int ty = tile % p.tiles_y;
    const int img = tile / p.tiles_y;
    const int x0 = tx * p.tw, y0 = ty * p.th;
    const int cpt = p.cin_bytes >> 5;  // 32-byte channel chunks (one MMA K-step) per tap
    const int n_chunks = 9 * cpt;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&acc_bar), 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    int issued = 0;
    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        for (int k = 0; k < n_chunks; ++k) {
            const int s = k % kStages;
            const uint32_t ph = (uint32_t)(k / kStages) & 1u;
            if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u)) {
                failed = 1;
                break;
            }
            const uint32_t a_dst = base + (uint32_t)s * stage_bytes;
            const uint32_t fb = smem_u32(&full_bar[s]);
            mbar_expect_tx(fb, a_bytes + b_bytes);
            const int tap = k / cpt, cc = k - tap * cpt;
            const int dy = tap / 3, dx = tap - 3 * (tap / 3);
            const int plane = img * (p.cin_bytes >> 4) + 2 * cc;
            tma_load_4d(a_dst, &tmap_x, 0, x0 + dx - 1, y0 + dy - 1, plane, fb);
            tma_load_4d(a_dst + a_bytes / 2, &tmap_x, 0, x0 + dx - 1, y0 + dy - 1, plane + 1, fb);
            tma_load_2d(a_dst + a_bytes, &tmap_w, tap * p.cin_bytes + cc * 32, 0, fb);
            issued = k + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = FP8 ? e4m3_idesc(128, p.cout_pad) : bf16_idesc(128, p.cout_pad);
        int k = 0;
        for (; k < n_chunks; ++k) {
            const int s = k % kStages;
            const uint32_t ph = (uint32_t)(k / kStages) & 1u;
            if (!mbar_wait(smem_u32(&full_bar[s]), ph)) {
                failed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a_src = base + (uint32_t)s * stage_bytes;
            const uint64_t adesc = noswz_desc(a_src, a_bytes / 2), bdesc = sw32_desc(a_src + a_bytes);
            mma_issue<FP8>(tmem, adesc, bdesc, idesc, k > 0 ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty_bar[s]))
                         : "memory");
        }
        if (k == n_chunks)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&acc_bar))
                         : "memory");
    }
    __syncwarp();

    // ---- epilogue: every thread owns one accumulator row (one pixel)
    const bool acc_ok = mbar_wait(smem_u32(&acc_bar), 0u);
    if (!acc_ok) failed = 1;
    __syncwarp();
    tc_fence_after();
    const int m = warp * 32 + lane;
    const int xx = m % p.tw, yy = m / p.tw;
    const int x = x0 + xx, y = y0 + yy;
    const bool valid = acc_ok && x < p.W && y < p.H;
    const float dq = dequant_factor(p);
    float amax = 0.0f;
    for (int c0 = 0; c0 < p.cout_pad; c0 += 16) {
        uint32_t v[16];
        // collective load of 16 accumulator columns of this warp's 32 lanes
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (valid && c0 < p.cout_valid)
            epilogue16<PB>(p, v, c0, img, x, y, p.bias ? p.bias + c0 : nullptr, dq, &amax);
        __syncwarp();
    }
    publish_amax(p.out_amax, amax, 0xffffffffu);

    // ---- teardown
    tc_fence_before();
    __syncthreads();
    if (failed) {
        if (threadIdx.x == 0) atomicExch(p.err, 1u);
        // wait (bounded) for this CTA's own TMA copies still in flight
        if (warp == 0 && lane == 0) {
            for (int k = 0; k < issued; ++k) {
                const int s = k % kStages;
                if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)(k / kStages) & 1u)) break;
            }
        }
        __syncthreads();
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Row-tile form, for images at least 48 pixels wide (128-pixel row tiles).
// A persistent CTA keeps a slice of Nc output channels of the layer's weights
// resident in shared memory for its whole life ([chunk][tap][Nc][16 ch],
// 32-byte swizzle, one TMA load per chunk) and loops over tiles of R output
// rows x 128 pixels.  Per 16-channel input chunk the tile's halo, R + 2 rows x
// 130 pixels of two 8-channel planes, arrives once: each halo row is one
// contiguous run in the planar activation layout, copied with one bulk copy
// (large requests instead of one per 16-byte pixel), the part outside the
// image zero-filled.  Rows are 16 bytes per pixel and unswizzled, so any row
// starts a valid 8-row core matrix: the A operand of output row r and tap
// (dy, dx) is the window starting at halo row (r + dy) * 130 + dx, and 9 R
// MMAs (M = 128, N = Nc, K = 16) per chunk read (R + 2) / R input rows per
// output row instead of 9.
//   warp 0          weight TMA (lane 0), halo row copies (one lane per row),
//   warp 1 lane 0   MMA issuer; accumulators of tile i in TMEM buffer i & 1,
//   warps 2..9      epilogue: TMEM lane quarter warp % 4, and the two warps of
//                   a quarter take alternate 16-column chunks of each row.
constexpr int kRowThreads = 320;
constexpr int kEpiWarps = kRowThreads / 32 - 2;
constexpr int kEpiSplit = kEpiWarps / 4;  // epilogue warps per TMEM lane quarter
constexpr int kRowMaxStages = 6;
constexpr int kHaloW = 130;
constexpr int kMaxRows = 4;


// EV: the epilogue variant, 0 plain, 1 also the 2x2 max-pool of the output (kStore), 2 the pool
// gradient routed through the pool (kDgradPoolBwd)
template <int R, bool FP8, bool MP, int EV>
__global__ void __launch_bounds__(kRowThreads, 2) conv_tc_rows_kernel(const __grid_constant__ CUtensorMap tmap_wh,
                                                                   const ConvParams p, const RowPlan rp) {
    // The setup that reads nothing the preceding kernel writes (barriers, bias, tensor memory and the
    // weight load: the weights and biases are packed once) runs before the wait on that kernel, so it
    // overlaps the preceding kernel's tail when the launch is programmatically dependent.
    pdl_allow_dependents();
    extern __shared__ uint8_t smem_raw[];
    __shared__ float s_bias[256];
    __shared__ __align__(8) uint64_t full_bar[kRowMaxStages], empty_bar[kRowMaxStages], accf_bar[2], acce_bar[2],
        w_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t wbase = base + (uint32_t)rp.stages * rp.stage_bytes;
    const int S = rp.stages, Nc = rp.nc;
    const int n_chunks = p.cin_bytes >> 5;
    const uint32_t w_chunk = 9u * (uint32_t)Nc * 32u;  // bytes of one chunk's weights, all taps
    const int slice = blockIdx.x % rp.n_slices;
    const int n0 = slice * Nc;
    const int first = blockIdx.x / rp.n_slices, step = gridDim.x / rp.n_slices;
    const bool has_work = first < rp.n_tiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&accf_bar[b]), 1);
            mbar_init(smem_u32(&acce_bar[b]), kEpiWarps);
        }
        mbar_init(smem_u32(&w_bar), 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int c = threadIdx.x; c < Nc; c += blockDim.x) s_bias[c] = p.bias ? p.bias[n0 + c] : 0.0f;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(rp.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    auto tile_origin = [&](int t, int* img, int* x0, int* y0) {
        const int tx = t % p.tiles_x;
        t /= p.tiles_x;
        *y0 = (t % p.tiles_y) * R;
        *img = t / p.tiles_y;
        *x0 = tx * 128;
    };

    int issued = 0;
    bool w_issued = false;
    if (warp == 0 && has_work && lane == 0) {
        const uint32_t wb = smem_u32(&w_bar);
        mbar_expect_tx(wb, (uint32_t)n_chunks * w_chunk);
        for (int c = 0; c < n_chunks; ++c) tma_load_4d(wbase + (uint32_t)c * w_chunk, &tmap_wh, 0, n0, 0, c, wb);
        w_issued = true;
    }
    pdl_wait();  // activations, masks and outputs: after the preceding kernel has completed
    if (warp == 0) {
        if (has_work) {
            // Halo rows by plain bulk copies: lane l < 2 (R + 2) owns row l % (R + 2)
            // of plane l / (R + 2); the part of the row outside the image is
            // zero-filled with shared-memory stores made visible to the async
            // proxy before the stage's barrier is armed.
            const int rows = R + 2;
            const bool mine = lane < 2 * rows;
            const int q = lane / rows, hr = lane - q * rows;
            const size_t plane_bytes = (size_t)p.H * p.W * 16;
            const uint8_t* x_bytes = reinterpret_cast<const uint8_t*>(p.x);
            int g = 0;
            for (int t = first; t < rp.n_tiles; t += step) {
                int img, x0, y0;
                tile_origin(t, &img, &x0, &y0);
                const int y = y0 - 1 + hr;
                const int xa = x0 - 1 < 0 ? 0 : x0 - 1, xb = x0 + 129 > p.W ? p.W : x0 + 129;
                const bool row_in = mine && y >= 0 && y < p.H && xb > xa;
                const uint32_t n_bytes = row_in ? (uint32_t)(xb - xa) * 16u : 0u;
                const int lead = row_in ? xa - (x0 - 1) : kHaloW;  // zero pixels [0, lead)
                const int tail = row_in ? xb - (x0 - 1) : kHaloW;  // zero pixels [tail, 130)
                const uint32_t total = __reduce_add_sync(0xffffffffu, n_bytes);
                int c = 0;
                for (; c < n_chunks; ++c, ++g) {
                    const int s = g % S;
                    int ok = 1;
                    if (lane == 0) ok = mbar_wait(smem_u32(&empty_bar[s]), ((uint32_t)(g / S) & 1u) ^ 1u) ? 1 : 0;
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) {
                        if (lane == 0) failed = 1;
                        break;
                    }
                    const uint32_t row_smem = base + (uint32_t)s * rp.stage_bytes + (uint32_t)q * rp.plane_bytes +
                                              (uint32_t)hr * (uint32_t)kHaloW * 16u;
                    if (mine) {
                        for (int x = 0; x < lead; ++x)
                            asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(row_smem + 16u * x), "r"(0)
                                         : "memory");
                        for (int x = tail; x < kHaloW; ++x)
                            asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(row_smem + 16u * x), "r"(0)
                                         : "memory");
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    const uint32_t fb = smem_u32(&full_bar[s]);
                    if (lane == 0) mbar_expect_tx(fb, total);
                    __syncwarp();
                    if (n_bytes > 0) {
                        const uint8_t* src = x_bytes + (size_t)(img * (p.cin_bytes >> 4) + 2 * c + q) * plane_bytes +
                                             ((size_t)y * p.W + xa) * 16;
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                row_smem + 16u * (uint32_t)lead),
                            "l"(src), "r"(n_bytes), "r"(fb)
                            : "memory");
                    }
                    issued = g + 1;
                }
                if (c < n_chunks || failed) break;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && has_work) {
            const uint32_t idesc = FP8 ? e4m3_idesc(128, Nc) : bf16_idesc(128, Nc);
            bool ok = mbar_wait(smem_u32(&w_bar), 0u);
            if (!ok) failed = 1;
            int g = 0, i = 0;
            for (int t = first; ok && t < rp.n_tiles && !failed; t += step, ++i) {
                const int b = i & 1;
                if (!mbar_wait(smem_u32(&acce_bar[b]), ((uint32_t)(i >> 1) & 1u) ^ 1u)) {
                    failed = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d0 = tmem + (uint32_t)(b * R) * rp.acc_stride;
                int c = 0;
                for (; c < n_chunks; ++c, ++g) {
                    const int s = g % S;
                    if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)(g / S) & 1u)) {
                        failed = 1;
                        break;
                    }
                    tc_fence_after();
                    // descriptors of the stage's halo and the chunk's weights; each MMA adds a
                    // compile-time offset (in 16-byte units) to the start-address field, which
                    // stays below 2^14 for any shared-memory address
                    const uint64_t a0 = noswz_desc(base + (uint32_t)s * rp.stage_bytes, rp.plane_bytes);
                    const uint64_t b0 = sw32_desc(wbase + (uint32_t)c * w_chunk);
                    const uint64_t b_step = (uint64_t)((uint32_t)Nc * 2u);  // Nc x 32 bytes per tap, in 16-byte units
                    const uint32_t acc0 = c > 0 ? 1u : 0u;
                    // MMAs grouped by A window: halo row hr and column shift dx feed output rows
                    // r = hr - dy for every tap row dy with 0 <= r < R, so the window is read from
                    // shared memory once (collector fill) and reused by the following MMAs.  The
                    // first MMA into accumulator r of chunk 0 is (hr = r, dx = 0, dy = 0).
#pragma unroll
                    for (int hr = 0; hr < R + 2; ++hr) {
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
                            const uint64_t adesc = a0 + (uint64_t)(hr * kHaloW + dx);
                            const int dy_lo = hr - R + 1 > 0 ? hr - R + 1 : 0, dy_hi = hr < 2 ? hr : 2;
#pragma unroll
                            for (int dy = dy_lo; dy <= dy_hi; ++dy) {
                                const uint32_t d = d0 + (uint32_t)(hr - dy) * rp.acc_stride;
                                const uint64_t bdesc = b0 + (uint64_t)(dy * 3 + dx) * b_step;
                                const uint32_t acc = (dx == 0 && dy == 0) ? acc0 : 1u;
                                if (dy_lo == dy_hi) mma_issue<FP8, kAPlain>(d, adesc, bdesc, idesc, acc);
                                else if (dy == dy_lo) mma_issue<FP8, kAFill>(d, adesc, bdesc, idesc, acc);
                                else if (dy == dy_hi) mma_issue<FP8, kALast>(d, adesc, bdesc, idesc, acc);
                                else mma_issue<FP8, kAUse>(d, adesc, bdesc, idesc, acc);
                            }
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&empty_bar[s]))
                                 : "memory");
                }
                if (c < n_chunks) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&accf_bar[b]))
                             : "memory");
            }
        }
        __syncwarp();
    } else {
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int m = q * 32 + lane;
        float amax = 0.0f;
        // this warp's 16-column chunks of a row: 16 h, 16 (h + kEpiSplit), ...,
        // drained two per TMEM-load wait
        const int cfirst = 16 * h, cstep = 16 * kEpiSplit;
        // MP (ReLU-masked input gradients with at most 64 channels per CTA): the
        // mask words of the next row are loaded while the current row drains
        // (and those of a tile's first row before its accumulator wait), so
        // their latency does not stall the epilogue
        const bool pref = MP && p.mode == kDgradMask && Nc <= 2 * cstep;
        uint4 na0{}, na1{}, nb0{}, nb1{};  // next row's mask words of chunks cfirst (a) and cfirst + cstep (b)
        auto load_row = [&](int img, int x, int y) {
            uint4 w[2];
            if (cfirst < Nc && x < p.W && y < p.H && n0 + cfirst < p.cout_valid) {
                load_mask16(p, n0 + cfirst, img, x, y, w);
                na0 = w[0];
                na1 = w[1];
            }
            if (cfirst + cstep < Nc && x < p.W && y < p.H && n0 + cfirst + cstep < p.cout_valid) {
                load_mask16(p, n0 + cfirst + cstep, img, x, y, w);
                nb0 = w[0];
                nb1 = w[1];
            }
        };
        // 2x2 max-pool of the stored values: the two pixels of a window are neighbouring
        // lanes, its two rows consecutive rows of this thread (R even, tiles start on even
        // rows and columns); the maxima are taken on the stored BF16 values
        // (EV 1: the instantiation for the convolutions that feed a pooling layer)
        const bool pool = EV == 1 && R % 2 == 0 && p.pool_out != nullptr && p.mode == kStore && Nc <= 2 * cstep;
        float pool_amax = 0.0f;
        uint32_t ha[8], hb[8];  // the even row's stored values of chunks c0 / c1, packed BF16 pairs
        int i = 0;
        for (int t = first; t < rp.n_tiles; t += step, ++i) {
            const int b = i & 1;
            int img, x0, y0;
            tile_origin(t, &img, &x0, &y0);
            const int x = x0 + m;
            if (pref) load_row(img, x, y0);
            const bool ok = mbar_wait(smem_u32(&accf_bar[b]), (uint32_t)(i >> 1) & 1u);
            __syncwarp();
            if (!__all_sync(0xffffffffu, ok)) {
                failed = 1;
                break;
            }
            tc_fence_after();
            const float dq = dequant_factor(p);
            constexpr int kRowUnroll = MP || EV != 0 ? 1 : R;  // prefetch / pool registers leave no room to unroll
#pragma unroll kRowUnroll
            for (int r = 0; r < R; ++r) {
                const int y = y0 + r;
                const bool valid = x < p.W && y < p.H;
                const uint32_t tr = tmem + (uint32_t)(b * R + r) * rp.acc_stride + ((uint32_t)(q * 32) << 16);
                const uint4 ca0 = na0, ca1 = na1, cb0 = nb0, cb1 = nb1;
                if (pref && r + 1 < R) load_row(img, x, y + 1);
                for (int c0 = cfirst; c0 < Nc; c0 += 2 * cstep) {
                    uint32_t v[32];
                    const int c1 = c0 + cstep;
                    const bool two = c1 < Nc;
                    tmem_ld16_async(tr + (uint32_t)c0, v);
                    if (two) tmem_ld16_async(tr + (uint32_t)c1, v + 16);
                    tmem_wait_ld();
                    uint32_t ka[8], kb[8];
                    const bool va = valid && n0 + c0 < p.cout_valid, vb = two && valid && n0 + c1 < p.cout_valid;
                    if (va) epilogue16<EV == 2>(p, v, n0 + c0, img, x, y, s_bias + c0, dq, &amax, pref, ca0, ca1, ka);
                    if (vb)
                        epilogue16<EV == 2>(p, v + 16, n0 + c1, img, x, y, s_bias + c1, dq, &amax, pref, cb0, cb1, kb);
                    if (pool) {
                        if ((r & 1) == 0) {
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                ha[k] = ka[k];
                                hb[k] = kb[k];
                            }
                        } else {
                            const int Hp = p.H >> 1, Wp = p.W >> 1;
                            auto pool_store = [&](const uint32_t* h, const uint32_t* k, int c, bool ok) {
                                uint32_t w[8];
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&h[j]);
                                    __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&k[j]);
                                    a = __hmax2(a, b);
                                    uint32_t u = *reinterpret_cast<uint32_t*>(&a);
                                    const uint32_t o = __shfl_xor_sync(0xffffffffu, u, 1);
                                    a = __hmax2(a, *reinterpret_cast<const __nv_bfloat162*>(&o));
                                    w[j] = *reinterpret_cast<uint32_t*>(&a);
                                }
                                if ((lane & 1) == 0 && ok) {
                                    __nv_bfloat16* dst = p.pool_out + plane_off(img, p.pool_ctotal >> 3, c >> 3, Hp, Wp,
                                                                                y >> 1, x >> 1);
                                    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
                                    *reinterpret_cast<uint4*>(dst + (size_t)Hp * Wp * 8) =
                                        make_uint4(w[4], w[5], w[6], w[7]);
                                    if (p.pool_amax) {
#pragma unroll
                                        for (int j = 0; j < 8; ++j) {
                                            const float2 f2 = __bfloat1622float2(
                                                *reinterpret_cast<const __nv_bfloat162*>(&w[j]));
                                            pool_amax = fmaxf(pool_amax, fmaxf(fabsf(f2.x), fabsf(f2.y)));
                                        }
                                    }
                                }
                            };
                            pool_store(ha, ka, n0 + c0, va);
                            pool_store(hb, kb, n0 + c1, vb);
                        }
                    }
                    __syncwarp();
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce_bar[b]));
        }
        publish_amax(p.out_amax, amax, 0xffffffffu);
        if (pool) publish_amax(p.pool_amax, pool_amax, 0xffffffffu);
    }

    tc_fence_before();
    __syncthreads();
    if (failed) {
        if (threadIdx.x == 0) atomicExch(p.err, 1u);
        if (warp == 0 && lane == 0) {  // let this CTA's copies in flight land before it exits
            if (w_issued) mbar_wait(smem_u32(&w_bar), 0u);
            for (int g = 0; g < issued; ++g)
                if (!mbar_wait(smem_u32(&full_bar[g % S]), (uint32_t)(g / S) & 1u)) break;
        }
        __syncthreads();
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(rp.tmem_cols)
                     : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn(const char** why) {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    if (!fn) *why = "cuTensorMapEncodeTiled is not available from the driver";
    return fn;
}

struct DeviceLimits {
    int sms = 0;
    uint32_t rows_smem_max = 0;  // dynamic shared memory one row-tile CTA may request
    uint32_t rows_smem_two = 0;  // dynamic shared memory per CTA with two CTAs on an SM
};

const DeviceLimits& device_limits() {
    static std::once_flag once;
    static DeviceLimits L;
    std::call_once(once, [] {
        int dev = 0, optin = 0, per_sm = 0, reserved = 0;
        cudaFuncAttributes fa{};
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&L.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, conv_tc_rows_kernel<4, false, false, 0>) != cudaSuccess ||
            optin <= (int)fa.sharedSizeBytes) {
            L.sms = 0;
            return;
        }
        L.rows_smem_max = (uint32_t)(optin - (int)fa.sharedSizeBytes);
        const int two = per_sm / 2 - (int)fa.sharedSizeBytes - reserved;
        L.rows_smem_two = two > 0 ? (uint32_t)two : 0u;
    });
    return L;
}

uint32_t pow2_at_least(uint32_t v) {
    uint32_t c = 32;
    while (c < v) c <<= 1;
    return c;
}

// Row-tile plan: the fewest channel slices whose resident weights leave room
// for two halo stages; per slice the most rows per tile (up to kMaxRows) that
// fit tensor memory (two buffers of R accumulators) and still give 1.5 tiles
// per SM; two CTAs per SM where both fit in shared memory and tensor memory.
bool plan_rows(const ConvParams& p, RowPlan* out) {
    if (p.tw != 128 || p.th != 1) return false;
    const DeviceLimits& lim = device_limits();
    const int sms = lim.sms;
    if (sms <= 0) return false;
    const uint32_t kSmemMax = lim.rows_smem_max, kAlign = 1024u;
    const int n_chunks = p.cin_bytes / 32;
    for (int n_slices = 1; 16 * n_slices <= p.cout_pad; ++n_slices) {
        if (p.cout_pad % (16 * n_slices) != 0) continue;
        const int nc = p.cout_pad / n_slices;
        const uint32_t acc_stride = pow2_at_least((uint32_t)nc);
        const uint32_t w_bytes = (uint32_t)n_chunks * 9u * (uint32_t)nc * 32u;
        // the largest R that fits, except that a plan of two CTAs per SM is
        // preferred to one of a single CTA with a larger R
        RowPlan single{};
        bool have_single = false;
        for (int R = kMaxRows; R >= 1; R >>= 1) {
            const uint32_t tmem_cols = pow2_at_least(2u * (uint32_t)R * acc_stride);
            if (tmem_cols > 512u) continue;
            RowPlan rp{};
            rp.rows = R;
            rp.nc = nc;
            rp.n_slices = n_slices;
            rp.plane_bytes = ((uint32_t)(R + 2) * kHaloW * 16u + 127u) & ~127u;
            rp.stage_bytes = (2u * rp.plane_bytes + 1023u) & ~1023u;
            rp.acc_stride = acc_stride;
            rp.tmem_cols = tmem_cols;
            if (w_bytes + 2u * rp.stage_bytes + kAlign > kSmemMax) continue;
            rp.n_tiles = p.n_img * ((p.H + R - 1) / R) * p.tiles_x;
            if (R > 1 && 2 * n_slices * rp.n_tiles < 3 * sms) continue;
            // two CTAs per SM (their MMA streams interleave on the tensor core) as
            // soon as each fits a two-stage halo ring beside its weights
            const bool two = w_bytes + 2u * rp.stage_bytes + kAlign <= lim.rows_smem_two && 2u * tmem_cols <= 512u;
            const uint32_t budget = two ? lim.rows_smem_two : kSmemMax;
            int S = (int)((budget - kAlign - w_bytes) / rp.stage_bytes);
            rp.stages = S > kRowMaxStages ? kRowMaxStages : S;
            rp.smem_bytes = (uint32_t)rp.stages * rp.stage_bytes + w_bytes + kAlign;
            const int per_slice = (two ? 2 : 1) * sms / n_slices;
            rp.grid = n_slices * (per_slice < rp.n_tiles ? per_slice : rp.n_tiles);
            if (two || R == 1) {
                *out = have_single && !two ? single : rp;
                return true;
            }
            if (!have_single) {
                single = rp;
                have_single = true;
            }
        }
        if (have_single) {
            *out = single;
            return true;
        }
    }
    return false;
}

size_t conv_smem_bytes(int cout_pad) {
    const size_t stage = ((size_t)128 * 32 + (size_t)cout_pad * 32 + 1023) & ~(size_t)1023;
    return kStages * stage + 1024;
}

}  // namespace

bool encode_plane_rows_map(CUtensorMap* map, const void* base, int W, int H, long long n_planes, int box_px,
                           int box_rows, int box_planes, const char** why) {
    auto enc = encode_fn(why);
    if (!enc) return false;
    // BF16 8-channel planes [plane][H][W][16 B] as rows of 8-byte elements (two per pixel), so that a box
    // row of box_px pixels is one contiguous run for the copy engine
    const cuuint64_t dims[3] = {(cuuint64_t)W * 2, (cuuint64_t)H, (cuuint64_t)n_planes};
    const cuuint64_t str[2] = {(cuuint64_t)W * 16, (cuuint64_t)H * W * 16};
    const cuuint32_t box[3] = {(cuuint32_t)box_px * 2, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
    const cuuint32_t ones[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, const_cast<void*>(base), dims, str, box, ones,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *why = "plane-row tensor map rejected by the driver";
        return false;
    }
    return true;
}

// 128-pixel row tiles from 48 pixels up (narrower rows would leave most of each
// tile's MMA rows empty); below that the smallest power of two covering W
int conv_pick_tile_w(int W) {
    if (W >= 48) return 128;
    int tw = 64;
    while (tw > 8 && tw / 2 >= W) tw /= 2;
    return tw;
}

bool conv_make_desc(ConvDesc* d, const void* x, const void* w, const char** why) {
    auto enc = encode_fn(why);
    if (!enc) return false;
    const ConvParams& p = d->p;
    // The maps move bytes: activations are planes of 16-byte pixel rows
    // ([img * cin_bytes / 16 + plane][H][W][16 B]), weights are K-major rows
    // of 9 * cin_bytes bytes, BF16 or E4M3 alike.
    const cuuint64_t xdims[4] = {16, (cuuint64_t)p.W, (cuuint64_t)p.H, (cuuint64_t)p.n_img * (p.cin_bytes / 16)};
    const cuuint64_t xstr[3] = {16, (cuuint64_t)p.W * 16, (cuuint64_t)p.H * p.W * 16};
    const cuuint32_t xbox[4] = {16, (cuuint32_t)p.tw, (cuuint32_t)p.th, 1};
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    CUresult r = enc(&d->tmap_x, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, const_cast<void*>(x), xdims, xstr, xbox, ones,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *why = "activation tensor map rejected by the driver";
        return false;
    }
    const cuuint64_t wdims[2] = {(cuuint64_t)9 * p.cin_bytes, (cuuint64_t)p.cout_pad};
    const cuuint64_t wstr[1] = {(cuuint64_t)9 * p.cin_bytes};
    const cuuint32_t wbox[2] = {32, (cuuint32_t)p.cout_pad};
    r = enc(&d->tmap_w, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(w), wdims, wstr, wbox, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *why = "weight tensor map rejected by the driver";
        return false;
    }
    d->p.x = x;
    d->rows_form = plan_rows(d->p, &d->rp);
    if (d->rows_form) {
        const RowPlan& rp = d->rp;
        d->p.tiles_y = (p.H + rp.rows - 1) / rp.rows;
        // The same K-major weights [cout][tap][cin] viewed as (32 bytes of
        // channels, cout, tap, chunk): one box lands in shared memory as
        // [tap][nc][32 B].
        const cuuint64_t hdims[4] = {32, (cuuint64_t)p.cout_pad, 9, (cuuint64_t)(p.cin_bytes / 32)};
        const cuuint64_t hstr[3] = {(cuuint64_t)9 * p.cin_bytes, (cuuint64_t)p.cin_bytes, 32};
        const cuuint32_t hwbox[4] = {32, (cuuint32_t)rp.nc, 9, 1};
        r = enc(&d->tmap_wh, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, const_cast<void*>(w), hdims, hstr, hwbox, ones,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            *why = "halo weight tensor map rejected by the driver";
            return false;
        }
    }
    return true;
}

template <bool FP8, bool MP, int EV>
static void set_rows_smem(int bytes, cudaError_t* err) {
    const void* fs[3] = {(const void*)conv_tc_rows_kernel<1, FP8, MP, EV>,
                         (const void*)conv_tc_rows_kernel<2, FP8, MP, EV>,
                         (const void*)conv_tc_rows_kernel<4, FP8, MP, EV>};
    for (const void* f : fs)
        if (*err == cudaSuccess && bytes > 0)
            *err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <bool FP8, bool MP, int EV>
static void launch_rows(const ConvDesc& d, cudaStream_t stream) {
    const dim3 g(d.rp.grid), t(kRowThreads);
    const size_t sm = d.rp.smem_bytes;
    if (d.rp.rows == 4)
        launch_k_dependent(conv_tc_rows_kernel<4, FP8, MP, EV>, g, t, sm, stream, d.tmap_wh, d.p, d.rp);
    else if (d.rp.rows == 2)
        launch_k_dependent(conv_tc_rows_kernel<2, FP8, MP, EV>, g, t, sm, stream, d.tmap_wh, d.p, d.rp);
    else launch_k_dependent(conv_tc_rows_kernel<1, FP8, MP, EV>, g, t, sm, stream, d.tmap_wh, d.p, d.rp);
}

bool conv_mask_prefetch(const ConvDesc& d) { return d.rows_form && d.p.mode == kDgradMask && d.rp.nc <= 64; }

cudaError_t conv_launch(const ConvDesc& d, cudaStream_t stream) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        const int lim = (int)device_limits().rows_smem_max;
        const int tile = (int)conv_smem_bytes(256);
        const void* generic[4] = {(const void*)conv_tc_kernel<false, false>, (const void*)conv_tc_kernel<true, false>,
                                  (const void*)conv_tc_kernel<false, true>, (const void*)conv_tc_kernel<true, true>};
        for (const void* f : generic)
            if (attr_err == cudaSuccess)
                attr_err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, tile);
        set_rows_smem<false, false, 0>(lim, &attr_err);
        set_rows_smem<true, false, 0>(lim, &attr_err);
        set_rows_smem<false, true, 0>(lim, &attr_err);
        set_rows_smem<true, true, 0>(lim, &attr_err);
        set_rows_smem<false, false, 1>(lim, &attr_err);
        set_rows_smem<true, false, 1>(lim, &attr_err);
        set_rows_smem<false, false, 2>(lim, &attr_err);
        set_rows_smem<true, false, 2>(lim, &attr_err);
    });
    if (attr_err != cudaSuccess) return attr_err;
    if (d.rows_form) {
        // masked input gradients whose mask words fit the prefetch registers take the prefetching variant
        const bool mp = conv_mask_prefetch(d);
        const bool pl = d.p.pool_out != nullptr;  // conv_make_desc keeps it only where the plan can pool
        const bool pb = d.p.mode == kDgradPoolBwd;
        if (d.p.fp8) {
            if (mp) launch_rows<true, true, 0>(d, stream);
            else if (pl) launch_rows<true, false, 1>(d, stream);
            else if (pb) launch_rows<true, false, 2>(d, stream);
            else launch_rows<true, false, 0>(d, stream);
        } else {
            if (mp) launch_rows<false, true, 0>(d, stream);
            else if (pl) launch_rows<false, false, 1>(d, stream);
            else if (pb) launch_rows<false, false, 2>(d, stream);
            else launch_rows<false, false, 0>(d, stream);
        }
        return cudaGetLastError();
    }
    const int n_tiles = d.p.n_img * d.p.tiles_y * d.p.tiles_x;
    const size_t smem = conv_smem_bytes(d.p.cout_pad);
    const bool pb = d.p.mode == kDgradPoolBwd;
    if (d.p.fp8) {
        if (pb) launch_k(conv_tc_kernel<true, true>, n_tiles, kConvThreads, smem, stream, d.tmap_x, d.tmap_w, d.p);
        else launch_k(conv_tc_kernel<true, false>, n_tiles, kConvThreads, smem, stream, d.tmap_x, d.tmap_w, d.p);
    } else {
        if (pb) launch_k(conv_tc_kernel<false, true>, n_tiles, kConvThreads, smem, stream, d.tmap_x, d.tmap_w, d.p);
        else launch_k(conv_tc_kernel<false, false>, n_tiles, kConvThreads, smem, stream, d.tmap_x, d.tmap_w, d.p);
    }
    return cudaGetLastError();
}

}  // namespace mcdi
