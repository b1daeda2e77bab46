// tcgen05 implicit-GEMM 3x3 convolution (see tc_conv.cuh).
//
// One CTA computes a tile of 128 output pixels (tw x th) for all output
// channels: D[128 x cout_pad] (FP32, in tensor memory) = sum over the 9 taps
// and over input-channel chunks of 16 of
//   A[128 pixels x 16 ch] (the input shifted by the tap, zero outside the
//   image: TMA out-of-bounds fill) x B[cout_pad x 16 ch]^T (weights).
// Every chunk is one tcgen05.mma (M = 128, N = cout_pad, K = 16, BF16 inputs,
// FP32 accumulation).  Operands are staged by TMA into 32-byte-swizzled shared
// memory through a ring of kStages buffers guarded by mbarriers:
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

namespace mcdi {
namespace {

constexpr int kStages = 6;
constexpr int kConvThreads = 128;
constexpr uint64_t kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false after kWaitNs without the phase completing
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 255u) == 0u && global_ns() - t0 > kWaitNs) return false;
    }
}

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

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

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

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M x N.
__host__ __device__ constexpr uint32_t bf16_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void store16_bf16(__nv_bfloat16* dst, const float* f) {
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t*>(&h);
    }
    uint4* d = reinterpret_cast<uint4*>(dst);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// bias / activation / mask and store of 16 output channels of one pixel
__device__ __forceinline__ void epilogue16(const ConvParams& p, const uint32_t* v, int c0, int img, int x, int y,
                                           size_t pix) {
    float f[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i] = __uint_as_float(v[i]);
    if (p.mode == kDgradMask || p.mode == kDgradPlain) {
        if (p.mode == kDgradMask) {
            const uint4* mk4 = reinterpret_cast<const uint4*>(p.mask + pix * p.mask_ctotal + p.mask_coff + c0);
            const uint4 m0 = mk4[0], m1 = mk4[1];
            const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&mw[i]);
                if (!(__bfloat162float(h.x) > 0.0f)) f[2 * i] = 0.0f;
                if (!(__bfloat162float(h.y) > 0.0f)) f[2 * i + 1] = 0.0f;
            }
        }
        store16_bf16(p.out + pix * p.out_ctotal + p.out_coff + c0, f);
        return;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        f[i] += p.bias ? __ldg(p.bias + c0 + i) : 0.0f;
        if (p.relu) f[i] = fmaxf(f[i], 0.0f);
    }
    if (p.mode == kStoreF32) {
        p.out_f32[pix] = make_float4(f[0], f[1], f[2], 0.0f);
    } else if (p.mode == kStoreUp2) {
        const int W2 = 2 * p.W, H2 = 2 * p.H;
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const size_t q = ((size_t)img * H2 + 2 * y + j) * W2 + 2 * x + i;
                store16_bf16(p.out + q * p.out_ctotal + p.out_coff + c0, f);
            }
    } else {
        store16_bf16(p.out + pix * p.out_ctotal + p.out_coff + c0, f);
    }
}

__global__ void __launch_bounds__(kConvThreads) conv_tc_kernel(const __grid_constant__ CUtensorMap tmap_x,
                                                               const __grid_constant__ CUtensorMap tmap_w,
                                                               const ConvParams p) {
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
    const int cpt = p.cin_pad >> 4;  // channel chunks per tap
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
            tma_load_4d(a_dst, &tmap_x, cc * 16, x0 + dx - 1, y0 + dy - 1, img, fb);
            tma_load_2d(a_dst + a_bytes, &tmap_w, tap * p.cin_pad + cc * 16, 0, fb);
            issued = k + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = bf16_idesc(128, p.cout_pad);
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
            const uint64_t adesc = sw32_desc(a_src), bdesc = sw32_desc(a_src + a_bytes);
            const uint32_t accum = k > 0 ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
                : "memory");
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
    const size_t pix = ((size_t)img * p.H + y) * p.W + x;
    for (int c0 = 0; c0 < p.cout_pad; c0 += 16) {
        uint32_t v[16];
        // collective load of 16 accumulator columns of this warp's 32 lanes
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (valid && c0 < p.cout_valid) epilogue16(p, v, c0, img, x, y, pix);
        __syncwarp();
    }

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

size_t conv_smem_bytes(int cout_pad) {
    const size_t stage = ((size_t)128 * 32 + (size_t)cout_pad * 32 + 1023) & ~(size_t)1023;
    return kStages * stage + 1024;
}

}  // namespace

int conv_pick_tile_w(int W) {
    int tw = 128;
    while (tw > 8 && tw / 2 >= W) tw /= 2;
    return tw;
}

bool conv_make_desc(ConvDesc* d, const __nv_bfloat16* x, const __nv_bfloat16* w, const char** why) {
    auto enc = encode_fn(why);
    if (!enc) return false;
    const ConvParams& p = d->p;
    const cuuint64_t xdims[4] = {(cuuint64_t)p.cin_pad, (cuuint64_t)p.W, (cuuint64_t)p.H, (cuuint64_t)p.n_img};
    const cuuint64_t xstr[3] = {(cuuint64_t)p.cin_pad * 2, (cuuint64_t)p.W * p.cin_pad * 2,
                                (cuuint64_t)p.H * p.W * p.cin_pad * 2};
    const cuuint32_t xbox[4] = {16, (cuuint32_t)p.tw, (cuuint32_t)p.th, 1};
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    CUresult r = enc(&d->tmap_x, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(x), xdims, xstr,
                     xbox, ones, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *why = "activation tensor map rejected by the driver";
        return false;
    }
    const cuuint64_t wdims[2] = {(cuuint64_t)9 * p.cin_pad, (cuuint64_t)p.cout_pad};
    const cuuint64_t wstr[1] = {(cuuint64_t)9 * p.cin_pad * 2};
    const cuuint32_t wbox[2] = {16, (cuuint32_t)p.cout_pad};
    r = enc(&d->tmap_w, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(w), wdims, wstr, wbox, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *why = "weight tensor map rejected by the driver";
        return false;
    }
    return true;
}

cudaError_t conv_launch(const ConvDesc& d, cudaStream_t stream) {
    const size_t smem = conv_smem_bytes(d.p.cout_pad);
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)conv_smem_bytes(256));
    });
    if (attr_err != cudaSuccess) return attr_err;
    const int grid = d.p.n_img * d.p.tiles_y * d.p.tiles_x;
    conv_tc_kernel<<<grid, kConvThreads, smem, stream>>>(d.tmap_x, d.tmap_w, d.p);
    return cudaGetLastError();
}

}  // namespace mcdi
