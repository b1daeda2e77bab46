// Device helpers of the tcgen05 kernels (sm_103a): shared-memory addresses,
// bounded mbarrier waits, tensor-core fences and tensor-memory loads, and the
// instruction descriptor of BF16 MMAs with FP32 accumulation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mcdi {

constexpr uint64_t kWaitNs = 2000000000ull;

static __device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

static __device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

static __device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

static __device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

static __device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
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
static __device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 255u) == 0u && global_ns() - t0 > kWaitNs) return false;
    }
}

static __device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

static __device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M x N.
static __host__ __device__ constexpr uint32_t bf16_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The same with both A and B MN-major (bits 15 and 16): in shared memory each
// operand's M (or N) index runs within 16-byte rows and its K index across
// rows, i.e. core matrices of 8 K-rows x 16 bytes.
static __host__ __device__ constexpr uint32_t bf16_idesc_mn(int M, int N) {
    return bf16_idesc(M, N) | (1u << 15) | (1u << 16);
}

// Shared-memory descriptor of an MN-major operand without swizzle: core
// matrices of 8 K-rows of 16 bytes (8 BF16 along M or N, rows 16 bytes
// apart); K-adjacent core matrices `k_stride` bytes apart (the leading byte
// offset field) and MN-adjacent ones `mn_stride` bytes apart (the stride byte
// offset field) -- for this no-swizzle MN-major form the two fields trade the
// roles they have in the swizzled and K-major forms.
static __device__ __forceinline__ uint64_t mn_desc(uint32_t saddr, uint32_t k_stride, uint32_t mn_stride) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((k_stride >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((mn_stride >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version; swizzle mode 0 (none)
    return d;
}

static __device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

static __device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

static __device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

}  // namespace mcdi
