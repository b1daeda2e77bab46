// Read sweep over a buffer small enough to stay in L2: the denominator of the
// shadow-ray tracer's L2 request bandwidth (the tracer's working set, BVH and
// triangles, is L2-resident at the headline scene size).
#include "internal.h"

namespace mcdi {
namespace {

constexpr int kSweepThreads = 512;

// Every thread reads 16-byte words with ld.global.cg (cached in L2, not L1)
// in a grid-stride loop, `passes` times over the buffer; the xor of what it
// read reaches *sink only if it equals a value no buffer of zeros gives, so
// the loads cannot be dropped.
__global__ void __launch_bounds__(kSweepThreads) read_sweep_kernel(const uint4* __restrict__ buf, long long n16,
                                                                   int passes, unsigned* __restrict__ sink) {
    pdl_prologue();
    uint32_t acc = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p) {
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
            uint32_t a, b, c, d;
            asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
                         : "l"(buf + i));
            acc ^= a ^ b ^ c ^ d;
        }
    }
    if (acc == 0x9e3779b9u) *sink = acc;
}

}  // namespace

cudaError_t launch_read_sweep(const void* buf, size_t bytes, int passes, unsigned* sink, cudaStream_t stream) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    launch_k(read_sweep_kernel, sms * 4, kSweepThreads, 0, stream, static_cast<const uint4*>(buf),
             (long long)(bytes / 16), passes, sink);
    return cudaGetLastError();
}

}  // namespace mcdi
