// Final colour from the separated, denoised light terms (Sec. 4.2: the image
// is composed as c = k_d * D(c_d) + D(c_s), with the demodulated diffuse term
// re-modulated by the diffuse reflectance).
#include "internal.h"

namespace mcdi {
namespace {

__global__ void composite_kernel(const float4* __restrict__ kd, const float4* __restrict__ dd,
                                 const float4* __restrict__ ds, long long n, float4* __restrict__ c) {
    pdl_prologue();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 k = kd[i], a = dd[i], b = ds[i];
    c[i] = make_float4(k.x * a.x + b.x, k.y * a.y + b.y, k.z * a.z + b.z, 0.0f);
}

}  // namespace

cudaError_t launch_composite(const float* kd, const float* dd, const float* ds, long long n, float* c,
                             cudaStream_t s) {
    launch_k(composite_kernel, (int)((n + 255) / 256), 256, 0, s, reinterpret_cast<const float4*>(kd),
             reinterpret_cast<const float4*>(dd), reinterpret_cast<const float4*>(ds), n, reinterpret_cast<float4*>(c));
    return cudaGetLastError();
}

}  // namespace mcdi
