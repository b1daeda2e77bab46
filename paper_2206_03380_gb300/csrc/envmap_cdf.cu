// Piecewise-constant 2D sampling distribution of the light probe (Sec. 4.1:
// light importance sampling; the distribution is rebuilt whenever the probe
// changes).  Texel weights w_ij = max(Y, 0) sin(theta_j) with Y = (r+g+b)/3 and
// theta_j the band-centre polar angle; prefix sums are accumulated in FP64
// (block-wide warp-shuffle scans) and the normalised tables stored in FP32.
#include "common.cuh"
#include "internal.h"

namespace mcdi {
namespace {

constexpr int kCdfThreads = 256;

// Exclusive block scan of one double per thread; returns the exclusive prefix
// and writes the block total to *total (all threads).
template <int THREADS>
__device__ double block_exclusive_scan(double v, double* total) {
    __shared__ double warp_off[THREADS / 32];
    __shared__ double block_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double n = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += n;
    }
    double ex = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) ex = 0.0;
    if (lane == 31) warp_off[warp] = inc;  // warp total
    __syncthreads();
    if (warp == 0) {
        const double w = lane < THREADS / 32 ? warp_off[lane] : 0.0;
        double winc = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double n = __shfl_up_sync(0xffffffffu, winc, off);
            if (lane >= off) winc += n;
        }
        double wex = __shfl_up_sync(0xffffffffu, winc, 1);
        if (lane == 0) wex = 0.0;
        __syncwarp();
        if (lane < THREADS / 32) warp_off[lane] = wex;
        if (lane == 31) block_total = winc;
    }
    __syncthreads();
    *total = block_total;
    return warp_off[warp] + ex;
}

// One block per probe row j: conditional CDF of the row and its sum R_j.
__global__ void __launch_bounds__(kCdfThreads) row_cdf_kernel(const float4* __restrict__ env, int W, int H,
                                                               float* __restrict__ cond, double* __restrict__ row_sum) {
    pdl_prologue();
    const int j = blockIdx.x;
    const int chunk = (W + kCdfThreads - 1) / kCdfThreads;
    const int i0 = min(W, threadIdx.x * chunk), i1 = min(W, i0 + chunk);
    const double s = sin(3.14159265358979323846 * (j + 0.5) / H);
    const float4* row = env + (size_t)j * W;
    double local = 0.0;
    for (int i = i0; i < i1; ++i) {
        const float4 t = row[i];
        const double Y = ((double)t.x + (double)t.y + (double)t.z) / 3.0;
        local += (Y > 0.0 ? Y : 0.0) * s;
    }
    double R;
    double run = block_exclusive_scan<kCdfThreads>(local, &R);
    float* c = cond + (size_t)j * (W + 1);
    for (int i = i0; i < i1; ++i) {
        if (R > 0.0) {
            c[i] = (float)(run / R);
            const float4 t = row[i];
            const double Y = ((double)t.x + (double)t.y + (double)t.z) / 3.0;
            run += (Y > 0.0 ? Y : 0.0) * s;
        } else {
            c[i] = (float)((double)i / W);
        }
    }
    if (threadIdx.x == 0) {
        c[W] = 1.0f;
        row_sum[j] = R;
    }
}

constexpr int kMargThreads = 1024;

// Single block: marginal CDF over the row sums and the normaliser T.
__global__ void __launch_bounds__(kMargThreads) marg_cdf_kernel(const double* __restrict__ row_sum, int H,
                                                                 float* __restrict__ marg, double* __restrict__ total) {
    pdl_prologue();
    const int chunk = (H + kMargThreads - 1) / kMargThreads;
    const int j0 = min(H, threadIdx.x * chunk), j1 = min(H, j0 + chunk);
    double local = 0.0;
    for (int j = j0; j < j1; ++j) local += row_sum[j];
    double T;
    double run = block_exclusive_scan<kMargThreads>(local, &T);
    for (int j = j0; j < j1; ++j) {
        if (T > 0.0) {
            marg[j] = (float)(run / T);
            run += row_sum[j];
        } else {
            marg[j] = (float)((double)j / H);
        }
    }
    if (threadIdx.x == 0) {
        marg[H] = 1.0f;
        *total = T;
    }
}

}  // namespace

cudaError_t launch_envmap_cdf(const float* env, int W, int H, float* cond, float* marg, double* row_sum,
                              double* total, cudaStream_t stream) {
    launch_k(row_cdf_kernel, H, kCdfThreads, 0, stream, reinterpret_cast<const float4*>(env), W, H, cond, row_sum);
    launch_k(marg_cdf_kernel, 1, kMargThreads, 0, stream, row_sum, H, marg, total);
    return cudaGetLastError();
}

}  // namespace mcdi
