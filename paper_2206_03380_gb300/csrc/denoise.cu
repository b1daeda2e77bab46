// The differentiable denoiser (Sec. 4.2 "Neural denoisers", App. B): a U-Net
// of 3x3 convolutions applied to the demodulated diffuse term c_d and the
// specular term c_s, each with the k_d and normal planes as guides.  Forward
// and input-gradient backward (Sec. 4.2's gradient-sharing identity
// dL/dX = dL/dO conv F^T is what the backward convolutions compute); the
// paper's main results lock the denoiser weights, and the weight gradient of
// its live-trained variant (App. B) runs on request from the stored
// activations and gradients (wgrad.cu).
//
// Precision: BF16 operands, or E4M3 operands with per-tensor scaling (every
// convolution input and weight tensor quantised as round(v 448 / amax) just
// before use, FP32 accumulation rescaled by the two amax / 448 factors); the
// stored activations and gradients stay BF16 either way.
//
// Layout: BF16 activations in 8-channel planes, channels padded to multiples
// of 16 (E4M3 copies: 16-channel planes, padded to multiples of 32).  Skip
// connections are never copied: the encoder's second convolution of a level
// stores straight into the channel slice of that level's concatenation buffer,
// and the decoder's second convolution stores its 2x nearest-upsampled output
// into the other slice one level up ([upsampled | skip], as in the reading of
// the network).  Max-pooling and the small backward routing steps are
// memory-bound kernels of their own.
#include <cuda_fp8.h>
#include <algorithm>
#include <stdio.h>

#include "internal.h"
#include "tc_conv.cuh"

namespace mcdi {

// ---------------------------------------------------------------- plan
struct ConvSpec {
    int ci, co, level;
};
// enc1a enc1b enc2a enc2b enc3a enc3b bot_a bot_b dec3a dec3b dec2a dec2b dec1a dec1b out
static const ConvSpec kPlan[kUnetConvs] = {
    {9, 32, 0},   {32, 32, 0},  {32, 48, 1}, {48, 48, 1}, {48, 64, 2}, {64, 64, 2}, {64, 96, 3}, {96, 96, 3},
    {160, 64, 2}, {64, 64, 2},  {112, 48, 1}, {48, 48, 1}, {80, 32, 0}, {32, 32, 0}, {32, 3, 0}};

static int pad16(int c) { return (c + 15) & ~15; }

static int pad32(int c) { return (c + 31) & ~31; }

UnetWeightLayout unet_weight_layout() {
    UnetWeightLayout L{};
    size_t o = 0;
    for (int i = 0; i < kUnetConvs; ++i) {
        const int cip = pad16(kPlan[i].ci), cop = pad16(kPlan[i].co);
        L.wk[i] = o;
        o = align256(o + (size_t)cop * 9 * cip * 2);
        L.wf[i] = o;
        o = align256(o + (size_t)cip * 9 * cop * 2);
        L.bias[i] = o;
        o = align256(o + (size_t)cop * 4);
        L.wk8[i] = o;  // E4M3 [cop][9][pad32(ci)]
        o = align256(o + (size_t)cop * 9 * pad32(kPlan[i].ci));
        L.wf8[i] = o;  // E4M3 [cip][9][pad32(co)]
        o = align256(o + (size_t)cip * 9 * pad32(kPlan[i].co));
    }
    L.amax = o;  // one float per convolution: amax of its weights
    o = align256(o + kUnetConvs * sizeof(float));
    L.total = o;
    size_t n = 0;
    for (int i = 0; i < kUnetConvs; ++i) n += (size_t)kPlan[i].co * kPlan[i].ci * 9 + kPlan[i].co;
    L.n_params = n;
    return L;
}

// activation buffers (forward) and gradient buffers (backward)
enum Act { X0, A1, CAT1, P1, A2, CAT2, P2, A3, CAT3, P3, B1, D3A, D2A, D1A, D1B, kActs };
static const int kActC[kActs] = {16, 32, 80, 32, 48, 112, 48, 64, 160, 64, 96, 64, 48, 32, 32};
static const int kActLvl[kActs] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 2, 1, 0, 0};
// (the gradient at each pool's output is never stored: the convolution that computes it routes it through
// the pool into g_E directly, kDgradPoolBwd)
enum Grad { GY, GD1B, GD1A, GCAT1, GD2B, GD2A, GCAT2, GD3B, GD3A, GCAT3, GB2, GB1, GE3, GA3, GE2, GA2, GE1, GA1,
            kGrads };
static const int kGradC[kGrads] = {16, 32, 32, 80, 48, 48, 112, 64, 64, 160, 96, 96, 64, 64, 48, 48, 32, 32};
static const int kGradLvl[kGrads] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0};

static size_t level_pixels(int n, int H, int W, int l) { return (size_t)n * (H >> l) * (W >> l); }

template <int K>
static void layout_of(const int* C, const int* lvl, int n, int H, int W, size_t* off, size_t* total) {
    size_t o = 0;
    for (int i = 0; i < K; ++i) {
        off[i] = o;
        o = align256(o + level_pixels(n, H, W, lvl[i]) * C[i] * 2);
    }
    *total = o;
}

// E4M3 copies of the convolution inputs are made just before each convolution
// into one scratch region (largest input), followed by the amax slots.
static const int kFwdIn[kUnetConvs][2] = {{0, 16}, {0, 32}, {1, 32}, {1, 48}, {2, 48}, {2, 64}, {3, 64}, {3, 96},
                                          {2, 160}, {2, 64}, {1, 112}, {1, 48}, {0, 80}, {0, 32}, {0, 32}};
static const int kBwdIn[kUnetConvs][2] = {{0, 16}, {0, 32}, {0, 32}, {1, 48}, {1, 48}, {2, 64}, {2, 64}, {3, 96},
                                          {3, 96}, {2, 64}, {2, 64}, {1, 48}, {1, 48}, {0, 32}, {0, 32}};
constexpr int kAmaxSlots = 64;  // one per tensor: an Act (forward) or Grad (backward) index
static_assert(kActs <= kAmaxSlots && kGrads <= kAmaxSlots, "amax slots");

static size_t e4m3_scratch(const int (*in)[2], int n, int H, int W) {
    size_t m = 0;
    for (int i = 0; i < kUnetConvs; ++i) {
        const size_t b = level_pixels(n, H, W, in[i][0]) * pad32(in[i][1]);
        m = b > m ? b : m;
    }
    return m;
}

struct Fp8Region {
    size_t q, amax, total;
};

static Fp8Region fp8_region(size_t base, const int (*in)[2], int n, int H, int W) {
    Fp8Region r;
    r.q = align256(base);
    r.amax = align256(r.q + e4m3_scratch(in, n, H, W));
    r.total = align256(r.amax + kAmaxSlots * sizeof(float));
    return r;
}

size_t unet_act_bytes(int n, int H, int W, int precision) {
    size_t off[kActs], t;
    layout_of<kActs>(kActC, kActLvl, n, H, W, off, &t);
    return precision == MCDI_DENOISE_E4M3 ? fp8_region(t, kFwdIn, n, H, W).total : t;
}

size_t unet_grad_bytes(int n, int H, int W, int precision) {
    size_t off[kGrads], t;
    layout_of<kGrads>(kGradC, kGradLvl, n, H, W, off, &t);
    return precision == MCDI_DENOISE_E4M3 ? fp8_region(t, kBwdIn, n, H, W).total : t;
}

namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ int pad16_dev(int c) { return (c + 15) & ~15; }

// ---------------------------------------------------------------- small kernels
// Activations and gradients are BF16 in 8-channel planes: a C-channel tensor
// at H x W is [img][C / 8][H][W][8], so a warp's 32 pixels of one group are
// 512 contiguous bytes and a tensor-map box of one group is a run of 16-byte
// rows.
__device__ __forceinline__ size_t poff(int img, int G, int g, int H, int W, int y, int x) {
    return ((((size_t)img * G + g) * H + y) * W + x) * 8;
}

__device__ __forceinline__ void ld8(const bf16* p, float* f) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[i]);
        f[2 * i] = __bfloat162float(h.x);
        f[2 * i + 1] = __bfloat162float(h.y);
    }
}

__device__ __forceinline__ void st8(bf16* p, const float* f) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

// max |v| of 8 values about to be stored as BF16, folded into a running max
__device__ __forceinline__ float max8(float m, const float* f) {
#pragma unroll
    for (int c = 0; c < 8; ++c) m = fmaxf(m, fabsf(f[c]));
    return m;
}

// A thread's running max |value| of what it stored, published for the E4M3
// consumer of the tensor (float bits in *amax, null in BF16 mode): rounded to
// BF16 like the stored values (monotonic, so it is the max over the stored
// tensor), reduced over the warp, one atomic per warp.  Every lane of the
// warp calls it.
__device__ __forceinline__ void warp_amax(unsigned* amax, float m) {
    if (amax == nullptr) return;
    const unsigned w = __reduce_max_sync(0xffffffffu, __float_as_uint(__bfloat162float(__float2bfloat16_rn(m))));
    if ((threadIdx.x & 31) == 0 && w) atomicMax(amax, w);
}

// network input: [term.rgb, k_d.rgb, normal.xyz, 0 x 7] per pixel (16
// channels, two planes); image i uses guide planes of image i % n_aux
__global__ void pack_input_kernel(const float4* __restrict__ term, const float4* __restrict__ kd,
                                  const float4* __restrict__ nrm, int n_img, int n_aux, int HW, bf16* __restrict__ x,
                                  unsigned* amax) {
    pdl_prologue();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.0f;
    if (i < (long long)n_img * HW) {
        const int img = (int)(i / HW), p = (int)(i - (long long)img * HW);
        const long long g = (long long)(img % n_aux) * HW + p;
        const float4 t = term[i], k = kd[g], n = nrm[g];
        const float f0[8] = {t.x, t.y, t.z, k.x, k.y, k.z, n.x, n.y}, f1[8] = {n.z, 0, 0, 0, 0, 0, 0, 0};
        st8(x + (((size_t)img * 2 + 0) * HW + p) * 8, f0);
        st8(x + (((size_t)img * 2 + 1) * HW + p) * 8, f1);
        m = max8(max8(m, f0), f1);
    }
    warp_amax(amax, m);
}

// upstream gradient (rgb of float4) -> 16-channel BF16 (channels 3..15 zero)
__global__ void pack_grad_kernel(const float4* __restrict__ gy, int n_img, int HW, bf16* __restrict__ g,
                                 unsigned* amax) {
    pdl_prologue();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.0f;
    if (i < (long long)n_img * HW) {
        const int img = (int)(i / HW), p = (int)(i - (long long)img * HW);
        const float4 v = gy[i];
        const float f0[8] = {v.x, v.y, v.z, 0, 0, 0, 0, 0}, f1[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        st8(g + (((size_t)img * 2 + 0) * HW + p) * 8, f0);
        st8(g + (((size_t)img * 2 + 1) * HW + p) * 8, f1);
        m = max8(m, f0);
    }
    warp_amax(amax, m);
}

// thread index -> (img, group, y, x) with x fastest
__device__ __forceinline__ bool split_index(long long i, int groups, int H, int W, int* img, int* g, int* y, int* x,
                                            int n) {
    if (i >= (long long)n * groups * H * W) return false;
    *x = (int)(i % W);
    i /= W;
    *y = (int)(i % H);
    i /= H;
    *g = (int)(i % groups);
    *img = (int)(i / groups);
    return true;
}

// 2x2 max-pool of channels [coff, coff + C) of src (Ctot channels, H x W) into dst (C channels)
__global__ void maxpool2_kernel(const bf16* __restrict__ src, int Ctot, int coff, int C, int n, int H, int W,
                                bf16* __restrict__ dst, unsigned* amax) {
    pdl_prologue();
    const int Ho = H >> 1, Wo = W >> 1;
    int img, g, yo, xo;
    float a = 0.0f;
    if (split_index((long long)blockIdx.x * blockDim.x + threadIdx.x, C >> 3, Ho, Wo, &img, &g, &yo, &xo, n)) {
        float m[8], v[8];
        const bf16* s = src + poff(img, Ctot >> 3, (coff >> 3) + g, H, W, 2 * yo, 2 * xo);
        for (int k = 0; k < 4; ++k) {
            ld8(s + ((size_t)(k >> 1) * W + (k & 1)) * 8, v);
#pragma unroll
            for (int c = 0; c < 8; ++c) m[c] = k == 0 ? v[c] : fmaxf(m[c], v[c]);
        }
        st8(dst + poff(img, C >> 3, g, Ho, Wo, yo, xo), m);
        a = max8(a, m);
    }
    warp_amax(amax, a);
}

// gradient through "nearest 2x upsample then ReLU output": g_low = sum of the
// 2x2 block of g_cat[0 : C] times [activation > 0], the activation read from
// the upsampled copy in cat (top-left of the block)
__global__ void up2_bwd_kernel(const bf16* __restrict__ gcat, const bf16* __restrict__ cat, int Ctot, int C, int n,
                               int Hl, int Wl, bf16* __restrict__ glow, unsigned* amax) {
    pdl_prologue();
    int img, g, y, x;
    float m = 0.0f;
    if (split_index((long long)blockIdx.x * blockDim.x + threadIdx.x, C >> 3, Hl, Wl, &img, &g, &y, &x, n)) {
        const int H2 = 2 * Hl, W2 = 2 * Wl;
        const size_t o = poff(img, Ctot >> 3, g, H2, W2, 2 * y, 2 * x);
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0}, v[8], a[8];
        for (int k = 0; k < 4; ++k) {
            ld8(gcat + o + ((size_t)(k >> 1) * W2 + (k & 1)) * 8, v);
#pragma unroll
            for (int c = 0; c < 8; ++c) s[c] += v[c];
        }
        ld8(cat + o, a);
#pragma unroll
        for (int c = 0; c < 8; ++c) s[c] = a[c] > 0.0f ? s[c] : 0.0f;
        st8(glow + poff(img, C >> 3, g, Hl, Wl, y, x), s);
        m = max8(m, s);
    }
    warp_amax(amax, m);
}


// fp32 [co][ci][3][3] + [co] (the plan's parameters, concatenated) -> packed
// BF16 K-major forward weights [co_pad][tap][ci_pad], flipped transposed
// weights for the input gradient [ci_pad][tap'][co_pad] with tap' = 8 - tap,
// and zero-padded FP32 biases
__global__ void pack_weights_kernel(const float* __restrict__ W, const float* __restrict__ b, int ci, int co,
                                    bf16* __restrict__ wk, bf16* __restrict__ wf, float* __restrict__ bias) {
    pdl_prologue();
    const int cip = pad16_dev(ci), cop = pad16_dev(co);
    const long long n = (long long)cop * 9 * cip;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int c_in = (int)(i % cip);
        const int tap = (int)((i / cip) % 9);
        const int c_out = (int)(i / (9LL * cip));
        const float v = (c_in < ci && c_out < co) ? W[((size_t)c_out * ci + c_in) * 9 + tap] : 0.0f;
        wk[i] = __float2bfloat16_rn(v);
        wf[((size_t)c_in * 9 + (8 - tap)) * cop + c_out] = __float2bfloat16_rn(v);
    }
    if (i < cop) bias[i] = i < co ? b[i] : 0.0f;
}

// ---------------------------------------------------------------- E4M3
__device__ __forceinline__ float e4m3_scale(float amax) { return amax > 0.0f ? 448.0f / amax : 0.0f; }

// 16 floats -> 16 E4M3 codes (round to nearest even, saturating), one uint4
__device__ __forceinline__ uint4 to_e4m3x16(const float* f, float s) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(f[4 * i] * s, f[4 * i + 1] * s), __NV_SATFINITE, __NV_E4M3);
        const uint32_t hi =
            __nv_cvt_float2_to_fp8x2(make_float2(f[4 * i + 2] * s, f[4 * i + 3] * s), __NV_SATFINITE, __NV_E4M3);
        w[i] = lo | (hi << 16);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// BF16 tensor (C channels, 8-channel planes) -> E4M3 copy (pad32(C) channels,
// 16-channel planes), scale 448 / amax
__global__ void quant_e4m3_kernel(const bf16* __restrict__ x, int C, int n, int HW, const float* __restrict__ amax,
                                  uint8_t* __restrict__ q) {
    pdl_prologue();
    const int G16 = ((C + 31) & ~31) >> 4;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * G16 * HW) return;
    const int p = (int)(i % HW);
    const long long r = i / HW;
    const int g = (int)(r % G16), img = (int)(r / G16);
    const float s = e4m3_scale(*amax);
    float f[16];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int b = 2 * g + h;
        if (b < (C >> 3)) ld8(x + (((size_t)img * (C >> 3) + b) * HW + p) * 8, f + 8 * h);
        else
#pragma unroll
            for (int k = 0; k < 8; ++k) f[8 * h + k] = 0.0f;
    }
    reinterpret_cast<uint4*>(q)[((size_t)img * G16 + g) * HW + p] = to_e4m3x16(f, s);
}

__global__ void amax_f32_kernel(const float* __restrict__ w, long long n, unsigned* __restrict__ amax) {
    pdl_prologue();
    unsigned m = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(w[i])));
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(amax, m);
}

// E4M3 forward weights [cop][9][pad32(ci)] and flipped transposed backward
// weights [cip][9][pad32(co)], scale 448 / amax of the convolution's weights
__global__ void pack_weights_e4m3_kernel(const float* __restrict__ W, int ci, int co, const float* __restrict__ amax,
                                         uint8_t* __restrict__ wk8, uint8_t* __restrict__ wf8) {
    pdl_prologue();
    const int cip = pad16_dev(ci), cop = pad16_dev(co), ci32 = (ci + 31) & ~31, co32 = (co + 31) & ~31;
    const int cmax_o = co32 > cop ? co32 : cop, cmax_i = ci32 > cip ? ci32 : cip;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)cmax_o * 9 * cmax_i) return;
    const int c_in = (int)(i % cmax_i);
    const int tap = (int)((i / cmax_i) % 9);
    const int c_out = (int)(i / (9LL * cmax_i));
    const float v = (c_in < ci && c_out < co) ? W[((size_t)c_out * ci + c_in) * 9 + tap] : 0.0f;
    const uint8_t b = (uint8_t)__nv_cvt_float_to_fp8(v * e4m3_scale(*amax), __NV_SATFINITE, __NV_E4M3);
    if (c_out < cop && c_in < ci32) wk8[((size_t)c_out * 9 + tap) * ci32 + c_in] = b;
    if (c_in < cip && c_out < co32) wf8[((size_t)c_in * 9 + (8 - tap)) * co32 + c_out] = b;
}

}  // namespace

// ---------------------------------------------------------------- orchestration
// Launch-plan recorder (mcdi_denoise_record_plan): per host thread, one record
// of kPlanRecordInts ints per convolution launched while it is set.
struct PlanRecorder {
    int* rec = nullptr;
    int cap = 0;
    int* count = nullptr;
};
static thread_local PlanRecorder t_plan;

void set_plan_recorder(int* rec, int cap, int* count) {
    t_plan.rec = rec;
    t_plan.cap = cap;
    t_plan.count = count;
    if (count) *count = 0;
}

struct Unet {
    const char* wbase;
    UnetWeightLayout L;
    int n, H, W;
    unsigned* err;
    bool fp8 = false;
    uint8_t* q = nullptr;     // E4M3 copy of the current convolution's input
    float* amax = nullptr;    // one slot per tensor (Act or Grad index), zeroed at the start of a pass
    // where a producer publishes the amax of tensor k (null in BF16 mode or k < 0)
    unsigned* out(int k) const { return fp8 && k >= 0 ? reinterpret_cast<unsigned*>(amax + k) : nullptr; }
};

struct Wsel {  // which packed weights: convolution i, forward or flipped (input gradient)
    int i;
    bool dgrad;
};

static const bf16* wk_of(const Unet& u, int i) { return reinterpret_cast<const bf16*>(u.wbase + u.L.wk[i]); }
static const bf16* wf_of(const Unet& u, int i) { return reinterpret_cast<const bf16*>(u.wbase + u.L.wf[i]); }
static const float* b_of(const Unet& u, int i) { return reinterpret_cast<const float*>(u.wbase + u.L.bias[i]); }

static int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

#define CHECK(e)                          \
    do {                                  \
        cudaError_t _e = (e);             \
        if (_e != cudaSuccess) return _e; \
    } while (0)

static ConvDesc conv_desc(int n, int H, int W, int cin_pad, int cin_bytes, const float* bias, int cout_pad,
                          int cout_valid, int mode, int relu, bf16* out, int out_ctotal, int out_coff, float4* out_f32,
                          const bf16* mask, int mask_ctotal, int mask_coff, unsigned* err) {
    ConvDesc d{};
    ConvParams& p = d.p;
    p.n_img = n;
    p.H = H;
    p.W = W;
    p.tw = conv_pick_tile_w(p.W);
    p.th = 128 / p.tw;
    p.tiles_x = (p.W + p.tw - 1) / p.tw;
    p.tiles_y = (p.H + p.th - 1) / p.th;
    p.cin_pad = cin_pad;
    p.cin_bytes = cin_bytes;
    p.cout_pad = cout_pad;
    p.cout_valid = cout_valid;
    p.mode = mode;
    p.relu = relu;
    p.bias = bias;
    p.out = out;
    p.out_ctotal = out_ctotal;
    p.out_coff = out_coff;
    p.out_f32 = out_f32;
    p.mask = mask;
    p.mask_ctotal = mask_ctotal;
    p.mask_coff = mask_coff;
    p.err = err;
    return d;
}

// One convolution of the network on a BF16 input (tensor x_slot, written by
// producers that published its amax) into tensor out_slot (-1: no E4M3
// consumer).  In E4M3 mode the input is first quantised with its amax and the
// E4M3 weights are used.
struct PoolTo {  // a 2x2 max-pool of the convolution's output, into tensor `slot`
    bf16* out = nullptr;
    int ctotal = 0;
    int slot = -1;
    bool* done = nullptr;  // set when the convolution's epilogue wrote it
};

static cudaError_t run_conv(Unet& u, int level, const bf16* x, int x_slot, int cin_pad, Wsel w, const float* bias,
                            int cout_pad, int cout_valid, int mode, int relu, bf16* out, int out_slot, int out_ctotal,
                            int out_coff, float4* out_f32, const bf16* mask, int mask_ctotal, int mask_coff,
                            cudaStream_t s, const char** why, PoolTo pool = PoolTo{}, const bf16* gskip = nullptr) {
    const int Hl = u.H >> level, Wl = u.W >> level;
    ConvDesc d = conv_desc(u.n, Hl, Wl, cin_pad, 2 * cin_pad, bias, cout_pad, cout_valid, mode, relu, out, out_ctotal,
                           out_coff, out_f32, mask, mask_ctotal, mask_coff, u.err);
    d.p.gskip = gskip;
    d.p.out_amax = u.out(out_slot);
    const void* xin = x;
    const void* win = w.dgrad ? (const void*)wf_of(u, w.i) : (const void*)wk_of(u, w.i);
    if (u.fp8) {
        if (x_slot < 0 || x_slot >= kAmaxSlots) {
            *why = "denoiser: bad amax slot";
            return cudaErrorInvalidValue;
        }
        const float* am = u.amax + x_slot;
        const int c32 = pad32(cin_pad);
        launch_k(quant_e4m3_kernel, blocks_for((long long)u.n * (c32 / 16) * Hl * Wl, 256), 256, 0, s, x, cin_pad, u.n,
                 Hl * Wl, am, u.q);
        CHECK(cudaGetLastError());
        xin = u.q;
        win = u.wbase + (w.dgrad ? u.L.wf8[w.i] : u.L.wk8[w.i]);
        d.p.cin_pad = c32;
        d.p.cin_bytes = c32;
        d.p.fp8 = 1;
        d.p.x_amax = am;
        d.p.w_amax = reinterpret_cast<const float*>(u.wbase + u.L.amax) + w.i;
    }
    if (!conv_make_desc(&d, xin, win, why)) return cudaErrorInvalidValue;
    if (pool.out && d.rows_form && d.rp.rows % 2 == 0 && d.rp.nc <= 64 && mode == kStore) {
        d.p.pool_out = pool.out;
        d.p.pool_ctotal = pool.ctotal;
        d.p.pool_amax = u.out(pool.slot);
        *pool.done = true;
    }
    if (t_plan.rec && t_plan.count && *t_plan.count < t_plan.cap) {
        int* r = t_plan.rec + (size_t)kPlanRecordInts * (*t_plan.count)++;
        r[0] = w.dgrad ? 1 : 0;
        r[1] = w.i;
        r[2] = level;
        r[3] = d.rows_form ? 1 : 0;
        r[4] = d.rows_form ? d.rp.rows : 0;
        r[5] = conv_mask_prefetch(d) ? 1 : 0;
        r[6] = d.p.pool_out != nullptr ? 1 : 0;
        r[7] = d.p.fp8;
    }
    return conv_launch(d, s);
}

cudaError_t launch_unet_pack_weights(const float* params, void* weights, cudaStream_t s) {
    const UnetWeightLayout L = unet_weight_layout();
    char* base = static_cast<char*>(weights);
    float* amax = reinterpret_cast<float*>(base + L.amax);
    CHECK(cudaMemsetAsync(amax, 0, kUnetConvs * sizeof(float), s));
    size_t off = 0;
    for (int i = 0; i < kUnetConvs; ++i) {
        const int ci = kPlan[i].ci, co = kPlan[i].co;
        const long long n = (long long)pad16(co) * 9 * pad16(ci);
        const long long nw = (long long)co * ci * 9;
        launch_k(pack_weights_kernel, blocks_for(n, 256), 256, 0, s, params + off, params + off + (size_t)co * ci * 9,
                 ci, co, reinterpret_cast<bf16*>(base + L.wk[i]), reinterpret_cast<bf16*>(base + L.wf[i]),
                 reinterpret_cast<float*>(base + L.bias[i]));
        launch_k(amax_f32_kernel, std::min(blocks_for(nw, 256), 256), 256, 0, s, params + off, nw,
                 reinterpret_cast<unsigned*>(amax + i));
        const long long n8 = (long long)std::max(pad32(co), pad16(co)) * 9 * std::max(pad32(ci), pad16(ci));
        launch_k(pack_weights_e4m3_kernel, blocks_for(n8, 256), 256, 0, s, params + off, ci, co, amax + i,
                 reinterpret_cast<uint8_t*>(base + L.wk8[i]), reinterpret_cast<uint8_t*>(base + L.wf8[i]));
        off += (size_t)co * ci * 9 + co;
    }
    return cudaGetLastError();
}

cudaError_t launch_unet_fwd(const void* weights, int precision, int n, int H, int W, const float* term,
                            const float* kd, const float* nrm, int n_aux, float* y, void* acts, unsigned* err,
                            cudaStream_t s, const char** why) {
    Unet u{static_cast<const char*>(weights), unet_weight_layout(), n, H, W, err};
    size_t off[kActs], tot;
    layout_of<kActs>(kActC, kActLvl, n, H, W, off, &tot);
    char* a = static_cast<char*>(acts);
    if (precision == MCDI_DENOISE_E4M3) {
        const Fp8Region r = fp8_region(tot, kFwdIn, n, H, W);
        u.fp8 = true;
        u.q = reinterpret_cast<uint8_t*>(a + r.q);
        u.amax = reinterpret_cast<float*>(a + r.amax);
        CHECK(cudaMemsetAsync(u.amax, 0, kAmaxSlots * sizeof(float), s));
    }
    auto A = [&](int k) { return reinterpret_cast<bf16*>(a + off[k]); };
    const long long HW = (long long)H * W;
    launch_k(pack_input_kernel, blocks_for(n * HW, 256), 256, 0, s, reinterpret_cast<const float4*>(term),
             reinterpret_cast<const float4*>(kd), reinterpret_cast<const float4*>(nrm), n, n_aux, (int)HW, A(X0),
             u.out(X0));
    CHECK(cudaGetLastError());
    auto pool = [&](const bf16* src, int Ctot, int coff, int C, int level, int dst_slot) {
        const int Hl = H >> level, Wl = W >> level;
        const long long work = (long long)n * (Hl / 2) * (Wl / 2) * (C / 8);
        launch_k(maxpool2_kernel, blocks_for(work, 256), 256, 0, s, src, Ctot, coff, C, n, Hl, Wl, A(dst_slot),
                 u.out(dst_slot));
        return cudaGetLastError();
    };
    // level 0
    CHECK(run_conv(u, 0, A(X0), X0, 16, Wsel{0, false}, b_of(u, 0), 32, 32, kStore, 1, A(A1), A1, 32, 0, nullptr,
                   nullptr, 0, 0, s, why));
    bool pooled = false;
    CHECK(run_conv(u, 0, A(A1), A1, 32, Wsel{1, false}, b_of(u, 1), 32, 32, kStore, 1, A(CAT1), CAT1, 80, 48, nullptr,
                   nullptr, 0, 0, s, why, PoolTo{A(P1), 32, P1, &pooled}));
    if (!pooled) CHECK(pool(A(CAT1), 80, 48, 32, 0, P1));
    // level 1
    CHECK(run_conv(u, 1, A(P1), P1, 32, Wsel{2, false}, b_of(u, 2), 48, 48, kStore, 1, A(A2), A2, 48, 0, nullptr,
                   nullptr, 0, 0, s, why));
    pooled = false;
    CHECK(run_conv(u, 1, A(A2), A2, 48, Wsel{3, false}, b_of(u, 3), 48, 48, kStore, 1, A(CAT2), CAT2, 112, 64,
                   nullptr, nullptr, 0, 0, s, why, PoolTo{A(P2), 48, P2, &pooled}));
    if (!pooled) CHECK(pool(A(CAT2), 112, 64, 48, 1, P2));
    // level 2
    CHECK(run_conv(u, 2, A(P2), P2, 48, Wsel{4, false}, b_of(u, 4), 64, 64, kStore, 1, A(A3), A3, 64, 0, nullptr,
                   nullptr, 0, 0, s, why));
    pooled = false;
    CHECK(run_conv(u, 2, A(A3), A3, 64, Wsel{5, false}, b_of(u, 5), 64, 64, kStore, 1, A(CAT3), CAT3, 160, 96,
                   nullptr, nullptr, 0, 0, s, why, PoolTo{A(P3), 64, P3, &pooled}));
    if (!pooled) CHECK(pool(A(CAT3), 160, 96, 64, 2, P3));
    // bottleneck (level 3): second conv stores its 2x upsample into the level-2 concatenation
    CHECK(run_conv(u, 3, A(P3), P3, 64, Wsel{6, false}, b_of(u, 6), 96, 96, kStore, 1, A(B1), B1, 96, 0, nullptr,
                   nullptr, 0, 0, s, why));
    CHECK(run_conv(u, 3, A(B1), B1, 96, Wsel{7, false}, b_of(u, 7), 96, 96, kStoreUp2, 1, A(CAT3), CAT3, 160, 0,
                   nullptr, nullptr, 0, 0, s, why));
    // decoder
    CHECK(run_conv(u, 2, A(CAT3), CAT3, 160, Wsel{8, false}, b_of(u, 8), 64, 64, kStore, 1, A(D3A), D3A, 64, 0,
                   nullptr, nullptr, 0, 0, s, why));
    CHECK(run_conv(u, 2, A(D3A), D3A, 64, Wsel{9, false}, b_of(u, 9), 64, 64, kStoreUp2, 1, A(CAT2), CAT2, 112, 0,
                   nullptr, nullptr, 0, 0, s, why));
    CHECK(run_conv(u, 1, A(CAT2), CAT2, 112, Wsel{10, false}, b_of(u, 10), 48, 48, kStore, 1, A(D2A), D2A, 48, 0,
                   nullptr, nullptr, 0, 0, s, why));
    CHECK(run_conv(u, 1, A(D2A), D2A, 48, Wsel{11, false}, b_of(u, 11), 48, 48, kStoreUp2, 1, A(CAT1), CAT1, 80, 0,
                   nullptr, nullptr, 0, 0, s, why));
    CHECK(run_conv(u, 0, A(CAT1), CAT1, 80, Wsel{12, false}, b_of(u, 12), 32, 32, kStore, 1, A(D1A), D1A, 32, 0,
                   nullptr, nullptr, 0, 0, s, why));
    CHECK(run_conv(u, 0, A(D1A), D1A, 32, Wsel{13, false}, b_of(u, 13), 32, 32, kStore, 1, A(D1B), D1B, 32, 0,
                   nullptr, nullptr, 0, 0, s, why));
    CHECK(run_conv(u, 0, A(D1B), D1B, 32, Wsel{14, false}, b_of(u, 14), 16, 3, kStoreF32, 0, nullptr, -1, 0, 0,
                   reinterpret_cast<float4*>(y), nullptr, 0, 0, s, why));
    return cudaSuccess;
}

cudaError_t launch_unet_bwd(const void* weights, int precision, int n, int H, int W, const void* acts,
                            const float* gy, float* gx_term, void* grad_ws, unsigned* err, cudaStream_t s,
                            const char** why) {
    Unet u{static_cast<const char*>(weights), unet_weight_layout(), n, H, W, err};
    size_t aoff[kActs], goff[kGrads], t;
    layout_of<kActs>(kActC, kActLvl, n, H, W, aoff, &t);
    layout_of<kGrads>(kGradC, kGradLvl, n, H, W, goff, &t);
    const char* a = static_cast<const char*>(acts);
    char* g = static_cast<char*>(grad_ws);
    if (precision == MCDI_DENOISE_E4M3) {
        const Fp8Region r = fp8_region(t, kBwdIn, n, H, W);
        u.fp8 = true;
        u.q = reinterpret_cast<uint8_t*>(g + r.q);
        u.amax = reinterpret_cast<float*>(g + r.amax);
        CHECK(cudaMemsetAsync(u.amax, 0, kAmaxSlots * sizeof(float), s));
    }
    auto A = [&](int k) { return reinterpret_cast<const bf16*>(a + aoff[k]); };
    auto G = [&](int k) { return reinterpret_cast<bf16*>(g + goff[k]); };
    const long long P0 = (long long)n * H * W;
    launch_k(pack_grad_kernel, blocks_for(P0, 256), 256, 0, s, reinterpret_cast<const float4*>(gy), n, H * W, G(GY),
             u.out(GY));
    CHECK(cudaGetLastError());
    auto up_bwd = [&](const bf16* gcat, const bf16* cat, int Ctot, int C, int low_level, int glow) {
        const int Hl = H >> low_level, Wl = W >> low_level;
        const long long work = (long long)n * Hl * Wl * (C / 8);
        launch_k(up2_bwd_kernel, blocks_for(work, 256), 256, 0, s, gcat, cat, Ctot, C, n, Hl, Wl, G(glow), u.out(glow));
        return cudaGetLastError();
    };
    // out (32 -> 3): dgrad through the ReLU of dec1b
    CHECK(run_conv(u, 0, G(GY), GY, 16, Wsel{14, true}, nullptr, 32, 32, kDgradMask, 0, G(GD1B), GD1B, 32, 0, nullptr,
                   A(D1B), 32, 0, s, why));
    CHECK(run_conv(u, 0, G(GD1B), GD1B, 32, Wsel{13, true}, nullptr, 32, 32, kDgradMask, 0, G(GD1A), GD1A, 32, 0,
                   nullptr, A(D1A), 32, 0, s, why));
    CHECK(run_conv(u, 0, G(GD1A), GD1A, 32, Wsel{12, true}, nullptr, 80, 80, kDgradPlain, 0, G(GCAT1), -1, 80, 0,
                   nullptr, nullptr, 0, 0, s, why));
    CHECK(up_bwd(G(GCAT1), A(CAT1), 80, 48, 1, GD2B));
    CHECK(run_conv(u, 1, G(GD2B), GD2B, 48, Wsel{11, true}, nullptr, 48, 48, kDgradMask, 0, G(GD2A), GD2A, 48, 0,
                   nullptr, A(D2A), 48, 0, s, why));
    CHECK(run_conv(u, 1, G(GD2A), GD2A, 48, Wsel{10, true}, nullptr, 112, 112, kDgradPlain, 0, G(GCAT2), -1, 112, 0,
                   nullptr, nullptr, 0, 0, s, why));
    CHECK(up_bwd(G(GCAT2), A(CAT2), 112, 64, 2, GD3B));
    CHECK(run_conv(u, 2, G(GD3B), GD3B, 64, Wsel{9, true}, nullptr, 64, 64, kDgradMask, 0, G(GD3A), GD3A, 64, 0,
                   nullptr, A(D3A), 64, 0, s, why));
    CHECK(run_conv(u, 2, G(GD3A), GD3A, 64, Wsel{8, true}, nullptr, 160, 160, kDgradPlain, 0, G(GCAT3), -1, 160, 0,
                   nullptr, nullptr, 0, 0, s, why));
    CHECK(up_bwd(G(GCAT3), A(CAT3), 160, 96, 3, GB2));
    CHECK(run_conv(u, 3, G(GB2), GB2, 96, Wsel{7, true}, nullptr, 96, 96, kDgradMask, 0, G(GB1), GB1, 96, 0, nullptr,
                   A(B1), 96, 0, s, why));
    // the input gradient of the level-2 pool, routed through the pool into g_E3 by the epilogue
    CHECK(run_conv(u, 3, G(GB1), GB1, 96, Wsel{6, true}, nullptr, 64, 64, kDgradPoolBwd, 0, G(GE3), GE3, 64, 0, nullptr,
                   A(CAT3), 160, 96, s, why, PoolTo{}, G(GCAT3)));
    CHECK(run_conv(u, 2, G(GE3), GE3, 64, Wsel{5, true}, nullptr, 64, 64, kDgradMask, 0, G(GA3), GA3, 64, 0, nullptr,
                   A(A3), 64, 0, s, why));
    CHECK(run_conv(u, 2, G(GA3), GA3, 64, Wsel{4, true}, nullptr, 48, 48, kDgradPoolBwd, 0, G(GE2), GE2, 48, 0, nullptr,
                   A(CAT2), 112, 64, s, why, PoolTo{}, G(GCAT2)));
    CHECK(run_conv(u, 1, G(GE2), GE2, 48, Wsel{3, true}, nullptr, 48, 48, kDgradMask, 0, G(GA2), GA2, 48, 0, nullptr,
                   A(A2), 48, 0, s, why));
    CHECK(run_conv(u, 1, G(GA2), GA2, 48, Wsel{2, true}, nullptr, 32, 32, kDgradPoolBwd, 0, G(GE1), GE1, 32, 0, nullptr,
                   A(CAT1), 80, 48, s, why, PoolTo{}, G(GCAT1)));
    CHECK(run_conv(u, 0, G(GE1), GE1, 32, Wsel{1, true}, nullptr, 32, 32, kDgradMask, 0, G(GA1), GA1, 32, 0, nullptr,
                   A(A1), 32, 0, s, why));
    // the input gradient of the term channels (0..2) straight out of the last convolution's epilogue, as float4
    CHECK(run_conv(u, 0, G(GA1), GA1, 32, Wsel{0, true}, nullptr, 16, 3, kStoreF32, 0, nullptr, -1, 0, 0,
                   reinterpret_cast<float4*>(gx_term), nullptr, 0, 0, s, why));
    return cudaGetLastError();
}

// ---------------------------------------------------------------- weight gradient
// Per convolution, its forward input and the gradient at its pre-activation
// output (ReLU-masked where the layer has one): both are left in place by the
// forward (activations) and the input-gradient backward (gradient buffers).
static const int kWgX[kUnetConvs] = {X0, A1, P1, A2, P2, A3, P3, B1, CAT3, D3A, CAT2, D2A, CAT1, D1A, D1B};
static const int kWgG[kUnetConvs] = {GA1, GE1, GA2, GE2, GA3, GE3, GB1, GB2, GD3A, GD3B, GD2A, GD2B, GD1A, GD1B, GY};

size_t unet_wgrad_bytes(int n, int H, int W) {
    size_t m = 0;
    for (int k = 0; k < kUnetConvs; ++k) {
        const int l = kPlan[k].level;
        m = std::max(m, wgrad_scratch_bytes(kActC[kWgX[k]], kGradC[kWgG[k]], n, H >> l, W >> l));
    }
    return m;
}

cudaError_t launch_unet_wgrad(const void* acts, const void* grad_ws, int n, int H, int W, float* gw, void* scratch,
                              unsigned* err, cudaStream_t s, const char** why) {
    size_t aoff[kActs], goff[kGrads], t;
    layout_of<kActs>(kActC, kActLvl, n, H, W, aoff, &t);
    layout_of<kGrads>(kGradC, kGradLvl, n, H, W, goff, &t);
    size_t o = 0;  // parameter order: W[co][ci][3][3], then b[co], per convolution
    for (int k = 0; k < kUnetConvs; ++k) {
        const int l = kPlan[k].level;
        const cudaError_t e =
            launch_wgrad(static_cast<const char*>(acts) + aoff[kWgX[k]], kActC[kWgX[k]],
                         static_cast<const char*>(grad_ws) + goff[kWgG[k]], kGradC[kWgG[k]], n, H >> l, W >> l,
                         kPlan[k].ci, kPlan[k].co, scratch, gw + o, err, s, why);
        if (e != cudaSuccess) return e;
        o += (size_t)kPlan[k].co * kPlan[k].ci * 9 + kPlan[k].co;
    }
    return cudaGetLastError();
}

cudaError_t launch_conv3x3(const void* x, int n, int H, int W, int cin_pad, const void* w, const float* bias,
                           int cout_pad, int relu, void* y, unsigned* err, cudaStream_t s, const char** why) {
    ConvDesc d = conv_desc(n, H, W, cin_pad, 2 * cin_pad, bias, cout_pad, cout_pad, kStore, relu, static_cast<bf16*>(y),
                           cout_pad, 0, nullptr, nullptr, 0, 0, err);
    if (!conv_make_desc(&d, x, w, why)) return cudaErrorInvalidValue;
    return conv_launch(d, s);
}

cudaError_t launch_conv3x3_e4m3(const void* x, int n, int H, int W, int cin_pad, const void* w, const float* x_amax,
                                const float* w_amax, const float* bias, int cout_pad, int relu, void* y, unsigned* err,
                                cudaStream_t s, const char** why) {
    ConvDesc d = conv_desc(n, H, W, cin_pad, cin_pad, bias, cout_pad, cout_pad, kStore, relu, static_cast<bf16*>(y),
                           cout_pad, 0, nullptr, nullptr, 0, 0, err);
    d.p.fp8 = 1;
    d.p.x_amax = x_amax;
    d.p.w_amax = w_amax;
    if (!conv_make_desc(&d, x, w, why)) return cudaErrorInvalidValue;
    return conv_launch(d, s);
}

}  // namespace mcdi
