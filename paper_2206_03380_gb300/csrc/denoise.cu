// The differentiable denoiser (Sec. 4.2 "Neural denoisers", App. B): a U-Net
// of 3x3 convolutions applied to the demodulated diffuse term c_d and the
// specular term c_s, each with the k_d and normal planes as guides.  Forward
// and input-gradient backward (the paper's main results lock the denoiser
// weights, so no weight gradient is formed; Sec. 4.2's gradient-sharing
// identity dL/dX = dL/dO conv F^T is what the backward convolutions compute).
//
// Layout: NHWC BF16 activations, channels padded to multiples of 16.  Skip
// connections are never copied: the encoder's second convolution of a level
// stores straight into the channel slice of that level's concatenation buffer,
// and the decoder's second convolution stores its 2x nearest-upsampled output
// into the other slice one level up ([upsampled | skip], as in the reading of
// the network).  Max-pooling and the small backward routing steps are
// memory-bound kernels of their own.
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
    }
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
enum Grad { GY, GD1B, GD1A, GCAT1, GD2B, GD2A, GCAT2, GD3B, GD3A, GCAT3, GB2, GB1, GP3, GE3, GA3, GP2, GE2, GA2,
            GP1, GE1, GA1, GX0, kGrads };
static const int kGradC[kGrads] = {16, 32, 32, 80, 48, 48, 112, 64, 64, 160, 96, 96, 64, 64, 64, 48, 48, 48,
                                   32, 32, 32, 16};
static const int kGradLvl[kGrads] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0};

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

size_t unet_act_bytes(int n, int H, int W) {
    size_t off[kActs], t;
    layout_of<kActs>(kActC, kActLvl, n, H, W, off, &t);
    return t;
}

size_t unet_grad_bytes(int n, int H, int W) {
    size_t off[kGrads], t;
    layout_of<kGrads>(kGradC, kGradLvl, n, H, W, off, &t);
    return t;
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

// network input: [term.rgb, k_d.rgb, normal.xyz, 0 x 7] per pixel (16
// channels, two planes); image i uses guide planes of image i % n_aux
__global__ void pack_input_kernel(const float4* __restrict__ term, const float4* __restrict__ kd,
                                  const float4* __restrict__ nrm, int n_img, int n_aux, int HW, bf16* __restrict__ x) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n_img * HW) return;
    const int img = (int)(i / HW), p = (int)(i - (long long)img * HW);
    const long long g = (long long)(img % n_aux) * HW + p;
    const float4 t = term[i], k = kd[g], n = nrm[g];
    const float f0[8] = {t.x, t.y, t.z, k.x, k.y, k.z, n.x, n.y}, f1[8] = {n.z, 0, 0, 0, 0, 0, 0, 0};
    st8(x + (((size_t)img * 2 + 0) * HW + p) * 8, f0);
    st8(x + (((size_t)img * 2 + 1) * HW + p) * 8, f1);
}

// upstream gradient (rgb of float4) -> 16-channel BF16 (channels 3..15 zero)
__global__ void pack_grad_kernel(const float4* __restrict__ gy, int n_img, int HW, bf16* __restrict__ g) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n_img * HW) return;
    const int img = (int)(i / HW), p = (int)(i - (long long)img * HW);
    const float4 v = gy[i];
    const float f0[8] = {v.x, v.y, v.z, 0, 0, 0, 0, 0}, f1[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    st8(g + (((size_t)img * 2 + 0) * HW + p) * 8, f0);
    st8(g + (((size_t)img * 2 + 1) * HW + p) * 8, f1);
}

// input gradient of the network (channels 0..2 = the term) -> float4
__global__ void unpack_grad_kernel(const bf16* __restrict__ g, int n_img, int HW, float4* __restrict__ gx) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n_img * HW) return;
    const int img = (int)(i / HW), p = (int)(i - (long long)img * HW);
    float f[8];
    ld8(g + ((size_t)img * 2 * HW + p) * 8, f);
    gx[i] = make_float4(f[0], f[1], f[2], 0.0f);
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
                                bf16* __restrict__ dst) {
    const int Ho = H >> 1, Wo = W >> 1;
    int img, g, yo, xo;
    if (!split_index((long long)blockIdx.x * blockDim.x + threadIdx.x, C >> 3, Ho, Wo, &img, &g, &yo, &xo, n)) return;
    float m[8], v[8];
    const bf16* s = src + poff(img, Ctot >> 3, (coff >> 3) + g, H, W, 2 * yo, 2 * xo);
    for (int k = 0; k < 4; ++k) {
        ld8(s + ((size_t)(k >> 1) * W + (k & 1)) * 8, v);
#pragma unroll
        for (int c = 0; c < 8; ++c) m[c] = k == 0 ? v[c] : fmaxf(m[c], v[c]);
    }
    st8(dst + poff(img, C >> 3, g, Ho, Wo, yo, xo), m);
}

// gradient through "nearest 2x upsample then ReLU output": g_low = sum of the
// 2x2 block of g_cat[0 : C] times [activation > 0], the activation read from
// the upsampled copy in cat (top-left of the block)
__global__ void up2_bwd_kernel(const bf16* __restrict__ gcat, const bf16* __restrict__ cat, int Ctot, int C, int n,
                               int Hl, int Wl, bf16* __restrict__ glow) {
    int img, g, y, x;
    if (!split_index((long long)blockIdx.x * blockDim.x + threadIdx.x, C >> 3, Hl, Wl, &img, &g, &y, &x, n)) return;
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
}

// gradient of an encoder output E (stored in cat at channel offset ecoff) that
// feeds both the skip slice and the 2x2 max-pool: g_E = (g_cat skip slice +
// pool gradient routed to the window's first maximum) * [E > 0]
__global__ void pool_bwd_kernel(const bf16* __restrict__ gcat, const bf16* __restrict__ cat, int Ctot, int ecoff,
                                int C, const bf16* __restrict__ gpool, int n, int H, int W, bf16* __restrict__ gE) {
    int img, g, y, x;
    if (!split_index((long long)blockIdx.x * blockDim.x + threadIdx.x, C >> 3, H, W, &img, &g, &y, &x, n)) return;
    const int xo = x >> 1, yo = y >> 1, me = (x & 1) + 2 * (y & 1);
    const int G = Ctot >> 3, ge = (ecoff >> 3) + g;
    const size_t w0 = poff(img, G, ge, H, W, 2 * yo, 2 * xo);
    float win[4][8];
    for (int k = 0; k < 4; ++k) ld8(cat + w0 + ((size_t)(k >> 1) * W + (k & 1)) * 8, win[k]);
    float gs[8], gp[8];
    ld8(gcat + poff(img, G, ge, H, W, y, x), gs);
    ld8(gpool + poff(img, C >> 3, g, H >> 1, W >> 1, yo, xo), gp);
    float out[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        int arg = 0;
        for (int k = 1; k < 4; ++k)
            if (win[k][c] > win[arg][c]) arg = k;
        const float v = gs[c] + (arg == me ? gp[c] : 0.0f);
        out[c] = win[me][c] > 0.0f ? v : 0.0f;
    }
    st8(gE + poff(img, C >> 3, g, H, W, y, x), out);
}

// fp32 [co][ci][3][3] + [co] (the plan's parameters, concatenated) -> packed
// BF16 K-major forward weights [co_pad][tap][ci_pad], flipped transposed
// weights for the input gradient [ci_pad][tap'][co_pad] with tap' = 8 - tap,
// and zero-padded FP32 biases
__global__ void pack_weights_kernel(const float* __restrict__ W, const float* __restrict__ b, int ci, int co,
                                    bf16* __restrict__ wk, bf16* __restrict__ wf, float* __restrict__ bias) {
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

}  // namespace

// ---------------------------------------------------------------- orchestration
struct Unet {
    const char* wbase;
    UnetWeightLayout L;
    int n, H, W;
    unsigned* err;
};

static const bf16* wk_of(const Unet& u, int i) { return reinterpret_cast<const bf16*>(u.wbase + u.L.wk[i]); }
static const bf16* wf_of(const Unet& u, int i) { return reinterpret_cast<const bf16*>(u.wbase + u.L.wf[i]); }
static const float* b_of(const Unet& u, int i) { return reinterpret_cast<const float*>(u.wbase + u.L.bias[i]); }

static cudaError_t run_conv(const Unet& u, int level, const bf16* x, int cin_pad, const bf16* w, const float* bias,
                            int cout_pad, int cout_valid, int mode, int relu, bf16* out, int out_ctotal, int out_coff,
                            float4* out_f32, const bf16* mask, int mask_ctotal, int mask_coff, cudaStream_t s,
                            const char** why) {
    ConvDesc d{};
    ConvParams& p = d.p;
    p.n_img = u.n;
    p.H = u.H >> level;
    p.W = u.W >> level;
    p.tw = conv_pick_tile_w(p.W);
    p.th = 128 / p.tw;
    p.tiles_x = (p.W + p.tw - 1) / p.tw;
    p.tiles_y = (p.H + p.th - 1) / p.th;
    p.cin_pad = cin_pad;
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
    p.err = u.err;
    if (!conv_make_desc(&d, x, w, why)) return cudaErrorInvalidValue;
    return conv_launch(d, s);
}

static int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

#define CHECK(e)                          \
    do {                                  \
        cudaError_t _e = (e);             \
        if (_e != cudaSuccess) return _e; \
    } while (0)

cudaError_t launch_unet_pack_weights(const float* params, void* weights, cudaStream_t s) {
    const UnetWeightLayout L = unet_weight_layout();
    char* base = static_cast<char*>(weights);
    size_t off = 0;
    for (int i = 0; i < kUnetConvs; ++i) {
        const int ci = kPlan[i].ci, co = kPlan[i].co;
        const long long n = (long long)pad16(co) * 9 * pad16(ci);
        pack_weights_kernel<<<blocks_for(n, 256), 256, 0, s>>>(
            params + off, params + off + (size_t)co * ci * 9, ci, co, reinterpret_cast<bf16*>(base + L.wk[i]),
            reinterpret_cast<bf16*>(base + L.wf[i]), reinterpret_cast<float*>(base + L.bias[i]));
        off += (size_t)co * ci * 9 + co;
    }
    return cudaGetLastError();
}

cudaError_t launch_unet_fwd(const void* weights, int n, int H, int W, const float* term, const float* kd,
                            const float* nrm, int n_aux, float* y, void* acts, unsigned* err, cudaStream_t s,
                            const char** why) {
    Unet u{static_cast<const char*>(weights), unet_weight_layout(), n, H, W, err};
    size_t off[kActs], tot;
    layout_of<kActs>(kActC, kActLvl, n, H, W, off, &tot);
    char* a = static_cast<char*>(acts);
    auto A = [&](int k) { return reinterpret_cast<bf16*>(a + off[k]); };
    const long long HW = (long long)H * W;
    pack_input_kernel<<<blocks_for(n * HW, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(term),
                                                               reinterpret_cast<const float4*>(kd),
                                                               reinterpret_cast<const float4*>(nrm), n, n_aux,
                                                               (int)HW, A(X0));
    CHECK(cudaGetLastError());
    auto pool = [&](const bf16* src, int Ctot, int coff, int C, int level, bf16* dst) {
        const int Hl = H >> level, Wl = W >> level;
        const long long work = (long long)n * (Hl / 2) * (Wl / 2) * (C / 8);
        maxpool2_kernel<<<blocks_for(work, 256), 256, 0, s>>>(src, Ctot, coff, C, n, Hl, Wl, dst);
        return cudaGetLastError();
    };
    // level 0
    CHECK(run_conv(u, 0, A(X0), 16, wk_of(u, 0), b_of(u, 0), 32, 32, kStore, 1, A(A1), 32, 0, nullptr, nullptr, 0, 0,
                   s, why));
    CHECK(run_conv(u, 0, A(A1), 32, wk_of(u, 1), b_of(u, 1), 32, 32, kStore, 1, A(CAT1), 80, 48, nullptr, nullptr, 0,
                   0, s, why));
    CHECK(pool(A(CAT1), 80, 48, 32, 0, A(P1)));
    // level 1
    CHECK(run_conv(u, 1, A(P1), 32, wk_of(u, 2), b_of(u, 2), 48, 48, kStore, 1, A(A2), 48, 0, nullptr, nullptr, 0, 0,
                   s, why));
    CHECK(run_conv(u, 1, A(A2), 48, wk_of(u, 3), b_of(u, 3), 48, 48, kStore, 1, A(CAT2), 112, 64, nullptr, nullptr, 0,
                   0, s, why));
    CHECK(pool(A(CAT2), 112, 64, 48, 1, A(P2)));
    // level 2
    CHECK(run_conv(u, 2, A(P2), 48, wk_of(u, 4), b_of(u, 4), 64, 64, kStore, 1, A(A3), 64, 0, nullptr, nullptr, 0, 0,
                   s, why));
    CHECK(run_conv(u, 2, A(A3), 64, wk_of(u, 5), b_of(u, 5), 64, 64, kStore, 1, A(CAT3), 160, 96, nullptr, nullptr, 0,
                   0, s, why));
    CHECK(pool(A(CAT3), 160, 96, 64, 2, A(P3)));
    // bottleneck (level 3): second conv stores its 2x upsample into the level-2 concatenation
    CHECK(run_conv(u, 3, A(P3), 64, wk_of(u, 6), b_of(u, 6), 96, 96, kStore, 1, A(B1), 96, 0, nullptr, nullptr, 0, 0,
                   s, why));
    CHECK(run_conv(u, 3, A(B1), 96, wk_of(u, 7), b_of(u, 7), 96, 96, kStoreUp2, 1, A(CAT3), 160, 0, nullptr, nullptr,
                   0, 0, s, why));
    // decoder
    CHECK(run_conv(u, 2, A(CAT3), 160, wk_of(u, 8), b_of(u, 8), 64, 64, kStore, 1, A(D3A), 64, 0, nullptr, nullptr,
                   0, 0, s, why));
    CHECK(run_conv(u, 2, A(D3A), 64, wk_of(u, 9), b_of(u, 9), 64, 64, kStoreUp2, 1, A(CAT2), 112, 0, nullptr,
                   nullptr, 0, 0, s, why));
    CHECK(run_conv(u, 1, A(CAT2), 112, wk_of(u, 10), b_of(u, 10), 48, 48, kStore, 1, A(D2A), 48, 0, nullptr, nullptr,
                   0, 0, s, why));
    CHECK(run_conv(u, 1, A(D2A), 48, wk_of(u, 11), b_of(u, 11), 48, 48, kStoreUp2, 1, A(CAT1), 80, 0, nullptr,
                   nullptr, 0, 0, s, why));
    CHECK(run_conv(u, 0, A(CAT1), 80, wk_of(u, 12), b_of(u, 12), 32, 32, kStore, 1, A(D1A), 32, 0, nullptr, nullptr,
                   0, 0, s, why));
    CHECK(run_conv(u, 0, A(D1A), 32, wk_of(u, 13), b_of(u, 13), 32, 32, kStore, 1, A(D1B), 32, 0, nullptr, nullptr,
                   0, 0, s, why));
    CHECK(run_conv(u, 0, A(D1B), 32, wk_of(u, 14), b_of(u, 14), 16, 3, kStoreF32, 0, nullptr, 0, 0,
                   reinterpret_cast<float4*>(y), nullptr, 0, 0, s, why));
    return cudaSuccess;
}

cudaError_t launch_unet_bwd(const void* weights, int n, int H, int W, const void* acts, const float* gy,
                            float* gx_term, void* grad_ws, unsigned* err, cudaStream_t s, const char** why) {
    Unet u{static_cast<const char*>(weights), unet_weight_layout(), n, H, W, err};
    size_t aoff[kActs], goff[kGrads], t;
    layout_of<kActs>(kActC, kActLvl, n, H, W, aoff, &t);
    layout_of<kGrads>(kGradC, kGradLvl, n, H, W, goff, &t);
    const char* a = static_cast<const char*>(acts);
    char* g = static_cast<char*>(grad_ws);
    auto A = [&](int k) { return reinterpret_cast<const bf16*>(a + aoff[k]); };
    auto G = [&](int k) { return reinterpret_cast<bf16*>(g + goff[k]); };
    const long long P0 = (long long)n * H * W;
    pack_grad_kernel<<<blocks_for(P0, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(gy), n, H * W, G(GY));
    CHECK(cudaGetLastError());
    auto up_bwd = [&](const bf16* gcat, const bf16* cat, int Ctot, int C, int low_level, bf16* glow) {
        const int Hl = H >> low_level, Wl = W >> low_level;
        const long long work = (long long)n * Hl * Wl * (C / 8);
        up2_bwd_kernel<<<blocks_for(work, 256), 256, 0, s>>>(gcat, cat, Ctot, C, n, Hl, Wl, glow);
        return cudaGetLastError();
    };
    auto pool_bwd = [&](const bf16* gcat, const bf16* cat, int Ctot, int ecoff, int C, const bf16* gpool, int level,
                        bf16* gE) {
        const int Hl = H >> level, Wl = W >> level;
        const long long work = (long long)n * Hl * Wl * (C / 8);
        pool_bwd_kernel<<<blocks_for(work, 256), 256, 0, s>>>(gcat, cat, Ctot, ecoff, C, gpool, n, Hl, Wl, gE);
        return cudaGetLastError();
    };
    // out (32 -> 3): dgrad through the ReLU of dec1b
    CHECK(run_conv(u, 0, G(GY), 16, wf_of(u, 14), nullptr, 32, 32, kDgradMask, 0, G(GD1B), 32, 0, nullptr, A(D1B), 32,
                   0, s, why));
    CHECK(run_conv(u, 0, G(GD1B), 32, wf_of(u, 13), nullptr, 32, 32, kDgradMask, 0, G(GD1A), 32, 0, nullptr, A(D1A),
                   32, 0, s, why));
    CHECK(run_conv(u, 0, G(GD1A), 32, wf_of(u, 12), nullptr, 80, 80, kDgradPlain, 0, G(GCAT1), 80, 0, nullptr,
                   nullptr, 0, 0, s, why));
    CHECK(up_bwd(G(GCAT1), A(CAT1), 80, 48, 1, G(GD2B)));
    CHECK(run_conv(u, 1, G(GD2B), 48, wf_of(u, 11), nullptr, 48, 48, kDgradMask, 0, G(GD2A), 48, 0, nullptr, A(D2A),
                   48, 0, s, why));
    CHECK(run_conv(u, 1, G(GD2A), 48, wf_of(u, 10), nullptr, 112, 112, kDgradPlain, 0, G(GCAT2), 112, 0, nullptr,
                   nullptr, 0, 0, s, why));
    CHECK(up_bwd(G(GCAT2), A(CAT2), 112, 64, 2, G(GD3B)));
    CHECK(run_conv(u, 2, G(GD3B), 64, wf_of(u, 9), nullptr, 64, 64, kDgradMask, 0, G(GD3A), 64, 0, nullptr, A(D3A),
                   64, 0, s, why));
    CHECK(run_conv(u, 2, G(GD3A), 64, wf_of(u, 8), nullptr, 160, 160, kDgradPlain, 0, G(GCAT3), 160, 0, nullptr,
                   nullptr, 0, 0, s, why));
    CHECK(up_bwd(G(GCAT3), A(CAT3), 160, 96, 3, G(GB2)));
    CHECK(run_conv(u, 3, G(GB2), 96, wf_of(u, 7), nullptr, 96, 96, kDgradMask, 0, G(GB1), 96, 0, nullptr, A(B1), 96,
                   0, s, why));
    CHECK(run_conv(u, 3, G(GB1), 96, wf_of(u, 6), nullptr, 64, 64, kDgradPlain, 0, G(GP3), 64, 0, nullptr, nullptr, 0,
                   0, s, why));
    CHECK(pool_bwd(G(GCAT3), A(CAT3), 160, 96, 64, G(GP3), 2, G(GE3)));
    CHECK(run_conv(u, 2, G(GE3), 64, wf_of(u, 5), nullptr, 64, 64, kDgradMask, 0, G(GA3), 64, 0, nullptr, A(A3), 64,
                   0, s, why));
    CHECK(run_conv(u, 2, G(GA3), 64, wf_of(u, 4), nullptr, 48, 48, kDgradPlain, 0, G(GP2), 48, 0, nullptr, nullptr, 0,
                   0, s, why));
    CHECK(pool_bwd(G(GCAT2), A(CAT2), 112, 64, 48, G(GP2), 1, G(GE2)));
    CHECK(run_conv(u, 1, G(GE2), 48, wf_of(u, 3), nullptr, 48, 48, kDgradMask, 0, G(GA2), 48, 0, nullptr, A(A2), 48,
                   0, s, why));
    CHECK(run_conv(u, 1, G(GA2), 48, wf_of(u, 2), nullptr, 32, 32, kDgradPlain, 0, G(GP1), 32, 0, nullptr, nullptr, 0,
                   0, s, why));
    CHECK(pool_bwd(G(GCAT1), A(CAT1), 80, 48, 32, G(GP1), 0, G(GE1)));
    CHECK(run_conv(u, 0, G(GE1), 32, wf_of(u, 1), nullptr, 32, 32, kDgradMask, 0, G(GA1), 32, 0, nullptr, A(A1), 32,
                   0, s, why));
    CHECK(run_conv(u, 0, G(GA1), 32, wf_of(u, 0), nullptr, 16, 16, kDgradPlain, 0, G(GX0), 16, 0, nullptr, nullptr, 0,
                   0, s, why));
    unpack_grad_kernel<<<blocks_for(P0, 256), 256, 0, s>>>(G(GX0), n, H * W, reinterpret_cast<float4*>(gx_term));
    return cudaGetLastError();
}

cudaError_t launch_conv3x3(const void* x, int n, int H, int W, int cin_pad, const void* w, const float* bias,
                           int cout_pad, int relu, void* y, unsigned* err, cudaStream_t s, const char** why) {
    Unet u{nullptr, {}, n, H, W, err};
    return run_conv(u, 0, static_cast<const bf16*>(x), cin_pad, static_cast<const bf16*>(w), bias, cout_pad, cout_pad,
                    kStore, relu, static_cast<bf16*>(y), cout_pad, 0, nullptr, nullptr, 0, 0, s, why);
}

}  // namespace mcdi
