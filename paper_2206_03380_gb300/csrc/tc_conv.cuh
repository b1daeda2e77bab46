// 3x3 convolution as an implicit GEMM on the 5th-generation tensor cores
// (tcgen05, sm_103a): the denoiser's building block (Sec. 4.2 neural denoiser,
// App. B).  Activations are NHWC BF16 with channels padded to multiples of 16.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mcdi {

enum ConvEpilogue : int {
    kStore = 0,       // out = bf16(act(acc + bias)) into a channel slice
    kStoreUp2 = 1,    // same value written to the 2x2 block of a 2x larger output
    kStoreF32 = 2,    // out float4 = (acc + bias) channels 0..2, w = 0 (final layer)
    kDgradMask = 3,   // out = bf16(acc * [mask > 0])  (input gradient through a ReLU)
    kDgradPlain = 4,  // out = bf16(acc)
};

struct ConvParams {
    int n_img, H, W;           // spatial size of input and output (up2: output is 2H x 2W)
    int tw, th;                // pixel tile, tw * th = 128
    int tiles_x, tiles_y;
    int cin_pad;               // input channels (multiple of 16) = MMA K per tap
    int cout_pad;              // MMA N (multiple of 16, <= 256)
    int cout_valid;            // channels written
    int mode;
    int relu;
    const float* bias;         // [cout_pad] or null
    __nv_bfloat16* out;        // NHWC
    int out_ctotal, out_coff;
    float4* out_f32;           // [n_img][H][W] (kStoreF32)
    const __nv_bfloat16* mask; // NHWC, same spatial size as the output
    int mask_ctotal, mask_coff;
    unsigned* err;             // device error word (set on a wait timeout)
};

// Host helpers (tc_conv.cu).
struct ConvDesc {
    CUtensorMap tmap_x;
    CUtensorMap tmap_w;
    ConvParams p;
};

// Encodes the tensor maps of an NHWC BF16 input (n_img, H, W, cin_pad) and a
// K-major BF16 weight matrix [cout_pad][9 * cin_pad]; returns false (with a
// message) when the driver rejects them.
bool conv_make_desc(ConvDesc* d, const __nv_bfloat16* x, const __nv_bfloat16* w, const char** why);

cudaError_t conv_launch(const ConvDesc& d, cudaStream_t stream);

int conv_pick_tile_w(int W);

}  // namespace mcdi
