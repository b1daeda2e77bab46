// 3x3 convolution as an implicit GEMM on the 5th-generation tensor cores
// (tcgen05, sm_103a): the denoiser's building block (Sec. 4.2 neural denoiser,
// App. B).  Activations are BF16 in 8-channel planes, [img][C / 8][H][W][8],
// with C padded to a multiple of 16.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pdl.cuh"

namespace mcdi {

enum ConvEpilogue : int {
    kStore = 0,       // out = bf16(act(acc + bias)) into a channel slice
    kStoreUp2 = 1,    // same value written to the 2x2 block of a 2x larger output
    kStoreF32 = 2,    // out float4 = (acc + bias) channels 0..2, w = 0 (final layer)
    kDgradMask = 3,   // out = bf16(acc * [mask > 0])  (input gradient through a ReLU)
    kDgradPlain = 4,  // out = bf16(acc)
    // input gradient of a 2x2 max-pool's output, routed on: with gp = bf16(acc) and E (`mask`, twice the
    // size) the pooled tensor, out (twice the size) = (skip gradient `gskip` + gp at the window's first
    // maximum) * [E > 0] for the four pixels of the window
    kDgradPoolBwd = 5,
};

struct ConvParams {
    int n_img, H, W;           // spatial size of input and output (up2: output is 2H x 2W)
    int tw, th;                // pixel tile, tw * th = 128
    int tiles_x, tiles_y;
    int cin_pad;               // input channels (multiple of 16 for BF16, of 32 for FP8)
    int cin_bytes;             // bytes of one pixel's input channels (multiple of 32: one MMA K-step)
    int fp8;                   // 1: E4M3 operands (kind::f8f6f4), else BF16 (kind::f16)
    const float* x_amax;       // FP8: device amax of the unquantised input (scale 448 / amax)
    const float* w_amax;       // FP8: device amax of the unquantised weights
    int cout_pad;              // MMA N (multiple of 16, <= 256)
    int cout_valid;            // channels written
    int mode;
    int relu;
    const void* x;             // input activations (the row-tile form copies halo rows directly)
    const float* bias;         // [cout_pad] or null
    __nv_bfloat16* out;        // 8-channel planes, out_ctotal channels
    int out_ctotal, out_coff;
    float4* out_f32;           // [n_img][H][W] (kStoreF32)
    const __nv_bfloat16* mask; // 8-channel planes, same spatial size as the output (kDgradPoolBwd: twice it)
    int mask_ctotal, mask_coff;
    const __nv_bfloat16* gskip; // kDgradPoolBwd: the skip gradient, laid out as `mask`
    unsigned* err;             // device error word (set on a wait timeout)
    unsigned* out_amax;        // nullable: max |stored value| of the output (float bits), for E4M3 consumers
    // nullable (kStore in the row-tile form with an even number of rows per tile, at most 64 channels per
    // CTA): the 2x2 max-pool of the stored channels, into 8-channel planes of pool_ctotal channels at
    // (H / 2, W / 2), output channel c at pool channel c; pool_amax as out_amax for the pooled tensor
    __nv_bfloat16* pool_out;
    int pool_ctotal;
    unsigned* pool_amax;
};

// Launch plan of the row-tile form (tiles of `rows` x 128 pixels, weights of
// `nc` output channels resident per CTA).
struct RowPlan {
    int rows;                // output rows per tile (R)
    int nc;                  // output channels per CTA (MMA N); n_slices * nc = cout_pad
    int n_slices;
    int stages;              // halo ring depth
    int n_tiles;             // tiles per channel slice
    int grid;                // CTAs (a multiple of n_slices)
    uint32_t plane_bytes;    // halo plane stride in shared memory: (R + 2) rows x 130 pixels x 16 bytes, 128-aligned
    uint32_t stage_bytes;    // two planes, 1024-byte aligned
    uint32_t acc_stride;     // TMEM columns between the accumulators of two rows
    uint32_t tmem_cols;      // TMEM columns allocated (two buffers of R accumulators)
    uint32_t smem_bytes;     // dynamic shared memory
};

// Host helpers (tc_conv.cu).
struct ConvDesc {
    CUtensorMap tmap_x;
    CUtensorMap tmap_w;
    CUtensorMap tmap_wh;  // row-tile form: one 16-channel chunk of all 9 taps' weights, [tap][nc][16]
    bool rows_form;
    RowPlan rp;
    ConvParams p;
};

// Encodes the tensor maps of an input (n_img, H, W; planes of 16-byte pixel
// rows, cin_bytes per pixel) and a K-major weight matrix
// [cout_pad][9 * cin_bytes bytes]; for 128-pixel-wide row
// tiles whose weights fit in shared memory it also plans the row-tile form and
// encodes its maps.  Returns false (with a message) when the driver rejects a
// map.
bool conv_make_desc(ConvDesc* d, const void* x, const void* w, const char** why);

// Runs the persistent row-tile kernel when planned, else one CTA per tile.
cudaError_t conv_launch(const ConvDesc& d, cudaStream_t stream);

// Whether conv_launch runs the row-tile variant that prefetches the ReLU-mask
// words of the next row (masked input gradients whose mask words fit its registers).
bool conv_mask_prefetch(const ConvDesc& d);

// Tensor map over BF16 8-channel planes [plane][H][W][16 B] (n_planes =
// images x planes), rank 3 with 8-byte elements: coordinates (2 x, y, plane).
// A box of box_planes x box_rows x box_px pixels (box_px <= 128) lands in
// shared memory as [plane][row][px][16 B]; loads outside the tensor read
// zeros.
bool encode_plane_rows_map(CUtensorMap* map, const void* base, int W, int H, long long n_planes, int box_px,
                           int box_rows, int box_planes, const char** why);
int conv_pick_tile_w(int W);

}  // namespace mcdi
