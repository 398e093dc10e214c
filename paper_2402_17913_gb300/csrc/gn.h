// Internal interface of the learned initial-guess network (gn_kernels.cu,
// gn_host.cu).
//
// The network is the bias-free 3-level, 16-channel 3D U-Net of the learned
// warm start: 3x3x3 cross-correlations with zero padding, ReLU, 2x2x2 average
// pooling, copy upsampling and skip additions.  Activations live in HBM as
// BF16 "NDHWC16": [n][z][y][x][16 channels] (32 bytes per voxel, channel
// fastest); layers with fewer channels (the 2-channel input, the 1-channel
// output) are zero-padded to 16.  Weights are kept in FP32 as [27][16][16]
// (tap t = (dz+1)*9 + (dy+1)*3 + (dx+1), input channel, output channel) and
// packed to BF16 tensor-core operands after every update.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>

#include "npmg_internal.cuh"

namespace npmg {
namespace gn {

constexpr int kC = 16;                  // channels of every activation tensor
constexpr int kTaps = 27;
constexpr int kLayers = 9;
constexpr int kWElems = kTaps * kC * kC;  // 6912 FP32 weights per (padded) layer
constexpr int kPackBytes = kTaps * 512;   // one packed BF16 operand set per layer

// Forward / data-gradient convolution tile: M = 16 x 8 voxels per MMA, kTZ
// z-planes per CTA iteration.
constexpr int kTX = 16, kTY = 8, kTZ = 2;
// Weight-gradient tile.
constexpr int kWTX = 16, kWTY = 8, kWTZ = 4;

// Epilogues of the convolution kernel.
enum Epi {
  kEpiF32 = 0,    // out: float [vox][16] = acc
  kEpiRelu = 1,   // out: bf16 [vox][16] = max(acc, 0)
  kEpiLin = 2,    // out: bf16 [vox][16] = acc
  kEpiMask = 3,   // out: bf16 [vox][16] = acc where mask[vox][c] > 0, else 0
  kEpiOut0 = 4,   // out: float [vox] = acc[channel 0] * scale[n]
};

// Kernels launched by this file's launchers (process-wide).
extern std::atomic<int64_t> g_launches;

struct Dims {
  int n, nx, ny, nz;
  size_t vox() const { return (size_t)nx * ny * nz; }
};

// Encodes the 5D tensor map (16 channels, x, y, z, n) of an NDHWC16 BF16
// tensor with a box of 16 channels x bx x by x bz x 1, 32-byte swizzled
// (rows of one voxel; halves exchanged on rows with address bit 7 set).
bool encode_act(CUtensorMap* m, const void* base, const Dims& d, int bx, int by, int bz);

// y = conv(x, W) with the packed operand `wpack` (kPackBytes, 16-byte
// aligned), epilogue `epi`; *err is set when a bounded wait expires.
cudaError_t launch_conv(const void* x, const void* wpack, void* out, int epi, const void* mask, const float* scale,
                        const Dims& d, int* err, cudaStream_t s);
// partials[b][27*16*16] of dW[t][ci][co] = sum_v x[v + o_t][ci] g[v][co];
// returns the number of blocks used (<= max_blocks) in *nblocks.
cudaError_t launch_wgrad(const void* x, const void* g, float* partials, int max_blocks, int* nblocks, const Dims& d,
                         int* err, cudaStream_t s);
// dw[e] (+)= scale * sum_b partials[b][e], e < kWElems; fixed order.
cudaError_t launch_wgrad_reduce(const float* partials, int nblocks, float* dw, float scale, bool accumulate,
                                cudaStream_t s);

// Elementwise kernels on NDHWC16 BF16 tensors (d = the fine level).
cudaError_t launch_pool(const void* fine, void* coarse, const Dims& d, cudaStream_t s);
cudaError_t launch_up_add(const void* coarse, const void* fine, void* out, const Dims& d, cudaStream_t s);
cudaError_t launch_upbwd_mask(const void* gfine, const void* act_coarse, void* out_coarse, const Dims& d,
                              cudaStream_t s);
cudaError_t launch_poolbwd_add_mask(const void* gskip, const void* gcoarse, const void* act, void* out,
                                    const Dims& d, cudaStream_t s);

// Input / output / loss.  A sample n reads field f of sample index
// idx[n] (idx == nullptr: n) at base + idx * sample_stride (floats).
struct Fields {
  const float* b;
  const float* p;
  const float* t;      // target dp (L2 loss only)
  const float* fluid;  // 1 on fluid cells, 0 on solid (residual loss; nullptr = all fluid)
  size_t stride;       // floats between samples
  const int* idx;      // device sample indices or nullptr
};
// rms[s] = rms of b over sample s, rms[n + s] = rms of p (pooled: over all
// samples), 1 for an all-zero field; inv_rms = 1 / rms.  partials: 2 * n *
// 64 floats.
cudaError_t launch_rms(const Fields& f, const Dims& d, bool pooled, float* partials, float* rms, float* inv_rms,
                       cudaStream_t s);
// x0 = (b * inv_rms[s], p * inv_rms[n + s], 0, ...)
cudaError_t launch_pack_input(const Fields& f, const float* inv_rms, void* x0, const Dims& d, cudaStream_t s);
// L2 loss: gy[vox][16] = (y - t * inv_rms) in channel 0, 0 elsewhere;
// *loss = 0.5 * mean of the squares (float64, fixed-order sum).
cudaError_t launch_loss_grad(const float* y, const Fields& f, const float* inv_rms, void* gy, double* partials,
                             double* loss, const Dims& d, cudaStream_t s);
// Residual loss: r = (A_crop y - b * inv_rms) on interior fluid cells (0
// elsewhere), *loss = 0.5 * sum r^2 / (n * vox); gy = A_crop r in channel 0.
cudaError_t launch_residual_loss_grad(const float* y, const Fields& f, const float* inv_rms, float inv_h2, float* r,
                                      void* gy, double* partials, double* loss, const Dims& d, cudaStream_t s);

// Adam update of every padded layer (update == false: pack only) and the
// BF16 operand packing for the forward (wf) and data-gradient (wd) kernels.
struct AdamArgs {
  // betas, 1 - betas (each rounded from float64), eps; c1 = 1 / (1 - b1^t),
  // c2 = 1 / (1 - b2^t)
  float lr, b1, b2, omb1, omb2, eps, c1, c2;
};
cudaError_t launch_adam_pack(float* w, float* m, float* v, const float* grad, bool update, AdamArgs a, void* wf,
                             void* wd, cudaStream_t s);

// Crop extraction: dataset sample (b, p^n = p - dp, dp, fluid) from full
// fields (solid: uint8, nullable).
cudaError_t launch_crop(const float* b, const float* p_next, const float* dp, const uint8_t* solid,
                        const int64_t full[3], const int64_t crop[3], const int64_t origin[3], float* dst,
                        cudaStream_t s);

// Packs one FP32 layer [27][16][16] into the forward and data-gradient
// operands (building-block convolutions).
cudaError_t launch_pack_layer(const float* w, void* wf, void* wd, cudaStream_t s);

}  // namespace gn
}  // namespace npmg
