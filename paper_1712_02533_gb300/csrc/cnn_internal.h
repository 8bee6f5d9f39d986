// Internal interface between the learned initialiser (cnn.cu) and the series
// engine (engine.cu); not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/reg.h"

struct reg_cnn;
// Forward of B pairs x (device, B x 2 x S x S) into y (device, B x 2 x S/4 x
// S/4) on stream st; tc: the 32-channel layers on the tensor cores.
reg_status cnn_forward(reg_cnn *h, const float *x, int B, float *y, cudaStream_t st, bool tc);
int64_t cnn_output_side(const reg_cnn *h);
int cnn_input_side(const reg_cnn *h);
int cnn_max_batch(const reg_cnn *h);
// The tensor-core layers exchange activations as BF16 in a channel-group
// planar layout, [b][c / 8][y][x][c % 8] (16 bytes per pixel and group of 8
// channels): "planar" below.
//
// Weight and bias gradient of a 32 -> 32 layer of stride S on the tensor cores
// (tcgen05) into grad (the layer's W then b): in the layer's input (planar, B
// x 32 x H x H), gz the output gradient (FP32 NCHW); part: device scratch of
// cnn_wgrad32_umma_part_floats() floats; err: the tcgen05 error word.
reg_status cnn_wgrad32_umma(const uint16_t *in, int H, const float *gz, int B, int S, float *grad, float *part,
                            cudaStream_t st, int *err);
int cnn_wgrad32_umma_part_floats();
// 32 -> 32 channel 3x3 convolution (zero padding 1, stride S = 1 or 2) with
// bias and ReLU on the fifth-generation tensor cores (tcgen05.mma, accumulator
// in TMEM, BF16 operands, FP32 accumulation): in (planar, B x 32 x H x H, read
// by TMA; H even for S = 2), out (B x 32 x Ho x Ho) planar, or FP32 NCHW with
// out_f32; theta: the layer's W then b; wpack: device buffer of
// cnn_conv32_umma_words() words, 16-byte aligned, holding the packed weights
// (pack: pack theta into it first, else it holds them from an earlier call);
// err: a device word set to nonzero when a wait of the kernel ran out (the
// result is then invalid).
reg_status cnn_conv32_umma(const uint16_t *in, int H, const float *theta, void *out, bool out_f32, int B, int S,
                           cudaStream_t st, uint32_t *wpack, bool pack, int *err);
// Data gradient of a stride-1 32 -> 32 layer on the tensor cores: gx (FP32
// NCHW, B x 32 x H x H) = (mask > 0) * conv(gz, W flipped and transposed), gz
// (FP32 NCHW) the gradient with respect to the layer's pre-activation output,
// mask the activation below (planar).
reg_status cnn_dgrad32_umma(const float *gz, int H, const float *theta, const uint16_t *mask, float *gx, int B,
                            cudaStream_t st, uint32_t *wpack, bool pack, int *err);
// Data gradient of a stride-2 32 -> 32 layer on the tensor cores: gz (FP32
// NCHW, B x 32 x Hg x Hg) the gradient with respect to the layer's
// pre-activation output, gx (FP32 NCHW, B x 32 x 2Hg x 2Hg) = (mask > 0) *
// the transposed convolution, mask the activation below (planar, side 2 Hg);
// wpack as cnn_dgrad32_umma's (the same packing).
reg_status cnn_dgrad32s2_umma(const float *gz, int Hg, const float *theta, const uint16_t *mask, float *gx, int B,
                              cudaStream_t st, uint32_t *wpack, bool pack, int *err);
int cnn_conv32_umma_words();
// The last layer (32 -> 2, stride 1, no ReLU) on the same kernel with N = 16
// (output rows 2..15 zero): in planar (B x 32 x H x H), out FP32 NCHW (B x 2 x
// H x H); wpack: cnn_last_umma_words() words.
reg_status cnn_last_umma(const uint16_t *in, int H, const float *theta, float *out, int B, cudaStream_t st,
                         uint32_t *wpack, bool pack, int *err);
int cnn_last_umma_words();
// The first layer (2 -> 32, stride 2, ReLU) on the tensor cores: x FP32 NCHW
// (B x 2 x H x H, H even), rounded to BF16; out planar (B x 32 x H/2 x H/2);
// wpack: cnn_first_umma_words() words.
reg_status cnn_first_umma(const float *x, int H, const float *theta, uint16_t *out, int B, cudaStream_t st,
                          uint32_t *wpack, bool pack, int *err);
int cnn_first_umma_words();
// After the handle's stream has been synchronised: REG_ECUDA if a tcgen05
// kernel reported a wait that ran out since the last check (and clear it).
reg_status cnn_check_device_error(reg_cnn *h);
// Record an error message for reg_last_error().
reg_status reg_internal_fail(reg_status st, const char *msg);
