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
// 32 -> 32 channel 3x3 convolution with ReLU on the tensor cores (BF16 operands,
// FP32 accumulation): in (B x 32 x H x H), out (B x 32 x Ho x Ho), stride S;
// theta: the layer's W then b; wpack: device scratch of cnn_conv32_tc_words()
// words for the packed weights.
reg_status cnn_conv32_tc(const float *in, int H, const float *theta, float *out, int B, int S, cudaStream_t st,
                         uint32_t *wpack);
int cnn_conv32_tc_words();
// Data gradient of a stride-1 32 -> 32 layer on the tensor cores: gx (B x 32 x
// H x H) = mask(> 0) * conv(gz, W flipped and transposed), gz the gradient with
// respect to the layer's pre-activation output.
reg_status cnn_dgrad32_tc(const float *gz, int H, const float *theta, const float *mask, float *gx, int B,
                          cudaStream_t st, uint32_t *wpack);
// Weight and bias gradient of a 32 -> 32 layer of stride S on the tensor cores
// into grad (the layer's W then b); part: device scratch of
// (cnn_wgrad32_tc_blocks() + 1) x 32 x 288 floats.
reg_status cnn_wgrad32_tc(const float *in, int H, const float *gz, int B, int S, float *grad, float *part,
                          cudaStream_t st);
int cnn_wgrad32_tc_blocks();
// Record an error message for reg_last_error().
reg_status reg_internal_fail(reg_status st, const char *msg);
