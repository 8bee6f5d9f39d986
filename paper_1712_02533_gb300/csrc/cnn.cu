// The learned initialiser: a small convolutional network that predicts a coarse
// initial displacement for a frame pair, trained on the GPU on displacements
// that the plain method computes (its forward, backward and update kernels).
//
// Network: input 2 x S x S (reference, template; normalised), six 3x3
// convolutions with zero padding 1 -- 2->32 stride 2, 32->32 stride 2, three
// 32->32 stride 1, 32->2 stride 1 -- with a ReLU after every layer but the
// last; output 2 x S/4 x S/4, the displacement in input pixels at input pixels
// (4i, 4j).  Loss: mean squared difference to a target displacement.
// Parameters: one flat float vector, layer by layer W (O x C x 3 x 3) then b.
//
// Layout: the FP32 path keeps activations NCHW in float, one buffer per layer,
// on the CUDA cores.  The tensor-core path runs with BF16 operands and FP32
// accumulation: the forward of all six layers and the data and weight
// gradients of the four 32 -> 32 layers on tcgen05 with TMEM accumulators;
// the outputs of layers 0..4 are then BF16 in a channel-group planar layout
// [b][c / 8][y][x][c % 8], the operand layout of those kernels.  The remaining
// gradients (the first and last layers' weights, whose few channels make them
// bandwidth work, and the last layer's data) run on the CUDA cores in FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/reg.h"
#include "cnn_internal.h"

namespace {

constexpr int NL = 6;
struct LayerShape {
    int C, O, S;
};
constexpr LayerShape LAYERS[NL] = {{2, 32, 2}, {32, 32, 2}, {32, 32, 1}, {32, 32, 1}, {32, 32, 1}, {32, 2, 1}};

constexpr int64_t layer_params(int k) { return (int64_t)LAYERS[k].O * LAYERS[k].C * 9 + LAYERS[k].O; }
int64_t param_offset(int k)
{
    int64_t o = 0;
    for (int j = 0; j < k; j++) o += layer_params(j);
    return o;
}
int64_t total_params() { return param_offset(NL); }


// ---------------------------------------------------------------------------
// Forward: one thread per output pixel (b, y, x) computes all O channels.
// ---------------------------------------------------------------------------
template <int C, int O, int S, bool RELU>
__global__ void __launch_bounds__(128) k_conv_fwd(const float *__restrict__ in, int H, const float *__restrict__ theta,
                                                  float *__restrict__ out, int Ho, int total)
{
    // weights as [c][tap][o], so that one vector load brings the weights of
    // several output channels for an input value
    __shared__ __align__(16) float w[O * C * 9];
    __shared__ float bias[O];
    for (int i = threadIdx.x; i < O * C * 9; i += blockDim.x) {
        const int o = i / (C * 9), ck = i - o * (C * 9);
        w[ck * O + o] = theta[i];
    }
    for (int i = threadIdx.x; i < O; i += blockDim.x) bias[i] = theta[O * C * 9 + i];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    const int x = p % Ho, y = (p / Ho) % Ho, b = p / (Ho * Ho);
    float acc[O];
#pragma unroll
    for (int o = 0; o < O; o++) acc[o] = bias[o];
    for (int c = 0; c < C; c++) {
        const float *src = in + ((int64_t)b * C + c) * H * H;
        float v[9];
#pragma unroll
        for (int dy = 0; dy < 3; dy++)
#pragma unroll
            for (int dx = 0; dx < 3; dx++) {
                const int iy = S * y + dy - 1, ix = S * x + dx - 1;
                v[dy * 3 + dx] = (iy >= 0 && iy < H && ix >= 0 && ix < H) ? src[iy * H + ix] : 0.f;
            }
        // per output channel the products are added in the order (c, tap)
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const float *wk = w + (c * 9 + k) * O;
            if constexpr (O % 4 == 0) {
#pragma unroll
                for (int q = 0; q < O / 4; q++) {
                    const float4 wv = reinterpret_cast<const float4 *>(wk)[q];
                    acc[4 * q] = fmaf(wv.x, v[k], acc[4 * q]);
                    acc[4 * q + 1] = fmaf(wv.y, v[k], acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(wv.z, v[k], acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(wv.w, v[k], acc[4 * q + 3]);
                }
            } else if constexpr (O == 2) {
                const float2 wv = *reinterpret_cast<const float2 *>(wk);
                acc[0] = fmaf(wv.x, v[k], acc[0]);
                acc[1] = fmaf(wv.y, v[k], acc[1]);
            } else {
#pragma unroll
                for (int o = 0; o < O; o++) acc[o] = fmaf(wk[o], v[k], acc[o]);
            }
        }
    }
#pragma unroll
    for (int o = 0; o < O; o++)
        if (RELU) acc[o] = fmaxf(acc[o], 0.f);
#pragma unroll
    for (int o = 0; o < O; o++) out[(((int64_t)b * O + o) * Ho + y) * Ho + x] = acc[o];
}

// ---------------------------------------------------------------------------
// Backward, data: gx[b, c, iy, ix] = sum over (o, dy, dx) with S oy + dy - 1 = iy
// and S ox + dx - 1 = ix of W[o, c, dy, dx] gz[b, o, oy, ox], times the ReLU
// mask of the layer below (its output a > 0).  One thread per input pixel.
// ---------------------------------------------------------------------------
// MASK_PLANAR: a_below is BF16 in the planar layout of the tensor-core layers
// (C = 32) instead of FP32 NCHW.
template <int C, int O, int S, bool MASK_PLANAR = false>
__global__ void __launch_bounds__(128) k_conv_bwd_data(const float *__restrict__ gz, int Ho,
                                                       const float *__restrict__ theta,
                                                       const void *__restrict__ a_below, float *__restrict__ gx,
                                                       int H, int total)
{
    // weights as [o][tap][c], so that one vector load brings the weights of
    // several input channels for an output gradient value
    __shared__ __align__(16) float w[O * C * 9];
    for (int i = threadIdx.x; i < O * C * 9; i += blockDim.x) {
        const int o = i / (C * 9), r = i - o * (C * 9), c = r / 9, k = r - c * 9;
        w[(o * 9 + k) * C + c] = theta[i];
    }
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    const int ix = p % H, iy = (p / H) % H, b = p / (H * H);
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; c++) acc[c] = 0.f;
#pragma unroll
    for (int dy = 0; dy < 3; dy++) {
        const int ty = iy + 1 - dy;
        if (ty < 0 || ty % S != 0 || ty / S >= Ho) continue;
        const int oy = ty / S;
#pragma unroll
        for (int dx = 0; dx < 3; dx++) {
            const int tx = ix + 1 - dx;
            if (tx < 0 || tx % S != 0 || tx / S >= Ho) continue;
            const int ox = tx / S;
            for (int o = 0; o < O; o++) {
                const float g = gz[(((int64_t)b * O + o) * Ho + oy) * Ho + ox];
                const float *wk = w + (o * 9 + dy * 3 + dx) * C;
                if constexpr (C % 4 == 0) {
#pragma unroll
                    for (int q = 0; q < C / 4; q++) {
                        const float4 wv = reinterpret_cast<const float4 *>(wk)[q];
                        acc[4 * q] = fmaf(wv.x, g, acc[4 * q]);
                        acc[4 * q + 1] = fmaf(wv.y, g, acc[4 * q + 1]);
                        acc[4 * q + 2] = fmaf(wv.z, g, acc[4 * q + 2]);
                        acc[4 * q + 3] = fmaf(wv.w, g, acc[4 * q + 3]);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < C; c++) acc[c] = fmaf(wk[c], g, acc[c]);
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < C; c++) {
        const int64_t i = (((int64_t)b * C + c) * H + iy) * H + ix;
        bool pos;
        if (MASK_PLANAR) {
            const uint16_t v = reinterpret_cast<const uint16_t *>(
                a_below)[(((int64_t)(4 * b + c / 8) * H + iy) * H + ix) * 8 + (c & 7)];
            pos = v != 0 && !(v & 0x8000u);
        } else {
            pos = reinterpret_cast<const float *>(a_below)[i] > 0.f;
        }
        gx[i] = pos ? acc[c] : 0.f;
    }
}

// ---------------------------------------------------------------------------
// Backward, weights: gW[o, c, dy, dx] = sum_{b, y, x} gz[b, o, y, x]
// in_pad[b, c, S y + dy, S x + dx] and gb[o] = sum gz[b, o, ., .].  One block per
// (o, c), a fixed-order reduction (deterministic).
// ---------------------------------------------------------------------------
//
// With split > 1 the pixels are cut into `split` contiguous parts, one block
// each (grid O C split), and each block writes its 10 sums to part; the
// layers with few (o, c) pairs (2 -> 32, 32 -> 2) keep the GPU busy that way,
// and k_bwd_weight_sum adds the parts in order.
template <int C, int O, int S>
__global__ void __launch_bounds__(256) k_conv_bwd_weight(const float *__restrict__ in, int H,
                                                         const float *__restrict__ gz, int Ho, int B,
                                                         float *__restrict__ grad, int split,
                                                         float *__restrict__ part)
{
    const int oc = blockIdx.x / split, sp = blockIdx.x % split;
    const int o = oc / C, c = oc % C;
    float acc[10];
#pragma unroll
    for (int k = 0; k < 10; k++) acc[k] = 0.f;
    const int per = Ho * Ho, total = B * per;
    const int chunk = (total + split - 1) / split, p0 = sp * chunk, p1 = min(total, p0 + chunk);
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const int b = p / per, q = p % per, y = q / Ho, x = q % Ho;
        const float g = gz[((int64_t)b * O + o) * per + q];
        const float *src = in + ((int64_t)b * C + c) * H * H;
#pragma unroll
        for (int dy = 0; dy < 3; dy++)
#pragma unroll
            for (int dx = 0; dx < 3; dx++) {
                const int iy = S * y + dy - 1, ix = S * x + dx - 1;
                float v = 0.f;
                if (iy >= 0 && iy < H && ix >= 0 && ix < H) v = src[iy * H + ix];
                acc[dy * 3 + dx] = fmaf(g, v, acc[dy * 3 + dx]);
            }
        acc[9] += g;
    }
    __shared__ float red[8][10];
#pragma unroll
    for (int k = 0; k < 10; k++) {
        float v = acc[k];
        for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        float t = 0.f;
        for (int w = 0; w < 8; w++) t += red[w][threadIdx.x];
        if (split > 1) {
            part[(int64_t)blockIdx.x * 10 + threadIdx.x] = t;
        } else {
            if (threadIdx.x < 9) grad[(o * C + c) * 9 + threadIdx.x] = t;
            else if (c == 0) grad[O * C * 9 + o] = t;
        }
    }
}

// The parts of k_conv_bwd_weight in order (one thread per (o, c) and sum).
template <int C, int O>
__global__ void k_bwd_weight_sum(const float *__restrict__ part, int split, float *__restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= O * C * 10) return;
    const int oc = i / 10, k = i % 10, o = oc / C, c = oc % C;
    float t = 0.f;
    for (int sp = 0; sp < split; sp++) t += part[((int64_t)oc * split + sp) * 10 + k];
    if (k < 9) grad[(o * C + c) * 9 + k] = t;
    else if (c == 0) grad[O * C * 9 + o] = t;
}

// ---------------------------------------------------------------------------
// Weight gradients of the 2 -> 32 (stride 2) and 32 -> 2 layers.  Their
// arithmetic intensity is a few FLOPs per byte (two input channels, or two
// output channels), so they stay on the CUDA cores in FP32, but each input
// element is read from global memory once: a block stages a tile of the output
// gradient and the input window the tile needs, and its threads form all the
// layer's weight and bias sums from shared memory.  Each block works through a
// fixed sequence of tiles (tile = block + k grid) and writes one partial
// record; k_wgrad_parts_sum adds the records in block order, so the result is
// deterministic for a given grid.
// ---------------------------------------------------------------------------
constexpr int WF_TR = 2, WF_TW = 64, WF_NP = WF_TR * WF_TW;  // first layer: 2 output rows x 64 columns
constexpr int WF_XR = 2 * WF_TR + 1, WF_XC = 2 * WF_TW + 1;  // its input window: 5 x 129
constexpr int WF_GS = WF_NP + 1;                              // row stride of the staged gradient
constexpr int WF_REC = 32 * 2 * 9 + 32;                       // weights (o, c, tap), then biases

// First layer: gW[o][c][dy][dx] = sum gz[b][o][y][x] x[b][c][2 y + dy - 1][2 x + dx - 1],
// gb[o] = sum gz[b][o][y][x]; x FP32 NCHW (B x 2 x H x H), gz FP32 NCHW (B x
// 32 x Ho x Ho).  Thread (og, ps) = (t % 8, t / 8) sums output channels
// 4 og .. 4 og + 3 over the tile pixels ps + 32 k.
__global__ void __launch_bounds__(256, 2) k_wgrad_first(const float *__restrict__ x, int H,
                                                     const float *__restrict__ gz, int Ho, int B,
                                                     float *__restrict__ part)
{
    __shared__ float xs[2][WF_XR][WF_XC];
    __shared__ float gs[32 * WF_GS];  // [o][pixel]
    __shared__ float red[8][8][4 * 19];
    const int t = threadIdx.x, og = t & 7, ps = t >> 3;
    float acc[4][19];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 19; j++) acc[i][j] = 0.f;
    const int tx_n = (Ho + WF_TW - 1) / WF_TW, ty_n = (Ho + WF_TR - 1) / WF_TR, nt = B * tx_n * ty_n;
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const int b = tile / (tx_n * ty_n), r = tile % (tx_n * ty_n);
        const int y0 = (r / tx_n) * WF_TR, x0 = (r % tx_n) * WF_TW;
        __syncthreads();  // the previous tile's reads are done
        // a thread's loads are issued in groups before their stores: the
        // input window (up to 6), then the gradient in two groups of 8
        constexpr int NG = 32 * WF_NP / 256 / 2, NX = (2 * WF_XR * WF_XC + 255) / 256;
        {
            float xv[NX];
#pragma unroll
            for (int k = 0; k < NX; k++) {
                const int i = t + 256 * k, c = i / (WF_XR * WF_XC), rr = (i / WF_XC) % WF_XR, cc = i % WF_XC;
                const int iy = 2 * y0 - 1 + rr, ix = 2 * x0 - 1 + cc;
                xv[k] = (i < 2 * WF_XR * WF_XC && iy >= 0 && iy < H && ix >= 0 && ix < H)
                            ? x[(((int64_t)b * 2 + c) * H + iy) * H + ix] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < NX; k++) {
                const int i = t + 256 * k;
                if (i < 2 * WF_XR * WF_XC) (&xs[0][0][0])[i] = xv[k];
            }
        }
#pragma unroll
        for (int half = 0; half < 2; half++) {
            float gv[NG];
#pragma unroll
            for (int k = 0; k < NG; k++) {
                const int i = t + 256 * (NG * half + k), o = i / WF_NP, p = i % WF_NP;
                const int y = y0 + p / WF_TW, xx = x0 + p % WF_TW;
                gv[k] = (y < Ho && xx < Ho) ? gz[(((int64_t)b * 32 + o) * Ho + y) * Ho + xx] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < NG; k++) {
                const int i = t + 256 * (NG * half + k);
                gs[(i / WF_NP) * WF_GS + i % WF_NP] = gv[k];
            }
        }
        __syncthreads();
#pragma unroll 1
        for (int k = 0; k < WF_NP / 32; k++) {
            const int p = ps + 32 * k, py = p / WF_TW, px = p % WF_TW;
            float gv[4];
#pragma unroll
            for (int i = 0; i < 4; i++) gv[i] = gs[(4 * og + i) * WF_GS + p];
#pragma unroll
            for (int c = 0; c < 2; c++)
#pragma unroll
                for (int dy = 0; dy < 3; dy++)
#pragma unroll
                    for (int dx = 0; dx < 3; dx++) {
                        const float v = xs[c][2 * py + dy][2 * px + dx];
#pragma unroll
                        for (int i = 0; i < 4; i++) acc[i][c * 9 + dy * 3 + dx] = fmaf(gv[i], v, acc[i][c * 9 + dy * 3 + dx]);
                    }
#pragma unroll
            for (int i = 0; i < 4; i++) acc[i][18] += gv[i];
        }
    }
    // the lanes l, l ^ 8, l ^ 16, l ^ 24 of a warp share og; then the 8 warps
    const int lane = t & 31, w = t >> 5;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 19; j++) {
            float v = acc[i][j];
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            if (lane < 8) red[w][lane][i * 19 + j] = v;
        }
    __syncthreads();
    for (int e = t; e < WF_REC; e += 256) {
        // weights (o, c, tap) at (2 o + c) 9 + tap, then the biases
        const int o = e < 576 ? e / 18 : e - 576, j = e < 576 ? e % 18 : 18;
        float sum = 0.f;
        for (int w2 = 0; w2 < 8; w2++) sum += red[w2][o >> 2][(o & 3) * 19 + j];
        part[(int64_t)blockIdx.x * WF_REC + e] = sum;
    }
}

constexpr int WL_TR = 4, WL_TW = 32, WL_NP = WL_TR * WL_TW;  // last layer: 4 output rows x 32 columns
constexpr int WL_AR = WL_TR + 2, WL_AC = WL_TW + 2;          // its input window: 6 x 34
constexpr int WL_CS = WL_AR * WL_AC + 1;                     // channel stride (odd: no bank conflicts)
constexpr int WL_REC = 2 * 32 * 9 + 2;

// Last layer: gW[o][c][dy][dx] = sum gz[b][o][y][x] a[b][c][y + dy - 1][x + dx - 1],
// gb[o] = sum gz[b][o][y][x]; a the planar BF16 input (B x 32 x H x H), gz FP32
// NCHW (B x 2 x H x H).  Thread (c, seg) = (t % 32, t / 32) walks 16 pixels of
// tile row seg / 2 with a sliding 3 x 3 window of channel c.
__global__ void __launch_bounds__(256) k_wgrad_last(const uint4 *__restrict__ a, int H, const float *__restrict__ gz,
                                                    int B, float *__restrict__ part)
{
    __shared__ float as[32 * WL_CS];
    __shared__ float gs[2][WL_NP];
    __shared__ float red[8][32][18];
    __shared__ float redb[8][2];
    const int t = threadIdx.x, c = t & 31, seg = t >> 5, r = seg >> 1, xs0 = (seg & 1) * 16;
    float acc[18], gb0 = 0.f, gb1 = 0.f;
#pragma unroll
    for (int j = 0; j < 18; j++) acc[j] = 0.f;
    const int tx_n = (H + WL_TW - 1) / WL_TW, ty_n = (H + WL_TR - 1) / WL_TR, nt = B * tx_n * ty_n;
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const int b = tile / (tx_n * ty_n), rr0 = tile % (tx_n * ty_n);
        const int y0 = (rr0 / tx_n) * WL_TR, x0 = (rr0 % tx_n) * WL_TW;
        __syncthreads();
        // all of a thread's loads are issued before its stores
        constexpr int NA = (4 * WL_AR * WL_AC + 255) / 256;
        float g[2];
        uint4 qa[NA];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const int i = t + 256 * k, o = i / WL_NP, p = i % WL_NP, y = y0 + p / WL_TW, xx = x0 + p % WL_TW;
            g[k] = (y < H && xx < H) ? gz[(((int64_t)b * 2 + o) * H + y) * H + xx] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < NA; k++) {
            const int i = t + 256 * k, cg = i / (WL_AR * WL_AC), rr = (i / WL_AC) % WL_AR, cc = i % WL_AC;
            const int iy = y0 - 1 + rr, ix = x0 - 1 + cc;
            qa[k] = make_uint4(0u, 0u, 0u, 0u);
            if (i < 4 * WL_AR * WL_AC && iy >= 0 && iy < H && ix >= 0 && ix < H)
                qa[k] = a[((int64_t)(4 * b + cg) * H + iy) * H + ix];
        }
#pragma unroll
        for (int k = 0; k < 2; k++) (&gs[0][0])[t + 256 * k] = g[k];
#pragma unroll
        for (int k = 0; k < NA; k++) {
            const int i = t + 256 * k, cg = i / (WL_AR * WL_AC), rr = (i / WL_AC) % WL_AR, cc = i % WL_AC;
            if (i >= 4 * WL_AR * WL_AC) continue;
            const uint32_t wv[4] = {qa[k].x, qa[k].y, qa[k].z, qa[k].w};
            float *dst = as + (8 * cg) * WL_CS + rr * WL_AC + cc;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                dst[(2 * j) * WL_CS] = __uint_as_float(wv[j] << 16);
                dst[(2 * j + 1) * WL_CS] = __uint_as_float(wv[j] & 0xFFFF0000u);
            }
        }
        __syncthreads();
        const float *ac = as + c * WL_CS + r * WL_AC + xs0;
        float win[3][3];
#pragma unroll
        for (int dy = 0; dy < 3; dy++) {
            win[dy][0] = ac[dy * WL_AC];
            win[dy][1] = ac[dy * WL_AC + 1];
        }
#pragma unroll 4
        for (int px = 0; px < 16; px++) {
#pragma unroll
            for (int dy = 0; dy < 3; dy++) win[dy][2] = ac[dy * WL_AC + px + 2];
            const int p = r * WL_TW + xs0 + px;
            const float g0 = gs[0][p], g1 = gs[1][p];
#pragma unroll
            for (int dy = 0; dy < 3; dy++)
#pragma unroll
                for (int dx = 0; dx < 3; dx++) {
                    acc[dy * 3 + dx] = fmaf(g0, win[dy][dx], acc[dy * 3 + dx]);
                    acc[9 + dy * 3 + dx] = fmaf(g1, win[dy][dx], acc[9 + dy * 3 + dx]);
                }
            gb0 += g0;
            gb1 += g1;
#pragma unroll
            for (int dy = 0; dy < 3; dy++) {
                win[dy][0] = win[dy][1];
                win[dy][1] = win[dy][2];
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 18; j++) red[seg][c][j] = acc[j];
    if (c == 0) {
        redb[seg][0] = gb0;
        redb[seg][1] = gb1;
    }
    __syncthreads();
    for (int e = t; e < WL_REC; e += 256) {
        // weights (o, c, tap) at (32 o + c) 9 + tap, then the biases
        float sum = 0.f;
        if (e < 576) {
            const int o = e / 288, cc = (e % 288) / 9, tap = e % 9;
            for (int w2 = 0; w2 < 8; w2++) sum += red[w2][cc][o * 9 + tap];
        } else {
            for (int w2 = 0; w2 < 8; w2++) sum += redb[w2][e - 576];
        }
        part[(int64_t)blockIdx.x * WL_REC + e] = sum;
    }
}

// grad[e] = sum over blocks of part[block][e], e < rec: one block per entry,
// a fixed-order tree.
__global__ void __launch_bounds__(256) k_wgrad_parts_sum(const float *__restrict__ part, int nblk, int rec,
                                                         float *__restrict__ grad)
{
    __shared__ float red[8];
    const int e = blockIdx.x, t = threadIdx.x;
    float s = 0.f;
    for (int k = t; k < nblk; k += 256) s += part[(int64_t)k * rec + e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((t & 31) == 0) red[t >> 5] = s;
    __syncthreads();
    if (t == 0) {
        float tot = 0.f;
        for (int w = 0; w < 8; w++) tot += red[w];
        grad[e] = tot;
    }
}

// Grid of the two kernels above: two blocks per SM, at most one per tile.
int wgrad_small_grid(int n_tiles)
{
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        nsm = 152;
    return std::max(1, std::min(n_tiles, 2 * nsm));
}

// Mean squared error: per-block partial sums (double), then one block adds them
// in order; gy = 2 (y - t) / N.
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, int64_t n, float *__restrict__ gy,
                      double *__restrict__ partial)
{
    double s = 0.0;
    const float inv = 2.f / (float)n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        s += (double)d * d;
        gy[i] = inv * d;
    }
    __shared__ double red[8];
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += red[w];
        partial[blockIdx.x] = tot;
    }
}

__global__ void __launch_bounds__(256) k_sum_partials(const double *partial, int n, double scale, double *out)
{
    // fixed order: thread t adds entries t, t + 256, ...; then the warps' sums
    // by shuffles and the eight warp totals in order
    __shared__ double red[8];
    const int t = threadIdx.x;
    double s = 0.0;
    for (int i = t; i < n; i += 256) s += partial[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((t & 31) == 0) red[t >> 5] = s;
    __syncthreads();
    if (t == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; w++) tot += red[w];
        *out = tot * scale;
    }
}

// Adam with bias correction (step t >= 1).
__global__ void k_adam(float *__restrict__ theta, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

template <int C, int O, int S, bool RELU>
void fwd(const float *in, int H, const float *theta, float *out, int B, cudaStream_t st)
{
    const int Ho = (H + 2 - 3) / S + 1, total = B * Ho * Ho;
    k_conv_fwd<C, O, S, RELU><<<(total + 127) / 128, 128, 0, st>>>(in, H, theta, out, Ho, total);
}

template <int C, int O, int S>
void bwd(const float *in, int H, const float *gz, const float *theta, const float *a_below, float *gx, float *grad,
         int B, cudaStream_t st, float *part)
{
    const int Ho = (H + 2 - 3) / S + 1;
    // (o, c) pairs times parts of the pixel range: about a thousand blocks
    const int split = (O * C >= 512) ? 1 : std::min(64, 1024 / (O * C));
    k_conv_bwd_weight<C, O, S><<<O * C * split, 256, 0, st>>>(in, H, gz, Ho, B, grad, split, part);
    if (split > 1) k_bwd_weight_sum<C, O><<<(O * C * 10 + 255) / 256, 256, 0, st>>>(part, split, grad);
    if (gx) {
        const int total = B * H * H;
        k_conv_bwd_data<C, O, S><<<(total + 127) / 128, 128, 0, st>>>(gz, Ho, theta, a_below, gx, H, total);
    }
}

}  // namespace

struct reg_cnn {
    cudaStream_t stream = nullptr;
    int side = 0, max_batch = 0;
    int64_t n = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    float *act[NL] = {nullptr};  // layer outputs (post-ReLU, the last one raw)
    float *g0 = nullptr, *g1 = nullptr;  // gradient ping-pong (largest activation)
    float *gy = nullptr;
    double *partial = nullptr, *loss = nullptr;
    uint16_t *actb[5] = {nullptr};  // tensor-core path: outputs of layers 0..4, BF16 planar [b][c/8][y][x][c%8]
    uint32_t *wpack_u = nullptr;  // the 32 -> 32 layers' weights in the tcgen05 operand layout
    uint32_t *wpack_d = nullptr;  // the same, flipped and transposed for the data gradients
    uint32_t *wpack_first = nullptr, *wpack_last = nullptr;  // the first and last layers, tcgen05 layouts
    // parameter version (set_params, adam_step) and the version each packed
    // copy was made from (forward: layers 0..5): the packing runs only after a change
    int64_t version = 0, packed_fwd[6] = {-1, -1, -1, -1, -1, -1}, packed_dgrad[4] = {-1, -1, -1, -1};
    int *uerr = nullptr;          // error word of the tcgen05 kernels (a wait ran out): device view
    int *uerr_host = nullptr;     // the same word, pinned host memory mapped into the device
    float *wpart = nullptr;     // per-block partial weight gradients of the tensor-core training
    int64_t step = 0;
};

namespace {

reg_status cnn_fail(reg_status st, const char *msg) { return reg_internal_fail(st, msg); }

#define CKC(x)                                                          \
    do {                                                                \
        cudaError_t e_ = (x);                                           \
        if (e_ != cudaSuccess) return cnn_fail(REG_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

int out_side(int k, int side)
{
    int H = side;
    for (int j = 0; j <= k; j++) H = (H + 2 - 3) / LAYERS[j].S + 1;
    return H;
}

int in_side(int k, int side) { return k == 0 ? side : out_side(k - 1, side); }

int64_t act_elems(int k, int side) { return (int64_t)LAYERS[k].O * out_side(k, side) * out_side(k, side); }

}  // namespace

int64_t cnn_output_side(const reg_cnn *h) { return out_side(NL - 1, h->side); }

reg_status cnn_check_device_error(reg_cnn *h)
{
    volatile int *w = h->uerr_host;
    const int e = *w;
    if (e == 0) return REG_OK;
    *w = 0;
    return cnn_fail(REG_ECUDA, e == 1   ? "tcgen05 convolution: a copy did not complete in time"
                               : e == 2 ? "tcgen05 convolution: the tensor-core work did not complete in time"
                                        : "tcgen05 convolution: shared memory not 128-byte aligned");
}
int cnn_input_side(const reg_cnn *h) { return h->side; }
int cnn_max_batch(const reg_cnn *h) { return h->max_batch; }

// Forward of a batch of pairs x (device, B x 2 x side x side) into y (device,
// B x 2 x side/4 x side/4) on the given stream; the layer outputs stay in the
// handle for a backward pass.
reg_status cnn_forward(reg_cnn *h, const float *x, int B, float *y, cudaStream_t st, bool tc)
{
    const int S = h->side;
    const float *a = x;
    for (int k = 0; k < NL; k++) {
        const int H = in_side(k, S);
        const float *th = h->theta + param_offset(k);
        float *out = (k == NL - 1 && y) ? y : h->act[k];
        if (tc) {
            // tensor-core path, all six layers on tcgen05: layer 0 from the FP32
            // input, the others from the BF16 planar activations, which layers
            // 0..4 write; layer 5 writes the FP32 output
            const bool pack = h->packed_fwd[k] != h->version;
            reg_status rs;
            if (k == 0)
                rs = cnn_first_umma(a, H, th, h->actb[0], B, st, h->wpack_first, pack, h->uerr);
            else if (k == NL - 1)
                rs = cnn_last_umma(h->actb[k - 1], H, th, out, B, st, h->wpack_last, pack, h->uerr);
            else
                rs = cnn_conv32_umma(h->actb[k - 1], H, th, h->actb[k], false, B, LAYERS[k].S, st,
                                     h->wpack_u + (k - 1) * cnn_conv32_umma_words(), pack, h->uerr);
            if (rs != REG_OK) return rs;
            h->packed_fwd[k] = h->version;
        } else {
            switch (k) {
            case 0: fwd<2, 32, 2, true>(a, H, th, out, B, st); break;
            case 1: fwd<32, 32, 2, true>(a, H, th, out, B, st); break;
            case 2:
            case 3:
            case 4: fwd<32, 32, 1, true>(a, H, th, out, B, st); break;
            default: fwd<32, 2, 1, false>(a, H, th, out, B, st); break;
            }
        }
        if (k == NL - 1 && y && y != h->act[k])
            CKC(cudaMemcpyAsync(h->act[k], y, sizeof(float) * act_elems(k, S) * B, cudaMemcpyDeviceToDevice, st));
        a = out;
    }
    CKC(cudaGetLastError());
    return REG_OK;
}

extern "C" {

int64_t reg_cnn_num_params(void) { return total_params(); }
reg_status reg_cnn_loss_grad_tc(reg_cnn_t h, const float *x, const float *target, int32_t batch, double *loss,
                                float *grad_out);

reg_status reg_cnn_create(int32_t side, int32_t max_batch, void *cuda_stream, reg_cnn_t *out)
{
    if (!out || side < 16 || side % 4 != 0 || side > 4096 || max_batch < 1) return cnn_fail(REG_EINVAL, "bad argument");
    reg_cnn *h = new reg_cnn();
    h->stream = (cudaStream_t)cuda_stream;
    h->side = side;
    h->max_batch = max_batch;
    h->n = total_params();
    auto alloc = [&](void **p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    bool ok = alloc((void **)&h->theta, sizeof(float) * h->n) && alloc((void **)&h->grad, sizeof(float) * h->n) &&
              alloc((void **)&h->m, sizeof(float) * h->n) && alloc((void **)&h->v, sizeof(float) * h->n);
    int64_t big = 0;
    for (int k = 0; k < NL && ok; k++) {
        ok = alloc((void **)&h->act[k], sizeof(float) * act_elems(k, side) * max_batch);
        if (ok && k < 5) ok = alloc((void **)&h->actb[k], sizeof(uint16_t) * act_elems(k, side) * max_batch);
        big = std::max(big, act_elems(k, side));
    }
    big = std::max(big, (int64_t)2 * side * side);
    ok = ok && alloc((void **)&h->g0, sizeof(float) * big * max_batch) &&
         alloc((void **)&h->g1, sizeof(float) * big * max_batch) &&
         alloc((void **)&h->gy, sizeof(float) * act_elems(NL - 1, side) * max_batch) &&
         alloc((void **)&h->partial, sizeof(double) * 1024) && alloc((void **)&h->loss, sizeof(double)) &&
         alloc((void **)&h->wpack_u, sizeof(uint32_t) * 4 * cnn_conv32_umma_words()) &&
         alloc((void **)&h->wpack_d, sizeof(uint32_t) * 4 * cnn_conv32_umma_words()) &&
         alloc((void **)&h->wpack_first, sizeof(uint32_t) * cnn_first_umma_words()) &&
         alloc((void **)&h->wpack_last, sizeof(uint32_t) * cnn_last_umma_words()) &&
         cudaHostAlloc((void **)&h->uerr_host, sizeof(int), cudaHostAllocMapped) == cudaSuccess &&
         cudaHostGetDevicePointer((void **)&h->uerr, h->uerr_host, 0) == cudaSuccess &&
         alloc((void **)&h->wpart, sizeof(float) * (size_t)std::max(cnn_wgrad32_umma_part_floats(), 2 * 1024 * 608));
    if (!ok) {
        reg_cnn_destroy(h);
        return cnn_fail(REG_ENOMEM, "device allocation failed");
    }
    cudaMemsetAsync(h->theta, 0, sizeof(float) * h->n, h->stream);
    cudaMemsetAsync(h->m, 0, sizeof(float) * h->n, h->stream);
    cudaMemsetAsync(h->v, 0, sizeof(float) * h->n, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        reg_cnn_destroy(h);
        return cnn_fail(REG_ECUDA, "init");
    }
    *reinterpret_cast<volatile int *>(h->uerr_host) = 0;
    *out = h;
    return REG_OK;
}

reg_status reg_cnn_set_params(reg_cnn_t h, const float *theta, int32_t on_device)
{
    if (!h || !theta) return cnn_fail(REG_EINVAL, "bad argument");
    CKC(cudaMemcpyAsync(h->theta, theta, sizeof(float) * h->n,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    CKC(cudaMemsetAsync(h->m, 0, sizeof(float) * h->n, h->stream));
    CKC(cudaMemsetAsync(h->v, 0, sizeof(float) * h->n, h->stream));
    h->step = 0;
    h->version++;
    CKC(cudaStreamSynchronize(h->stream));
    return REG_OK;
}

reg_status reg_cnn_get_params(reg_cnn_t h, float *theta, int32_t on_device)
{
    if (!h || !theta) return cnn_fail(REG_EINVAL, "bad argument");
    CKC(cudaMemcpyAsync(theta, h->theta, sizeof(float) * h->n,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    CKC(cudaStreamSynchronize(h->stream));
    return REG_OK;
}

reg_status reg_cnn_forward(reg_cnn_t h, const float *x, int32_t batch, float *y, int32_t tensor_cores)
{
    if (!h || !x || !y || batch < 1 || batch > h->max_batch) return cnn_fail(REG_EINVAL, "bad argument");
    reg_status st = cnn_forward(h, x, batch, y, h->stream, tensor_cores != 0);
    if (st != REG_OK) return st;
    CKC(cudaStreamSynchronize(h->stream));
    return cnn_check_device_error(h);
}

static reg_status loss_grad(reg_cnn_t h, const float *x, const float *target, int32_t batch, double *loss,
                            float *grad_out, bool tc);

reg_status reg_cnn_loss_grad(reg_cnn_t h, const float *x, const float *target, int32_t batch, double *loss,
                             float *grad_out)
{
    return loss_grad(h, x, target, batch, loss, grad_out, false);
}

reg_status reg_cnn_loss_grad_tc(reg_cnn_t h, const float *x, const float *target, int32_t batch, double *loss,
                                float *grad_out)
{
    return loss_grad(h, x, target, batch, loss, grad_out, true);
}

// Loss and gradient; tc: the forward of all six layers, the four 32 -> 32
// layers' weight and data gradients on the tensor cores (BF16 operands, FP32
// accumulation); the weight gradients of the 2 -> 32 and 32 -> 2 layers
// (k_wgrad_first, k_wgrad_last) and the last layer's data gradient on the CUDA
// cores in FP32.
static reg_status loss_grad(reg_cnn_t h, const float *x, const float *target, int32_t batch, double *loss,
                            float *grad_out, bool tc)
{
    if (!h || !x || !target || batch < 1 || batch > h->max_batch) return cnn_fail(REG_EINVAL, "bad argument");
    cudaStream_t st = h->stream;
    const int S = h->side, B = batch;
    reg_status rs = cnn_forward(h, x, B, nullptr, st, tc);
    if (rs != REG_OK) return rs;
    const int64_t ny = act_elems(NL - 1, S) * B;
    const int nb = (int)std::min<int64_t>(1024, (ny + 255) / 256);
    k_mse<<<nb, 256, 0, st>>>(h->act[NL - 1], target, ny, h->gy, h->partial);
    k_sum_partials<<<1, 256, 0, st>>>(h->partial, nb, 1.0 / (double)ny, h->loss);
    const float *gz = h->gy;
    float *bufs[2] = {h->g0, h->g1};
    for (int k = NL - 1; k >= 0; k--) {
        const int H = in_side(k, S);
        const float *in = k == 0 ? x : h->act[k - 1];
        const float *th = h->theta + param_offset(k);
        float *gr = h->grad + param_offset(k);
        float *gx = k == 0 ? nullptr : bufs[k & 1];
        const float *below = k == 0 ? nullptr : h->act[k - 1];
        if (tc && k >= 1 && k <= 4) {
            // the layer's input and the mask below: BF16 planar
            const uint16_t *inb = h->actb[k - 1];
            rs = cnn_wgrad32_umma(inb, H, gz, B, LAYERS[k].S, gr, h->wpart, st, h->uerr);
            if (rs != REG_OK) return rs;
            const bool pack = h->packed_dgrad[k - 1] != h->version;
            uint32_t *wp = h->wpack_d + (k - 1) * cnn_conv32_umma_words();
            if (LAYERS[k].S == 1) rs = cnn_dgrad32_umma(gz, H, th, inb, gx, B, st, wp, pack, h->uerr);
            else rs = cnn_dgrad32s2_umma(gz, H / 2, th, inb, gx, B, st, wp, pack, h->uerr);
            if (rs != REG_OK) return rs;
            h->packed_dgrad[k - 1] = h->version;
            gz = gx;
            continue;
        }
        if (tc && k == NL - 1) {
            // the last layer's input (and the mask below) is the planar BF16
            // output of layer 4
            const int nt = B * ((H + WL_TW - 1) / WL_TW) * ((H + WL_TR - 1) / WL_TR), grid = wgrad_small_grid(nt);
            k_wgrad_last<<<grid, 256, 0, st>>>(reinterpret_cast<const uint4 *>(h->actb[k - 1]), H, gz, B, h->wpart);
            k_wgrad_parts_sum<<<WL_REC, 256, 0, st>>>(h->wpart, grid, WL_REC, gr);
            const int total = B * H * H;
            k_conv_bwd_data<32, 2, 1, true><<<(total + 127) / 128, 128, 0, st>>>(gz, H, th, h->actb[k - 1], gx, H, total);
            gz = gx;
            continue;
        }
        if (tc && k == 0) {
            const int Ho = H / 2, nt = B * ((Ho + WF_TW - 1) / WF_TW) * ((Ho + WF_TR - 1) / WF_TR);
            const int grid = wgrad_small_grid(nt);
            k_wgrad_first<<<grid, 256, 0, st>>>(x, H, gz, Ho, B, h->wpart);
            k_wgrad_parts_sum<<<WF_REC, 256, 0, st>>>(h->wpart, grid, WF_REC, gr);
            continue;
        }
        switch (k) {
        case 0: bwd<2, 32, 2>(in, H, gz, th, below, gx, gr, B, st, h->wpart); break;
        case 1: bwd<32, 32, 2>(in, H, gz, th, below, gx, gr, B, st, h->wpart); break;
        case 2:
        case 3:
        case 4: bwd<32, 32, 1>(in, H, gz, th, below, gx, gr, B, st, h->wpart); break;
        default: bwd<32, 2, 1>(in, H, gz, th, below, gx, gr, B, st, h->wpart); break;
        }
        gz = gx;
    }
    CKC(cudaGetLastError());
    if (loss) CKC(cudaMemcpyAsync(loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad_out) CKC(cudaMemcpyAsync(grad_out, h->grad, sizeof(float) * h->n, cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    return cnn_check_device_error(h);
}

reg_status reg_cnn_adam_step(reg_cnn_t h, double lr, double beta1, double beta2, double eps)
{
    if (!h || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return cnn_fail(REG_EINVAL, "bad argument");
    h->step++;
    h->version++;
    const double c1 = 1.0 - std::pow(beta1, (double)h->step), c2 = 1.0 - std::pow(beta2, (double)h->step);
    k_adam<<<(int)std::min<int64_t>(1024, (h->n + 255) / 256), 256, 0, h->stream>>>(
        h->theta, h->grad, h->m, h->v, h->n, (float)lr, (float)beta1, (float)beta2, (float)eps, (float)c1, (float)c2);
    CKC(cudaGetLastError());
    CKC(cudaStreamSynchronize(h->stream));
    return REG_OK;
}

reg_status reg_cnn_destroy(reg_cnn_t h)
{
    if (!h) return REG_OK;
    cudaFree(h->theta);
    cudaFree(h->grad);
    cudaFree(h->m);
    cudaFree(h->v);
    for (int k = 0; k < NL; k++) cudaFree(h->act[k]);
    for (int k = 0; k < 5; k++) cudaFree(h->actb[k]);
    cudaFree(h->g0);
    cudaFree(h->g1);
    cudaFree(h->gy);
    cudaFree(h->wpack_u);
    cudaFree(h->wpack_d);
    cudaFree(h->wpack_first);
    cudaFree(h->wpack_last);
    if (h->uerr_host) cudaFreeHost(h->uerr_host);
    cudaFree(h->wpart);
    cudaFree(h->partial);
    cudaFree(h->loss);
    delete h;
    return REG_OK;
}

}  // extern "C"
