// Weight gradients of the learned initialiser's 32 -> 32 channel layers on the
// tensor cores (BF16 operands, FP32 accumulation, mma.sync m16n8k16), and the
// bias gradients of those layers.  (Their forward and stride-1 data gradients
// run on tcgen05 in cnn_umma.cu.)
#include <cuda_bf16.h>

#include <algorithm>

#include "cnn_internal.h"

namespace {

constexpr int TC_C = 32, TC_O = 32, TC_K = TC_C * 9;
constexpr int TC_TH = 8, TC_TW = 16;  // output tile (rows, columns)
// the input tile of an output tile, with its halo
__host__ __device__ constexpr int in_rows(int S) { return S * (TC_TH - 1) + 3; }
__host__ __device__ constexpr int in_cols(int S) { return S * (TC_TW - 1) + 3; }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const uint32_t l = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return l | (h << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// Weight gradient of a 32 -> 32 layer on the tensor cores:
//   gW[o][n] = sum_p gz[o][p] A[p][n],  n = (3 dy + dx) * 32 + c,
// A the im2col of the layer's input (A[p][n] = in_pad[c][S y + dy][S x + dx]
// for output pixel p = (y, x)), an implicit GEMM with M = 32 output channels,
// N = 288 and the reduction over all output pixels of the batch, BF16
// operands and FP32 accumulation (mma.sync m16n8k16).  A block walks output
// tiles of 8 x 16 pixels (grid-stride), stages per tile the output gradient as
// BF16 pairs of pixels and the input tile with its halo (from the BF16 planar
// activations [b][c / 8][y][x][c % 8]) as [c][y][x], and keeps the
// 32 x 288 partial in registers: each warp holds both m-tiles of 16 channels
// and 9 of the 36 n-tiles.  The partials of the blocks are summed in a fixed
// order by k_wgrad_reduce (deterministic).
// ---------------------------------------------------------------------------
constexpr int WG_PW = 68;  // words per output channel row of the staged gradient: 64 pixel pairs + pad

template <int S>
__global__ void __launch_bounds__(128) k_wgrad32_tc(const uint4 *__restrict__ in, int H, const float *__restrict__ gz,
                                                    int Ho, int tiles_x, int tiles_y, int n_tiles,
                                                    float *__restrict__ part)
{
    constexpr int IR = in_rows(S), IC = in_cols(S);
    __shared__ uint32_t gs[TC_O * WG_PW];
    __shared__ __nv_bfloat16 xs[TC_C * IR * IC];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    float acc[2][9][4];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int j = 0; j < 9; j++)
#pragma unroll
            for (int i = 0; i < 4; i++) acc[m][j][i] = 0.f;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int tx = tile % tiles_x, rest = tile / tiles_x;
        const int ty = rest % tiles_y, b = rest / tiles_y;
        const int oy0 = ty * TC_TH, ox0 = tx * TC_TW;
        const int iy0 = S * oy0 - 1, ix0 = S * ox0 - 1;
        __syncthreads();  // the previous tile's operands are no longer read
        // output gradient: pixel pair q of channel o -> pixels 2q, 2q+1 of the tile
        for (int i = tid; i < TC_O * 64; i += blockDim.x) {
            const int o = i / 64, q = i % 64, py = q / 8, px = 2 * (q % 8);
            const int oy = oy0 + py, ox = ox0 + px;
            float v0 = 0.f, v1 = 0.f;
            if (oy < Ho) {
                const float *r = gz + (((int64_t)b * TC_O + o) * Ho + oy) * Ho;
                if (ox < Ho) v0 = r[ox];
                if (ox + 1 < Ho) v1 = r[ox + 1];
            }
            gs[o * WG_PW + q] = pack_bf16(v0, v1);
        }
        // input tile with its halo, BF16, [c][iy][ix], from the planar input
        // (one 16-byte group of 8 channels per item)
        for (int i = tid; i < (TC_C / 8) * IR * IC; i += blockDim.x) {
            const int ix = i % IC, r2 = i / IC, iy = r2 % IR, cg = r2 / IR;
            const int gy = iy0 + iy, gx = ix0 + ix;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gy >= 0 && gy < H && gx >= 0 && gx < H) v = in[((int64_t)(4 * b + cg) * H + gy) * H + gx];
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
            __nv_bfloat16 *dst = xs + ((8 * cg) * IR + iy) * IC + ix;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                dst[(2 * j) * IR * IC] = __ushort_as_bfloat16((unsigned short)(w[j] & 0xFFFFu));
                dst[(2 * j + 1) * IR * IC] = __ushort_as_bfloat16((unsigned short)(w[j] >> 16));
            }
        }
        __syncthreads();
#pragma unroll 1
        for (int ks = 0; ks < TC_TH; ks++) {  // one output row of 16 pixels per k-step
            uint32_t a[2][4];
#pragma unroll
            for (int m = 0; m < 2; m++) {
                const uint32_t *r0 = gs + (16 * m + g) * WG_PW + 8 * ks + t;
                const uint32_t *r1 = r0 + 8 * WG_PW;
                a[m][0] = r0[0];
                a[m][1] = r1[0];
                a[m][2] = r0[4];
                a[m][3] = r1[4];
            }
#pragma unroll
            for (int j = 0; j < 9; j++) {
                const int n = (9 * warp + j) * 8 + g;  // im2col column of this thread's B element
                const int tap = n >> 5, c = n & 31, dy = tap / 3, dx = tap - 3 * dy;
                const __nv_bfloat16 *row = xs + (c * IR + S * ks + dy) * IC + dx;
                const uint32_t b0 = (uint32_t)__bfloat16_as_ushort(row[S * (2 * t)]) |
                                    ((uint32_t)__bfloat16_as_ushort(row[S * (2 * t + 1)]) << 16);
                const uint32_t b1 = (uint32_t)__bfloat16_as_ushort(row[S * (2 * t + 8)]) |
                                    ((uint32_t)__bfloat16_as_ushort(row[S * (2 * t + 9)]) << 16);
#pragma unroll
                for (int m = 0; m < 2; m++) mma_bf16(acc[m][j], a[m], b0, b1);
            }
        }
    }
    // this block's partial: part[block][o][n]
    float *dst = part + (int64_t)blockIdx.x * TC_O * TC_K;
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int j = 0; j < 9; j++) {
            const int n = (9 * warp + j) * 8 + 2 * t, o = 16 * m + g;
            *reinterpret_cast<float2 *>(dst + o * TC_K + n) = make_float2(acc[m][j][0], acc[m][j][1]);
            *reinterpret_cast<float2 *>(dst + (o + 8) * TC_K + n) = make_float2(acc[m][j][2], acc[m][j][3]);
        }
}

// Sum of the blocks' partials in block order; scatter to the parameter layout
// W[o][c][dy][dx] (n = (3 dy + dx) * 32 + c).
__global__ void k_wgrad_reduce(const float *__restrict__ part, int nblk, float *__restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= TC_O * TC_K) return;
    float s = 0.f;
    for (int k = 0; k < nblk; k++) s += part[(int64_t)k * TC_O * TC_K + i];
    const int o = i / TC_K, n = i % TC_K, tap = n >> 5, c = n & 31;
    grad[(o * TC_C + c) * 9 + tap] = s;
}

// Bias gradient: gb[o] = sum over the batch's output pixels of gz.  Block
// (o, part) sums one contiguous part of channel o's B x per values into
// bpart; k_bias_grad_sum adds the parts in order (deterministic).
constexpr int BG_SPLIT = 32;

__global__ void k_bias_grad(const float *__restrict__ gz, int per, int B, float *__restrict__ bpart)
{
    const int o = blockIdx.x / BG_SPLIT, sp = blockIdx.x % BG_SPLIT;
    const int total = B * per, chunk = (total + BG_SPLIT - 1) / BG_SPLIT;
    const int q0 = sp * chunk, q1 = min(total, q0 + chunk);
    float s = 0.f;
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        const int b = q / per, p = q - b * per;
        s += gz[((int64_t)b * TC_O + o) * per + p];
    }
    __shared__ float red[8];
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += red[w];
        bpart[blockIdx.x] = tot;
    }
}

__global__ void k_bias_grad_sum(const float *__restrict__ bpart, float *__restrict__ gb)
{
    const int o = threadIdx.x;
    if (o >= TC_O) return;
    float t = 0.f;
    for (int sp = 0; sp < BG_SPLIT; sp++) t += bpart[o * BG_SPLIT + sp];
    gb[o] = t;
}

template <int S>
reg_status launch_wgrad(const uint4 *in, int H, const float *gz, int B, float *grad, float *part, int max_blocks,
                        cudaStream_t st)
{
    const int Ho = (H + 2 - 3) / S + 1;
    const int tx = (Ho + TC_TW - 1) / TC_TW, ty = (Ho + TC_TH - 1) / TC_TH, nt = B * tx * ty;
    const int nblk = std::min(nt, max_blocks);
    k_wgrad32_tc<S><<<nblk, 128, 0, st>>>(in, H, gz, Ho, tx, ty, nt, part);
    k_wgrad_reduce<<<(TC_O * TC_K + 255) / 256, 256, 0, st>>>(part, nblk, grad);
    // the bias parts after the weight partials in the scratch (part has room:
    // max_blocks x 32 x 288 floats, the weight partials use nblk of them)
    float *bpart = part + (int64_t)nblk * TC_O * TC_K;
    k_bias_grad<<<TC_O * BG_SPLIT, 256, 0, st>>>(gz, Ho * Ho, B, bpart);
    k_bias_grad_sum<<<1, 32, 0, st>>>(bpart, grad + TC_O * TC_K);
    if (cudaGetLastError() != cudaSuccess) return reg_internal_fail(REG_ECUDA, "tensor-core weight gradient launch");
    return REG_OK;
}

}  // namespace

// Blocks of the weight-gradient kernel: three resident per SM (its register
// limit) on every SM of the current device.
int cnn_wgrad32_tc_blocks()
{
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        nsm = 152;
    return 3 * nsm;
}

reg_status cnn_wgrad32_tc(const uint16_t *in, int H, const float *gz, int B, int S, float *grad, float *part,
                          cudaStream_t st)
{
    const uint4 *inq = reinterpret_cast<const uint4 *>(in);
    if (S == 1) return launch_wgrad<1>(inq, H, gz, B, grad, part, cnn_wgrad32_tc_blocks(), st);
    if (S == 2) return launch_wgrad<2>(inq, H, gz, B, grad, part, cnn_wgrad32_tc_blocks(), st);
    return reg_internal_fail(REG_EINVAL, "tensor-core weight gradient: stride must be 1 or 2");
}
