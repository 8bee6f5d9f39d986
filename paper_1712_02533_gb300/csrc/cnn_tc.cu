// Tensor-core forward of the learned initialiser's 32 -> 32 channel layers:
// a 3x3 convolution (zero padding 1, stride 1 or 2) with bias and ReLU as an
// implicit GEMM, D[pixel][o] = sum_k A[pixel][k] W[o][k] with
// k = (c, dy, dx) = 9 c + 3 dy + dx (K = 288 = 18 steps of 16).  Operands are
// BF16 (activations rounded when loaded, weights rounded into shared memory),
// accumulation FP32 (mma.sync m16n8k16).  One warp computes 16 output pixels
// (consecutive in the flattened batch x row x column order) for all 32 output
// channels (four n-tiles of 8).
#include <cuda_bf16.h>

#include "cnn_internal.h"

namespace {

constexpr int TC_C = 32, TC_O = 32, TC_K = TC_C * 9;
// Shared-memory row of one output channel's weights, in BF16 pairs: 144 pairs
// padded to 148 so that the eight rows a fragment load touches (o = 8j + g)
// fall into distinct banks.
constexpr int TC_WROW = TC_K / 2 + 4;

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

// Input value at reduction index k for output pixel (b, y, x) (zero outside).
__device__ __forceinline__ float a_elem(const float *in, int H, int S, int b, int y, int x, int k, bool valid)
{
    const int c = k / 9, r = k - 9 * c, dy = r / 3, dx = r - 3 * dy;
    const int iy = S * y + dy - 1, ix = S * x + dx - 1;
    if (!valid || iy < 0 || iy >= H || ix < 0 || ix >= H) return 0.f;
    return in[(((int64_t)b * TC_C + c) * H + iy) * H + ix];
}

__global__ void __launch_bounds__(128) k_conv32_tc(const float *__restrict__ in, int H,
                                                   const float *__restrict__ theta, float *__restrict__ out, int Ho,
                                                   int S, int B)
{
    __shared__ uint32_t wsm[TC_O * TC_WROW];  // W[o][k] as BF16 pairs (k, k+1)
    __shared__ float bias[TC_O];
    for (int i = threadIdx.x; i < TC_O * TC_K / 2; i += blockDim.x) {
        const int o = i / (TC_K / 2), q = i - o * (TC_K / 2);
        wsm[o * TC_WROW + q] = pack_bf16(theta[2 * i], theta[2 * i + 1]);
    }
    for (int i = threadIdx.x; i < TC_O; i += blockDim.x) bias[i] = theta[TC_O * TC_K + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int total = B * Ho * Ho;
    const int p0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 16;
    if (p0 >= total) return;  // warp-uniform
    // the two pixels of this lane's A rows: g and g + 8
    int pb[2], py[2], px[2];
    bool pv[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int p = p0 + g + 8 * h;
        pv[h] = p < total;
        const int q = pv[h] ? p : 0;
        px[h] = q % Ho;
        py[h] = (q / Ho) % Ho;
        pb[h] = q / (Ho * Ho);
    }
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int i = 0; i < 4; i++) acc[j][i] = 0.f;
    for (int k0 = 0; k0 < TC_K; k0 += 16) {
        uint32_t a[4];
        const int ka = k0 + 2 * t, kb = ka + 8;
        a[0] = pack_bf16(a_elem(in, H, S, pb[0], py[0], px[0], ka, pv[0]),
                         a_elem(in, H, S, pb[0], py[0], px[0], ka + 1, pv[0]));
        a[1] = pack_bf16(a_elem(in, H, S, pb[1], py[1], px[1], ka, pv[1]),
                         a_elem(in, H, S, pb[1], py[1], px[1], ka + 1, pv[1]));
        a[2] = pack_bf16(a_elem(in, H, S, pb[0], py[0], px[0], kb, pv[0]),
                         a_elem(in, H, S, pb[0], py[0], px[0], kb + 1, pv[0]));
        a[3] = pack_bf16(a_elem(in, H, S, pb[1], py[1], px[1], kb, pv[1]),
                         a_elem(in, H, S, pb[1], py[1], px[1], kb + 1, pv[1]));
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int o = 8 * j + g;
            mma_bf16(acc[j], a, wsm[o * TC_WROW + (ka >> 1)], wsm[o * TC_WROW + (kb >> 1)]);
        }
    }
    // D fragment: (row g, cols 2t, 2t+1) and (row g+8, same cols) of each n-tile
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int h = i >> 1, o = 8 * j + 2 * t + (i & 1);
            if (!pv[h]) continue;
            out[(((int64_t)pb[h] * TC_O + o) * Ho + py[h]) * Ho + px[h]] = fmaxf(acc[j][i] + bias[o], 0.f);
        }
}

}  // namespace

reg_status cnn_conv32_tc(const float *in, int H, const float *theta, float *out, int B, int S, cudaStream_t st)
{
    const int Ho = (H + 2 - 3) / S + 1;
    const int tiles = (B * Ho * Ho + 15) / 16;
    k_conv32_tc<<<(tiles + 3) / 4, 128, 0, st>>>(in, H, theta, out, Ho, S, B);
    if (cudaGetLastError() != cudaSuccess) return reg_internal_fail(REG_ECUDA, "tensor-core convolution launch");
    return REG_OK;
}
