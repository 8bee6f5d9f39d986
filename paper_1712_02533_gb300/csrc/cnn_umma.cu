// The learned initialiser's convolutions on the fifth-generation tensor cores:
// tcgen05.mma with the accumulator in tensor memory (TMEM), BF16 operands,
// FP32 accumulation.  All six layers of the tensor-core forward run here: the
// four 32 -> 32 layers and the last layer (32 -> 2) from TMA-loaded tiles,
// the first layer (2 -> 32) from tiles the CTA's threads stage; the data
// gradients of the four 32 -> 32 layers (stride 1, and stride 2 as four
// parity classes of stride-1 GEMMs); and their weight gradients, GEMMs whose
// reduction runs over the batch's pixels (k_wgrad32_umma).
//
// Implicit GEMM per output tile of 16 rows x 8 columns of one image:
//   D[m][o] = sum_k A[m][k] W[o][k],   m = 8 (tile row) + (tile column),
//   k = (3 dy + dx) * C + c,           M = 128, N = 32 (last layer: 16, of which
// the 2 output channels are real), K = 9 C in steps of 16,
// A[m][k] = in_pad[c][S y + dy][S x + dx] for output pixel (y, x) of tile row m.
//
// Activations between layers are BF16 in a channel-group planar layout,
// [b][cg][y][x][8 channels] (cg = c / 8): 16 bytes per pixel and channel
// group.  It is the K-major operand layout of the tensor cores, so a tile's
// input needs no conversion.
//
// Shared-memory operands in the K-major layout without swizzling: "core
// matrices" of 8 rows x 16 bytes (8 BF16 values along k), each stored as 128
// contiguous bytes, rows 16 bytes apart.  A descriptor gives the start address
// and two strides: between core matrices adjacent along M (or N) and along K.
//   - Weights, packed by k_pack_umma when the parameters change: [tap][cg][o][8
//     channels] BF16.  For a k-step (tap, half h) the operand starts at
//     ((4 tap + 2 h) N) 16 bytes; N-stride 128 B, K-stride 16 N bytes.  They
//     reach shared memory by a bulk asynchronous copy (cp.async.bulk).
//   - The input tile with its halo, [cg][halo row][halo column][8 channels].
//     Every 8 output pixels of a tile row read 8 consecutive halo columns for
//     any tap, so each tap of the 3 x 3 window is the same operand with a
//     shifted start address: tap (dy, dx) starts at halo row dy, column dx.
//     The 32-channel layers load the tile with one TMA tensor copy
//     (cp.async.bulk.tensor, 18 rows x 10 columns x 4 groups; zeros outside
//     the image).  With stride 2 the output columns x read halo columns
//     2 x + dx, so the halo is loaded as two copies, the columns of one
//     parity each (a view of the activations with the column split into
//     (x / 2, x % 2)), and a tap starts in the copy of its parity dx & 1 at
//     column dx >> 1; the M-stride then covers two halo rows.
//   - The first layer has 2 input channels, padded to one group of 8: a
//     k-step of 16 takes two taps, whose core matrices the descriptor's
//     K-stride joins (the ninth tap pairs with zero weights), 5 MMAs a tile.
//
// The TMA-fed layers split each CTA into a copy warp, an MMA warp and four
// epilogue warps that hand tiles on through mbarriers (NS halo stages, two
// TMEM accumulators); each epilogue warp reads its 32 TMEM lanes (= tile rows
// 32 w .. 32 w + 31) with tcgen05.ld and writes bias + ReLU as planar BF16, or
// the last layer's two channels as FP32 NCHW.  The kernels whose threads stage
// their tiles (the first layer; the data gradient of a 32 -> 32 layer, which
// runs the same GEMM on the output gradient, FP32 NCHW, with flipped and
// transposed weights, times the ReLU mask of the layer below) keep one thread
// issuing the MMAs, two halo buffers and two accumulators, so that a tile's
// MMAs run while the next is staged and the previous one is written.  Every
// wait on an mbarrier is bounded (one second of the global timer); a wait that
// runs out sets the error word, the CTA stops issuing work, frees its TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "cnn_internal.h"

namespace {

constexpr int UC = 32;                     // channels of the 32-channel layers
constexpr int UTH = 16, UTW = 8;           // output tile: 16 rows x 8 columns = the 128 rows of the MMA
constexpr uint64_t U_WAIT_NS = 1000000000ull;

// packed weights of a layer with N output rows and 32 input channels
template <int N>
struct Wts {
    static constexpr int bytes = 9 * 4 * N * 16;
};
// the first layer: 5 k-steps of two taps, 2 halves of 8 channels, 32 outputs
constexpr int L0_STEPS = 5;
constexpr int L0_WBYTES = L0_STEPS * 2 * UC * 16;
// TMEM columns: two FP32 accumulators of N columns (at least 32 columns)
template <int N>
__host__ __device__ constexpr int tmem_cols()
{
    return 2 * N < 32 ? 32 : 2 * N;
}

// The staged input tile of stride S with G channel groups: per copy (one, or
// one per column parity with stride 2) [cg][rows][cols][16 bytes].  A TMA
// tensor copy writes to a 128-byte aligned shared-memory address, so each
// copy starts on a multiple of 128 bytes.
template <int S, int G = 4>
struct Halo {
    static constexpr int rows = S * (UTH - 1) + 3;           // 18 or 33
    static constexpr int cols = S == 1 ? UTW + 2 : UTW + 1;  // 10, or 9 per parity
    static constexpr int cg_bytes = rows * cols * 16;        // 2880 or 4752
    static constexpr int copy_bytes = G * cg_bytes;          // what one copy writes
    static constexpr int copy_stride = (copy_bytes + 127) / 128 * 128;
    static constexpr int bytes = S * copy_stride;
    static constexpr int sbo = S * cols * 16;                // M-stride: one output row = S halo rows
    // start of tap (dy, dx) in channel group cg, relative to the buffer
    __host__ __device__ static constexpr int tap_offset(int dy, int dx, int cg)
    {
        return (S == 1 ? 0 : (dx & 1) * copy_stride) + cg * cg_bytes + (dy * cols + (S == 1 ? dx : dx >> 1)) * 16;
    }
};

// shared memory: [weights][halo buffers][mbarriers: weights, 2 full, 2 MMA][TMEM
// address][bias], the halo buffers 128-byte aligned.
template <int WB, int HB, int NBUF>
struct Smem {
    static constexpr int nbuf = NBUF;
    static constexpr int w = 0;
    static constexpr int halo = (WB + 127) / 128 * 128;
    static constexpr int bars = halo + nbuf * HB;  // 8-byte aligned
    static constexpr int taddr = bars + 5 * 8;
    static constexpr int bias = taddr + 8;
    static constexpr int bytes = bias + UC * 4;
    static_assert(halo % 128 == 0 && HB % 128 == 0, "TMA destinations must be 128-byte aligned");
};
using DgradSmem = Smem<Wts<UC>::bytes, Halo<1>::bytes, 2>;
using L0Smem = Smem<L0_WBYTES, Halo<2, 1>::bytes, 2>;

// The warp-specialised forward: [weights][NS halo stages][mbarriers: weights,
// full[NS], empty[NS], accumulator full[2], accumulator empty[2]][TMEM
// address][abort flag][bias].  Stride 1 keeps four stages (three CTAs per
// SM), stride 2 two.
template <int S, int N>
struct WsSmem {
    static constexpr int ns = S == 1 ? 4 : 2;
    static constexpr int w = 0;
    static constexpr int halo = (Wts<N>::bytes + 127) / 128 * 128;
    static constexpr int bars = halo + ns * Halo<S>::bytes;
    static constexpr int nbars = 1 + 2 * ns + 4;
    static constexpr int taddr = bars + nbars * 8;
    static constexpr int abort = taddr + 4;
    static constexpr int bias = taddr + 8;
    static constexpr int bytes = bias + UC * 4;
    static_assert(halo % 128 == 0 && Halo<S>::bytes % 128 == 0, "TMA destinations must be 128-byte aligned");
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; false after one
// second of the global timer.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > U_WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// mbar_wait that also gives up when another role of the CTA set the abort flag.
__device__ __forceinline__ bool mbar_wait_ab(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag || global_ns() - t0 > U_WAIT_NS) return false;
    }
    return true;
}

// Shared-memory matrix descriptor, no swizzling: start address, K-direction
// (leading) and M/N-direction (stride) byte offsets between core matrices, all
// in units of 16 bytes; bits 46..48 hold the fixed value 0b001.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16 for M = 128 and N: FP32 accumulator
// (bits 4-5 = 1), BF16 A and B (bits 7-9 and 10-12 = 1), both K-major (bits
// 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
template <int N>
__device__ __forceinline__ constexpr uint32_t idesc()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
}

template <int N>
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc<N>()), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// N consecutive FP32 columns (16 or 32) of this thread's TMEM lane.
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[N])
{
    uint32_t r[N];
    if constexpr (N == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    } else {
        static_assert(N == 16, "16 or 32 columns");
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < N; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

// W[o][c][dy][dx] (FP32, O output and 32 input channels) -> [tap][cg][n][8
// channels] (BF16), n < N, rows n >= O zero.  DGRAD: the data gradient of a
// stride-1 32 -> 32 layer as a forward convolution of the output gradient
// with K'[c][o][tap] = W[o][c][8 - tap] (output channel c, reduction channel o).
template <bool DGRAD, int N, int O>
__global__ void k_pack_umma(const float *__restrict__ theta, uint32_t *__restrict__ wpack)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // one pair of reduction channels
    if (i >= Wts<N>::bytes / 4) return;
    const int jp = i & 3, n = (i >> 2) % N, r = (i >> 2) / N, cg = r & 3, tap = r >> 2;
    const int k0 = 8 * cg + 2 * jp;  // reduction channel of the low half
    float lo = 0.f, hi = 0.f;
    if (DGRAD) {
        lo = theta[((int64_t)k0 * UC + n) * 9 + (8 - tap)];
        hi = theta[((int64_t)(k0 + 1) * UC + n) * 9 + (8 - tap)];
    } else if (n < O) {
        lo = theta[((int64_t)n * UC + k0) * 9 + tap];
        hi = theta[((int64_t)n * UC + k0 + 1) * 9 + tap];
    }
    wpack[i] = pack2(lo, hi);
}

// The first layer's taps in k-step order: step j takes taps l0_tap(j, 0) and
// l0_tap(j, 1) (-1: zero weights), chosen so that the second one lies at a
// higher address of the stride-2 halo (the K-stride is unsigned).
__host__ __device__ constexpr int l0_tap(int j, int h)
{
    // (dy, dx) = (0,0)+(0,2), (1,0)+(1,2), (2,0)+(2,2), (0,1)+(1,1), (2,1)
    return j < 3 ? 3 * j + 2 * h : (j == 3 ? 1 + 3 * h : (h == 0 ? 7 : -1));
}

// W[o][c][dy][dx] of the first layer (32 x 2 x 3 x 3) -> [step][half][o][8
// channels] (BF16), channels 2..7 and the missing tap zero.
__global__ void k_pack_l0(const float *__restrict__ theta, uint32_t *__restrict__ wpack)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L0_WBYTES / 4) return;
    const int jp = i & 3, o = (i >> 2) & 31, h = (i >> 7) & 1, j = i >> 8;
    const int tap = l0_tap(j, h);
    float lo = 0.f, hi = 0.f;
    if (tap >= 0 && jp == 0) {
        lo = theta[(o * 2 + 0) * 9 + tap];
        hi = theta[(o * 2 + 1) * 9 + tap];
    }
    wpack[i] = pack2(lo, hi);
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

// The 18 MMAs of one tile of a 32-input-channel layer: halo buffer at hbase,
// accumulator at d.
template <int S, int N>
__device__ __forceinline__ void issue_tile_mmas(uint32_t hbase, uint32_t wbase, uint32_t d)
{
    using HL = Halo<S>;
#pragma unroll
    for (int ks = 0; ks < 18; ks++) {
        const int tap = ks >> 1, h = ks & 1, dy = tap / 3, dx = tap - 3 * dy;
        umma_bf16<N>(d, sdesc(hbase + HL::tap_offset(dy, dx, 2 * h), HL::cg_bytes, HL::sbo),
                     sdesc(wbase + (4 * tap + 2 * h) * N * 16, N * 16, 128), ks > 0);
    }
}

// The 5 MMAs of one tile of the first layer (two taps a k-step).
__device__ __forceinline__ void issue_l0_mmas(uint32_t hbase, uint32_t wbase, uint32_t d)
{
    using HL = Halo<2, 1>;
#pragma unroll
    for (int j = 0; j < L0_STEPS; j++) {
        const int t0 = l0_tap(j, 0), t1 = l0_tap(j, 1);
        const int a0 = HL::tap_offset(t0 / 3, t0 % 3, 0);
        // the second tap's core matrices; the missing one reads the next column
        // (in bounds) against zero weights
        const int a1 = t1 >= 0 ? HL::tap_offset(t1 / 3, t1 % 3, 0) : a0 + 16;
        umma_bf16<UC>(d, sdesc(hbase + a0, a1 - a0, HL::sbo), sdesc(wbase + j * 2 * UC * 16, UC * 16, 128), j > 0);
    }
}

// The 18 MMAs of one tile of the data gradient of a stride-2 32 -> 32 layer.
// An input pixel (2 i + py, 2 j + px) takes the taps dy with 2 i + py + 1 - dy
// even: dy = 1 (output row i) for py = 0, dy = 0 (row i + 1) and dy = 2 (row i)
// for py = 1, and likewise along x.  Each parity class q = 2 py + px is then a
// stride-1 GEMM over the output gradient on the class grid (i, j), with 1, 2, 2
// or 4 taps at offsets 0 and +1: in the halo of the stride-1 data gradient
// (origin one row and column before the tile) offset delta is tap row or column
// 1 + delta.  The weights are those of the stride-1 packing (flipped: packed
// tap p holds W[.][.][8 - p]), so tap (dy, dx) reads packed tap 8 - (3 dy + dx).
// Class q accumulates into columns d + 32 q.
__device__ __forceinline__ void issue_dgrad2_mmas(uint32_t hbase, uint32_t wbase, uint32_t d)
{
    using HL = Halo<1>;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int py = q >> 1, px = q & 1;
        int first = 1;
#pragma unroll
        for (int ty = 0; ty < 1 + py; ty++) {
            const int dy = py ? 2 * ty : 1, hy = dy == 0 ? 2 : 1;
#pragma unroll
            for (int tx = 0; tx < 1 + px; tx++) {
                const int dx = px ? 2 * tx : 1, hx = dx == 0 ? 2 : 1, p = 8 - (3 * dy + dx);
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    umma_bf16<UC>(d + 32 * q, sdesc(hbase + HL::tap_offset(hy, hx, 2 * h), HL::cg_bytes, HL::sbo),
                                  sdesc(wbase + (4 * p + 2 * h) * UC * 16, UC * 16, 128), first ? 0u : 1u);
                    first = 0;
                }
            }
        }
    }
}

// Common setup: TMEM columns, mbarriers, bias (nb entries), and the weights'
// bulk copy (wbytes, a multiple of 32).
template <class SM, int COLS>
__device__ __forceinline__ uint32_t umma_setup(uint8_t *smem, const float *bias_g, int nb, const uint32_t *wpack,
                                               int wbytes)
{
    const int tid = threadIdx.x;
    const uint32_t s_base = smem_u32(smem);
    const uint32_t bar_w = s_base + SM::bars;
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_base + SM::taddr),
                     "r"(COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 5; i++) mbar_init(bar_w + 8 * i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    float *bias = reinterpret_cast<float *>(smem + SM::bias);
    if (tid < UC) bias[tid] = (bias_g && tid < nb) ? bias_g[tid] : 0.f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        mbar_expect_tx(bar_w, wbytes);
#pragma unroll
        for (int h = 0; h < 2; h++)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    s_base + SM::w + h * (wbytes / 2)),
                "l"(reinterpret_cast<const uint8_t *>(wpack) + h * (wbytes / 2)), "r"(wbytes / 2), "r"(bar_w)
                : "memory");
    }
    return *reinterpret_cast<volatile uint32_t *>(smem + SM::taddr);
}

template <int COLS>
__device__ __forceinline__ void umma_teardown(uint32_t tmem)
{
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
    }
}

__device__ __forceinline__ void tile_coords(int tile, int tiles_x, int tiles_y, int &b, int &ty, int &tx)
{
    const int per_img = tiles_x * tiles_y;
    b = tile / per_img;
    const int r = tile - b * per_img;
    ty = r / tiles_x;
    tx = r - ty * tiles_x;
}

// The epilogue's store of one output pixel's NR channels v (bias added): as
// planar BF16 (32 channels) after ReLU, or FP32 NCHW (ReLU if RELU).
template <int NR, bool RELU, bool OUT_F32>
__device__ __forceinline__ void store_pixel(void *out, float *v, const float *bias, int b, int Ho, int oy, int ox)
{
#pragma unroll
    for (int o = 0; o < NR; o++) {
        v[o] += bias[o];
        if (RELU) v[o] = fmaxf(v[o], 0.f);
    }
    if (OUT_F32) {
        float *o32 = reinterpret_cast<float *>(out);
        const int64_t o0 = ((int64_t)b * NR * Ho + oy) * Ho + ox, plane = (int64_t)Ho * Ho;
#pragma unroll
        for (int o = 0; o < NR; o++) o32[o0 + o * plane] = v[o];
    } else {
        static_assert(OUT_F32 || NR == UC, "planar output has 32 channels");
        uint4 *o16 = reinterpret_cast<uint4 *>(out);
#pragma unroll
        for (int cg = 0; cg < NR / 8; cg++) {
            const float *q = v + 8 * cg;
            o16[((int64_t)(4 * b + cg) * Ho + oy) * Ho + ox] =
                make_uint4(pack2(q[0], q[1]), pack2(q[2], q[3]), pack2(q[4], q[5]), pack2(q[6], q[7]));
        }
    }
}

// Forward of a layer with 32 input channels: input by TMA from the planar
// BF16 activations (tensor map tin), N output rows of which NR are written
// (bias, ReLU if RELU) as planar BF16 or FP32 NCHW.  The CTA's roles are split
// over six warps, each waiting on its own mbarriers: warp 4 (one lane) issues
// the weights' bulk copy and the tiles' TMA copies into NS stages, warp 5 (one
// lane) issues each tile's 18 MMAs into one of two TMEM accumulators once its
// stage is full and the accumulator has been read, and commits them to the
// stage's "empty" and the accumulator's "full" barriers; warps 0..3 read the
// accumulator (their 32 TMEM lanes each), hand it back (one arrival per warp)
// and store the tile.  A wait that runs out (one second) or sees another
// role's abort sets the error word and the abort flag and ends that role.
template <int S, int N, int NR, bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(192) k_conv_umma_ws(const __grid_constant__ CUtensorMap tin,
                                                      const float *__restrict__ bias_g,
                                                      const uint32_t *__restrict__ wpack, void *__restrict__ out,
                                                      int Ho, int tiles_x, int tiles_y, int n_tiles,
                                                      int *__restrict__ err)
{
    using HL = Halo<S>;
    using SM = WsSmem<S, N>;
    constexpr int NS = SM::ns, COLS = tmem_cols<N>();
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t s_base = smem_u32(smem);
    if (s_base & 127u) {  // the TMA destinations would not be 128-byte aligned
        if (tid == 0) *reinterpret_cast<volatile int *>(err) = 3;
        return;
    }
    const uint32_t bar_w = s_base + SM::bars, bar_full = bar_w + 8, bar_empty = bar_full + 8 * NS;
    const uint32_t bar_accf = bar_empty + 8 * NS, bar_acce = bar_accf + 16;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + SM::abort);
    float *bias = reinterpret_cast<float *>(smem + SM::bias);
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_base + SM::taddr),
                     "r"(COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bar_w, 1);
        for (int i = 0; i < NS; i++) {
            mbar_init(bar_full + 8 * i, 1);
            mbar_init(bar_empty + 8 * i, 1);
        }
        for (int i = 0; i < 2; i++) {
            mbar_init(bar_accf + 8 * i, 1);
            mbar_init(bar_acce + 8 * i, 4);  // one arrival per epilogue warp
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < UC) bias[tid] = tid < NR ? bias_g[tid] : 0.f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(smem + SM::taddr);
    const int my_tiles = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto fail = [&](int code) {
        *reinterpret_cast<volatile int *>(err) = code;
        *abort_flag = 1;
    };
    if (warp == 4) {
        if (lane == 0) {
            mbar_expect_tx(bar_w, Wts<N>::bytes);
#pragma unroll
            for (int h = 0; h < 2; h++)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        s_base + SM::w + h * (Wts<N>::bytes / 2)),
                    "l"(reinterpret_cast<const uint8_t *>(wpack) + h * (Wts<N>::bytes / 2)),
                    "r"(Wts<N>::bytes / 2), "r"(bar_w)
                    : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tin)) : "memory");
            for (int i = 0; i < my_tiles; i++) {
                const int st = i % NS;
                // the stage's last tile (i - NS) has been multiplied
                if (i >= NS && !mbar_wait_ab(bar_empty + 8 * st, ((i / NS) - 1) & 1, abort_flag)) {
                    fail(1);
                    break;
                }
                int b, ty, tx;
                tile_coords(blockIdx.x + i * gridDim.x, tiles_x, tiles_y, b, ty, tx);
                const int iy0 = S * UTH * ty - 1;
                const uint32_t dst = s_base + SM::halo + st * HL::bytes, bar = bar_full + 8 * st;
                mbar_expect_tx(bar, S * HL::copy_bytes);
                if (S == 1) {
                    tma_load_4d(dst, &tin, 0, UTW * tx - 1, iy0, 4 * b, bar);
                } else {
                    tma_load_5d(dst, &tin, 0, 1, UTW * tx - 1, iy0, 4 * b, bar);
                    tma_load_5d(dst + HL::copy_stride, &tin, 0, 0, UTW * tx, iy0, 4 * b, bar);
                }
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            bool ok = my_tiles == 0 || mbar_wait_ab(bar_w, 0, abort_flag);
            if (!ok) fail(1);
            for (int i = 0; ok && i < my_tiles; i++) {
                const int st = i % NS, a = i & 1;
                if (!mbar_wait_ab(bar_full + 8 * st, (i / NS) & 1, abort_flag)) {
                    fail(1);
                    break;
                }
                // the accumulator's last tile (i - 2) has been read
                if (i >= 2 && !mbar_wait_ab(bar_acce + 8 * a, ((i >> 1) - 1) & 1, abort_flag)) {
                    fail(2);
                    break;
                }
                tc_fence_after();
                issue_tile_mmas<S, N>(s_base + SM::halo + st * HL::bytes, s_base + SM::w, tmem + a * N);
                umma_commit(bar_empty + 8 * st);
                umma_commit(bar_accf + 8 * a);
            }
        }
    } else {
        for (int i = 0; i < my_tiles; i++) {
            const int a = i & 1;
            const bool ok = mbar_wait_ab(bar_accf + 8 * a, (i >> 1) & 1, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) fail(2);
                break;
            }
            tc_fence_after();
            float v[N];
            tmem_ld<N>(tmem + ((uint32_t)(32 * warp) << 16) + a * N, v);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_acce + 8 * a);
            int b, ty, tx;
            tile_coords(blockIdx.x + i * gridDim.x, tiles_x, tiles_y, b, ty, tx);
            const int m = 32 * warp + lane, oy = ty * UTH + (m >> 3), ox = tx * UTW + (m & 7);
            if (oy < Ho && ox < Ho) store_pixel<NR, RELU, OUT_F32>(out, v, bias, b, Ho, oy, ox);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
    }
}

// Positive entries of a planar BF16 activation: 32 bits, one per channel.
__device__ __forceinline__ uint32_t positive_mask(const uint4 *act, int b, int H, int y, int x)
{
    uint32_t m = 0;
#pragma unroll
    for (int cg = 0; cg < 4; cg++) {
        const uint4 q = act[((int64_t)(4 * b + cg) * H + y) * H + x];
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t lo = w[j] & 0xFFFFu, hi = w[j] >> 16;
            m |= (uint32_t)(lo != 0 && !(lo & 0x8000u)) << (8 * cg + 2 * j);
            m |= (uint32_t)(hi != 0 && !(hi & 0x8000u)) << (8 * cg + 2 * j + 1);
        }
    }
    return m;
}

// Kernels whose tiles the CTA's threads stage from FP32 NCHW input, rounded
// to BF16 (the previous tile's MMAs waited on in the last epilogue):
//   ST_DGRAD1: the data gradient of a stride-1 32 -> 32 layer, gz (the
//     gradient with respect to the layer's pre-activation output) in, gx =
//     the GEMM with flipped and transposed weights where the planar BF16
//     activation below (mask) is positive, else 0;
//   ST_FIRST: the first layer's forward (2 input channels, stride 2, padded to
//     one group of 8), bias + ReLU out as planar BF16;
//   ST_DGRAD2: the data gradient of a stride-2 32 -> 32 layer: tiles of the
//     class grid (side H, the output gradient's), the four parity classes of
//     a tile in four accumulators (issue_dgrad2_mmas), gx of side Ho = 2 H
//     written as pairs of adjacent columns (px = 0, 1), masked as ST_DGRAD1.
constexpr int ST_DGRAD1 = 0, ST_FIRST = 1, ST_DGRAD2 = 2;
template <int MODE>
__host__ __device__ constexpr int staged_cols()
{
    return MODE == ST_DGRAD2 ? 2 * 4 * UC : tmem_cols<UC>();
}

template <int MODE>
__global__ void __launch_bounds__(128) k_conv_umma_staged(const float *__restrict__ in, int H,
                                                          const uint32_t *__restrict__ wpack,
                                                          const float *__restrict__ bias_g,
                                                          const uint4 *__restrict__ mask, void *__restrict__ out,
                                                          int Ho, int tiles_x, int tiles_y, int n_tiles,
                                                          int *__restrict__ err)
{
    constexpr bool L0 = MODE == ST_FIRST;
    constexpr int S = L0 ? 2 : 1, G = L0 ? 1 : 4;
    using HL = Halo<S, G>;
    using SM = std::conditional_t<L0, L0Smem, DgradSmem>;
    constexpr int COLS = staged_cols<MODE>(), ACC = COLS / 2;  // two accumulators of ACC columns
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t s_base = smem_u32(smem);
    const uint32_t bar_w = s_base + SM::bars, bar_mma = bar_w + 24;
    const float *bias = reinterpret_cast<const float *>(smem + SM::bias);
    const uint32_t tmem = umma_setup<SM, COLS>(smem, L0 ? bias_g : nullptr, UC, wpack, L0 ? L0_WBYTES : Wts<UC>::bytes);
    int bad = 0;
    int it = 0, prev = -1;
    for (int tile = blockIdx.x;; tile += gridDim.x, ++it) {
        const bool have = tile < n_tiles;
        const int buf = it & 1;
        if (have) {
            int b, ty, tx;
            tile_coords(tile, tiles_x, tiles_y, b, ty, tx);
            const int iy0 = S * UTH * ty - 1, ix0 = S * UTW * tx - 1;
            uint8_t *hbuf = smem + SM::halo + buf * HL::bytes;
            constexpr int C = L0 ? 2 : UC;
            const float *img = in + (int64_t)b * C * H * H;
            const int64_t plane = (int64_t)H * H;
            if (L0) {
                // halo columns ix0 + 2 j (copy 0) and ix0 + 1 + 2 j (copy 1), j < 9
                for (int i = tid; i < 2 * HL::rows * HL::cols; i += 128) {
                    const int j = i % HL::cols, r3 = i / HL::cols, iy = r3 % HL::rows, par = r3 / HL::rows;
                    const int gy = iy0 + iy, gxx = ix0 + par + 2 * j;
                    uint4 v = make_uint4(0u, 0u, 0u, 0u);
                    if (gy >= 0 && gy < H && gxx >= 0 && gxx < H) {
                        const float *p = img + (int64_t)gy * H + gxx;
                        v.x = pack2(p[0], p[plane]);
                    }
                    *reinterpret_cast<uint4 *>(hbuf + par * HL::copy_stride + (iy * HL::cols + j) * 16) = v;
                }
            } else {
                for (int i = tid; i < 4 * HL::rows * HL::cols; i += 128) {
                    const int ix = i % HL::cols, r3 = i / HL::cols, iy = r3 % HL::rows, cg = r3 / HL::rows;
                    const int gy = iy0 + iy, gxx = ix0 + ix;
                    uint4 v = make_uint4(0u, 0u, 0u, 0u);
                    if (gy >= 0 && gy < H && gxx >= 0 && gxx < H) {
                        const float *p = img + (int64_t)(8 * cg) * plane + (int64_t)gy * H + gxx;
                        v = make_uint4(pack2(p[0], p[plane]), pack2(p[2 * plane], p[3 * plane]),
                                       pack2(p[4 * plane], p[5 * plane]), pack2(p[6 * plane], p[7 * plane]));
                    }
                    *reinterpret_cast<uint4 *>(hbuf + cg * HL::cg_bytes + (iy * HL::cols + ix) * 16) = v;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        tc_fence_before();
        __syncthreads();
        if (have && tid == 0 && !bad) {
            tc_fence_after();
            if (it == 0 && !mbar_wait(bar_w, 0)) {
                *reinterpret_cast<volatile int *>(err) = 1;
            } else {
                const uint32_t hbase = s_base + SM::halo + buf * HL::bytes;
                if (MODE == ST_FIRST) issue_l0_mmas(hbase, s_base + SM::w, tmem + buf * ACC);
                else if (MODE == ST_DGRAD2) issue_dgrad2_mmas(hbase, s_base + SM::w, tmem + buf * ACC);
                else issue_tile_mmas<1, UC>(hbase, s_base + SM::w, tmem + buf * ACC);
            }
            umma_commit(bar_mma + 8 * buf);
        }
        if (prev >= 0) {
            const int pb = buf ^ 1;
            const bool ok = bad ? true : mbar_wait(bar_mma + 8 * pb, ((it - 1) >> 1) & 1);
            if (!ok) *reinterpret_cast<volatile int *>(err) = 2;
            bad = __syncthreads_or(!ok || bad);
            if (!bad) {
                tc_fence_after();
                int b, ty, tx;
                tile_coords(prev, tiles_x, tiles_y, b, ty, tx);
                const int m = 32 * warp + lane;
                const uint32_t lanes = (uint32_t)(32 * warp) << 16;
                if (MODE == ST_DGRAD2) {
                    // class grid pixel (i, j) -> input pixels (2 i + py, 2 j + px)
                    const int i = ty * UTH + (m >> 3), j = tx * UTW + (m & 7);
                    float *gx = reinterpret_cast<float *>(out);
                    const int64_t plane = (int64_t)Ho * Ho;
#pragma unroll 1
                    for (int py = 0; py < 2; py++) {
                        float v0[UC], v1[UC];
                        tmem_ld<UC>(tmem + lanes + pb * ACC + 32 * (2 * py), v0);
                        tmem_ld<UC>(tmem + lanes + pb * ACC + 32 * (2 * py + 1), v1);
                        if (i < H && j < H) {
                            const int iy = 2 * i + py, ix = 2 * j;
                            const uint32_t m0 = positive_mask(mask, b, Ho, iy, ix);
                            const uint32_t m1 = positive_mask(mask, b, Ho, iy, ix + 1);
                            float2 *o2 = reinterpret_cast<float2 *>(gx + ((int64_t)b * UC * Ho + iy) * Ho + ix);
#pragma unroll
                            for (int o = 0; o < UC; o++)
                                o2[o * (plane / 2)] = make_float2(((m0 >> o) & 1u) ? v0[o] : 0.f,
                                                                  ((m1 >> o) & 1u) ? v1[o] : 0.f);
                        }
                    }
                } else {
                    float v[UC];
                    tmem_ld<UC>(tmem + lanes + pb * ACC, v);
                    const int oy = ty * UTH + (m >> 3), ox = tx * UTW + (m & 7);
                    if (oy < Ho && ox < Ho) {
                        if (L0) {
                            store_pixel<UC, true, false>(out, v, bias, b, Ho, oy, ox);
                        } else {
                            float *gx = reinterpret_cast<float *>(out);
                            const uint32_t pm = positive_mask(mask, b, Ho, oy, ox);
                            const int64_t o0 = ((int64_t)b * UC * Ho + oy) * Ho + ox, plane = (int64_t)Ho * Ho;
#pragma unroll
                            for (int o = 0; o < UC; o++) gx[o0 + o * plane] = ((pm >> o) & 1u) ? v[o] : 0.f;
                        }
                    }
                }
            }
        }
        if (!have || bad) break;
        prev = tile;
    }
    umma_teardown<COLS>(tmem);
}

// Weight gradient of a 32 -> 32 layer (stride S) on the tensor cores:
//   gW[o][c][dy][dx] = sum_p gz[o][p] in_pad[c][S y + dy][S x + dx],
// the sum over all output pixels p = (y, x) of the batch, as GEMMs with the
// pixels as the reduction: for every output row y of a tile of WG_TH x WG_TW
// pixels and every dy, one MMA with K = the row's 16 pixels,
//   D_dy[o][(dx, c)] += A[o][k] B_dy[(dx, c)][k],   M = 128, N = 96,
// A = the output gradient (BF16; rows 32..127 read padding, so lanes 32..127
// of D are unused), B_dy = the input row S y + dy at the columns S x + dx - 1.
// Both operands are K-major core matrices staged by the CTA's threads:
//   A: [tile row][k half][8-channel group of o][8 o x 8 pixels], 1536 B of
//      padding after it for the unused rows;
//   B: [dx, 8-channel group of c][input row of the tile][k half][8 c x 8
//      pixels], one copy per dx (so that every MMA reads 16-byte aligned core
//      matrices), from the planar BF16 input.
// The three accumulators D_0, D_1, D_2 take TMEM columns 0, 96 and 192, so
// column 32 (3 dy + dx) + c holds tap (dy, dx) of channel c.  The CTA walks
// its tiles (tile = block + k grid) with two staging buffers, so that the MMAs
// of one tile run while the next is staged; the bias sums (of the unrounded
// FP32 gradient) are formed from the staging registers.  Each CTA writes one
// record in the parameter layout ((o 32 + c) 9 + tap, then the 32 biases);
// k_wgrad_umma_reduce adds the records in block order.
constexpr int WG_TH = 8, WG_TW = 16, WG_N = 96, WG_COLS = 512;
constexpr int WG_REC = UC * UC * 9 + UC;

template <int S>
struct WgSmem {
    static constexpr int ir = S * (WG_TH - 1) + 3;      // input rows of a tile
    static constexpr int a_bytes = WG_TH * 1024 + 1536;  // 8 rows x 2 halves x 4 groups x 128 B + padding
    static constexpr int b_bytes = 12 * ir * 256;        // 12 groups x rows x 2 halves x 128 B
    static constexpr int a0 = 0, b0 = 2 * a_bytes;
    static constexpr int bars = b0 + 2 * b_bytes;        // MMA done, per buffer
    static constexpr int taddr = bars + 16;
    static constexpr int red = taddr + 16;               // bias sums: [warp][8 o][4 groups]
    static constexpr int bytes = red + 8 * 8 * 4 * 4;
    static_assert(a_bytes % 128 == 0 && b_bytes % 128 == 0, "core matrices 16-byte aligned");
};

template <int S>
__global__ void __launch_bounds__(256, 1) k_wgrad32_umma(const uint4 *__restrict__ in, int H,
                                                         const float *__restrict__ gz, int Ho, int tiles_x,
                                                         int tiles_y, int n_tiles, float *__restrict__ part,
                                                         int *__restrict__ err)
{
    using SM = WgSmem<S>;
    constexpr int IR = SM::ir, NB = (96 * IR + 255) / 256;
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t s_base = smem_u32(smem), bar_mma = s_base + SM::bars;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_base + SM::taddr),
                     "r"(WG_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bar_mma, 1);
        mbar_init(bar_mma + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(smem + SM::taddr);
    // A items: jp = pixel pair, r = o % 8 (consecutive lanes: conflict-free
    // stores), then k half, tile row and group og = o / 8 (= slot k / 2)
    const int a_jp = tid & 3, a_r = (tid >> 2) & 7;
    float bsum[4] = {0.f, 0.f, 0.f, 0.f};
    int bad = 0, it = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
        const int buf = it & 1;
        int b, ty, tx;
        tile_coords(tile, tiles_x, tiles_y, b, ty, tx);
        const int oy0 = ty * WG_TH, ox0 = tx * WG_TW;
        // the gradient's and the input's values of this tile, loaded before
        // the buffer is free
        float2 av[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int item = tid + 256 * k, kap = (item >> 5) & 1, y = (item >> 6) & 7, o = 8 * (item >> 9) + a_r;
            const int oy = oy0 + y, ox = ox0 + 8 * kap + 2 * a_jp;
            float2 v = make_float2(0.f, 0.f);
            if (oy < Ho) {
                const float *row = gz + (((int64_t)b * UC + o) * Ho + oy) * Ho;
                if (ox < Ho) v.x = row[ox];
                if (ox + 1 < Ho) v.y = row[ox + 1];
            }
            av[k] = v;
        }
        uint4 q0[NB], q1[NB];
#pragma unroll
        for (int k = 0; k < NB; k++) {
            const int item = tid + 256 * k, jp = item & 3, kap = (item >> 2) & 1, r2 = item >> 3;
            const int ir = r2 % IR, g = r2 / IR, dx = g >> 2, cg = g & 3;
            const int iy = S * oy0 - 1 + ir, x = ox0 + 8 * kap + 2 * jp;
            const int ix0 = S * x + dx - 1, ix1 = S * (x + 1) + dx - 1;
            q0[k] = q1[k] = make_uint4(0u, 0u, 0u, 0u);
            if (item < 96 * IR && iy >= 0 && iy < H) {
                const uint4 *row = in + ((int64_t)(4 * b + cg) * H + iy) * H;
                if (ix0 >= 0 && ix0 < H) q0[k] = row[ix0];
                if (ix1 >= 0 && ix1 < H) q1[k] = row[ix1];
            }
        }
        if (it >= 2) {
            // the MMAs of tile it - 2 have read this buffer
            const bool ok = bad ? true : mbar_wait(bar_mma + 8 * buf, ((it - 2) >> 1) & 1);
            if (!ok) *reinterpret_cast<volatile int *>(err) = 3;
            bad = __syncthreads_or(!ok || bad);
            if (bad) break;
        }
        uint8_t *abuf = smem + SM::a0 + buf * SM::a_bytes;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int item = tid + 256 * k, kap = (item >> 5) & 1, y = (item >> 6) & 7, og = item >> 9;
            bsum[k >> 1] += av[k].x + av[k].y;
            *reinterpret_cast<uint32_t *>(abuf + ((y * 2 + kap) * 4 + og) * 128 + a_r * 16 + a_jp * 4) =
                pack2(av[k].x, av[k].y);
        }
        uint8_t *bbuf = smem + SM::b0 + buf * SM::b_bytes;
#pragma unroll
        for (int k = 0; k < NB; k++) {
            const int item = tid + 256 * k, jp = item & 3, kap = (item >> 2) & 1, r2 = item >> 3;
            if (item >= 96 * IR) continue;
            const int ir = r2 % IR, g = r2 / IR;
            uint8_t *cm = bbuf + ((g * IR + ir) * 2 + kap) * 128 + jp * 4;
            const uint32_t w0[4] = {q0[k].x, q0[k].y, q0[k].z, q0[k].w}, w1[4] = {q1[k].x, q1[k].y, q1[k].z, q1[k].w};
            // wd[c]: channel c of the two pixels (row c of the core matrix)
            uint32_t wd[8];
#pragma unroll
            for (int c = 0; c < 8; c++) wd[c] = __byte_perm(w0[c >> 1], w1[c >> 1], (c & 1) ? 0x7632 : 0x5410);
            // rotated by the lane group (rot = lane / 4), so that the 8 lane
            // groups of a store instruction write 8 different rows: 32 banks
            const int rot = lane >> 2;
#pragma unroll
            for (int sh = 1; sh < 8; sh <<= 1) {
                uint32_t t[8];
#pragma unroll
                for (int i = 0; i < 8; i++) t[i] = (rot & sh) ? wd[(i + sh) & 7] : wd[i];
#pragma unroll
                for (int i = 0; i < 8; i++) wd[i] = t[i];
            }
#pragma unroll
            for (int i = 0; i < 8; i++) *reinterpret_cast<uint32_t *>(cm + ((i + rot) & 7) * 16) = wd[i];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t abase = s_base + SM::a0 + buf * SM::a_bytes, bbase = s_base + SM::b0 + buf * SM::b_bytes;
#pragma unroll 1
            for (int y = 0; y < WG_TH; y++)
#pragma unroll
                for (int dy = 0; dy < 3; dy++)
                    umma_bf16<WG_N>(tmem + WG_N * dy, sdesc(abase + y * 1024, 512, 128),
                                    sdesc(bbase + (S * y + dy) * 256, 128, IR * 256), (it > 0 || y > 0) ? 1u : 0u);
            umma_commit(bar_mma + 8 * buf);
        }
    }
    // the last tile's MMAs (and so all of them) are done
    if (!bad && it > 0) {
        const int last = it - 1;
        const bool ok = mbar_wait(bar_mma + 8 * (last & 1), (last >> 1) & 1);
        if (!ok) *reinterpret_cast<volatile int *>(err) = 3;
        bad = __syncthreads_or(!ok);
    }
    float *rec = part + (int64_t)blockIdx.x * WG_REC;
    if (warp == 0) {
        // lane o of the accumulators: column 32 (3 dy + dx) + c = tap (dy, dx), channel c
        tc_fence_after();
#pragma unroll 1
        for (int tap = 0; tap < 9; tap++) {
            float v[UC];
            if (!bad && it > 0) tmem_ld<UC>(tmem + 32 * tap, v);
            else
#pragma unroll
                for (int c = 0; c < UC; c++) v[c] = 0.f;
#pragma unroll
            for (int c = 0; c < UC; c++) rec[(lane * UC + c) * 9 + tap] = v[c];
        }
    }
    // bias: the four lanes of a pixel-pair group, then the eight warps
    float *red = reinterpret_cast<float *>(smem + SM::red);
#pragma unroll
    for (int g = 0; g < 4; g++) {
        float v = bsum[g];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        if (a_jp == 0) red[(warp * 8 + a_r) * 4 + g] = v;
    }
    __syncthreads();
    if (tid < UC) {
        float sum = 0.f;
        for (int w = 0; w < 8; w++) sum += red[(w * 8 + (tid & 7)) * 4 + (tid >> 3)];
        rec[UC * UC * 9 + tid] = sum;
    }
    umma_teardown<WG_COLS>(tmem);
}

// grad[e] = the records' sum in block order, one thread per entry.
__global__ void k_wgrad_umma_reduce(const float *__restrict__ part, int nblk, float *__restrict__ grad)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= WG_REC) return;
    float s = 0.f;
    for (int k = 0; k < nblk; k++) s += part[(int64_t)k * WG_REC + e];
    grad[e] = s;
}

// cuTensorMapEncodeTiled from the driver, found once.
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// Tensor map of B planar BF16 images of side H: [b][cg][y][x][8], as
// (8 channels, x, y, 4 b + cg) with boxes of one halo tile (stride 1), or as
// (8 channels, x % 2, x / 2, y, 4 b + cg) with boxes of one column parity
// (stride 2; H even).
bool encode_input_map(CUtensorMap *map, const void *act, int H, int B, int S)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t row = 16ull * H, img = 16ull * H * H;
    const cuuint32_t one[5] = {1, 1, 1, 1, 1};
    CUresult r;
    if (S == 1) {
        const cuuint64_t dims[4] = {8, (cuuint64_t)H, (cuuint64_t)H, 4ull * B};
        const cuuint64_t strides[3] = {16, row, img};
        const cuuint32_t box[4] = {8, Halo<1>::cols, Halo<1>::rows, 4};
        r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(act), dims, strides, box, one,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        if (H % 2) return false;
        const cuuint64_t dims[5] = {8, 2, (cuuint64_t)H / 2, (cuuint64_t)H, 4ull * B};
        const cuuint64_t strides[4] = {16, 32, row, img};
        const cuuint32_t box[5] = {8, 1, Halo<2>::cols, Halo<2>::rows, 4};
        r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(act), dims, strides, box, one,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS;
}

// Launch shape: one CTA per tile up to the resident CTAs of every SM (by
// shared memory, and at most 512 / cols so that the TMEM allocations of the
// resident CTAs fit the SM's 512 columns and never wait on one another).
template <typename K>
bool grid_for(K kern, int bytes, int cols, int n_tiles, int &grid)
{
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
            cudaSuccess)
        return false;
    int dev = 0, nsm = 0, smem_sm = 0, smem_rsv = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
        return false;
    const int per_sm = std::max(1, std::min(std::min(512 / cols, 16), smem_sm / (bytes + smem_rsv)));
    grid = std::min(n_tiles, nsm * per_sm);
    return true;
}

template <int S, int N, int NR, bool RELU, bool OUT_F32>
reg_status launch_fwd(const uint16_t *in, int H, const float *theta, void *out, int B, cudaStream_t st,
                      uint32_t *wpack, bool pack, int *err)
{
    CUtensorMap map;
    if (!encode_input_map(&map, in, H, B, S))
        return reg_internal_fail(REG_ECUDA, "tcgen05 convolution: tensor map of the input");
    if (pack) k_pack_umma<false, N, NR><<<(Wts<N>::bytes / 4 + 255) / 256, 256, 0, st>>>(theta, wpack);
    const int Ho = (H + 2 - 3) / S + 1;
    const int tx = (Ho + UTW - 1) / UTW, ty = (Ho + UTH - 1) / UTH, nt = B * tx * ty;
    auto kern = k_conv_umma_ws<S, N, NR, RELU, OUT_F32>;
    constexpr int bytes = WsSmem<S, N>::bytes;
    int grid = 0;
    if (!grid_for(kern, bytes, tmem_cols<N>(), nt, grid))
        return reg_internal_fail(REG_ECUDA, "tcgen05 convolution: launch attributes");
    kern<<<grid, 192, bytes, st>>>(map, theta + NR * UC * 9, wpack, out, Ho, tx, ty, nt, err);
    if (cudaGetLastError() != cudaSuccess) return reg_internal_fail(REG_ECUDA, "tcgen05 convolution launch");
    return REG_OK;
}

}  // namespace

int cnn_conv32_umma_words() { return Wts<UC>::bytes / 4; }

reg_status cnn_conv32_umma(const uint16_t *in, int H, const float *theta, void *out, bool out_f32, int B, int S,
                           cudaStream_t st, uint32_t *wpack, bool pack, int *err)
{
    if (S == 1)
        return out_f32 ? launch_fwd<1, UC, UC, true, true>(in, H, theta, out, B, st, wpack, pack, err)
                       : launch_fwd<1, UC, UC, true, false>(in, H, theta, out, B, st, wpack, pack, err);
    if (S == 2)
        return out_f32 ? launch_fwd<2, UC, UC, true, true>(in, H, theta, out, B, st, wpack, pack, err)
                       : launch_fwd<2, UC, UC, true, false>(in, H, theta, out, B, st, wpack, pack, err);
    return reg_internal_fail(REG_EINVAL, "tcgen05 convolution: stride must be 1 or 2");
}

reg_status cnn_last_umma(const uint16_t *in, int H, const float *theta, float *out, int B, cudaStream_t st,
                         uint32_t *wpack, bool pack, int *err)
{
    return launch_fwd<1, 16, 2, false, true>(in, H, theta, out, B, st, wpack, pack, err);
}

reg_status cnn_first_umma(const float *x, int H, const float *theta, uint16_t *out, int B, cudaStream_t st,
                          uint32_t *wpack, bool pack, int *err)
{
    if (H % 2) return reg_internal_fail(REG_EINVAL, "tcgen05 first layer: odd input side");
    if (pack) k_pack_l0<<<(L0_WBYTES / 4 + 255) / 256, 256, 0, st>>>(theta, wpack);
    const int Ho = (H + 2 - 3) / 2 + 1;
    const int tx = (Ho + UTW - 1) / UTW, ty = (Ho + UTH - 1) / UTH, nt = B * tx * ty;
    int grid = 0;
    if (!grid_for(k_conv_umma_staged<ST_FIRST>, L0Smem::bytes, staged_cols<ST_FIRST>(), nt, grid))
        return reg_internal_fail(REG_ECUDA, "tcgen05 first layer: launch attributes");
    k_conv_umma_staged<ST_FIRST><<<grid, 128, L0Smem::bytes, st>>>(x, H, wpack, theta + UC * 2 * 9, nullptr, out, Ho, tx,
                                                               ty, nt, err);
    if (cudaGetLastError() != cudaSuccess) return reg_internal_fail(REG_ECUDA, "tcgen05 first layer launch");
    return REG_OK;
}

reg_status cnn_dgrad32_umma(const float *gz, int H, const float *theta, const uint16_t *mask, float *gx, int B,
                            cudaStream_t st, uint32_t *wpack, bool pack, int *err)
{
    if (pack) k_pack_umma<true, UC, UC><<<(Wts<UC>::bytes / 4 + 255) / 256, 256, 0, st>>>(theta, wpack);
    const int tx = (H + UTW - 1) / UTW, ty = (H + UTH - 1) / UTH, nt = B * tx * ty;
    int grid = 0;
    if (!grid_for(k_conv_umma_staged<ST_DGRAD1>, DgradSmem::bytes, staged_cols<ST_DGRAD1>(), nt, grid))
        return reg_internal_fail(REG_ECUDA, "tcgen05 data gradient: launch attributes");
    k_conv_umma_staged<ST_DGRAD1><<<grid, 128, DgradSmem::bytes, st>>>(gz, H, wpack, nullptr,
                                                                   reinterpret_cast<const uint4 *>(mask), gx, H, tx,
                                                                   ty, nt, err);
    if (cudaGetLastError() != cudaSuccess) return reg_internal_fail(REG_ECUDA, "tcgen05 data gradient launch");
    return REG_OK;
}

reg_status cnn_dgrad32s2_umma(const float *gz, int Hg, const float *theta, const uint16_t *mask, float *gx, int B,
                              cudaStream_t st, uint32_t *wpack, bool pack, int *err)
{
    if (pack) k_pack_umma<true, UC, UC><<<(Wts<UC>::bytes / 4 + 255) / 256, 256, 0, st>>>(theta, wpack);
    const int tx = (Hg + UTW - 1) / UTW, ty = (Hg + UTH - 1) / UTH, nt = B * tx * ty;
    int grid = 0;
    if (!grid_for(k_conv_umma_staged<ST_DGRAD2>, DgradSmem::bytes, staged_cols<ST_DGRAD2>(), nt, grid))
        return reg_internal_fail(REG_ECUDA, "tcgen05 stride-2 data gradient: launch attributes");
    k_conv_umma_staged<ST_DGRAD2><<<grid, 128, DgradSmem::bytes, st>>>(gz, Hg, wpack, nullptr,
                                                                     reinterpret_cast<const uint4 *>(mask), gx,
                                                                     2 * Hg, tx, ty, nt, err);
    if (cudaGetLastError() != cudaSuccess) return reg_internal_fail(REG_ECUDA, "tcgen05 stride-2 data gradient launch");
    return REG_OK;
}

namespace {

template <int S>
reg_status launch_wgrad_umma(const uint16_t *in, int H, const float *gz, int B, float *grad, float *part,
                             cudaStream_t st, int *err)
{
    const int Ho = (H + 2 - 3) / S + 1;
    const int tx = (Ho + WG_TW - 1) / WG_TW, ty = (Ho + WG_TH - 1) / WG_TH, nt = B * tx * ty;
    int grid = 0;
    if (!grid_for(k_wgrad32_umma<S>, WgSmem<S>::bytes, WG_COLS, nt, grid))
        return reg_internal_fail(REG_ECUDA, "tcgen05 weight gradient: launch attributes");
    k_wgrad32_umma<S><<<grid, 256, WgSmem<S>::bytes, st>>>(reinterpret_cast<const uint4 *>(in), H, gz, Ho, tx, ty, nt,
                                                          part, err);
    k_wgrad_umma_reduce<<<(WG_REC + 255) / 256, 256, 0, st>>>(part, grid, grad);
    if (cudaGetLastError() != cudaSuccess) return reg_internal_fail(REG_ECUDA, "tcgen05 weight gradient launch");
    return REG_OK;
}

}  // namespace

reg_status cnn_wgrad32_umma(const uint16_t *in, int H, const float *gz, int B, int S, float *grad, float *part,
                            cudaStream_t st, int *err)
{
    if (S == 1) return launch_wgrad_umma<1>(in, H, gz, B, grad, part, st, err);
    if (S == 2) return launch_wgrad_umma<2>(in, H, gz, B, grad, part, st, err);
    return reg_internal_fail(REG_EINVAL, "tcgen05 weight gradient: stride must be 1 or 2");
}

int cnn_wgrad32_umma_part_floats()
{
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        nsm = 152;
    return nsm * WG_REC;
}

int cnn_last_umma_words() { return Wts<16>::bytes / 4; }
int cnn_first_umma_words() { return L0_WBYTES / 4; }
