// CUDA kernels of libreg (sm_103a).
//
// Grid conventions: level l is the vertex grid of n = 2^l + 1 nodes per side;
// node (r, c) is row r (x_1), column c (x_0).  Displacements are kept in grid
// units of their level (1 unit = one node spacing h = 2^-l), which keeps the
// sub-node position of a sample exact in float: the integer node index and the
// small displacement are split before they are added.  Frames are stored
// normalised per level (FE mean 0, FE standard deviation 1): NCC is invariant
// under affine changes of either image and bilinear interpolation commutes
// with them, so the energy and its gradient are those of the raw frames.
//
// Energies are sums over cells of the Q1 element integrals (exact FE mass and
// stiffness forms); per-cell values are float, per-warp and per-tile sums
// float, and the per-operator sum over tiles is double (the global energy and
// normalisation reductions that the Armijo test compares).
#include <algorithm>

#include "reg_common.cuh"

namespace {

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <bool BF16>
__device__ __forceinline__ float ldimg(const void *p, int idx)
{
    if constexpr (BF16) {
        unsigned short raw = __ldg(reinterpret_cast<const unsigned short *>(p) + idx);
        return __uint_as_float(((unsigned)raw) << 16);
    } else {
        return __ldg(reinterpret_cast<const float *>(p) + idx);
    }
}

// Bilinear interpolant of a nodal image at grid point (c + vx, r + vy),
// clamped to the grid [0, n-1]^2 (= Omega).  Cell index floor(x), capped at
// n-2 (the right/top cell on the last node line).  Derivatives in grid units,
// zero in a clamped coordinate.
template <bool BF16, bool GRAD>
__device__ __forceinline__ float sample(const void *img, int n, int pitch, int c, int r, float vx, float vy,
                                        float *gx, float *gy)
{
    float fx = floorf(vx), fy = floorf(vy);
    int jx = c + (int)fx, jy = r + (int)fy;
    float ax = vx - fx, ay = vy - fy;
    bool clx = false, cly = false;
    if (jx < 0) {
        jx = 0; ax = 0.f; clx = true;
    } else if (jx >= n - 1) {
        clx = (jx > n - 1) || (ax > 0.f);
        jx = n - 2; ax = 1.f;
    }
    if (jy < 0) {
        jy = 0; ay = 0.f; cly = true;
    } else if (jy >= n - 1) {
        cly = (jy > n - 1) || (ay > 0.f);
        jy = n - 2; ay = 1.f;
    }
    int i0 = jy * pitch + jx;
    float t00 = ldimg<BF16>(img, i0), t01 = ldimg<BF16>(img, i0 + 1);
    float t10 = ldimg<BF16>(img, i0 + pitch), t11 = ldimg<BF16>(img, i0 + pitch + 1);
    float v = (1.f - ay) * ((1.f - ax) * t00 + ax * t01) + ay * ((1.f - ax) * t10 + ax * t11);
    if constexpr (GRAD) {
        *gx = clx ? 0.f : (1.f - ay) * (t01 - t00) + ay * (t11 - t10);
        *gy = cly ? 0.f : (1.f - ax) * (t10 - t00) + ax * (t11 - t01);
    }
    return v;
}

// sample() at a compensated displacement (exact cell choice at cell lines).
template <bool BF16, bool GRAD>
__device__ __forceinline__ float sample_df(const void *img, int n, int pitch, int c, int r, float4 u, float *gx,
                                           float *gy)
{
    int ix, iy;
    float ax, ay;
    df_split(u.x, u.z, ix, ax);
    df_split(u.y, u.w, iy, ay);
    int jx = c + ix, jy = r + iy;
    bool clx = false, cly = false;
    if (jx < 0) {
        jx = 0; ax = 0.f; clx = true;
    } else if (jx >= n - 1) {
        clx = (jx > n - 1) || (ax > 0.f);
        jx = n - 2; ax = 1.f;
    }
    if (jy < 0) {
        jy = 0; ay = 0.f; cly = true;
    } else if (jy >= n - 1) {
        cly = (jy > n - 1) || (ay > 0.f);
        jy = n - 2; ay = 1.f;
    }
    int i0 = jy * pitch + jx;
    float t00 = ldimg<BF16>(img, i0), t01 = ldimg<BF16>(img, i0 + 1);
    float t10 = ldimg<BF16>(img, i0 + pitch), t11 = ldimg<BF16>(img, i0 + pitch + 1);
    float v = (1.f - ay) * ((1.f - ax) * t00 + ax * t01) + ay * ((1.f - ax) * t10 + ax * t11);
    if constexpr (GRAD) {
        *gx = clx ? 0.f : (1.f - ay) * (t01 - t00) + ay * (t11 - t10);
        *gy = cly ? 0.f : (1.f - ax) * (t10 - t00) + ax * (t11 - t01);
    }
    return v;
}

// Bilinear interpolant of a float2 field (for composition), clamped.
__device__ __forceinline__ float2 sample2(const float2 *f, int n, int pitch, int c, int r, float vx, float vy)
{
    float fx = floorf(vx), fy = floorf(vy);
    int jx = c + (int)fx, jy = r + (int)fy;
    float ax = vx - fx, ay = vy - fy;
    if (jx < 0) { jx = 0; ax = 0.f; } else if (jx >= n - 1) { jx = n - 2; ax = 1.f; }
    if (jy < 0) { jy = 0; ay = 0.f; } else if (jy >= n - 1) { jy = n - 2; ay = 1.f; }
    int i0 = jy * pitch + jx;
    float2 a = f[i0], b = f[i0 + 1], cc = f[i0 + pitch], d = f[i0 + pitch + 1];
    float2 o;
    o.x = (1.f - ay) * ((1.f - ax) * a.x + ax * b.x) + ay * ((1.f - ax) * cc.x + ax * d.x);
    o.y = (1.f - ay) * ((1.f - ax) * a.y + ax * b.y) + ay * ((1.f - ax) * cc.y + ax * d.y);
    return o;
}

__device__ __forceinline__ int find_entry(const int *pref, int nent, int item)
{
    // largest e with pref[e] <= item
    int lo = 0, hi = nent - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(pref + mid) <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace

// ---------------------------------------------------------------------------
// Pyramid construction
// ---------------------------------------------------------------------------

// Frame (side x side px, pitch in elements) -> level-L vertex grid; last row
// and column repeated.  grid: (x tiles, y tiles, frames).
__global__ void k_embed(const float *__restrict__ frames, int64_t frame_stride, int64_t pitch, int side,
                        float *__restrict__ out, int64_t out_stride, int out_pitch)
{
    int f = blockIdx.z;
    int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    int n = side + 1;
    if (r >= n || c >= n) return;
    int rr = r < side ? r : side - 1, cc = c < side ? c : side - 1;
    out[f * out_stride + (int64_t)r * out_pitch + c] = frames[f * frame_stride + (int64_t)rr * pitch + cc];
}

// Restriction 1/16 [1 2 1; 2 4 2; 1 2 1] with mirrored boundary.
// grid: (x tiles, y tiles, items); fine/coarse images of item z at
// fine + z*fstride, coarse + z*cstride.
__global__ void k_restrict_img(const float *__restrict__ fine, int64_t fstride, int fpitch, int nf,
                               float *__restrict__ coarse, int64_t cstride, int cpitch)
{
    int z = blockIdx.z;
    int nc = (nf + 1) / 2;
    int J = blockIdx.x * blockDim.x + threadIdx.x, I = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= nc || J >= nc) return;
    const float *F = fine + z * fstride;
    const float w[3] = {0.25f, 0.5f, 0.25f};
    float s = 0.f;
#pragma unroll
    for (int a = -1; a <= 1; a++) {
        int r = 2 * I + a;
        r = r < 0 ? -r : (r > nf - 1 ? 2 * (nf - 1) - r : r);
#pragma unroll
        for (int b = -1; b <= 1; b++) {
            int c = 2 * J + b;
            c = c < 0 ? -c : (c > nf - 1 ? 2 * (nf - 1) - c : c);
            s += w[a + 1] * w[b + 1] * F[(int64_t)r * fpitch + c];
        }
    }
    coarse[z * cstride + (int64_t)I * cpitch + J] = s;
}

// Per image: FE mean (w^T F) and FE standard deviation ((F-mean)^T M (F-mean))^1/2,
// two passes over the cells, summed in double.  Each image's cell rows are cut into
// STATS_SPLIT parts, one block each (grid: parts, images); the parts' sums
// go to `part` and are added in order by k_image_stats_fin (deterministic).
constexpr int STATS_SPLIT = 32;

__device__ __forceinline__ double block_sum_d(double v, double *red)
{
    v = warp_sum_d(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
    __syncthreads();
    return t;
}

// pass 0: sum of the cell means; pass 1: sum of the cell mass forms of F - mean
__global__ void k_image_stats_part(const float *__restrict__ img, int64_t stride, int pitch, int n, int pass,
                                   const double *__restrict__ stats, double *__restrict__ part)
{
    const float *F = img + blockIdx.y * stride;
    __shared__ double red[32];
    const int rows = n - 1, per = (rows + STATS_SPLIT - 1) / STATS_SPLIT;
    const int r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
    // each cell's term in FP32, their sum in FP64 (GB300's FP64 rate is a
    // small fraction of its FP32 rate).  Pass 1 centres on the FP64 mean
    // rounded to FP32: the cell form's linear term in that offset sums to
    // zero (M 1 = w and sum w (F - mean) = 0), so only its square, ~1e-14 of
    // the variance, remains.
    // (a thread adds its few cells of a row in FP32, then the row's share in
    // FP64)
    const float mf = pass ? (float)stats[2 * blockIdx.y] : 0.f;
    double s = 0.0;
    for (int r = r0; r < r1; r++) {
        const float *row = F + (int64_t)r * pitch;
        float rs = 0.f;
        for (int c = threadIdx.x; c < n - 1; c += blockDim.x) {
            const float *p = row + c;
            if (!pass) {
                rs += 0.25f * ((p[0] + p[1]) + (p[pitch] + p[pitch + 1]));
            } else {
                const float a = p[0] - mf, b = p[1] - mf, cc = p[pitch + 1] - mf, d = p[pitch] - mf;  // cyclic
                rs += 4.f * (a * a + b * b + cc * cc + d * d) + 4.f * (a * b + b * cc + cc * d + d * a) +
                      2.f * (a * cc + b * d);
            }
        }
        s += (double)rs;
    }
    const double t = block_sum_d(s, red) * (pass ? 1.0 / 36.0 : 1.0);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * STATS_SPLIT + blockIdx.x] = t;
}

// One thread per image: the parts in order; pass 0 writes the mean, pass 1 sigma.
__global__ void k_image_stats_fin(int n_img, int n, int pass, const double *__restrict__ part, double *__restrict__ out)
{
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= n_img) return;
    double t = 0.0;
    for (int k = 0; k < STATS_SPLIT; k++) t += part[(int64_t)z * STATS_SPLIT + k];
    const double h2 = 1.0 / ((double)(n - 1) * (n - 1));
    if (!pass) out[2 * z] = t * h2;
    else out[2 * z + 1] = sqrt(t * h2);
}

void launch_image_stats(const float *img, int64_t stride, int pitch, int n, int n_img, double *part, double *out,
                        cudaStream_t st)
{
    for (int pass = 0; pass < 2; pass++) {
        k_image_stats_part<<<dim3(STATS_SPLIT, n_img), 256, 0, st>>>(img, stride, pitch, n, pass, out, part);
        k_image_stats_fin<<<(n_img + 127) / 128, 128, 0, st>>>(n_img, n, pass, part, out);
    }
}

int image_stats_part_doubles(int n_img) { return n_img * STATS_SPLIT; }

// F~ = (F - mean) / sigma into float or bf16 storage. grid (x, y, images).
__global__ void k_normalize(const float *__restrict__ img, int64_t stride, int pitch, int n, const double *stats,
                            void *out, int64_t ostride, int opitch, int bf16)
{
    int z = blockIdx.z;
    int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= n || c >= n) return;
    double m = stats[2 * z], s = stats[2 * z + 1];
    float v = (float)(((double)img[z * stride + (int64_t)r * pitch + c] - m) / s);
    int64_t o = z * ostride + (int64_t)r * opitch + c;
    if (bf16) reinterpret_cast<__nv_bfloat16 *>(out)[o] = __float2bfloat16_rn(v);
    else reinterpret_cast<float *>(out)[o] = v;
}

// M~ R~ of normalised frames at one level: the FE mass matrix in units of h^2,
// M1 (x) M1 with the 1D weights 1/6, 4/6, 1/6 (2/6 on the diagonal at the
// border), applied to the stored (float or bf16) image.  The weights are taken
// as the integers 36 M~ and the sum is divided by 36 once, so that no rounded
// weight biases every node the same way.  The gradient and trial passes take
// the NCC terms int R~ phi_i from it.
__global__ void k_mass_image(const void *img, int64_t stride, int pitch, int n, int bf16, float *out,
                             int64_t ostride)
{
    int z = blockIdx.z;
    int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= n || c >= n) return;
    const void *f = bf16 ? (const void *)(reinterpret_cast<const __nv_bfloat16 *>(img) + z * stride)
                         : (const void *)(reinterpret_cast<const float *>(img) + z * stride);
    auto w6 = [n](int i, int a) { return a == 0 ? ((i == 0 || i == n - 1) ? 2.f : 4.f) : 1.f; };
    float acc = 0.f;
    for (int a = -1; a <= 1; a++) {
        if (r + a < 0 || r + a >= n) continue;
        float row = 0.f;
        for (int bb = -1; bb <= 1; bb++) {
            if (c + bb < 0 || c + bb >= n) continue;
            const int i = (r + a) * pitch + (c + bb);
            row += w6(c, bb) * (bf16 ? ldimg<true>(f, i) : ldimg<false>(f, i));
        }
        acc += w6(r, a) * row;
    }
    out[z * ostride + (int64_t)r * pitch + c] = acc / 36.f;
}

// ---------------------------------------------------------------------------
// Operator initialisation: composition and restriction of the initial guess
// ---------------------------------------------------------------------------

// init 1: U0 = left; init 2: U0(x) = left(x) + right(x + left(x)) (phi_jk o phi_ij,
// right sampled bilinearly, clamped).  grid: (x tiles, y tiles, ops).
__global__ void k_compose(BatchDev b)
{
    const OpDesc &op = b.ops[blockIdx.z];
    if (op.init == 0) return;
    const LevelDesc &L = op.lv[op.nl - 1];
    int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= L.n || c >= L.n) return;
    float2 a = op.left[(int64_t)r * op.slot_pitch + c];
    if (op.init == 2) {
        float2 q = sample2(op.right, L.n, op.slot_pitch, c, r, a.x, a.y);
        a.x += q.x;
        a.y += q.y;
    }
    L.V[0][(int64_t)r * L.pitch + c].u = make_float4(a.x, a.y, 0.f, 0.f);
}

// Restrict U0 from level index k+1 to k (grid units halve).  grid (x, y, ops).
__global__ void k_restrict_u(BatchDev b, int step)
{
    const OpDesc &op = b.ops[blockIdx.z];
    int k = op.nl - 1 - step;  // destination level index
    if (op.init == 0 || k < 0) return;
    const LevelDesc &C = op.lv[k], &F = op.lv[k + 1];
    int J = blockIdx.x * blockDim.x + threadIdx.x, I = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= C.n || J >= C.n) return;
    int nf = F.n;
    const float w[3] = {0.25f, 0.5f, 0.25f};
    float sx = 0.f, sy = 0.f;
#pragma unroll
    for (int a = -1; a <= 1; a++) {
        int r = 2 * I + a;
        r = r < 0 ? -r : (r > nf - 1 ? 2 * (nf - 1) - r : r);
#pragma unroll
        for (int bb = -1; bb <= 1; bb++) {
            int c = 2 * J + bb;
            c = c < 0 ? -c : (c > nf - 1 ? 2 * (nf - 1) - c : c);
            float4 v = F.V[0][(int64_t)r * F.pitch + c].u;
            float ww = w[a + 1] * w[bb + 1];
            sx += ww * v.x;
            sy += ww * v.y;
        }
    }
    C.V[0][(int64_t)I * C.pitch + J].u = make_float4(0.5f * sx, 0.5f * sy, 0.f, 0.f);
}

// Identity initial guess: zero U0 on the coarsest level.  grid (x, y, ops).
__global__ void k_zero_u(BatchDev b)
{
    const OpDesc &op = b.ops[blockIdx.z];
    if (op.init != 0) return;
    const LevelDesc &C = op.lv[0];
    int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= C.n || c >= C.n) return;
    C.V[0][(int64_t)r * C.pitch + c].u = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_init_state(BatchDev b, int n_ops)
{
    int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_ops) return;
    OpState s;
    memset(&s, 0, sizeof(s));
    s.phase = PH_START;
    s.lvl = 0;
    s.cur = 0;
    s.src = 0;
    s.tau = b.tau_init;
    s.status = OPST_CONVERGED;
    b.st[o] = s;
}

// ---------------------------------------------------------------------------
// Work planning: compacted per-family op lists and tile prefix sums
// ---------------------------------------------------------------------------

// work items per operator: prolongation block tiles, gradient and trial strip tiles
__device__ __forceinline__ int node_tiles(int n) { return ((n + REG_TX - 1) / REG_TX) * ((n + REG_TY - 1) / REG_TY); }
__device__ __forceinline__ int grad_tiles(const LevelDesc &L)
{
    return ((L.n + REG_GW - 1) / REG_GW) * ((L.n + L.hg - 1) / L.hg);
}
__device__ __forceinline__ int trial_tiles(const LevelDesc &L)
{
    return ((L.n - 1 + REG_CW - 1) / REG_CW) * ((L.n - 1 + L.ht - 1) / L.ht);
}

// Block-wide exclusive scan of one int per thread (blockDim.x == 1024).
__device__ int block_excl_scan(int v, int *tmp, int *total)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = tmp[lane];
        int s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        tmp[lane] = s - t;
        if (lane == 31) tmp[32] = s;
    }
    __syncthreads();
    int res = x - v + tmp[w];
    *total = tmp[32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(1024) k_plan(BatchDev b)
{
    __shared__ int tmp[33];
    int n_ops = b.ctr[0];
    int offE[3] = {0, 0, 0}, offI[3] = {0, 0, 0};
    int active = 0;
    for (int base = 0; base < n_ops; base += 1024) {
        int o = base + threadIdx.x;
        int inP = 0, inG = 0, inT = 0, tP = 0, tG = 0, tT = 0;
        if (o < n_ops) {
            const OpState &s = b.st[o];
            const OpDesc &op = b.ops[o];
            const LevelDesc &L = op.lv[s.lvl];
            if (s.phase != PH_DONE) active++;
            if (s.phase == PH_PROLONG || s.phase == PH_FINAL) { inP = 1; tP = node_tiles(L.n); }
            if (s.phase == PH_GRAD) { inG = 1; tG = grad_tiles(L); }
            if (s.phase == PH_START || s.phase == PH_GRAD || s.phase == PH_TRIAL || s.phase == PH_PROLONG) {
                inT = 1; tT = trial_tiles(L);
            }
        }
        int tot;
        int eP = block_excl_scan(inP, tmp, &tot); int nP = tot;
        int eG = block_excl_scan(inG, tmp, &tot); int nG = tot;
        int eT = block_excl_scan(inT, tmp, &tot); int nT = tot;
        int iP = block_excl_scan(tP, tmp, &tot); int sP = tot;
        int iG = block_excl_scan(tG, tmp, &tot); int sG = tot;
        int iT = block_excl_scan(tT, tmp, &tot); int sT = tot;
        if (o < n_ops) {
            OpState &s = b.st[o];
            if (inP) { b.listP[offE[0] + eP] = o; b.prefP[offE[0] + eP] = offI[0] + iP; }
            if (inG) { b.listG[offE[1] + eG] = o; b.prefG[offE[1] + eG] = offI[1] + iG; s.g_entry = offE[1] + eG; }
            if (inT) { b.listT[offE[2] + eT] = o; b.prefT[offE[2] + eT] = offI[2] + iT; }
            s.g_begin = offI[1] + iG; s.g_end = s.g_begin + tG;
            s.t_begin = offI[2] + iT; s.t_end = s.t_begin + tT;
        }
        offE[0] += nP; offE[1] += nG; offE[2] += nT;
        offI[0] += sP; offI[1] += sG; offI[2] += sT;
    }
    // active ops
    int tot;
    block_excl_scan(active, tmp, &tot);
    if (threadIdx.x == 0) {
        b.prefP[offE[0]] = offI[0];
        b.prefG[offE[1]] = offI[1];
        b.prefT[offE[2]] = offI[2];
        b.ctr[1] = offE[0]; b.ctr[2] = offE[1]; b.ctr[3] = offE[2];
        b.ctr[4] = offI[0]; b.ctr[5] = offI[1]; b.ctr[6] = offI[2];
        b.ctr[7] = tot;
    }
}

// ---------------------------------------------------------------------------
// Work distribution of the step kernels: a fixed grid, each block takes one
// contiguous range of the step's work items (tiles of 32 x 32 nodes or
// cells), so that it locates its first op once and then walks forward.
// ---------------------------------------------------------------------------
namespace {

struct ItemWalker {
    const int *pref;
    int e, e_end;
    __device__ ItemWalker(const int *p, int nent, int first) : pref(p)
    {
        e = find_entry(p, nent, first);
        e_end = __ldg(p + e + 1);
    }
    // entry (index into the compacted op list) of a work item >= the previous one
    __device__ int entry(int item)
    {
        while (item >= e_end) {
            e++;
            e_end = __ldg(pref + e + 1);
        }
        return e;
    }
};

__device__ __forceinline__ void block_range(int items, int &b0, int &b1)
{
    int per = (items + gridDim.x - 1) / gridDim.x;
    b0 = blockIdx.x * per;
    b1 = min(items, b0 + per);
}

}  // namespace

// ---------------------------------------------------------------------------
// P: apply the pending step and prolongate to the next level (or write the
// finest-level result into the destination slot).  Tile: 32 x 32 fine nodes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(REG_THREADS, 4) k_prolong(BatchDev b)
{
    int nent = b.ctr[1], items = b.ctr[4];
    int b0, b1;
    block_range(items, b0, b1);
    if (b0 >= b1) return;
    ItemWalker wk(b.prefP, nent, b0);
    const int lx = threadIdx.x % REG_TX, ly = threadIdx.x / REG_TX;
    for (int item = b0; item < b1; item++) {
        int e = wk.entry(item);
        int o = b.listP[e];
        int t = item - b.prefP[e];
        const OpState &s = b.st[o];
        const OpDesc &op = b.ops[o];
        const LevelDesc &Lv = op.lv[s.lvl];
        const int n = Lv.n, tx = (n + REG_TX - 1) / REG_TX;
        const int r0 = (t / tx) * REG_TY, c = (t % tx) * REG_TX + lx;
        const float tau = (float)s.tau_acc;
        const bool fin = (s.phase == PH_FINAL);
        float corr = 0.f;  // judged ops: |final - learned start| over this thread's nodes
#pragma unroll
        for (int k = 0; k < REG_RPT; k++) {
            const int r = r0 + ly + k * REG_ROWSTEP;
            if (r >= n || c >= n) continue;
            if (fin) {
                const NodeRec &v = Lv.V[s.src][(int64_t)r * Lv.pitch + c];
                float4 u = v.u;
                if (tau != 0.f) {
                    float2 d = v.d;
                    u = df_add2(u, tau * d.x, tau * d.y);
                }
                const float2 res = make_float2(u.x + u.z, u.y + u.w);
                float2 &dst = op.out[(int64_t)r * op.slot_pitch + c];
                if (op.judge) {
                    const float2 g0 = dst;
                    corr += fabsf(res.x - g0.x) + fabsf(res.y - g0.y);
                }
                dst = res;
            } else {
                const LevelDesc &Cv = op.lv[s.lvl - 1];
                const NodeRec *V = Cv.V[s.src];
                int I = r >> 1, J = c >> 1, oi = r & 1, oj = c & 1;
                // 2 x bilinear prolongation (coarse grid unit = 2 fine units); the
                // weights 2, 1, 1/2 are exact, the sum is compensated
                float w2 = (oi ? 0.5f : 1.f) * (oj ? 0.5f : 1.f) * 2.f;
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int a = 0; a <= 1; a++)
#pragma unroll
                    for (int bb = 0; bb <= 1; bb++) {
                        if ((a && !oi) || (bb && !oj)) continue;
                        int64_t idx = (int64_t)(I + a) * Cv.pitch + (J + bb);
                        float4 u = V[idx].u;
                        if (tau != 0.f) {
                            float2 d = V[idx].d;
                            u = df_add2(u, tau * d.x, tau * d.y);
                        }
                        df_add(acc.x, acc.z, w2 * u.x);
                        df_add(acc.x, acc.z, w2 * u.z);
                        df_add(acc.y, acc.w, w2 * u.y);
                        df_add(acc.y, acc.w, w2 * u.w);
                    }
                Lv.V[0][(int64_t)r * Lv.pitch + c].u = acc;
            }
        }
        if (fin && op.judge) {  // block-uniform: the whole block works on this item
            const float w = warp_sum(corr);
            if ((threadIdx.x & 31) == 0) atomicAdd(&b.st[o].corr, (double)w);
        }
    }
}

// ---------------------------------------------------------------------------
// G: accept the pending step (u <- u + tau d) and compute the L2 gradient-flow
// direction at the new u:
//   dNCC/dThat_i = h^2 [ (M~ R~)_i / sigma_T - NCC (M~ (That - T_bar))_i / sigma_T^2 ]
//   psi_{i,c}    = -[...] dT_c(i) + lambda (K u_c)_i            (dE/du~ = h^2 psi)
//   d_{i,c}      = -psi_{i,c} / (h^2 omega_i)                  (d = -g / w, w = h^2 omega)
//   slope        = g^T d = -sum psi^2 / omega
//   Qud          = u^T K d = sum_i d_i . (K u)_i
// with M~ = M1 (x) M1 and K = K1 (x) M1 + M1 (x) K1 (1D mass M1 = [1 4 1] / 6,
// 2/6 on the diagonal at the border; 1D stiffness K1 = [-1 2 -1], 1 on the
// diagonal at the border), applied as separable stencils with the integer
// weights 6 M1 and 6 K1: along the column in registers, along the row by
// shuffles; the scale 1/36 or 1/6 is folded into per-tile coefficients, so that
// no rounded weight biases every node alike.  M~ R~ comes with the pyramid;
// 36 M~ That is stored for the trial passes of the search.  Strip tile: 30
// owned node columns by Lv.hg owned rows, one halo node around them.
// ---------------------------------------------------------------------------
template <bool BF16>
__global__ void __launch_bounds__(REG_STRIP_THREADS, 8) k_grad(BatchDev b)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (REG_STRIP_THREADS / 32);
    const int nent = b.ctr[2], items = b.ctr[5];
    for (int item = blockIdx.x * (REG_STRIP_THREADS / 32) + (threadIdx.x >> 5); item < items; item += nwarps) {
        const int e = find_entry(b.prefG, nent, item);
        const int o = b.listG[e];
        const int t = item - b.prefG[e];
        const OpState &s = b.st[o];
        const LevelDesc &Lv = b.ops[o].lv[s.lvl];
        const int n = Lv.n, pitch = Lv.pitch, ntx = (n + REG_GW - 1) / REG_GW, h = Lv.hg;
        const int r0 = (t / ntx) * h, c = (t % ntx) * REG_GW - 1 + lane;
        const int rLast = min(r0 + h - 1, n - 1);
        const bool colIn = c >= 0 && c < n;
        const bool own = colIn && lane >= 1 && lane <= REG_GW;
        const bool cEdge = (c == 0 || c == n - 1);
        const float cx6 = cEdge ? 2.f : 4.f;  // 6 M1 on the diagonal
        const float wx = cEdge ? 0.5f : 1.f, iwx = cEdge ? 2.f : 1.f;
        const float tau = (float)s.tau_acc;
        const NodeRec *Vs = Lv.V[s.src];
        NodeRec *Vc = Lv.V[s.cur];
        // the stencils run on the integer weights 6 M1 and 6 K1 (36 M~, 6 K); their
        // scale goes into these per-tile coefficients, each rounded once
        const float isig = (float)(1.0 / s.sigT);
        const float c36 = (float)(s.ncc / (s.sigT * s.sigT) / 36.0);  // NCC / sigma^2 / 36
        const float cT = (float)(s.ncc / (s.sigT * s.sigT) * s.Tbar);  // NCC / sigma^2 T_bar
        const float lam6 = (float)(b.lambda / 6.0);
        const float ih2 = 1.f / Lv.h2;  // exact: h^2 is a power of two
        // rows r-2 (suffix A) and r-1 (suffix M) of this column; row r is read
        // in the iteration and row r-1 is completed by it
        float tA = 0.f, tM = 0.f, kxAx = 0.f, kxAy = 0.f, kxMx = 0.f, kxMy = 0.f;
        float dyMx = 0.f, dyMy = 0.f, gxM = 0.f, gyM = 0.f, mrM = 0.f;
        float4 uM = make_float4(0.f, 0.f, 0.f, 0.f);
        float slope = 0.f, qud = 0.f;
        // the record and M~R~ of the next row are loaded while a row is worked on
        float4 nu = make_float4(0.f, 0.f, 0.f, 0.f), nd = nu;
        float nmr = 0.f;
        if (colIn && r0 - 1 >= 0) {
            const int64_t idx = (int64_t)(r0 - 1) * pitch + c;
            const float4 *rec = reinterpret_cast<const float4 *>(Vs + idx);
            nu = rec[0];
            nd = rec[1];
            nmr = Lv.MR[idx];
        }
        for (int r = r0 - 1; r <= rLast + 1; r++) {
            const bool in = colIn && r >= 0 && r < n;
            float4 u = nu;
            const float2 dp = make_float2(nd.x, nd.y);
            const float mr = nmr;
            if (colIn && r + 1 < n && r + 1 <= rLast + 1) {
                const int64_t idx = (int64_t)(r + 1) * pitch + c;
                const float4 *rec = reinterpret_cast<const float4 *>(Vs + idx);
                nu = rec[0];
                nd = rec[1];
                nmr = Lv.MR[idx];
            }
            float tv = 0.f, gx = 0.f, gy = 0.f;
            if (in) {
                if (tau != 0.f) u = df_add2(u, tau * dp.x, tau * dp.y);
                tv = sample_df<BF16, true>(Lv.T, n, pitch, c, r, u, &gx, &gy);
            } else {
                u = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            // u(r, c+1) - u(r, c) and u(r, c) - u(r-1, c), each from the hi and
            // lo parts (the stiffness terms are small differences of values of
            // several grid units); 0 where a node is missing
            float4 uR;
            uR.x = __shfl_down_sync(FULL, u.x, 1);
            uR.y = __shfl_down_sync(FULL, u.y, 1);
            uR.z = __shfl_down_sync(FULL, u.z, 1);
            uR.w = __shfl_down_sync(FULL, u.w, 1);
            const bool hasR = in && c + 1 < n, hasU = in && r >= 1 && r >= r0;
            const float dxx = hasR ? (uR.x - u.x) + (uR.z - u.z) : 0.f;
            const float dxy = hasR ? (uR.y - u.y) + (uR.w - u.w) : 0.f;
            const float dyx = hasU ? (u.x - uM.x) + (u.z - uM.z) : 0.f;
            const float dyy = hasU ? (u.y - uM.y) + (u.w - uM.w) : 0.f;
            // K1 along the row: [u(c) - u(c-1)] - [u(c+1) - u(c)]
            const float kxx = __shfl_up_sync(FULL, dxx, 1) - dxx;
            const float kxy = __shfl_up_sync(FULL, dxy, 1) - dxy;
            const int m = r - 1;
            if (m >= r0) {
                const bool mEdge = (m == 0 || m == n - 1);
                const float cy6 = mEdge ? 2.f : 4.f;
                // 36 M~ That at (m, c): 6 M1 down the column, then along the row
                const float vt = (tA + tv) + cy6 * tM;
                const float mt36 = (__shfl_up_sync(FULL, vt, 1) + __shfl_down_sync(FULL, vt, 1)) + cx6 * vt;
                // K1 along the column at m: [u(m) - u(m-1)] - [u(m+1) - u(m)]
                const float kyx = dyMx - dyx, kyy = dyMy - dyy;
                const float KYx = (__shfl_up_sync(FULL, kyx, 1) + __shfl_down_sync(FULL, kyx, 1)) + cx6 * kyx;
                const float KYy = (__shfl_up_sync(FULL, kyy, 1) + __shfl_down_sync(FULL, kyy, 1)) + cx6 * kyy;
                if (own) {
                    // 6 (K u)
                    const float kux = (kxAx + kxx) + cy6 * kxMx + KYx;
                    const float kuy = (kxAy + kxy) + cy6 * kxMy + KYy;
                    const float om = wx * (mEdge ? 0.5f : 1.f), iom = iwx * (mEdge ? 2.f : 1.f);
                    // dNCC/dThat / h^2 = (M~R~) / sigma - NCC (M~That - T_bar omega) / sigma^2
                    const float A = mrM * isig - c36 * mt36 + cT * om;
                    const float psx = -A * gxM + lam6 * kux, psy = -A * gyM + lam6 * kuy;
                    const float sc = ih2 * iom;
                    const float dnx = -psx * sc, dny = -psy * sc;
                    const int64_t idx = (int64_t)m * pitch + c;
                    float4 *rec = reinterpret_cast<float4 *>(Vc + idx);
                    rec[0] = uM;
                    rec[1] = make_float4(dnx, dny, mt36, mrM);
                    slope -= (psx * psx + psy * psy) * iom;
                    qud += dnx * kux + dny * kuy;
                }
            }
            tA = tM; tM = tv;
            kxAx = kxMx; kxAy = kxMy; kxMx = kxx; kxMy = kxy;
            dyMx = dyx; dyMy = dyy;
            gxM = gx; gyM = gy; mrM = mr; uM = u;
        }
        slope = warp_sum(slope);
        qud = warp_sum(qud / 6.f);
        if (lane < PG_STRIDE) b.partG[(int64_t)item * PG_STRIDE + lane] = lane == 0 ? slope : qud;
    }
}

// ---------------------------------------------------------------------------
// S: the H1-type smoother (Section "Gradient flow": d = -A^{-1} E'[phi], A
// selected to smooth).  A = M_s (x) M_s, the tensor-product Gram matrix of
// M_s = M1 + (s^2/2) K1 with s a number of grid spacings; in grid units of
// the level the direction is d = (T (x) T)^{-1} (omega d_L2), T = M_s / h the
// dimensionless tridiagonal matrix (off-diagonal 1/6 - s^2/2, diagonal
// 2/3 + s^2, 1/3 + s^2/2 at the ends) and d_L2 = -psi / (h^2 omega) the lumped
// direction of the gradient pass.  The Kronecker inverse is one tridiagonal
// solve along every row, then one along every column (Thomas elimination
// with the level's precomputed pivots).  The previous iterate's node records
// (not read again before the next gradient pass overwrites them) hold the
// intermediate fields.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 *sm_scratch(NodeRec *V, int64_t idx, int k)
{
    return reinterpret_cast<float2 *>(&V[idx].u) + k;  // k = 0: u.x, u.y; k = 1: u.z, u.w
}

// Rows: lane = one row of one operator, sequential over its columns.
__global__ void __launch_bounds__(128) k_smooth_rows(BatchDev b)
{
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * 4, nG = b.ctr[2];
    const float a = b.sm_a;
    for (int it = blockIdx.x * 4 + (threadIdx.x >> 5); it < nG * b.rch; it += nwarps) {
        const int e = it / b.rch, ch = it % b.rch;
        const int o = b.listG[e];
        const OpState &s = b.st[o];
        const LevelDesc &Lv = b.ops[o].lv[s.lvl];
        const int n = Lv.n, pitch = Lv.pitch, r = ch * 32 + lane;
        if (r >= n) continue;
        const NodeRec *Vc = Lv.V[s.cur];
        NodeRec *Vs = Lv.V[s.src];
        const float omr = (r == 0 || r == n - 1) ? 0.5f : 1.f;
        float2 y = make_float2(0.f, 0.f);
        for (int c = 0; c < n; c++) {
            const int64_t idx = (int64_t)r * pitch + c;
            const float2 d = Vc[idx].d;
            const float om = omr * ((c == 0 || c == n - 1) ? 0.5f : 1.f);
            const float m = Lv.sm_tab[c].y;
            y.x = (om * d.x - a * y.x) * m;
            y.y = (om * d.y - a * y.y) * m;
            *sm_scratch(Vs, idx, 0) = y;
        }
        float2 x = make_float2(0.f, 0.f);
        for (int c = n - 1; c >= 0; c--) {
            const int64_t idx = (int64_t)r * pitch + c;
            const float2 yc = *sm_scratch(Vs, idx, 0);
            const float cp = c < n - 1 ? Lv.sm_tab[c].x : 0.f;
            x.x = yc.x - cp * x.x;
            x.y = yc.y - cp * x.y;
            *sm_scratch(Vs, idx, 0) = x;
        }
    }
}

// Columns: a warp holds REG_GW owned columns and one halo column on each side
// (lanes 0 and 31), walks down for the elimination and up for the
// substitution; on the way up it writes d into the current records and sums
// the new slope g^T d = -h^4 sum omega d_L2 . d and u^T K d (6 K u by the
// integer stencils of the gradient pass, hi and lo parts of u differenced
// separately).
__global__ void __launch_bounds__(128) k_smooth_cols(BatchDev b)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * 4, nG = b.ctr[2];
    const float a = b.sm_a;
    for (int it = blockIdx.x * 4 + (threadIdx.x >> 5); it < nG * b.cch; it += nwarps) {
        const int e = it / b.cch, ch = it % b.cch;
        const int o = b.listG[e];
        const OpState &s = b.st[o];
        const LevelDesc &Lv = b.ops[o].lv[s.lvl];
        const int n = Lv.n, pitch = Lv.pitch;
        if (ch * REG_GW >= n) continue;  // warp-uniform
        const int c = ch * REG_GW - 1 + lane;
        const bool colIn = c >= 0 && c < n, own = colIn && lane >= 1 && lane <= REG_GW;
        NodeRec *Vc = Lv.V[s.cur];
        NodeRec *Vs = Lv.V[s.src];
        float2 y = make_float2(0.f, 0.f);
        if (colIn)
            for (int r = 0; r < n; r++) {
                const int64_t idx = (int64_t)r * pitch + c;
                const float2 x = *sm_scratch(Vs, idx, 0);
                const float m = Lv.sm_tab[r].y;
                y.x = (x.x - a * y.x) * m;
                y.y = (x.y - a * y.y) * m;
                *sm_scratch(Vs, idx, 1) = y;
            }
        const float cx6 = (c == 0 || c == n - 1) ? 2.f : 4.f;
        const float omc = (c == 0 || c == n - 1) ? 0.5f : 1.f;
        // rolling rows r+1 (P), r (C), r-1 (N) of u and of K1 along the row
        auto ldu = [&](int r) {
            return (colIn && r >= 0 && r < n) ? reinterpret_cast<const float4 *>(Vc + (int64_t)r * pitch + c)[0]
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        auto kx_of = [&](const float4 &u, int r) {
            // [u(c) - u(c-1)] - [u(c+1) - u(c)] along the row (0 past the grid)
            float4 uR;
            uR.x = __shfl_down_sync(FULL, u.x, 1);
            uR.y = __shfl_down_sync(FULL, u.y, 1);
            uR.z = __shfl_down_sync(FULL, u.z, 1);
            uR.w = __shfl_down_sync(FULL, u.w, 1);
            const bool rowIn = r >= 0 && r < n, hasR = colIn && rowIn && c + 1 < n;
            const float dxx = hasR ? (uR.x - u.x) + (uR.z - u.z) : 0.f;
            const float dxy = hasR ? (uR.y - u.y) + (uR.w - u.w) : 0.f;
            return make_float2(__shfl_up_sync(FULL, dxx, 1) - dxx, __shfl_up_sync(FULL, dxy, 1) - dxy);
        };
        float4 uP = make_float4(0.f, 0.f, 0.f, 0.f), uC = ldu(n - 1);
        float2 kP = make_float2(0.f, 0.f), kC = kx_of(uC, n - 1);
        float2 dnext = make_float2(0.f, 0.f);
        float sl = 0.f, qd = 0.f;
        for (int r = n - 1; r >= 0; r--) {
            const float4 uN = ldu(r - 1);
            const float2 kN = kx_of(uN, r - 1);
            float2 dn = make_float2(0.f, 0.f);
            const int64_t idx = (int64_t)r * pitch + c;
            if (colIn) {
                const float2 yr = *sm_scratch(Vs, idx, 1);
                const float cp = r < n - 1 ? Lv.sm_tab[r].x : 0.f;
                dn.x = yr.x - cp * dnext.x;
                dn.y = yr.y - cp * dnext.y;
            }
            dnext = dn;
            // K1 along the column at (r, c): [u(r) - u(r-1)] - [u(r+1) - u(r)]
            const bool hasU = colIn && r >= 1, hasD = colIn && r + 1 < n;
            const float kyx = (hasU ? (uC.x - uN.x) + (uC.z - uN.z) : 0.f) - (hasD ? (uP.x - uC.x) + (uP.z - uC.z) : 0.f);
            const float kyy = (hasU ? (uC.y - uN.y) + (uC.w - uN.w) : 0.f) - (hasD ? (uP.y - uC.y) + (uP.w - uC.w) : 0.f);
            const float KYx = (__shfl_up_sync(FULL, kyx, 1) + __shfl_down_sync(FULL, kyx, 1)) + cx6 * kyx;
            const float KYy = (__shfl_up_sync(FULL, kyy, 1) + __shfl_down_sync(FULL, kyy, 1)) + cx6 * kyy;
            if (own) {
                const float cy6 = (r == 0 || r == n - 1) ? 2.f : 4.f;
                const float kux = (kP.x + kN.x) + cy6 * kC.x + KYx;  // 6 (K u)
                const float kuy = (kP.y + kN.y) + cy6 * kC.y + KYy;
                const float om = omc * ((r == 0 || r == n - 1) ? 0.5f : 1.f);
                const float2 dl = Vc[idx].d;
                sl += om * (dl.x * dn.x + dl.y * dn.y);
                qd += dn.x * kux + dn.y * kuy;
                Vc[idx].d = dn;
            }
            uP = uC; uC = uN;
            kP = kC; kC = kN;
        }
        sl = warp_sum(sl);
        qd = warp_sum(qd / 6.f);
        if (lane == 0) {
            b.partS[((int64_t)e * b.cch + ch) * 2] = sl;
            b.partS[((int64_t)e * b.cch + ch) * 2 + 1] = qd;
        }
    }
}

void launch_smooth(int grid, cudaStream_t st, const BatchDev &b)
{
    k_smooth_rows<<<grid, 128, 0, st>>>(b);
    k_smooth_cols<<<grid, 128, 0, st>>>(b);
}

// Bilinear sampling helpers of the trial pass.
namespace {

struct Texel4 {
    int jx, jy;
    float ax, ay;
    bool clx, cly;
    float t00, t01, t10, t11;
};

__device__ __forceinline__ void locate(int n, int c, int r, float vx, float vy, int &jx, int &jy, float &ax,
                                       float &ay, bool &clx, bool &cly)
{
    float fx, fy;
    jx = c + floor_i(vx, fx);
    jy = r + floor_i(vy, fy);
    ax = vx - fx;
    ay = vy - fy;
    clx = cly = false;
    if (jx < 0) { jx = 0; ax = 0.f; clx = true; }
    else if (jx >= n - 1) { clx = (jx > n - 1) || (ax > 0.f); jx = n - 2; ax = 1.f; }
    if (jy < 0) { jy = 0; ay = 0.f; cly = true; }
    else if (jy >= n - 1) { cly = (jy > n - 1) || (ay > 0.f); jy = n - 2; ay = 1.f; }
}

template <bool BF16>
__device__ __forceinline__ void fetch(Texel4 &q, const void *img, int pitch)
{
    int i0 = q.jy * pitch + q.jx;
    q.t00 = ldimg<BF16>(img, i0);
    q.t01 = ldimg<BF16>(img, i0 + 1);
    q.t10 = ldimg<BF16>(img, i0 + pitch);
    q.t11 = ldimg<BF16>(img, i0 + pitch + 1);
}

__device__ __forceinline__ float bil(const Texel4 &q)
{
    return (1.f - q.ay) * ((1.f - q.ax) * q.t00 + q.ax * q.t01) + q.ay * ((1.f - q.ax) * q.t10 + q.ax * q.t11);
}

}  // namespace

// ---------------------------------------------------------------------------
// T: warp + energy as FE sums over a strip tile of 31 x 32 cells.
// Level-start pass (tau = 0), at u:
//   [0] int That / h^2 = sum omega_i That_i      [1] int That^2 / h^2 = That^T M~ That
//   [2] int That R~ / h^2 = sum (M~ R~)_i That_i   [3 MAXT] Quu, the Dirichlet form of u
// Trial pass: for every step size tau_j the change against the current u,
// delta_j = That(u + tau_j d) - That(u) per node:
//   [3j] sum omega delta   [3j+1] 2 sum (M~ That) delta + delta^T M~ delta
//   [3j+2] sum (M~ R~) delta
// and in the first pass of a search [3 MAXT + 2] Qdd, the Dirichlet form of d
// (the Dirichlet form of u + tau d is Quu + 2 tau Qud + tau^2 Qdd).
// When u and u + tau d lie in the same bilinear cell, delta is formed from the
// cell's four texels as
//   tau d_x [(1-a_y') (t01-t00) + a_y' (t11-t10)] + tau d_y [(1-a_x) (t10-t00) + a_x (t11-t01)],
// so that its float rounding is relative to delta itself (the quantity the
// Armijo test compares), not to That; a tiny move across a cell line is split
// into exact segments, and a move of 2^-10 grid units or more takes a fresh
// sample.
// Sums over nodes use per-node weights (omega and the stored M~ That, M~ R~);
// the quadratic forms are summed per cell.  With the cyclic corner order the
// element mass matrix is (1/36) [4 2 1 2; 2 4 2 1; 1 2 4 2; 2 1 2 4], and
//   36 v^T M~_e v = 4 P(top) + 4 P(bottom) + 2 top . [2 1; 1 2] bottom,
//   P(x0, x1) = x0 (x0 + x1) + x1^2,
// so each row's P is formed once for the two cells that share the row.  The
// cell's Dirichlet form is (P(p, q) + P(r, s)) / 3 per component, p, q the x
// differences of its top and bottom rows and r, s the y differences of its
// left and right columns.  Lane l holds node column c0 + l; lanes 0..30 own
// the cells to their right, lane 31 supplies the right corners.
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ float pform(float x0, float x1) { return x0 * (x0 + x1) + x1 * x1; }

struct StripGeom {
    int n, pitch, h, r0, rEnd, c;
    bool colIn, cellCol, nodeCol;
    float wx;
};

__device__ __forceinline__ StripGeom strip_geom(const LevelDesc &Lv, int t, int lane)
{
    StripGeom g;
    g.n = Lv.n;
    g.pitch = Lv.pitch;
    const int ntx = (g.n - 1 + REG_CW - 1) / REG_CW;
    g.h = Lv.ht;
    g.r0 = (t / ntx) * g.h;
    g.c = (t % ntx) * REG_CW + lane;
    g.rEnd = min(g.r0 + g.h, g.n - 1);
    g.colIn = g.c < g.n;
    g.cellCol = lane < REG_CW && g.c < g.n - 1;
    g.nodeCol = g.colIn && (lane < REG_CW || g.c == g.n - 1);
    g.wx = (g.c == 0 || g.c == g.n - 1) ? 0.5f : 1.f;
    return g;
}

// The 3 x 3 texel patch around the base cell of a node, extended towards the
// direction of its move, and the per-node terms of the exact change of the
// interpolant for moves of less than one cell (patch_delta).
struct Patch {
    float ax, ay;    // fractions of the base point in its cell (clamped coordinates: 0 or 1)
    float lx, ly;    // signed distance to the next cell line in the move direction
    float s0x, s1x;  // slope along x at a_y of the base cell and of its neighbour in the move direction
    float v0[3], v1[3];  // t(row + 1) - t(row) in the base row band and in the neighbour band,
                         // columns: base left, base right, neighbour outer
    bool nbx, nby;   // the neighbour cell exists (else the interpolant is flat beyond the border)
    bool posx, posy; // move direction
    int clx, cly;    // 0: inside; otherwise the raw cell index of the clamped base point (never 0)
    float rax, ray;  // raw fraction of a clamped base point
    float t0;        // the interpolant at the base point
};

template <bool BF16>
__device__ __forceinline__ void make_patch(Patch &P, const void *T, int n, int pitch, int c, int r, float4 u, float dx,
                                           float dy)
{
    int ix, iy;
    float fx, fy;
    df_split(u.x, u.z, ix, fx);
    df_split(u.y, u.w, iy, fy);
    int jx = c + ix, jy = r + iy;
    P.rax = fx;
    P.ray = fy;
    P.clx = P.cly = 0;
    float ax = fx, ay = fy;
    if (jx < 0) { P.clx = jx; jx = 0; ax = 0.f; }
    else if (jx >= n - 1) { if (jx > n - 1 || fx > 0.f) P.clx = jx; jx = n - 2; ax = 1.f; }
    if (jy < 0) { P.cly = jy; jy = 0; ay = 0.f; }
    else if (jy >= n - 1) { if (jy > n - 1 || fy > 0.f) P.cly = jy; jy = n - 2; ay = 1.f; }
    P.ax = ax;
    P.ay = ay;
    P.posx = dx >= 0.f;
    P.posy = dy >= 0.f;
    P.nbx = P.posx ? (jx + 1 <= n - 2) : (jx >= 1);
    P.nby = P.posy ? (jy + 1 <= n - 2) : (jy >= 1);
    const int cx2 = P.posx ? min(jx + 2, n - 1) : max(jx - 1, 0);
    const int ry2 = P.posy ? min(jy + 2, n - 1) : max(jy - 1, 0);
    const int rows[3] = {jy, jy + 1, ry2}, cols[3] = {jx, jx + 1, cx2};
    float t[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) t[a][b] = ldimg<BF16>(T, rows[a] * pitch + cols[b]);
    P.t0 = (1.f - ay) * ((1.f - ax) * t[0][0] + ax * t[0][1]) + ay * ((1.f - ax) * t[1][0] + ax * t[1][1]);
    P.lx = P.posx ? 1.f - ax : -ax;
    P.ly = P.posy ? 1.f - ay : -ay;
    P.s0x = (1.f - ay) * (t[0][1] - t[0][0]) + ay * (t[1][1] - t[1][0]);
    // neighbour cell along x: columns (1, 2) when moving right, (2, 0) when moving left
    const float nl0 = P.posx ? t[0][1] : t[0][2], nr0 = P.posx ? t[0][2] : t[0][0];
    const float nl1 = P.posx ? t[1][1] : t[1][2], nr1 = P.posx ? t[1][2] : t[1][0];
    P.s1x = P.nbx ? (1.f - ay) * (nr0 - nl0) + ay * (nr1 - nl1) : 0.f;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        P.v0[b] = t[1][b] - t[0][b];
        P.v1[b] = P.posy ? t[2][b] - t[1][b] : t[0][b] - t[2][b];
    }
}

// Change of the interpolant for the move (ex, ey) from the base point of P,
// split into a move along x in the base row band and a move along y at the new
// column; each part is a sum of segment lengths times the slope of the cell
// the segment lies in, so that its rounding is relative to the change itself
// (a single float fraction could not resolve a move far below its ulp across a
// cell line).  Past the grid border the interpolant is flat; a base point
// outside the grid contributes only the part of the move back inside.
// Returns false (and no value) for a move of a cell or more.
__device__ __forceinline__ bool patch_delta(const Patch &P, int n, float ex, float ey, float &del)
{
    bool ok = true;
    // x part
    float xpart, f;
    bool nbcol = false;  // the y part runs in the neighbour column cell
    if (P.clx) {
        ok = fabsf(ex) < 1.f;
        // length of the move inside the grid: from the left border (raw cell
        // -1) or back from the right border (raw cell n-1); 0 further out
        const float in = (P.clx == -1) ? fmaxf(P.rax + ex - 1.f, 0.f)
                                        : ((P.clx == n - 1) ? fminf(P.rax + ex, 0.f) : 0.f);
        xpart = in * P.s0x;
        f = P.ax + in;
    } else {
        const float ax1 = P.ax + ex;
        if (ax1 >= 0.f && ax1 < 1.f) {
            xpart = ex * P.s0x;
            f = ax1;
        } else {
            const float rest = ex - P.lx;  // length beyond the cell line
            ok = fabsf(rest) < 1.f;
            xpart = P.lx * P.s0x + rest * P.s1x;
            f = P.nbx ? (P.posx ? rest : 1.f + rest) : (P.posx ? 1.f : 0.f);
            nbcol = P.nbx;
        }
    }
    // y part at the new column: slopes of the base and neighbour row bands
    const float vl0 = nbcol ? (P.posx ? P.v0[1] : P.v0[2]) : P.v0[0];
    const float vr0 = nbcol ? (P.posx ? P.v0[2] : P.v0[0]) : P.v0[1];
    const float sy0 = (1.f - f) * vl0 + f * vr0;
    float ypart;
    if (P.cly) {
        ok = ok && fabsf(ey) < 1.f;
        const float in = (P.cly == -1) ? fmaxf(P.ray + ey - 1.f, 0.f)
                                        : ((P.cly == n - 1) ? fminf(P.ray + ey, 0.f) : 0.f);
        ypart = in * sy0;
    } else {
        const float ay1 = P.ay + ey;
        if (ay1 >= 0.f && ay1 < 1.f) {
            ypart = ey * sy0;
        } else {
            const float rest = ey - P.ly;
            ok = ok && fabsf(rest) < 1.f;
            const float vl1 = nbcol ? (P.posx ? P.v1[1] : P.v1[2]) : P.v1[0];
            const float vr1 = nbcol ? (P.posx ? P.v1[2] : P.v1[0]) : P.v1[1];
            const float sy1 = P.nby ? (1.f - f) * vl1 + f * vr1 : 0.f;
            ypart = P.ly * sy0 + rest * sy1;
        }
    }
    del = xpart + ypart;
    return ok;
}

// Level-start sums of one strip tile at u, accumulated in double: they seed
// every search of the level (the trial passes only add changes to them), and
// the pass runs once per level.
template <bool BF16>
__device__ __forceinline__ void start_tile(const OpState &s, const LevelDesc &Lv, const StripGeom &g, double *v)
{
    const unsigned FULL = 0xffffffffu;
    const NodeRec *V = Lv.V[s.cur];
    double s1 = 0.0, s3 = 0.0, q2 = 0.0, quu = 0.0;
    float tP = 0.f, tPR = 0.f, pux = 0.f, puy = 0.f;
    float4 uP = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int r = g.r0; r <= g.rEnd; r++) {
        float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
        float t0 = 0.f, mr = 0.f;
        if (g.colIn) {
            const int64_t idx = (int64_t)r * g.pitch + g.c;
            u = V[idx].u;
            mr = Lv.MR[idx];
            t0 = sample_df<BF16, false>(Lv.T, g.n, g.pitch, g.c, r, u, nullptr, nullptr);
        }
        if (g.nodeCol && (r < g.r0 + g.h || r == g.n - 1)) {
            const float w = g.wx * ((r == 0 || r == g.n - 1) ? 0.5f : 1.f);
            s1 += (double)(w * t0);
            s3 += (double)(mr * t0);
        }
        const float tR = __shfl_down_sync(FULL, t0, 1);
        float4 uR;
        uR.x = __shfl_down_sync(FULL, u.x, 1);
        uR.y = __shfl_down_sync(FULL, u.y, 1);
        uR.z = __shfl_down_sync(FULL, u.z, 1);
        uR.w = __shfl_down_sync(FULL, u.w, 1);
        const float qx = (uR.x - u.x) + (uR.z - u.z), qy = (uR.y - u.y) + (uR.w - u.w);
        const float rx = (u.x - uP.x) + (u.z - uP.z), ry = (u.y - uP.y) + (u.w - uP.w);
        const float sx = __shfl_down_sync(FULL, rx, 1), sy = __shfl_down_sync(FULL, ry, 1);
        if (g.cellCol) {
            const float wrow2 = (float)(2 * ((r > g.r0) + (r < g.rEnd)));
            q2 += (double)(wrow2 * pform(t0, tR));
            if (r > g.r0) {
                q2 += (double)(tP * (2.f * t0 + tR) + tPR * (t0 + 2.f * tR));
                quu += (double)(pform(pux, qx) + pform(rx, sx) + pform(puy, qy) + pform(ry, sy));
            }
        }
        tP = t0; tPR = tR;
        pux = qx; puy = qy; uP = u;
    }
    v[0] = s1;
    v[1] = q2 * (1.0 / 18.0);
    v[2] = s3;
    v[3] = quu * (1.0 / 3.0);
}

// Shared memory of one warp in the trial pass.  The row walk sums the nodes
// and cells that the polynomial moments cover and queues the rest: nodes whose
// largest move leaves their cell (or whose base point lies outside the grid),
// and cells with such a corner.  A window of up to TW rows is then finished
// cooperatively, one queued node or cell per lane, so that the exact path
// runs on full warps instead of on the few lanes of a row that need it.
constexpr int TW = 12;   // rows per window
constexpr int TQ = 96;   // queued nodes (a row adds at most 32)
constexpr int TC = 192;  // queued cells (a row adds at most 31)
template <int JM>
struct TrialScratch {
    float A[TW + 1][32], B[TW + 1][32];  // A, B of the window's rows; slot 0: the row before the window
    unsigned char qi[TW + 1][32];        // 1 + queue index of a node on the exact path, else 0
    unsigned short qn[TQ];               // queued nodes: slot << 5 | lane
    unsigned short qc[TC];               // queued cells: slot << 5 | lane (between slots slot-1 and slot)
    float dl[JM][TQ];                    // delta_j of the queued nodes
    float sn[3][JM][32];                 // per-lane node sums: omega delta, 36 M~That delta, M~R~ delta
    float sq[JM][32];                    // per-lane cell sums of 18 delta^T M~_e delta
};

// Exact change of the interpolant at one node for every step size, for a
// node whose largest move leaves its cell (or whose base point lies outside
// the grid): the moves that stay in the cell take the polynomial of the base
// cell, the others the texel patch, or a fresh sample for moves of a cell or
// more (whose rounding, ~1e-7 of That, is small against such a change).  The
// changes go to queue entry q and, for an owned node, into the node sums of
// the lane that computes them.
template <bool BF16, int JM>
__device__ __forceinline__ void node_deltas_exact(const LevelDesc &Lv, const float *tau, int J, int c, int r,
                                                  float4 u, float4 dm, float w, bool own, TrialScratch<JM> &sh,
                                                  int q, int lane)
{
    const int n = Lv.n, pitch = Lv.pitch;
    Patch P;
    make_patch<BF16>(P, Lv.T, n, pitch, c, r, u, dm.x, dm.y);
    const bool cl = P.clx || P.cly;
    // dThat/dx at a_y, dThat/dy at a_x and the mixed derivative of the base cell
    const float sy = P.v0[0] + P.ax * (P.v0[1] - P.v0[0]);
    const float A = dm.x * P.s0x + dm.y * sy;
    const float B = dm.x * dm.y * (P.v0[1] - P.v0[0]);
#pragma unroll
    for (int j = 0; j < JM; j++) {
        if (j < J) {
            const float ex = tau[j] * dm.x, ey = tau[j] * dm.y;
            const float ax1 = P.ax + ex, ay1 = P.ay + ey;
            float del;
            if (!cl && ax1 >= 0.f && ax1 < 1.f && ay1 >= 0.f && ay1 < 1.f) {
                del = tau[j] * (A + tau[j] * B);
            } else if (!patch_delta(P, n, ex, ey, del)) {
                Texel4 t;
                locate(n, c, r, (u.x + u.z) + ex, (u.y + u.w) + ey, t.jx, t.jy, t.ax, t.ay, t.clx, t.cly);
                fetch<BF16>(t, Lv.T, pitch);
                del = bil(t) - P.t0;
            }
            sh.dl[j][q] = del;
            if (own) {
                sh.sn[0][j][lane] += w * del;
                sh.sn[1][j][lane] += dm.z * del;
                sh.sn[2][j][lane] += dm.w * del;
            }
        }
    }
}

// Finish a window whose rows rlast-nrow+1 .. rlast sit in slots 1..nrow: the
// queued nodes from entry q0 on (one per lane), then the queued cells, whose
// corners take either a queued node's exact change or the polynomial of their
// A and B.  The last row moves to slot 0 with the changes of its queued nodes,
// for the cells between it and the next window.
template <bool BF16, int JM>
__device__ __forceinline__ void trial_flush(const LevelDesc &Lv, const StripGeom &g, const float4 *V,
                                            const float *tau, int J, TrialScratch<JM> &sh, int lane, int rlast,
                                            int nrow, int &q0, int &qn, int &qc)
{
    const unsigned FULL = 0xffffffffu;
    __syncwarp();
    for (int q = q0 + lane; q < qn; q += 32) {
        const int e = sh.qn[q], slot = e >> 5, ln = e & 31;
        const int r = rlast - nrow + slot, c = g.c - lane + ln;
        const int64_t idx = (int64_t)r * g.pitch + c;
        const float4 u = V[2 * idx], dm = V[2 * idx + 1];
        const bool own = (ln < REG_CW || c == g.n - 1) && (r < g.r0 + g.h || r == g.n - 1);
        const float w = ((c == 0 || c == g.n - 1) ? 0.5f : 1.f) * ((r == 0 || r == g.n - 1) ? 0.5f : 1.f);
        node_deltas_exact<BF16, JM>(Lv, tau, J, c, r, u, dm, w, own, sh, q, lane);
    }
    __syncwarp();
    for (int q = lane; q < qc; q += 32) {
        const int e = sh.qc[q], slot = e >> 5, ln = e & 31;
        const int itl = sh.qi[slot - 1][ln], itr = sh.qi[slot - 1][ln + 1];
        const int ibl = sh.qi[slot][ln], ibr = sh.qi[slot][ln + 1];
        const float Atl = sh.A[slot - 1][ln], Btl = sh.B[slot - 1][ln];
        const float Atr = sh.A[slot - 1][ln + 1], Btr = sh.B[slot - 1][ln + 1];
        const float Abl = sh.A[slot][ln], Bbl = sh.B[slot][ln];
        const float Abr = sh.A[slot][ln + 1], Bbr = sh.B[slot][ln + 1];
#pragma unroll
        for (int j = 0; j < JM; j++) {
            if (j < J) {
                const float t = tau[j];
                const float tl = itl ? sh.dl[j][itl - 1] : t * (Atl + t * Btl);
                const float tr = itr ? sh.dl[j][itr - 1] : t * (Atr + t * Btr);
                const float bl = ibl ? sh.dl[j][ibl - 1] : t * (Abl + t * Bbl);
                const float br = ibr ? sh.dl[j][ibr - 1] : t * (Abr + t * Bbr);
                sh.sq[j][lane] += 2.f * (pform(tl, tr) + pform(bl, br)) + tl * (2.f * bl + br) + tr * (bl + 2.f * br);
            }
        }
    }
    __syncwarp();
    // the last row becomes slot 0
    const int iq = sh.qi[nrow][lane];
    const unsigned m = __ballot_sync(FULL, iq != 0);
    const int np = __popc(m & ((1u << lane) - 1u));
    float keep[JM];
#pragma unroll
    for (int j = 0; j < JM; j++) keep[j] = (iq && j < J) ? sh.dl[j][iq - 1] : 0.f;
    const float a = sh.A[nrow][lane], b = sh.B[nrow][lane];
    __syncwarp();
    sh.A[0][lane] = a;
    sh.B[0][lane] = b;
    sh.qi[0][lane] = iq ? (unsigned char)(np + 1) : 0;
    if (iq) {
#pragma unroll
        for (int j = 0; j < JM; j++)
            if (j < J) sh.dl[j][np] = keep[j];
    }
    qn = q0 = __popc(m);
    qc = 0;
    __syncwarp();
}

// Trial sums of one strip tile for the step sizes tau_0..tau_{J-1}.  All step
// sizes move a node along the same ray u + tau d, and while the moved point
// stays in the base cell the change of the bilinear interpolant is exactly
//   delta(tau) = tau A + tau^2 B,  A = d . grad That (at the base point),
//   B = d_x d_y (t00 - t01 - t10 + t11),
// so the sums over such nodes and cells are polynomials in tau of per-node
// moments (sum omega A, sum omega B, ...; 18 A^T M~ A, 18 A^T M~ B, 18 B^T M~ B
// per cell) that are gathered once for all step sizes.  A node whose largest
// move leaves the cell, and every cell touching one, is summed exactly for each
// step size, in windows of rows finished by the whole warp (trial_flush).  The
// node record of the next row is loaded while the current row is worked on.
template <bool BF16, int JM>
__device__ __forceinline__ void steps_tile(const OpState &s, const LevelDesc &Lv, const StripGeom &g, float *v,
                                           TrialScratch<JM> &sh, int lane, unsigned &nexact)
{
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;
    const int J = min(s.ntr, JM);
    const bool withQ = (s.phase == PH_GRAD);
    const float4 *V = reinterpret_cast<const float4 *>(Lv.V[s.cur]);
    float tau[JM];
    float tmax = 0.f;
#pragma unroll
    for (int j = 0; j < JM; j++) {
        tau[j] = (j < J) ? (float)s.trial_tau[j] : 0.f;
        tmax = fmaxf(tmax, tau[j]);
#pragma unroll
        for (int k = 0; k < 3; k++) sh.sn[k][j][lane] = 0.f;
        sh.sq[j][lane] = 0.f;
    }
    // node moments (owned nodes that stay in their cell) and cell moments
    float mWA = 0.f, mWB = 0.f, mTA = 0.f, mTB = 0.f, mRA = 0.f, mRB = 0.f;
    float qaa = 0.f, qab = 0.f, qbb = 0.f;
    // the previous row: A, B here and at the right neighbour, its row forms
    float Ap = 0.f, ApR = 0.f, Bp = 0.f, BpR = 0.f, PaaP = 0.f, PabP = 0.f, PbbP = 0.f;
    bool slowP = false, slowPR = false;
    float qdd = 0.f, pdx = 0.f, pdy = 0.f, dPx = 0.f, dPy = 0.f;
    int q0 = 0, qn = 0, qc = 0, nrow = 0;  // queue state (warp-uniform)
    float4 nu = make_float4(0.f, 0.f, 0.f, 0.f), ndm = nu;  // record of the next row
    if (g.colIn) {
        const int64_t idx = (int64_t)g.r0 * g.pitch + g.c;
        nu = V[2 * idx];
        ndm = V[2 * idx + 1];
    }
    for (int r = g.r0; r <= g.rEnd; r++) {
        const float4 u = nu, dm = ndm;  // d = (dm.x, dm.y), 36 M~That = dm.z, M~R~ = dm.w
        if (g.colIn && r < g.rEnd) {
            const int64_t idx = (int64_t)(r + 1) * g.pitch + g.c;
            nu = V[2 * idx];
            ndm = V[2 * idx + 1];
        }
        const bool own = g.nodeCol && (r < g.r0 + g.h || r == g.n - 1);
        const float w = g.wx * ((r == 0 || r == g.n - 1) ? 0.5f : 1.f);
        float A = 0.f, B = 0.f;
        bool slow = false;
        if (g.colIn) {
            Texel4 q;
            int ix, iy;
            df_split(u.x, u.z, ix, q.ax);
            df_split(u.y, u.w, iy, q.ay);
            q.jx = g.c + ix;
            q.jy = r + iy;
            // a base point outside the grid, or a largest move that leaves the
            // cell (then every smaller one along the ray stays inside)
            const float ax1 = q.ax + tmax * dm.x, ay1 = q.ay + tmax * dm.y;
            slow = q.jx < 0 || q.jx > g.n - 2 || q.jy < 0 || q.jy > g.n - 2 || !(ax1 >= 0.f && ax1 < 1.f) ||
                   !(ay1 >= 0.f && ay1 < 1.f);
            if (!slow) {
                fetch<BF16>(q, Lv.T, g.pitch);
                const float dtx = q.t01 - q.t00, dtx1 = q.t11 - q.t10;
                const float sx = dtx + q.ay * (dtx1 - dtx);                            // dThat/dx
                const float sy = (q.t10 - q.t00) + q.ax * ((q.t11 - q.t01) - (q.t10 - q.t00));  // dThat/dy
                A = dm.x * sx + dm.y * sy;
                B = dm.x * dm.y * (dtx1 - dtx);
                if (own) {
                    mWA += w * A; mWB += w * B;
                    mTA += dm.z * A; mTB += dm.z * B;
                    mRA += dm.w * A; mRB += dm.w * B;
                }
            }
        }
        // this row's slot in the window; queue its nodes on the exact path
        const int slot = nrow + 1;
        const unsigned ms = __ballot_sync(FULL, slow);
        nexact += __popc(ms);
        const int pos = qn + __popc(ms & lt);
        sh.A[slot][lane] = A;
        sh.B[slot][lane] = B;
        sh.qi[slot][lane] = slow ? (unsigned char)(pos + 1) : 0;
        if (slow) sh.qn[pos] = (unsigned short)((slot << 5) | lane);
        qn += __popc(ms);
        // cells between rows r-1 and r, columns c and c+1
        const float AR = __shfl_down_sync(FULL, A, 1), BR = __shfl_down_sync(FULL, B, 1);
        const bool slowR = __shfl_down_sync(FULL, slow, 1);
        const float Paa = pform(A, AR), Pbb = pform(B, BR);
        const float Pab = A * B + AR * BR + 0.5f * (A * BR + AR * B);
        bool mixed = false;
        if (g.cellCol && r > g.r0) {
            if (!(slowP || slowPR || slow || slowR)) {
                const float ha = 2.f * A + AR, haR = A + 2.f * AR, hb = 2.f * B + BR, hbR = B + 2.f * BR;
                qaa += 2.f * (PaaP + Paa) + Ap * ha + ApR * haR;
                qbb += 2.f * (PbbP + Pbb) + Bp * hb + BpR * hbR;
                qab += 2.f * (PabP + Pab) + 0.5f * (Ap * hb + ApR * hbR + Bp * ha + BpR * haR);
            } else {
                mixed = true;
            }
        }
        const unsigned mc = __ballot_sync(FULL, mixed);
        if (mixed) sh.qc[qc + __popc(mc & lt)] = (unsigned short)((slot << 5) | lane);
        qc += __popc(mc);
        Ap = A; ApR = AR; Bp = B; BpR = BR;
        PaaP = Paa; PabP = Pab; PbbP = Pbb;
        slowP = slow; slowPR = slowR;
        if (withQ) {
            const float dRx = __shfl_down_sync(FULL, dm.x, 1), dRy = __shfl_down_sync(FULL, dm.y, 1);
            const float qx = dRx - dm.x, qy = dRy - dm.y;
            const float rx = dm.x - dPx, ry = dm.y - dPy;
            const float sx = __shfl_down_sync(FULL, rx, 1), sy = __shfl_down_sync(FULL, ry, 1);
            if (g.cellCol && r > g.r0) qdd += pform(pdx, qx) + pform(rx, sx) + pform(pdy, qy) + pform(ry, sy);
            pdx = qx; pdy = qy; dPx = dm.x; dPy = dm.y;
        }
        nrow++;
        if (nrow == TW || qn > TQ - 32 || qc > TC - 32 || r == g.rEnd) {
            if (qn > q0 || qc > 0) trial_flush<BF16, JM>(Lv, g, V, tau, J, sh, lane, r, nrow, q0, qn, qc);
            else {
                // nothing new queued (so the last row has no exact nodes): only
                // its A, B move to slot 0
                const float a = sh.A[nrow][lane], b = sh.B[nrow][lane];
                __syncwarp();
                sh.A[0][lane] = a;
                sh.B[0][lane] = b;
                sh.qi[0][lane] = 0;
                q0 = qn = 0;
                __syncwarp();
            }
            nrow = 0;
        }
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < JM; j++) {
        const float t = tau[j];
        v[3 * j] = t * (mWA + t * mWB) + sh.sn[0][j][lane];
        v[3 * j + 1] = (t * (mTA + t * mTB) + t * t * (qaa + t * (2.f * qab + t * qbb)) + sh.sn[1][j][lane] +
                        sh.sq[j][lane]) / 18.f;
        v[3 * j + 2] = t * (mRA + t * mRB) + sh.sn[2][j][lane];
    }
    v[3 * REG_MAX_TRIALS + 2] = qdd / 3.f;
}

// Warp sums of a tile's partial record; lane k stores entry k.
template <int JM>
__device__ __forceinline__ void write_partials(const BatchDev &b, int item, const float *v, int nused, int lane)
{
    const unsigned FULL = 0xffffffffu;
    if constexpr (JM <= 4) {
        // The (at most) 15 sums by one transpose-reduction: at each butterfly
        // step (lane offsets 16, 8, 4, 2) a lane keeps half of its values and
        // adds the partner's copy of them, so that after the last step (offset
        // 1) lanes 2 k and 2 k + 1 hold sum k.  Every sum pairs the same lanes
        // in the same order as warp_sum, so the totals are the same floats.
        float x[16];
#pragma unroll
        for (int k = 0; k < 12; k++) x[k] = (k < 3 * JM && k < nused) ? v[k] : 0.f;
#pragma unroll
        for (int k = 0; k < 3; k++) x[12 + k] = v[3 * REG_MAX_TRIALS + k];
        x[15] = 0.f;
#pragma unroll
        for (int o = 16, h = 8; h >= 1; o >>= 1, h >>= 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < h; i++) {
                const float send = up ? x[i] : x[h + i], keep = up ? x[h + i] : x[i];
                x[i] = keep + __shfl_xor_sync(FULL, send, o);
            }
        }
        x[0] += __shfl_xor_sync(FULL, x[0], 1);
        // entry e of the record: sums 0..11 from lanes 0, 2, .., 22; entries
        // 3 MAXT .. 3 MAXT + 2 from lanes 24, 26, 28; the rest zero
        const int src = lane < 12 ? 2 * lane : (lane >= 3 * REG_MAX_TRIALS ? 2 * (12 + lane - 3 * REG_MAX_TRIALS) : 0);
        const float tot = __shfl_sync(FULL, x[0], src & 31);
        const bool has = lane < 12 || (lane >= 3 * REG_MAX_TRIALS && lane < PT_STRIDE);
        if (lane < PT_STRIDE) b.partT[(int64_t)item * PT_STRIDE + lane] = has ? (double)tot : 0.0;
        return;
    }
    double mine = 0.0;
#pragma unroll
    for (int k = 0; k < PT_STRIDE; k++) {
        if ((k < 3 * JM && k < nused) || k >= 3 * REG_MAX_TRIALS) {
            const float tot = warp_sum(v[k]);
            if (lane == k) mine = tot;
        }
    }
    if (lane < PT_STRIDE) b.partT[(int64_t)item * PT_STRIDE + lane] = mine;
}

}  // namespace

template <bool BF16, int JM>
__global__ void __launch_bounds__(REG_STRIP_THREADS, 4) k_trial(BatchDev b)
{
    __shared__ TrialScratch<JM> scratch[REG_STRIP_THREADS / 32];
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (REG_STRIP_THREADS / 32);
    const int nent = b.ctr[3], items = b.ctr[6];
    for (int item = blockIdx.x * (REG_STRIP_THREADS / 32) + (threadIdx.x >> 5); item < items; item += nwarps) {
        const int e = find_entry(b.prefT, nent, item);
        const int o = b.listT[e];
        const OpState &s = b.st[o];
        const LevelDesc &Lv = b.ops[o].lv[s.lvl];
        const StripGeom g = strip_geom(Lv, item - b.prefT[e], lane);
        const bool start = (s.phase == PH_START || s.phase == PH_PROLONG);
        if (start) {
            // sums in double, reduced in double: [0..2] and the Dirichlet form of u
            double v[4];
            start_tile<BF16>(s, Lv, g, v);
            double mine = 0.0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const double tot = warp_sum_d(v[k]);
                if (lane == (k < 3 ? k : 3 * REG_MAX_TRIALS)) mine = tot;
            }
            if (lane < PT_STRIDE) b.partT[(int64_t)item * PT_STRIDE + lane] = mine;
        } else {
            float v[PT_STRIDE];
#pragma unroll
            for (int k = 0; k < PT_STRIDE; k++) v[k] = 0.f;
            unsigned nexact = 0;
            steps_tile<BF16, JM>(s, Lv, g, v, scratch[threadIdx.x >> 5], lane, nexact);
            write_partials<JM>(b, item, v, 3 * min(s.ntr, JM), lane);
            if (lane == 0 && nexact) atomicAdd(&b.work[KW_TEXACT], (unsigned long long)nexact);
        }
    }
}

// ---------------------------------------------------------------------------
// C: per-operator FP64 reduction and the Armijo state machine
// ---------------------------------------------------------------------------
namespace {

// NCC from the FE sums S1 = int That, S2 = int That^2, S3 = int That R~ (R~
// normalised: mean 0, FE sigma 1): NCC = S3 / sqrt(S2 - S1^2).
__device__ __forceinline__ double ncc_of(double S1, double S2, double S3)
{
    double var = S2 - S1 * S1;
    return S3 / (var > 0.0 ? sqrt(var) : 0.0);
}

__device__ void level_end(OpState &s, const OpDesc &op, int status, double pending)
{
    if (status == OPST_NONFINITE) s.nonfinite_seen = 1;
    s.status = status;
    s.tau_acc = pending;
    s.src = s.cur;
    if (s.lvl < op.nl - 1) {
        s.phase = PH_PROLONG;
        s.lvl += 1;
        s.cur = 0;
    } else {
        s.phase = PH_FINAL;
    }
}

// Lockstep replay: the step size the given search of iteration s.iter takes.
__device__ __forceinline__ double lock_step(const OpState &s, const OpDesc &op)
{
    return op.lock_tau[op.lock_off[s.lvl] + s.iter];
}

__device__ __forceinline__ int lock_count(const OpState &s, const OpDesc &op)
{
    return op.lock_off[s.lvl + 1] - op.lock_off[s.lvl];
}

__device__ void set_init_trials(OpState &s, const BatchDev &b, const OpDesc &op)
{
    if (op.lock_tau) {
        // replay: the one step size the reference sequence accepted here
        s.trial_tau[0] = lock_step(s, op);
        s.ntr = 1;
        s.search = SEARCH_INIT;
        return;
    }
    // sequential Armijo order: tau, then 2 tau (if accepted), else tau/2; the
    // pass covers the most likely continuations of both branches.
    int J = b.J;
    int k = 0;
    s.trial_tau[k++] = s.tau;
    double up = s.tau, dn = s.tau;
    while (k < J) {
        if (2.0 * up <= b.tau_max) { up *= 2.0; s.trial_tau[k++] = up; }
        if (k < J && 0.5 * dn >= b.tau_min) { dn *= 0.5; s.trial_tau[k++] = dn; }
        if (2.0 * up > b.tau_max && 0.5 * dn < b.tau_min) break;
    }
    s.ntr = k;
    s.search = SEARCH_INIT;
}

__device__ void schedule_grad(OpState &s, const BatchDev &b, const OpDesc &op, double pending)
{
    s.phase = PH_GRAD;
    s.tau_acc = pending;
    s.src = s.cur;
    s.cur = 1 - s.cur;
    set_init_trials(s, b, op);
}

}  // namespace

__device__ void control_op(const BatchDev &b, OpState &s, const OpDesc &op, int o, int ph, const double *S,
                           double slope, double qud);

__global__ void __launch_bounds__(256) k_control(BatchDev b)
{
    __shared__ double red[8][2];
    __shared__ double redT[9][PT_STRIDE];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int n_ops = b.ctr[0];
    // grid-stride over ops: one block per op, the block reduces the op's tile
    // partials, thread 0 runs the op's Armijo state machine
    for (int o = blockIdx.x; o < n_ops; o += gridDim.x) {
    OpState &s = b.st[o];
    const OpDesc &op = b.ops[o];
    int ph = s.phase;
    if (ph == PH_DONE) continue;
    if (threadIdx.x == 0) {
        // algorithmic work of this step (nodes of the level each kernel swept)
        unsigned long long nn = (unsigned long long)op.lv[s.lvl].n * op.lv[s.lvl].n;
        if (ph == PH_FINAL) atomicAdd(&b.work[KW_PFIN], nn);
        if (ph == PH_PROLONG) { atomicAdd(&b.work[KW_PPROL], nn); atomicAdd(&b.work[KW_TSTART], nn); }
        if (ph == PH_START) atomicAdd(&b.work[KW_TSTART], nn);
        if (ph == PH_GRAD) atomicAdd(&b.work[KW_G], nn);
        if (ph == PH_GRAD || ph == PH_TRIAL) {
            atomicAdd(&b.work[KW_T], nn);
            atomicAdd(&b.work[KW_TSAMPLES], nn * (unsigned long long)s.ntr);
        }
    }
    if (ph == PH_FINAL) {
        __syncthreads();
        if (threadIdx.x == 0) s.phase = PH_DONE;
        __syncthreads();
        continue;
    }
    // reduce the T partials (and G slope partials) of this op over the block:
    // thread t < 9 PT_STRIDE sums entry t % PT_STRIDE of every ninth record
    // from t / PT_STRIDE on, so that a warp's loads are consecutive doubles;
    // thread 0 then adds the nine partial sums of each entry in order
    // (deterministic)
    const int tb = s.t_begin, te = s.t_end;
    if (threadIdx.x < 9 * PT_STRIDE) {
        const int kk = threadIdx.x % PT_STRIDE, g = threadIdx.x / PT_STRIDE;
        double acc = 0.0;
        for (int it = tb + g; it < te; it += 9) acc += b.partT[(int64_t)it * PT_STRIDE + kk];
        redT[g][kk] = acc;
    }
    double slope = 0.0, qud = 0.0;
    if (ph == PH_GRAD) {
        for (int it = s.g_begin + threadIdx.x; it < s.g_end; it += blockDim.x) {
            slope += b.partG[(int64_t)it * PG_STRIDE];
            qud += b.partG[(int64_t)it * PG_STRIDE + 1];
        }
    }
    slope = warp_sum_d(slope);
    qud = warp_sum_d(qud);
    if (lane == 0) {
        red[wid][0] = slope;
        red[wid][1] = qud;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S[PT_STRIDE];
        for (int k = 0; k < PT_STRIDE; k++) {
            double v = 0.0;
            for (int g = 0; g < 9; g++) v += redT[g][k];
            S[k] = v;
        }
        slope = 0.0;
        qud = 0.0;
        for (int w = 0; w < 8; w++) {
            slope += red[w][0];
            qud += red[w][1];
        }
        control_op(b, s, op, o, ph, S, slope, qud);
    }
    __syncthreads();
    }
}

// The Armijo state machine of one operator after a step (thread 0 of its block).
__device__ void control_op(const BatchDev &b, OpState &s, const OpDesc &op, int o, int ph, const double *S,
                           double slope, double qud)
{
    const LevelDesc &Lv = op.lv[s.lvl];
    const double h2 = Lv.h2d;
    if (ph == PH_GRAD && b.smooth) {
        // the smoothed direction's slope and u^T K d (smoother partials, fixed order)
        double sl = 0.0, qd = 0.0;
        const int nch = (Lv.n + REG_GW - 1) / REG_GW;
        for (int ch = 0; ch < nch; ch++) {
            sl += b.partS[((int64_t)s.g_entry * b.cch + ch) * 2];
            qd += b.partS[((int64_t)s.g_entry * b.cch + ch) * 2 + 1];
        }
        slope = -h2 * h2 * sl;
        qud = qd;
    }
    if (ph == PH_GRAD) {
        // the Dirichlet forms of the new search: u^T K d from the gradient pass
        // (or the smoother), d^T K d from its first trial pass
        s.Qud = qud;
        s.Qdd = S[3 * REG_MAX_TRIALS + 2];
    }
    const double Qud = s.Qud, Qdd = s.Qdd;
    if (ph == PH_START || ph == PH_PROLONG) {
        s.S1 = h2 * S[0];
        s.S2 = h2 * S[1];
        s.S3 = h2 * S[2];
        s.Tbar = s.S1;
        double var = s.S2 - s.S1 * s.S1;
        s.sigT = var > 0.0 ? sqrt(var) : 0.0;
        s.ncc = ncc_of(s.S1, s.S2, s.S3);
        s.E = -s.ncc + 0.5 * b.lambda * h2 * S[3 * REG_MAX_TRIALS];
        s.iter = 0;
        s.tau = b.tau_init;
        s.evals += 1;
        if (!isfinite(s.E)) level_end(s, op, OPST_NONFINITE, 0.0);
        else if (op.lock_tau && lock_count(s, op) == 0) level_end(s, op, OPST_MAXITER, 0.0);
        else schedule_grad(s, b, op, 0.0);
        return;
    }
    if (ph == PH_GRAD) {
        s.iter += 1;
        s.iters_total += 1;
        s.slope = slope;
        if (!(slope < 0.0)) {
            level_end(s, op, slope == 0.0 ? OPST_ZERO_GRAD : OPST_NONFINITE, 0.0);
            return;
        }
    }
    s.evals += s.ntr;
    if (op.lock_tau) {
        // lockstep replay: take the given step whatever the test says (the
        // trace records the test), end the level after the last given step
        const double want = s.trial_tau[0];
        double S1 = s.S1 + h2 * S[0], S2 = s.S2 + h2 * S[1], S3 = s.S3 + h2 * S[2];
        double nc = ncc_of(S1, S2, S3);
        double dE = -(nc - s.ncc) + 0.5 * b.lambda * h2 * (2.0 * want * Qud + want * want * Qdd);
        s.trials_seq += 1;
        atomicAdd(&b.work[KW_TSEQ], (unsigned long long)Lv.n * Lv.n);
        bool acc = (dE <= b.sigma * want * s.slope);
        if (b.trace) {
            unsigned long long k = atomicAdd(b.trace_len, 1ull);
            if ((long long)k < b.trace_cap) {
                double *rec = b.trace + 7 * k;
                rec[0] = o; rec[1] = Lv.n; rec[2] = s.iter - 1; rec[3] = want;
                rec[4] = dE; rec[5] = b.sigma * want * s.slope; rec[6] = acc;
            }
        }
        s.E += dE;
        s.S1 = S1; s.S2 = S2; s.S3 = S3;
        s.Tbar = S1;
        double var = S2 - S1 * S1;
        s.sigT = var > 0.0 ? sqrt(var) : 0.0;
        s.ncc = nc;
        s.tau = want;
        if (s.iter >= lock_count(s, op)) level_end(s, op, OPST_MAXITER, want);
        else schedule_grad(s, b, op, want);
        return;
    }
    // Walk the sequential Armijo search over the step sizes evaluated this pass.
    for (int guard = 0; guard < 4 * REG_MAX_TRIALS + 8; guard++) {
        double want;
        if (s.search == SEARCH_INIT) want = s.tau;
        else if (s.search == SEARCH_WIDEN) want = 2.0 * s.btau;
        else want = 0.5 * s.sh_tau;
        bool finish = false, stall = false;
        if (s.search == SEARCH_WIDEN && want > b.tau_max) finish = true;
        if (s.search == SEARCH_SHRINK && want < b.tau_min) stall = true;
        if (!finish && !stall) {
            int j = -1;
            for (int k = 0; k < s.ntr; k++)
                if (s.trial_tau[k] == want) { j = k; break; }
            if (j < 0) {
                // continue the search in another pass
                int k = 0;
                double t = want;
                if (s.search == SEARCH_WIDEN) {
                    while (k < b.J && t <= b.tau_max) { s.trial_tau[k++] = t; t *= 2.0; }
                } else {
                    while (k < b.J && t >= b.tau_min) { s.trial_tau[k++] = t; t *= 0.5; }
                }
                s.ntr = k;
                s.phase = PH_TRIAL;
                return;
            }
            // energy change E(u + tau d) - E(u) from the accumulated sums at u
            double S1 = s.S1 + h2 * S[3 * j], S2 = s.S2 + h2 * S[3 * j + 1], S3 = s.S3 + h2 * S[3 * j + 2];
            double nc = ncc_of(S1, S2, S3);
            double dE = -(nc - s.ncc) + 0.5 * b.lambda * h2 * (2.0 * want * Qud + want * want * Qdd);
            s.trials_seq += 1;
            atomicAdd(&b.work[KW_TSEQ], (unsigned long long)Lv.n * Lv.n);
            bool acc = (dE <= b.sigma * want * s.slope);
            if (b.trace) {
                unsigned long long k = atomicAdd(b.trace_len, 1ull);
                if ((long long)k < b.trace_cap) {
                    double *rec = b.trace + 7 * k;
                    rec[0] = o; rec[1] = Lv.n; rec[2] = s.iter - 1; rec[3] = want;
                    rec[4] = dE; rec[5] = b.sigma * want * s.slope; rec[6] = acc;
                }
            }
            if (acc) { s.bS1 = S1; s.bS2 = S2; s.bS3 = S3; s.bncc = nc; s.bdE = dE; }
            if (s.search == SEARCH_INIT) {
                if (acc) { s.search = SEARCH_WIDEN; s.btau = want; }
                else { s.search = SEARCH_SHRINK; s.sh_tau = want; }
                continue;
            }
            if (s.search == SEARCH_WIDEN) {
                if (acc) { s.btau = want; continue; }
                finish = true;
            } else {
                if (acc) { s.btau = want; finish = true; }
                else { s.sh_tau = want; continue; }
            }
        }
        if (stall) {
            level_end(s, op, OPST_STALLED, 0.0);
            return;
        }
        if (finish) {
            double dec = -s.bdE;
            double scale = fabs(s.E) > 1.0 ? fabs(s.E) : 1.0;
            s.E += s.bdE;
            s.S1 = s.bS1; s.S2 = s.bS2; s.S3 = s.bS3;
            s.Tbar = s.S1;
            double var = s.S2 - s.S1 * s.S1;
            s.sigT = var > 0.0 ? sqrt(var) : 0.0;
            s.ncc = s.bncc;
            s.tau = s.btau;
            if (dec < b.eps * scale) level_end(s, op, OPST_CONVERGED, s.btau);
            else if (s.iter >= b.iter_max) level_end(s, op, OPST_MAXITER, s.btau);
            else schedule_grad(s, b, op, s.btau);
            return;
        }
    }
    atomicExch(&b.ctr[8], 1);  // the search did not terminate: internal error
    s.phase = PH_DONE;
}

// ---------------------------------------------------------------------------
// Series averaging (Section "Introduction": the frames f_i o phi_{0,i} of a
// registered series are averaged into one frame)
// ---------------------------------------------------------------------------

// Node (r, c) of the finest level: 1/m sum_k F_k(x + u_k(x)), F_k frame k's
// stored finest level with its normalisation undone (F = F~ sigma_k + mean_k),
// sampled bilinearly and clamped to the grid; u_k from fields[k] (float2 grid
// units of the finest level; null = the identity).  Sums in double.
template <bool BF16>
__global__ void k_average(const void *__restrict__ pyr, int64_t frame_block, int64_t img_off, int n, int pitch,
                          const double *__restrict__ fstats, const float2 *const *__restrict__ fields, int slot_pitch,
                          int m, float *__restrict__ out, int opitch)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= n || c >= n) return;
    double acc = 0.0;
    for (int k = 0; k < m; k++) {
        const float2 *f = fields[k];
        const float2 u = f ? f[(int64_t)r * slot_pitch + c] : make_float2(0.f, 0.f);
        const void *img = BF16 ? (const void *)(reinterpret_cast<const __nv_bfloat16 *>(pyr) + k * frame_block + img_off)
                               : (const void *)(reinterpret_cast<const float *>(pyr) + k * frame_block + img_off);
        const float v = sample<BF16, false>(img, n, pitch, c, r, u.x, u.y, nullptr, nullptr);
        acc += (double)v * fstats[2 * k + 1] + fstats[2 * k];
    }
    out[(int64_t)r * opitch + c] = (float)(acc / m);
}

void launch_average(int bf16, cudaStream_t st, const void *pyr, int64_t frame_block, int64_t img_off, int n,
                    int pitch, const double *fstats, const float2 *const *fields, int slot_pitch, int m, float *out,
                    int opitch)
{
    dim3 blk(32, 8), grid(cdiv(n, 32), cdiv(n, 8));
    if (bf16) k_average<true><<<grid, blk, 0, st>>>(pyr, frame_block, img_off, n, pitch, fstats, fields, slot_pitch, m, out, opitch);
    else k_average<false><<<grid, blk, 0, st>>>(pyr, frame_block, img_off, n, pitch, fstats, fields, slot_pitch, m, out, opitch);
}

// ---------------------------------------------------------------------------
// Rigid variant (Definition "Rigid transformation": phi(x) = R(alpha) x + t;
// Section "Gradient flow": no smoother in the rigid case)
// ---------------------------------------------------------------------------

// Rigid displacement of node (c, r) in grid units of a level of n nodes:
// u = (R(alpha) - I) x + t with a = cos(alpha) - 1, b = sin(alpha) and the
// translation (tx, ty) in grid units.
__device__ __forceinline__ float2 rigid_u(const RigidReq &q, int c, int r)
{
    return make_float2(fmaf(q.a, (float)c, fmaf(-q.b, (float)r, q.tx)), fmaf(q.b, (float)c, fmaf(q.a, (float)r, q.ty)));
}

// One block per 32 x 32 node tile of one operator (grid: tiles, ops).  For
// every requested parameter set j < q.n_e: the FE sums of the warped template
// That = T(x + u) over the tile (nodes and cells it owns): sum omega That,
// sum of the Q1 element mass forms of That, sum That M~R~ (multiplied by h^2
// on the host).  With q.grad: the data part of dE/dtheta at parameter set 0,
//   -sum_i dNCC/dThat_i (dT_0 du_0/dtheta + dT_1 du_1/dtheta),
//   dNCC/dThat_i = h^2 [ M~R~_i / sigma_T - NCC ((M~ That)_i - T_bar omega_i) / sigma_T^2 ],
// derivatives in Omega units.  That of the tile and a one-node halo is kept in
// shared memory for the cell forms and M~ That.
template <bool BF16>
__global__ void __launch_bounds__(256) k_rigid_eval(const RigidLevel *__restrict__ lv, const RigidReq *__restrict__ req,
                                                    double *__restrict__ part)
{
    constexpr int TS = 32, HS = TS + 2;
    __shared__ float sh[HS][HS + 1];
    __shared__ float red[8][RIGID_SUMS];
    const int o = blockIdx.y;
    const RigidLevel L = lv[o];
    const int n = L.n;
    const int tx = (n + TS - 1) / TS;
    const int tile = blockIdx.x;
    if (tile >= tx * tx) return;
    const int c0 = (tile % tx) * TS, r0 = (tile / tx) * TS;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double *out = part + ((int64_t)o * gridDim.x + tile) * RIGID_SUMS;
    const RigidReq *qs = req + (int64_t)o * REG_MAX_TRIALS;
    auto omega = [n](int i) { return (i == 0 || i == n - 1) ? 0.5f : 1.f; };
    auto w6 = [n](int i, int a) { return a == 0 ? ((i == 0 || i == n - 1) ? 2.f : 4.f) : 1.f; };
    const int nsets = qs[0].n_e;
    for (int j = 0; j < nsets; j++) {
        const RigidReq q = qs[j];
        const bool grad = (j == 0) && q.grad;
        // That on the tile plus a one-node halo (nodes outside the grid: 0)
        for (int k = threadIdx.x; k < HS * HS; k += blockDim.x) {
            const int rr = r0 - 1 + k / HS, cc = c0 - 1 + k % HS;
            float v = 0.f;
            if (rr >= 0 && rr < n && cc >= 0 && cc < n) {
                const float2 u = rigid_u(q, cc, rr);
                v = sample<BF16, false>(L.T, n, L.pitch, cc, rr, u.x, u.y, nullptr, nullptr);
            }
            sh[k / HS][k % HS] = v;
        }
        __syncthreads();
        float s1 = 0.f, s2 = 0.f, s3 = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
        for (int k = threadIdx.x; k < TS * TS; k += blockDim.x) {
            const int lr = k / TS, lc = k % TS, r = r0 + lr, c = c0 + lc;
            if (r >= n || c >= n) continue;
            const float t = sh[lr + 1][lc + 1];
            const float om = omega(r) * omega(c);
            const float mr = L.MR[(int64_t)r * L.pitch + c];
            s1 += om * t;
            s3 += t * mr;
            if (r < n - 1 && c < n - 1) {
                // cell (r, c): corners a=(r,c) b=(r,c+1) cc=(r+1,c+1) d=(r+1,c), element mass (1/36)[4 2 1 2; ...]
                const float A = t, B = sh[lr + 1][lc + 2], C = sh[lr + 2][lc + 2], D = sh[lr + 2][lc + 1];
                s2 += (4.f * (A * A + B * B + C * C + D * D) + 4.f * (A * B + B * C + C * D + D * A) +
                       2.f * (A * C + B * D)) * (1.f / 36.f);
            }
            if (grad) {
                // (36 M~ That)_i: integer weights, boundary rows/cols halved
                float mt = 0.f;
                for (int a = -1; a <= 1; a++) {
                    if (r + a < 0 || r + a >= n) continue;
                    float row = 0.f;
                    for (int b = -1; b <= 1; b++) {
                        if (c + b < 0 || c + b >= n) continue;
                        row += w6(c, b) * sh[lr + 1 + a][lc + 1 + b];
                    }
                    mt += w6(r, a) * row;
                }
                const float2 u = rigid_u(q, c, r);
                float dx, dy;
                sample<BF16, true>(L.T, n, L.pitch, c, r, u.x, u.y, &dx, &dy);
                // dNCC/dThat_i / h^2, times (n - 1) for derivatives in Omega units
                const float dn = (mr * q.inv_sig - q.ncc_over_var * (mt * (1.f / 36.f) - q.tbar * om)) * q.nm1;
                const float x0 = (float)c * q.h, x1 = (float)r * q.h;
                g0 -= dn * (dx * (-q.sa * x0 - q.ca * x1) + dy * (q.ca * x0 - q.sa * x1));
                g1 -= dn * dx;
                g2 -= dn * dy;
            }
        }
        float v[6] = {s1, s2, s3, g0, g1, g2};
        const int nv = grad ? 6 : 3;
        for (int m = 0; m < nv; m++) {
            float w = warp_sum(v[m]);
            if (lane == 0) red[wid][m] = w;
        }
        __syncthreads();
        if (threadIdx.x < nv) {
            double acc = 0.0;
            for (int w = 0; w < 8; w++) acc += red[w][threadIdx.x];
            out[(threadIdx.x < 3 ? 3 * j : 3 * REG_MAX_TRIALS - 3) + threadIdx.x] = acc;
        }
        __syncthreads();
    }
}

// Per operator: the tiles' partial sums in a fixed order (one block per op).
__global__ void k_rigid_reduce(const double *__restrict__ part, int tiles_stride, const RigidLevel *__restrict__ lv,
                               double *__restrict__ sums)
{
    const int o = blockIdx.x;
    const int n = lv[o].n, tx = (n + 31) / 32, tiles = tx * tx;
    __shared__ double red[RIGID_SUMS][8];
    for (int m = 0; m < RIGID_SUMS; m++) {
        double acc = 0.0;
        for (int t = threadIdx.x; t < tiles; t += blockDim.x) acc += part[((int64_t)o * tiles_stride + t) * RIGID_SUMS + m];
        acc = warp_sum_d(acc);
        if ((threadIdx.x & 31) == 0) red[m][threadIdx.x >> 5] = acc;
    }
    __syncthreads();
    if (threadIdx.x < RIGID_SUMS) {
        double acc = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) acc += red[threadIdx.x][w];
        sums[(int64_t)o * RIGID_SUMS + threadIdx.x] = acc;
    }
}

// The finest-level field of rigid parameters, in pixels (= grid units of the
// finest level), into a slot: u = (R(alpha) - I) x + t.
__global__ void k_rigid_fill(RigidReq q, int n, float2 *__restrict__ slot, int pitch)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= n || c >= n) return;
    slot[(int64_t)r * pitch + c] = rigid_u(q, c, r);
}

void launch_rigid(int bf16, int tiles, int n_ops, cudaStream_t st, const RigidLevel *lv, const RigidReq *req,
                  double *part, double *sums)
{
    dim3 grid(tiles, n_ops);
    if (bf16) k_rigid_eval<true><<<grid, 256, 0, st>>>(lv, req, part);
    else k_rigid_eval<false><<<grid, 256, 0, st>>>(lv, req, part);
    k_rigid_reduce<<<n_ops, 256, 0, st>>>(part, tiles, lv, sums);
}

void launch_rigid_fill(const RigidReq &q, int n, float2 *slot, int pitch, cudaStream_t st)
{
    k_rigid_fill<<<dim3(cdiv(n, 32), cdiv(n, 8)), dim3(32, 8), 0, st>>>(q, n, slot, pitch);
}

// ---------------------------------------------------------------------------
// Slot conversion helpers
// ---------------------------------------------------------------------------

// slot (float2, (side+1)^2 grid) -> planes (2 x side x side) for output
__global__ void k_slot_to_planes(const float2 *__restrict__ slot, int pitch, int side, float *__restrict__ out)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= side || c >= side) return;
    float2 v = slot ? slot[(int64_t)r * pitch + c] : make_float2(0.f, 0.f);
    out[(int64_t)r * side + c] = v.x;
    out[(int64_t)side * side + (int64_t)r * side + c] = v.y;
}

// Frames k0 .. k0 + gridDim.z - 1 of a series' deformations, planes (2 x side
// x side each) from their slots: frame k > 0 from slot k - 1 (slots slot_elems
// apart), frame 0 from slot0 (null: the identity, zero displacement).
__global__ void k_slots_to_planes(const float2 *__restrict__ slots, int64_t slot_elems, int k0,
                                  const float2 *__restrict__ slot0, int pitch, int side, float *__restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= side || c >= side) return;
    const int k = k0 + blockIdx.z;
    const float2 *slot = k == 0 ? slot0 : slots + (int64_t)(k - 1) * slot_elems;
    const float2 v = slot ? slot[(int64_t)r * pitch + c] : make_float2(0.f, 0.f);
    float *o = out + (int64_t)blockIdx.z * 2 * side * side;
    o[(int64_t)r * side + c] = v.x;
    o[(int64_t)side * side + (int64_t)r * side + c] = v.y;
}

// planes (2 x n x n) -> slot grid (n x n float2 with pitch)
__global__ void k_planes_to_slot(const float *__restrict__ in, int n, float2 *__restrict__ slot, int pitch)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= n || c >= n) return;
    slot[(int64_t)r * pitch + c] = make_float2(in[(int64_t)r * n + c], in[(int64_t)n * n + (int64_t)r * n + c]);
}

// Host launch wrappers for the templated kernels.
void launch_grad(int bf16, int grid, cudaStream_t st, const BatchDev &b)
{
    if (bf16) k_grad<true><<<grid, REG_STRIP_THREADS, 0, st>>>(b);
    else k_grad<false><<<grid, REG_STRIP_THREADS, 0, st>>>(b);
}

template <int JM>
static void launch_trial_j(int bf16, int grid, cudaStream_t st, const BatchDev &b)
{
    if (bf16) k_trial<true, JM><<<grid, REG_STRIP_THREADS, 0, st>>>(b);
    else k_trial<false, JM><<<grid, REG_STRIP_THREADS, 0, st>>>(b);
}

// J = trials per pass; the kernel instance holds room for the next power of two.
void launch_trial(int bf16, int J, int grid, cudaStream_t st, const BatchDev &b)
{
    if (J <= 1) launch_trial_j<1>(bf16, grid, st, b);
    else if (J <= 2) launch_trial_j<2>(bf16, grid, st, b);
    else if (J <= 4) launch_trial_j<4>(bf16, grid, st, b);
    else launch_trial_j<8>(bf16, grid, st, b);
}

// Resident blocks per SM of the step kernels.  Each asks for the smallest
// shared-memory carveout that still holds its register-limited number of
// blocks, which leaves the rest of the on-chip memory to L1 (the template
// gathers).
template <class K>
static int occupancy(K kernel, int threads, int carveout)
{
    int occ = 0;
    if (carveout < 0) {
        cudaFuncAttributes fa;
        int dev = 0, max_smem = 0, regs_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        cudaFuncGetAttributes(&fa, kernel);
        const int by_regs = fa.numRegs > 0 ? regs_sm / (fa.numRegs * threads) : 1;
        const size_t need = (size_t)by_regs * (fa.sharedSizeBytes + 1024);  // 1 KB reserved per block
        carveout = max_smem > 0 ? (int)std::min<size_t>(100, (need * 100 + max_smem - 1) / max_smem) : 100;
    }
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0);
    return occ;
}

int step_blocks_per_sm(int which, int J)
{
    int occ = 0;
    if (which == 0) {
        occ = occupancy(k_prolong, REG_THREADS, 0);
    } else if (which == 1) {
        occupancy(k_grad<true>, REG_STRIP_THREADS, 0);
        occ = occupancy(k_grad<false>, REG_STRIP_THREADS, 0);
    } else {
        if (J <= 1) { occupancy(k_trial<true, 1>, REG_STRIP_THREADS, -1); occ = occupancy(k_trial<false, 1>, REG_STRIP_THREADS, -1); }
        else if (J <= 2) { occupancy(k_trial<true, 2>, REG_STRIP_THREADS, -1); occ = occupancy(k_trial<false, 2>, REG_STRIP_THREADS, -1); }
        else if (J <= 4) { occupancy(k_trial<true, 4>, REG_STRIP_THREADS, -1); occ = occupancy(k_trial<false, 4>, REG_STRIP_THREADS, -1); }
        else { occupancy(k_trial<true, 8>, REG_STRIP_THREADS, -1); occ = occupancy(k_trial<false, 8>, REG_STRIP_THREADS, -1); }
    }
    cudaGetLastError();
    return occ;
}
