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

// 1D FE weights at node i for neighbour offset a in {-1,0,1}: mass (times 6/h)
// and stiffness (times h) of piecewise-linear hats with natural boundary.
__device__ __forceinline__ float m1w(int i, int a, int n)
{
    if (a == 0) return (i == 0 || i == n - 1) ? (2.f / 6.f) : (4.f / 6.f);
    int j = i + a;
    return (j >= 0 && j < n) ? (1.f / 6.f) : 0.f;
}
__device__ __forceinline__ float k1w(int i, int a, int n)
{
    if (a == 0) return (i == 0 || i == n - 1) ? 1.f : 2.f;
    int j = i + a;
    return (j >= 0 && j < n) ? -1.f : 0.f;
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
// two passes over the cells in double; one block per image.
__global__ void k_image_stats(const float *__restrict__ img, int64_t stride, int pitch, int n, double *out)
{
    const float *F = img + blockIdx.x * stride;
    __shared__ double red[32];
    __shared__ double mean_s;
    int cells = (n - 1) * (n - 1);
    double h2 = 1.0 / ((double)(n - 1) * (n - 1));
    double s = 0.0;
    for (int k = threadIdx.x; k < cells; k += blockDim.x) {
        int r = k / (n - 1), c = k % (n - 1);
        const float *p = F + (int64_t)r * pitch + c;
        s += 0.25 * ((double)p[0] + p[1] + p[pitch] + p[pitch + 1]);
    }
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum_d(v);
        if (threadIdx.x == 0) mean_s = v * h2;
    }
    __syncthreads();
    double m = mean_s;
    double q = 0.0;
    for (int k = threadIdx.x; k < cells; k += blockDim.x) {
        int r = k / (n - 1), c = k % (n - 1);
        const float *p = F + (int64_t)r * pitch + c;
        double a = p[0] - m, b = p[1] - m, cc = p[pitch + 1] - m, d = p[pitch] - m;  // cyclic a b c d
        q += (4.0 * (a * a + b * b + cc * cc + d * d) + 4.0 * (a * b + b * cc + cc * d + d * a) +
              2.0 * (a * cc + b * d)) / 36.0;
    }
    q = warp_sum_d(q);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = q;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum_d(v);
        if (threadIdx.x == 0) {
            out[2 * blockIdx.x] = m;
            out[2 * blockIdx.x + 1] = sqrt(v * h2);
        }
    }
}

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
    L.U[0][(int64_t)r * L.pitch + c] = make_float4(a.x, a.y, 0.f, 0.f);
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
            float4 v = F.U[0][(int64_t)r * F.pitch + c];
            float ww = w[a + 1] * w[bb + 1];
            sx += ww * v.x;
            sy += ww * v.y;
        }
    }
    C.U[0][(int64_t)I * C.pitch + J] = make_float4(0.5f * sx, 0.5f * sy, 0.f, 0.f);
}

// Identity initial guess: zero U0 on the coarsest level.  grid (x, y, ops).
__global__ void k_zero_u(BatchDev b)
{
    const OpDesc &op = b.ops[blockIdx.z];
    if (op.init != 0) return;
    const LevelDesc &C = op.lv[0];
    int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= C.n || c >= C.n) return;
    C.U[0][(int64_t)r * C.pitch + c] = make_float4(0.f, 0.f, 0.f, 0.f);
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

__device__ __forceinline__ int node_tiles(int n) { return ((n + REG_TX - 1) / REG_TX) * ((n + REG_TY - 1) / REG_TY); }
__device__ __forceinline__ int cell_tiles(int n) { return ((n - 1 + REG_TX - 1) / REG_TX) * ((n - 1 + REG_TY - 1) / REG_TY); }

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
            int n = op.lv[s.lvl].n;
            if (s.phase != PH_DONE) active++;
            if (s.phase == PH_PROLONG || s.phase == PH_FINAL) { inP = 1; tP = node_tiles(n); }
            if (s.phase == PH_GRAD) { inG = 1; tG = node_tiles(n); }
            if (s.phase == PH_START || s.phase == PH_GRAD || s.phase == PH_TRIAL || s.phase == PH_PROLONG) {
                inT = 1; tT = cell_tiles(n);
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
            if (inG) { b.listG[offE[1] + eG] = o; b.prefG[offE[1] + eG] = offI[1] + iG; }
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
#pragma unroll
        for (int k = 0; k < REG_RPT; k++) {
            const int r = r0 + ly + k * REG_ROWSTEP;
            if (r >= n || c >= n) continue;
            if (fin) {
                float4 u = Lv.U[s.src][(int64_t)r * Lv.pitch + c];
                if (tau != 0.f) {
                    float2 d = Lv.D[s.src][(int64_t)r * Lv.pitch + c];
                    u = df_add2(u, tau * d.x, tau * d.y);
                }
                op.out[(int64_t)r * op.slot_pitch + c] = make_float2(u.x + u.z, u.y + u.w);
            } else {
                const LevelDesc &Cv = op.lv[s.lvl - 1];
                const float4 *U = Cv.U[s.src];
                const float2 *D = Cv.D[s.src];
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
                        float4 u = U[idx];
                        if (tau != 0.f) {
                            float2 d = D[idx];
                            u = df_add2(u, tau * d.x, tau * d.y);
                        }
                        df_add(acc.x, acc.z, w2 * u.x);
                        df_add(acc.x, acc.z, w2 * u.z);
                        df_add(acc.y, acc.w, w2 * u.y);
                        df_add(acc.y, acc.w, w2 * u.w);
                    }
                Lv.U[0][(int64_t)r * Lv.pitch + c] = acc;
            }
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
// Tile: 32 x 32 nodes plus a one-node halo staged in shared memory.
// ---------------------------------------------------------------------------
template <bool BF16>
__global__ void __launch_bounds__(REG_THREADS, 4) k_grad(BatchDev b)
{
    constexpr int HX = REG_TX + 2, HY = REG_TY + 2, HN = HX * HY;
    __shared__ float4 su[HN];
    __shared__ float sT[HN], sR[HN], sgx[HN], sgy[HN];
    __shared__ float red[REG_THREADS / 32];
    int nent = b.ctr[2], items = b.ctr[5];
    int b0, b1;
    block_range(items, b0, b1);
    if (b0 >= b1) return;
    ItemWalker wk(b.prefG, nent, b0);
    const int lx = threadIdx.x % REG_TX, ly = threadIdx.x / REG_TX;
    for (int item = b0; item < b1; item++) {
        int e = wk.entry(item);
        int o = b.listG[e];
        int t = item - b.prefG[e];
        const OpState &s = b.st[o];
        const LevelDesc &Lv = b.ops[o].lv[s.lvl];
        const int n = Lv.n, pitch = Lv.pitch, tx = (n + REG_TX - 1) / REG_TX;
        const int r0 = (t / tx) * REG_TY, c0 = (t % tx) * REG_TX;
        const float tau = (float)s.tau_acc;
        const float4 *Us = Lv.U[s.src];
        const float2 *Ds = Lv.D[s.src];
        const float Tbar = (float)s.Tbar;
        const float isig = (float)(1.0 / s.sigT), ncc = (float)s.ncc, lam = (float)b.lambda;
        __syncthreads();
        // staging pass 1: the tile's own data (independent loads)
        for (int p = threadIdx.x; p < HN; p += REG_THREADS) {
            int r = r0 - 1 + p / HX, c = c0 - 1 + p % HX;
            float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
            float rv = 0.f;
            if (r >= 0 && r < n && c >= 0 && c < n) {
                int64_t idx = (int64_t)r * pitch + c;
                u = Us[idx];
                if (tau != 0.f) {
                    float2 d = Ds[idx];
                    u = df_add2(u, tau * d.x, tau * d.y);
                }
                rv = ldimg<BF16>(Lv.R, (int)idx);
            }
            su[p] = u; sR[p] = rv;
        }
        __syncthreads();
        // staging pass 2: the warped template and its derivative (gathers)
        for (int p = threadIdx.x; p < HN; p += REG_THREADS) {
            int r = r0 - 1 + p / HX, c = c0 - 1 + p % HX;
            float tv = 0.f, gx = 0.f, gy = 0.f;
            if (r >= 0 && r < n && c >= 0 && c < n)
                tv = sample_df<BF16, true>(Lv.T, n, pitch, c, r, su[p], &gx, &gy) - Tbar;
            sT[p] = tv; sgx[p] = gx; sgy[p] = gy;
        }
        __syncthreads();
        float contrib = 0.f;
        const int c = c0 + lx;
#pragma unroll
        for (int k = 0; k < REG_RPT; k++) {
            const int lr = ly + k * REG_ROWSTEP, r = r0 + lr;
            if (r >= n || c >= n) continue;
            float mT = 0.f, mR = 0.f, kux = 0.f, kuy = 0.f;
            const int pc = (lr + 1) * HX + lx + 1;
            const float4 u0 = su[pc];
#pragma unroll
            for (int a = -1; a <= 1; a++) {
                float wr = m1w(r, a, n), kr = k1w(r, a, n);
#pragma unroll
                for (int bb = -1; bb <= 1; bb++) {
                    float wc = m1w(c, bb, n), kc = k1w(c, bb, n);
                    int p = (lr + 1 + a) * HX + (lx + 1 + bb);
                    float wm = wr * wc, wkk = kr * wc + wr * kc;
                    mT += wm * sT[p];
                    mR += wm * sR[p];
                    // K has zero row sums: K u = sum w (u_p - u_0), the differences
                    // formed from the hi and lo parts separately
                    float4 up = su[p];
                    kux += wkk * ((up.x - u0.x) + (up.z - u0.z));
                    kuy += wkk * ((up.y - u0.y) + (up.w - u0.w));
                }
            }
            float A = mR * isig - ncc * mT * isig * isig;
            float psx = -A * sgx[pc] + lam * kux;
            float psy = -A * sgy[pc] + lam * kuy;
            float om = ((r == 0 || r == n - 1) ? 0.5f : 1.f) * ((c == 0 || c == n - 1) ? 0.5f : 1.f);
            float inv = 1.f / (Lv.h2 * om);
            int64_t idx = (int64_t)r * pitch + c;
            Lv.U[s.cur][idx] = su[pc];
            Lv.D[s.cur][idx] = make_float2(-psx * inv, -psy * inv);
            contrib -= (psx * psx + psy * psy) / om;
        }
        contrib = warp_sum(contrib);
        if (lx == 0) red[ly] = contrib;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
#pragma unroll
            for (int w = 0; w < REG_THREADS / 32; w++) tot += red[w];
            b.partG[item] = tot;
        }
    }
}

// ---------------------------------------------------------------------------
// T: warp + energy.
// Level-start pass (tau = 0): full sums at u, per cell (Q1 element)
//   [0] int That / h^2   [1] int That^2 / h^2   [2] int That R~ / h^2   [3 MAXT] Quu
// Trial pass: for every step size tau_j the change against the current u.
// Per node delta_j = That(u + tau_j d) - That(u); when both points lie in the
// same bilinear cell it is formed from the same four texels as
//   tau d_x [(1-a_y') (t01-t00) + a_y' (t11-t10)] + tau d_y [(1-a_x) (t10-t00) + a_x (t11-t01)],
// so that its float rounding is relative to delta itself (the quantity the
// Armijo test compares), not to That; across a cell line it is formed in
// double precision.
//   [3j] int delta / h^2   [3j+1] int delta (2 That + delta) / h^2   [3j+2] int delta R~ / h^2
// and the Dirichlet form of u + tau d as Quu + 2 tau Qud + tau^2 Qdd.
// Tile: 32 x 32 cells, i.e. 33 x 33 nodes staged in shared memory.
// ---------------------------------------------------------------------------
#define PT_STRIDE (3 * REG_MAX_TRIALS + 3)

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

// locate() for a compensated displacement (exact cell choice at cell lines)
__device__ __forceinline__ void locate_df(int n, int c, int r, float4 u, int &jx, int &jy, float &ax, float &ay,
                                          bool &clx, bool &cly)
{
    int ix, iy;
    df_split(u.x, u.z, ix, ax);
    df_split(u.y, u.w, iy, ay);
    jx = c + ix;
    jy = r + iy;
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

// Double-precision bilinear sample at grid point (X, Y), clamped like sample().
template <bool BF16>
__device__ double sample_d(const void *img, int n, int pitch, double X, double Y)
{
    if (X < 0.0) X = 0.0;
    if (X > n - 1) X = n - 1;
    if (Y < 0.0) Y = 0.0;
    if (Y > n - 1) Y = n - 1;
    int jx = (int)floor(X), jy = (int)floor(Y);
    if (jx > n - 2) jx = n - 2;
    if (jy > n - 2) jy = n - 2;
    double ax = X - jx, ay = Y - jy;
    int i0 = jy * pitch + jx;
    double t00 = ldimg<BF16>(img, i0), t01 = ldimg<BF16>(img, i0 + 1);
    double t10 = ldimg<BF16>(img, i0 + pitch), t11 = ldimg<BF16>(img, i0 + pitch + 1);
    return (1.0 - ay) * ((1.0 - ax) * t00 + ax * t01) + ay * ((1.0 - ax) * t10 + ax * t11);
}

// Change of the sample across a cell line (or at a clamp), in double: a float
// in-cell fraction cannot resolve sub-ulp moves across the line (1 - 2e-8
// rounds to 1), which would lose the energy change of the move.
template <bool BF16>
__device__ __noinline__ float cross_delta(const void *img, int n, int pitch, int c, int r, float4 u, float tau,
                                          float dx, float dy)
{
    double X0 = c + ((double)u.x + (double)u.z), Y0 = r + ((double)u.y + (double)u.w);
    double X1 = X0 + (double)tau * dx, Y1 = Y0 + (double)tau * dy;
    return (float)(sample_d<BF16>(img, n, pitch, X1, Y1) - sample_d<BF16>(img, n, pitch, X0, Y0));
}

// Change of the interpolant for a move (ex, ey) of less than one cell from an
// unclamped base point in cell (jx, jy) at fractions (ax, ay), when the move
// leaves the cell.  The move is split into its x part (along the row band of
// the base point) and its y part (at the new column); each part is a sum of
// segment lengths times the slope of the cell the segment lies in, so float
// rounding stays relative to the change itself even for moves far below one
// ulp of the fraction.  Past the grid border the interpolant is constant.
template <bool BF16>
__device__ __noinline__ float cross_delta_f32(const void *img, int n, int pitch, int jx, int jy, float ax, float ay,
                                              float ex, float ey)
{
    auto T = [&](int r, int c) { return ldimg<BF16>(img, r * pitch + c); };
    // slope along x of cell column i in row band jy at fraction ay (grid units)
    auto sx = [&](int i) {
        return (1.f - ay) * (T(jy, i + 1) - T(jy, i)) + ay * (T(jy + 1, i + 1) - T(jy + 1, i));
    };
    float dx = 0.f, ax1 = ax + ex;
    int cx = jx;  // cell column of the new x position
    if (ax1 >= 1.f) {
        dx = (1.f - ax) * sx(jx);
        if (jx + 1 <= n - 2) dx += (ex - (1.f - ax)) * sx(jx + 1);  // beyond the border: flat
        cx = jx + 1 <= n - 2 ? jx + 1 : jx;
        ax1 = jx + 1 <= n - 2 ? ex - (1.f - ax) : 1.f;
    } else if (ax1 < 0.f) {
        dx = -ax * sx(jx);
        if (jx - 1 >= 0) dx += (ex + ax) * sx(jx - 1);
        cx = jx - 1 >= 0 ? jx - 1 : jx;
        ax1 = jx - 1 >= 0 ? 1.f + (ex + ax) : 0.f;
    } else {
        dx = ex * sx(jx);
    }
    // slope along y of cell row j at column cell cx and fraction ax1
    auto sy = [&](int j) {
        return (1.f - ax1) * (T(j + 1, cx) - T(j, cx)) + ax1 * (T(j + 1, cx + 1) - T(j, cx + 1));
    };
    float dy = 0.f, ay1 = ay + ey;
    if (ay1 >= 1.f) {
        dy = (1.f - ay) * sy(jy);
        if (jy + 1 <= n - 2) dy += (ey - (1.f - ay)) * sy(jy + 1);
    } else if (ay1 < 0.f) {
        dy = -ay * sy(jy);
        if (jy - 1 >= 0) dy += (ey + ay) * sy(jy - 1);
    } else {
        dy = ey * sy(jy);
    }
    return dx + dy;
}

}  // namespace

template <int JM>
constexpr int trial_smem_bytes()
{
    return (REG_TX + 1) * (REG_TY + 1) *
           ((int)sizeof(float4) + (int)sizeof(float2) + 2 * (int)sizeof(float) + JM * (int)sizeof(float));
}

template <bool BF16, int JM>
__global__ void __launch_bounds__(REG_THREADS, 4) k_trial(BatchDev b)
{
    constexpr int HX = REG_TX + 1, HY = REG_TY + 1, HN = HX * HY;
    constexpr int NACC = 3 * JM + 3;
    extern __shared__ float4 dyn_smem[];
    float4 *su = reinterpret_cast<float4 *>(dyn_smem);
    float2 *sd = reinterpret_cast<float2 *>(su + HN);
    float *sR = reinterpret_cast<float *>(sd + HN);
    float *sT0 = sR + HN;
    float *sDel = sT0 + HN;  // [JM][HN]
    __shared__ float red[REG_THREADS / 32][NACC];
    int nent = b.ctr[3], items = b.ctr[6];
    int b0, b1;
    block_range(items, b0, b1);
    if (b0 >= b1) return;
    ItemWalker wk(b.prefT, nent, b0);
    const int lx = threadIdx.x % REG_TX, ly = threadIdx.x / REG_TX;
    for (int item = b0; item < b1; item++) {
        int e = wk.entry(item);
        int o = b.listT[e];
        int t = item - b.prefT[e];
        const OpState &s = b.st[o];
        const LevelDesc &Lv = b.ops[o].lv[s.lvl];
        const int n = Lv.n, pitch = Lv.pitch, tx = (n - 1 + REG_TX - 1) / REG_TX;
        const int r0 = (t / tx) * REG_TY, c0 = (t % tx) * REG_TX;
        const bool start = (s.phase == PH_START || s.phase == PH_PROLONG);
        const int J = start ? 0 : min(s.ntr, JM);
        float tau[JM];
#pragma unroll
        for (int j = 0; j < JM; j++) tau[j] = (j < J) ? (float)s.trial_tau[j] : 0.f;
        const float4 *U = Lv.U[s.cur];
        const float2 *D = Lv.D[s.cur];
        __syncthreads();
        // staging pass 1: the tile's own data (independent loads)
        for (int p = threadIdx.x; p < HN; p += REG_THREADS) {
            int r = r0 + p / HX, c = c0 + p % HX;
            float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 d = make_float2(0.f, 0.f);
            float rv = 0.f;
            if (r < n && c < n) {
                int64_t idx = (int64_t)r * pitch + c;
                u = U[idx];
                if (!start) d = D[idx];
                rv = ldimg<BF16>(Lv.R, (int)idx);
            }
            su[p] = u; sd[p] = d; sR[p] = rv;
        }
        __syncthreads();
        // staging pass 2: warped template at u and its changes for every step
        for (int p = threadIdx.x; p < HN; p += REG_THREADS) {
            int r = r0 + p / HX, c = c0 + p % HX;
            float t0 = 0.f;
            if (r < n && c < n) {
                const float4 u = su[p];
                const float2 d = sd[p];
                Texel4 q;
                locate_df(n, c, r, u, q.jx, q.jy, q.ax, q.ay, q.clx, q.cly);
                fetch<BF16>(q, Lv.T, pitch);
                t0 = bil(q);
#pragma unroll
                for (int j = 0; j < JM; j++) {
                    if (j < J) {
                        float ex = tau[j] * d.x, ey = tau[j] * d.y;
                        float ax1 = q.ax + ex, ay1 = q.ay + ey;
                        float del;
                        if (!(q.clx | q.cly) && ax1 >= 0.f && ax1 < 1.f && ay1 >= 0.f && ay1 < 1.f) {
                            del = ex * ((1.f - ay1) * (q.t01 - q.t00) + ay1 * (q.t11 - q.t10)) +
                                  ey * ((1.f - q.ax) * (q.t10 - q.t00) + q.ax * (q.t11 - q.t01));
                        } else if (fabsf(ex) < 0x1p-10f && fabsf(ey) < 0x1p-10f) {
                            // a tiny move across a cell line: exact segment split; from a
                            // clamped base point (outside the grid): double precision
                            if (!(q.clx | q.cly))
                                del = cross_delta_f32<BF16>(Lv.T, n, pitch, q.jx, q.jy, q.ax, q.ay, ex, ey);
                            else
                                del = cross_delta<BF16>(Lv.T, n, pitch, c, r, u, tau[j], d.x, d.y);
                        } else {
                            // a move of at least 2^-10 grid units: a fresh float sample;
                            // its rounding (~1e-7 of That) is small against delta
                            Texel4 w;
                            locate(n, c, r, (u.x + u.z) + ex, (u.y + u.w) + ey, w.jx, w.jy, w.ax, w.ay, w.clx, w.cly);
                            fetch<BF16>(w, Lv.T, pitch);
                            del = bil(w) - t0;
                        }
                        sDel[j * HN + p] = del;
                    }
                }
            }
            sT0[p] = t0;
        }
        __syncthreads();
        float acc[NACC];
#pragma unroll
        for (int k = 0; k < NACC; k++) acc[k] = 0.f;
        const int c = c0 + lx;
#pragma unroll
        for (int kk = 0; kk < REG_RPT; kk++) {
            const int lr = ly + kk * REG_ROWSTEP, r = r0 + lr;
            if (r >= n - 1 || c >= n - 1) continue;
            // cyclic corners a=(r,c) b=(r,c+1) c=(r+1,c+1) d=(r+1,c); element mass
            // matrix (1/36)[4 2 1 2; 2 4 2 1; 1 2 4 2; 2 1 2 4]
            const int pa = lr * HX + lx, pb = pa + 1, pc = pa + HX + 1, pd = pa + HX;
            float Ra = sR[pa], Rb = sR[pb], Rc = sR[pc], Rd = sR[pd];
            float MRa = (4.f * Ra + 2.f * Rb + Rc + 2.f * Rd) * (1.f / 36.f);
            float MRb = (2.f * Ra + 4.f * Rb + 2.f * Rc + Rd) * (1.f / 36.f);
            float MRc = (Ra + 2.f * Rb + 4.f * Rc + 2.f * Rd) * (1.f / 36.f);
            float MRd = (2.f * Ra + Rb + 2.f * Rc + 4.f * Rd) * (1.f / 36.f);
            float ta = sT0[pa], tb = sT0[pb], tc = sT0[pc], td = sT0[pd];
            if (start) {
                float Ma = 4.f * ta + 2.f * tb + tc + 2.f * td;
                float Mb = 2.f * ta + 4.f * tb + 2.f * tc + td;
                float Mc = ta + 2.f * tb + 4.f * tc + 2.f * td;
                float Md = 2.f * ta + tb + 2.f * tc + 4.f * td;
                acc[0] += 0.25f * (ta + tb + tc + td);
                acc[1] += (ta * Ma + tb * Mb + tc * Mc + td * Md) * (1.f / 36.f);
                acc[2] += ta * MRa + tb * MRb + tc * MRc + td * MRd;
            }
#pragma unroll
            for (int j = 0; j < JM; j++) {
                if (j < J) {
                    const float *dl = sDel + j * HN;
                    float da = dl[pa], db = dl[pb], dc = dl[pc], dd = dl[pd];
                    float wa = 2.f * ta + da, wb = 2.f * tb + db, wc = 2.f * tc + dc, wd = 2.f * td + dd;
                    float Ma = 4.f * wa + 2.f * wb + wc + 2.f * wd;
                    float Mb = 2.f * wa + 4.f * wb + 2.f * wc + wd;
                    float Mc = wa + 2.f * wb + 4.f * wc + 2.f * wd;
                    float Md = 2.f * wa + wb + 2.f * wc + 4.f * wd;
                    acc[3 * j + 0] += 0.25f * (da + db + dc + dd);
                    acc[3 * j + 1] += (da * Ma + db * Mb + dc * Mc + dd * Md) * (1.f / 36.f);
                    acc[3 * j + 2] += da * MRa + db * MRb + dc * MRc + dd * MRd;
                }
            }
            // Dirichlet form on the cell: (p^2 + pq + q^2 + r^2 + rs + s^2) / 3 with
            // p = v_b - v_a, q = v_c - v_d (x differences), r = v_d - v_a, s = v_c - v_b.
            float quu = 0.f, qud = 0.f, qdd = 0.f;
            const float4 Ua = su[pa], Ub = su[pb], Uc = su[pc], Ud = su[pd];
#pragma unroll
            for (int ch = 0; ch < 2; ch++) {
                // u differences from the hi and lo parts separately (the stiffness
                // terms are small differences of values of several grid units)
                float up = ch ? (Ub.y - Ua.y) + (Ub.w - Ua.w) : (Ub.x - Ua.x) + (Ub.z - Ua.z);
                float uq = ch ? (Uc.y - Ud.y) + (Uc.w - Ud.w) : (Uc.x - Ud.x) + (Uc.z - Ud.z);
                float ur = ch ? (Ud.y - Ua.y) + (Ud.w - Ua.w) : (Ud.x - Ua.x) + (Ud.z - Ua.z);
                float us = ch ? (Uc.y - Ub.y) + (Uc.w - Ub.w) : (Uc.x - Ub.x) + (Uc.z - Ub.z);
                float va = ch ? sd[pa].y : sd[pa].x, vb = ch ? sd[pb].y : sd[pb].x;
                float vc = ch ? sd[pc].y : sd[pc].x, vd = ch ? sd[pd].y : sd[pd].x;
                float dp = vb - va, dq = vc - vd, dr = vd - va, ds = vc - vb;
                quu += up * up + up * uq + uq * uq + ur * ur + ur * us + us * us;
                qud += up * dp + 0.5f * (up * dq + uq * dp) + uq * dq + ur * dr + 0.5f * (ur * ds + us * dr) + us * ds;
                qdd += dp * dp + dp * dq + dq * dq + dr * dr + dr * ds + ds * ds;
            }
            acc[3 * JM + 0] += quu * (1.f / 3.f);
            acc[3 * JM + 1] += qud * (1.f / 3.f);
            acc[3 * JM + 2] += qdd * (1.f / 3.f);
        }
        const int nused = start ? 3 : 3 * J;
#pragma unroll
        for (int k = 0; k < NACC; k++) {
            bool used = (k >= 3 * JM) || (k < nused);
            if (used) {
                float v = warp_sum(acc[k]);
                if (lx == 0) red[ly][k] = v;
            }
        }
        __syncthreads();
        if (threadIdx.x < PT_STRIDE) {
            int k = threadIdx.x;
            // map to the fixed partial layout: trials [0, 3 MAXT), Q terms at 3 MAXT
            int src = k < 3 * REG_MAX_TRIALS ? k : 3 * JM + (k - 3 * REG_MAX_TRIALS);
            bool used = (k >= 3 * REG_MAX_TRIALS) || (k < nused);
            double tot = 0.0;
            if (used) {
#pragma unroll
                for (int w = 0; w < REG_THREADS / 32; w++) tot += red[w][src];
            }
            b.partT[(int64_t)item * PT_STRIDE + k] = tot;
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

__device__ void set_init_trials(OpState &s, const BatchDev &b)
{
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

__device__ void schedule_grad(OpState &s, const BatchDev &b, double pending)
{
    s.phase = PH_GRAD;
    s.tau_acc = pending;
    s.src = s.cur;
    s.cur = 1 - s.cur;
    set_init_trials(s, b);
}

}  // namespace

__device__ void control_op(const BatchDev &b, OpState &s, const OpDesc &op, int o, int ph, const double *S,
                           double slope);

__global__ void __launch_bounds__(256) k_control(BatchDev b)
{
    __shared__ double red[8][PT_STRIDE + 1];
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
    // reduce the T partials (and G slope partials) of this op over the block
    double S[PT_STRIDE];
#pragma unroll
    for (int k = 0; k < PT_STRIDE; k++) S[k] = 0.0;
    const int tb = s.t_begin, te = s.t_end;
    for (int it = tb + threadIdx.x; it < te; it += blockDim.x) {
        const double *p = b.partT + (int64_t)it * PT_STRIDE;
#pragma unroll
        for (int k = 0; k < PT_STRIDE; k++) S[k] += p[k];
    }
    double slope = 0.0;
    if (ph == PH_GRAD) {
        for (int it = s.g_begin + threadIdx.x; it < s.g_end; it += blockDim.x) slope += b.partG[it];
    }
#pragma unroll
    for (int k = 0; k < PT_STRIDE; k++) {
        double v = warp_sum_d(S[k]);
        if (lane == 0) red[wid][k] = v;
    }
    slope = warp_sum_d(slope);
    if (lane == 0) red[wid][PT_STRIDE] = slope;
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k <= PT_STRIDE; k++) {
            double v = 0.0;
            for (int w = 0; w < 8; w++) v += red[w][k];
            if (k < PT_STRIDE) S[k] = v; else slope = v;
        }
        control_op(b, s, op, o, ph, S, slope);
    }
    __syncthreads();
    }
}

// The Armijo state machine of one operator after a step (thread 0 of its block).
__device__ void control_op(const BatchDev &b, OpState &s, const OpDesc &op, int o, int ph, const double *S,
                           double slope)
{
    const LevelDesc &Lv = op.lv[s.lvl];
    const double h2 = Lv.h2d;
    const double Qud = S[3 * REG_MAX_TRIALS + 1], Qdd = S[3 * REG_MAX_TRIALS + 2];
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
        else schedule_grad(s, b, 0.0);
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
            else schedule_grad(s, b, s.btau);
            return;
        }
    }
    atomicExch(&b.ctr[8], 1);  // the search did not terminate: internal error
    s.phase = PH_DONE;
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
    if (bf16) k_grad<true><<<grid, REG_THREADS, 0, st>>>(b);
    else k_grad<false><<<grid, REG_THREADS, 0, st>>>(b);
}

template <int JM>
static void launch_trial_j(int bf16, int grid, cudaStream_t st, const BatchDev &b)
{
    constexpr int sm = trial_smem_bytes<JM>();
    static bool init = false;
    if (!init) {
        cudaFuncSetAttribute(k_trial<false, JM>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_trial<true, JM>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        init = true;
    }
    if (bf16) k_trial<true, JM><<<grid, REG_THREADS, sm, st>>>(b);
    else k_trial<false, JM><<<grid, REG_THREADS, sm, st>>>(b);
}

// J = trials per pass; the kernel instance holds room for the next power of two.
void launch_trial(int bf16, int J, int grid, cudaStream_t st, const BatchDev &b)
{
    if (J <= 1) launch_trial_j<1>(bf16, grid, st, b);
    else if (J <= 2) launch_trial_j<2>(bf16, grid, st, b);
    else if (J <= 4) launch_trial_j<4>(bf16, grid, st, b);
    else launch_trial_j<8>(bf16, grid, st, b);
}

int trial_blocks_per_sm(int J);

// Resident blocks per SM of the step kernels (shared-memory carveout set to
// the maximum first, so that the occupancy reflects what a launch gets).
int step_blocks_per_sm(int which, int J)
{
    int occ = 0;
    if (which == 0) {
        cudaFuncSetAttribute(k_prolong, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_prolong, REG_THREADS, 0);
    } else if (which == 1) {
        cudaFuncSetAttribute(k_grad<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(k_grad<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_grad<false>, REG_THREADS, 0);
    } else {
        cudaFuncSetAttribute(k_trial<false, 1>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(k_trial<false, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(k_trial<false, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(k_trial<false, 8>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(k_trial<true, 1>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(k_trial<true, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(k_trial<true, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(k_trial<true, 8>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        // the dynamic shared memory exceeds the 48 KB default: opt in before sizing
        cudaFuncSetAttribute(k_trial<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, trial_smem_bytes<1>());
        cudaFuncSetAttribute(k_trial<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, trial_smem_bytes<2>());
        cudaFuncSetAttribute(k_trial<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, trial_smem_bytes<4>());
        cudaFuncSetAttribute(k_trial<false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, trial_smem_bytes<8>());
        cudaFuncSetAttribute(k_trial<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, trial_smem_bytes<1>());
        cudaFuncSetAttribute(k_trial<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, trial_smem_bytes<2>());
        cudaFuncSetAttribute(k_trial<true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, trial_smem_bytes<4>());
        cudaFuncSetAttribute(k_trial<true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, trial_smem_bytes<8>());
        occ = trial_blocks_per_sm(J);
    }
    cudaGetLastError();
    return occ;
}

int trial_blocks_per_sm(int J)
{
    int occ = 0;
    if (J <= 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trial<false, 1>, REG_THREADS, trial_smem_bytes<1>());
    else if (J <= 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trial<false, 2>, REG_THREADS, trial_smem_bytes<2>());
    else if (J <= 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trial<false, 4>, REG_THREADS, trial_smem_bytes<4>());
    else {
        cudaFuncSetAttribute(k_trial<false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, trial_smem_bytes<8>());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trial<false, 8>, REG_THREADS, trial_smem_bytes<8>());
    }
    return occ;
}
