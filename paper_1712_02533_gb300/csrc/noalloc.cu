// Energy of one frame pair at one grid level without any device allocation
// (reg_eval_energy_noalloc).  Some callers must not allocate device memory:
// for instance a plug-in running inside an acquisition pipeline whose host
// application has reserved the device memory up front, or a loop between
// frames that cannot afford the implicit synchronisation of cudaMalloc.  This
// entry point serves them: the caller passes the images, the displacement and
// the output; the only scratch is the file-scope device array below.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/reg.h"

namespace {

constexpr int NA_TX = 32, NA_TY = 32, NA_THREADS = 256;
constexpr int NA_SUMS = 6;  // per tile: int R, int That (pass 1); int Rc^2, int Tc^2, int Rc Tc, Dirichlet form (pass 2)
constexpr int NA_MAX_NODES = REG_NOALLOC_MAX_NODES;
constexpr int NA_MAX_TILES = ((NA_MAX_NODES - 1 + NA_TX - 1) / NA_TX) * ((NA_MAX_NODES - 1 + NA_TY - 1) / NA_TY);
constexpr int NA_OUT = NA_MAX_TILES * NA_SUMS;  // results: {E, NCC, reg, T_bar, sigma_T}, then R_bar

// Per-tile partial sums of the last call, then the results.  Every call
// overwrites the partials of all its tiles before reading them, so nothing has
// to start at zero; calls that overlap on the GPU race on this array.
static __device__ __align__(256) double g_noalloc_scratch[NA_OUT + 8];

__device__ __forceinline__ float bilinear_clamped(const float *T, int n, int pitch, int c, int r, float vx, float vy)
{
    float fx = floorf(vx), fy = floorf(vy);
    int jx = c + (int)fx, jy = r + (int)fy;
    float ax = vx - fx, ay = vy - fy;
    if (jx < 0) { jx = 0; ax = 0.f; } else if (jx >= n - 1) { jx = n - 2; ax = 1.f; }
    if (jy < 0) { jy = 0; ay = 0.f; } else if (jy >= n - 1) { jy = n - 2; ay = 1.f; }
    const float *p = T + (size_t)jy * pitch + jx;
    return (1.f - ay) * ((1.f - ax) * p[0] + ax * p[1]) + ay * ((1.f - ax) * p[pitch] + ax * p[pitch + 1]);
}

__device__ __forceinline__ float warp_sum(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One block per 32 x 32 tile of cells: FE integrals (Q1 element mass form) per
// tile, in double.  Pass 1 (centre == nullptr): int R and int That, for the
// means.  Pass 2: the second moments of the centred images R - R_bar and
// That - T_bar (centring first keeps the FP32 cell sums relative to the
// images' spread, not to their mean) and the Dirichlet form of u.
__global__ void __launch_bounds__(NA_THREADS) k_energy_tiles_noalloc(const float *R, const float *T, int n, int pitch,
                                                                     const float *u, const double *centre,
                                                                     double *scratch)
{
    const int tx = (n - 1 + NA_TX - 1) / NA_TX;
    const int c = (blockIdx.x % tx) * NA_TX + threadIdx.x % NA_TX;
    const int r0 = (blockIdx.x / tx) * NA_TY, ly = threadIdx.x / NA_TX;
    const size_t N = (size_t)n * n;
    const bool second = centre != nullptr;
    const float Rb = second ? (float)centre[5] : 0.f, Tb = second ? (float)centre[3] : 0.f;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int lr = ly; lr < NA_TY; lr += NA_THREADS / NA_TX) {
        const int r = r0 + lr;
        if (r >= n - 1 || c >= n - 1) continue;
        // cyclic corners a=(r,c) b=(r,c+1) c=(r+1,c+1) d=(r+1,c)
        const int cr[4] = {r, r, r + 1, r + 1}, cc[4] = {c, c + 1, c + 1, c};
        float Rv[4], Tv[4], ux[4], uy[4];
        for (int k = 0; k < 4; k++) {
            size_t i = (size_t)cr[k] * n + cc[k];
            ux[k] = u[i];
            uy[k] = u[N + i];
            Rv[k] = R[(size_t)cr[k] * pitch + cc[k]] - Rb;
            Tv[k] = bilinear_clamped(T, n, pitch, cc[k], cr[k], ux[k], uy[k]) - Tb;
        }
        if (!second) {
            acc[0] += 0.25f * (Rv[0] + Rv[1] + Rv[2] + Rv[3]);
            acc[1] += 0.25f * (Tv[0] + Tv[1] + Tv[2] + Tv[3]);
            continue;
        }
        // element mass matrix (1/36)[4 2 1 2; 2 4 2 1; 1 2 4 2; 2 1 2 4]
        auto mform = [](const float *v, const float *w) {
            float Mw0 = 4.f * w[0] + 2.f * w[1] + w[2] + 2.f * w[3];
            float Mw1 = 2.f * w[0] + 4.f * w[1] + 2.f * w[2] + w[3];
            float Mw2 = w[0] + 2.f * w[1] + 4.f * w[2] + 2.f * w[3];
            float Mw3 = 2.f * w[0] + w[1] + 2.f * w[2] + 4.f * w[3];
            return (v[0] * Mw0 + v[1] * Mw1 + v[2] * Mw2 + v[3] * Mw3) * (1.f / 36.f);
        };
        acc[0] += mform(Rv, Rv);
        acc[1] += mform(Tv, Tv);
        acc[2] += mform(Rv, Tv);
        // Dirichlet form (p^2 + pq + q^2 + r^2 + rs + s^2) / 3 per component
        for (int ch = 0; ch < 2; ch++) {
            const float *v = ch ? uy : ux;
            float p = v[1] - v[0], q = v[2] - v[3], rr = v[3] - v[0], s = v[2] - v[1];
            acc[3] += (p * p + p * q + q * q + rr * rr + rr * s + s * s) * (1.f / 3.f);
        }
    }
    __shared__ float red[NA_THREADS / 32][4];
    for (int k = 0; k < 4; k++) {
        float v = warp_sum(acc[k]);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < NA_THREADS / 32; w++) t += red[w][threadIdx.x];
        scratch[(size_t)blockIdx.x * NA_SUMS + (second ? 2 : 0) + threadIdx.x] = t;
    }
}

// One block: sums the tiles' partials in a fixed order.  Pass 1 forms the FE
// means R_bar = h^2 int R, T_bar = h^2 int That; pass 2 forms
// sigma^2 = h^2 int (F - F_bar)^2 (FE form), NCC = h^2 int Rc Tc / (sigma_R
// sigma_T) and E = -NCC + lambda/2 h^2 sum |grad u|^2 (Section "Spatial
// discretization").
__global__ void k_energy_finish_noalloc(int n_tiles, int n, double lambda, int second, double *scratch)
{
    __shared__ double red[32][4];
    const int base = second ? 2 : 0, cnt = second ? 4 : 2;
    double s[4] = {0, 0, 0, 0};
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x)
        for (int k = 0; k < cnt; k++) s[k] += scratch[(size_t)t * NA_SUMS + base + k];
    for (int k = 0; k < cnt; k++) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S[4] = {0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x / 32); w++)
            for (int k = 0; k < cnt; k++) S[k] += red[w][k];
        double h2 = 1.0 / ((double)(n - 1) * (n - 1));
        double *out = scratch + NA_OUT;
        if (!second) {
            out[5] = h2 * S[0];  // R_bar
            out[3] = h2 * S[1];  // T_bar
            return;
        }
        // the images were centred on the means rounded to float, c = F_bar + dF:
        // (F - c)^T M (G - c') = (F - F_bar)^T M (G - G_bar) + dF dG  (w^T 1 = 1)
        const double dR = (double)(float)out[5] - out[5], dT = (double)(float)out[3] - out[3];
        double vR = h2 * S[0] - dR * dR, vT = h2 * S[1] - dT * dT;
        double sR = vR > 0.0 ? sqrt(vR) : 0.0, sT = vT > 0.0 ? sqrt(vT) : 0.0;
        double ncc = (h2 * S[2] - dR * dT) / (sR * sT);
        double reg = 0.5 * lambda * h2 * S[3];
        out[0] = -ncc + reg;
        out[1] = ncc;
        out[2] = reg;
        out[4] = sT;
    }
}

std::mutex g_na_mu;
double *g_na_ptr[64] = {nullptr};  // device address of the scratch array, per device

}  // namespace

extern "C" reg_status reg_eval_energy_noalloc(const float *R, const float *T, int32_t n, int32_t pitch,
                                              const float *u_grid, double lambda, double *parts_out,
                                              int32_t out_on_device, void *cuda_stream)
{
    if (!R || !T || !u_grid || !parts_out) return REG_EINVAL;
    if (n < 3 || n > NA_MAX_NODES || pitch < n) return REG_EINVAL;  // beyond the scratch array
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return REG_ECUDA;
    double *scratch;
    {
        // First call on a device: the array's device address, with that device current.
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            e = cudaGetSymbolAddress((void **)&g_na_ptr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_na_ptr[dev] = nullptr;
                return REG_ECUDA;
            }
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int tiles = ((n - 1 + NA_TX - 1) / NA_TX) * ((n - 1 + NA_TY - 1) / NA_TY);
    // pass 1: means; pass 2: centred second moments and the regulariser
    k_energy_tiles_noalloc<<<tiles, NA_THREADS, 0, st>>>(R, T, n, pitch, u_grid, nullptr, scratch);
    k_energy_finish_noalloc<<<1, 1024, 0, st>>>(tiles, n, lambda, 0, scratch);
    k_energy_tiles_noalloc<<<tiles, NA_THREADS, 0, st>>>(R, T, n, pitch, u_grid, scratch + NA_OUT, scratch);
    k_energy_finish_noalloc<<<1, 1024, 0, st>>>(tiles, n, lambda, 1, scratch);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(parts_out, scratch + NA_OUT, 5 * sizeof(double),
                            out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? REG_OK : REG_ECUDA;
}
