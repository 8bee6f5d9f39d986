// Internal device data structures of libreg (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define REG_MAX_LEVELS 8
#define REG_MAX_TRIALS 8
#define REG_TX 32        // prolongation block tile width (nodes along x_0)
#define REG_TY 32        // prolongation block tile height
#define REG_THREADS 256  // threads per step-kernel block (8 warps)
#define REG_ROWSTEP (REG_THREADS / REG_TX)  // thread (lx, ly) handles rows ly + k REG_ROWSTEP
#define REG_RPT (REG_TY / REG_ROWSTEP)      // rows per thread
// Warp strips of the gradient and trial kernels: the 32 lanes of a warp hold 32
// adjacent node columns and walk down the rows of a tile together, so that
// vertical neighbours stay in registers and horizontal ones are a shuffle away.
#define REG_GW 30  // gradient tile: owned node columns (lanes 1..30; lanes 0, 31 are halo)
#define REG_CW 31  // trial tile: owned cell columns (lanes 0..30; lane 31 is the right corner)
#define REG_STRIP_THREADS 128  // threads per block of the strip kernels (warps work independently)
// Rows per strip tile at a level of n nodes per side (owned node rows of a
// gradient tile, owned cell rows of a trial tile): short strips on the coarse
// levels, where a tile's row walk is latency bound, long ones on the fine
// levels, where the halo rows cost bandwidth.
// Default strip rows of a level of n nodes per side (the tile autotuner may
// pick others per level): short strips where a tile's row walk is latency
// bound, long ones where there are enough tiles.
__host__ __device__ __forceinline__ int strip_rows(int n) { return n <= 65 ? 8 : (n <= 257 ? 16 : 32); }
#define PT_STRIDE (3 * REG_MAX_TRIALS + 3)  // doubles per trial-tile partial record
#define PG_STRIDE 2                         // doubles per gradient-tile partial record

// Phases of the per-operator state machine.
enum {
    PH_START = 0,    // evaluate the energy at the level's initial u (tau = 0)
    PH_GRAD = 1,     // apply the pending step, then gradient + first trial pass
    PH_TRIAL = 2,    // more step sizes of the same Armijo search
    PH_PROLONG = 3,  // apply pending step, prolongate to the next level, then START there
    PH_FINAL = 4,    // apply pending step on the finest level into the output slot
    PH_DONE = 5
};
enum { SEARCH_INIT = 0, SEARCH_WIDEN = 1, SEARCH_SHRINK = 2 };
enum { OPST_CONVERGED = 0, OPST_MAXITER = 1, OPST_STALLED = 2, OPST_NONFINITE = 3, OPST_ZERO_GRAD = 4 };

// Device work counters (nodes swept per kernel family, summed over steps).
enum { KW_G = 0,         // gradient pass nodes
       KW_T = 1,         // trial pass nodes (u, d, R, T read)
       KW_TSTART = 2,    // level-start energy nodes (u, R, T read)
       KW_TSAMPLES = 3,  // trial samples (nodes x step sizes)
       KW_PPROL = 4,     // prolongation: fine nodes written
       KW_PFIN = 5,      // final write: nodes
       KW_TEXACT = 6,    // trial nodes whose largest move leaves the cell (exact path)
       KW_TSEQ = 7,      // nodes x sequential Armijo trials decided (the one-at-a-time rule's trials)
       KW_COUNT = 8 };

// State of one operator at one node of a level, read and written as two
// 16-byte words: the displacement in grid units of the level as a float pair
// per component (value = (x, y) + (z, w), "double-float"), the descent
// direction d = -g / w, and the per-node weights of the current search
// (M~ That at u, M~ R~) that the trial passes use.
struct __align__(16) NodeRec {
    float4 u;
    float2 d;
    float mt;  // 36 M~ That (integer stencil weights, unscaled)
    float mr;  // M~ R~
};

struct LevelDesc {
    int n;            // nodes per side (2^l + 1)
    int pitch;        // row pitch in elements (float2 for U/D, scalar for images)
    int hg, ht;       // strip rows of the gradient and trial tiles at this level
    float h2;         // h^2 = 4^-l (as float for scaling, exact)
    double h2d;       // h^2 in double
    const void *R;    // normalised reference frame (mean 0, FE sigma 1) at this level
    const void *T;    // normalised template frame
    const float *MR;  // M~ R~: the reference frame times the FE mass matrix (units h^2)
    NodeRec *V[2];    // node records, double-buffered (the gradient pass reads one, writes the other)
    const float2 *sm_tab;  // H1-type smoother: Thomas coefficients (c'_i, m_i) of the level's 1D system
};

struct OpDesc {
    int nl;                 // number of levels
    int init;               // 0 identity, 1 copy left, 2 compose(left, right)
    const float2 *left;     // finest-level slot fields (px == grid units of level L)
    const float2 *right;
    float2 *out;            // destination slot (finest level)
    int slot_pitch;
    int judge;              // the output slot holds a learned start: measure the correction
    // Lockstep replay (diagnostic; null: free-running search).  Level k
    // (0 = coarsest) takes exactly the accepted step sizes
    // lock_tau[lock_off[k] .. lock_off[k+1]), one per gradient iteration, and
    // ends after the last of them.
    const double *lock_tau;
    int lock_off[REG_MAX_LEVELS + 1];
    LevelDesc lv[REG_MAX_LEVELS];  // index 0 = coarsest level m0
};

struct OpState {
    int phase, lvl, cur, src;
    int iter, iters_total, trials_seq, evals;
    int status, nonfinite_seen, search, ntr;
    int t_begin, t_end, g_begin, g_end;
    int g_entry;      // index in the gradient pass's op list of this step (smoother partials)
    double tau;       // base step of the current search
    double tau_acc;   // step to apply at the start of the next G/P pass
    double sh_tau;    // shrinking: last rejected step
    double E, Tbar, sigT, ncc;      // at the current u
    double S1, S2, S3;              // FE sums int That, int That^2, int That R~ at the current u
    double bS1, bS2, bS3, bncc, bdE;  // last accepted trial of the search
    double btau;
    double slope;
    double Qud, Qdd;  // Dirichlet forms u^T K d and d^T K d of the current search
    double trial_tau[REG_MAX_TRIALS];
    double corr;  // judged ops: sum over finest nodes of |u_final - u_start| (x + y, px)
};

// Device-side batch: everything the step kernels need, passed by value.
// Sizes that change per batch live in device memory (ctr) so that a captured
// graph stays valid across batches.
struct BatchDev {
    OpDesc *ops;
    OpState *st;
    int *listP, *listG, *listT;  // compacted op indices per family
    int *prefP, *prefG, *prefT;  // exclusive prefix of tile counts (n+1 entries)
    int *ctr;                    // [0] n_ops [1] nP [2] nG [3] nT [4] itemsP [5] itemsG [6] itemsT
                                 // [7] n_active [8] error flag
    double *partG;               // per G item: slope and u^T K d partials (PG_STRIDE)
    double *partT;               // per T item: 3 sums per step size, then 3 Dirichlet forms (PT_STRIDE)
    unsigned long long *work;    // per kernel family: nodes processed
    double *trace;               // optional Armijo trial records (7 doubles each)
    unsigned long long *trace_len;
    long long trace_cap;
    double lambda, sigma, tau_init, tau_max, tau_min, eps;
    int iter_max, J, bf16, pad;
    // H1-type smoother (smooth != 0): per gradient-pass op and column chunk of
    // REG_GW columns, the partial sums {sum omega d_L2 . d, sum d . 6 K u}
    double *partS;
    int smooth, rch, cch;  // row chunks of 32 and column chunks of REG_GW per op (maxima)
    float sm_a;            // off-diagonal of the dimensionless 1D system (1/6 - s^2/2)
};

// Rigid variant: one level of one operator, and one requested parameter set
// (element 0 of an operator's REG_MAX_TRIALS requests carries the count n_e
// and, with grad, the scalars of the gradient at that parameter set).
struct RigidLevel {
    int n, pitch;
    const void *T;     // normalised template at this level
    const float *MR;   // M~ R~ of the normalised reference
};
struct RigidReq {
    float a, b, tx, ty;           // cos(alpha) - 1, sin(alpha), translation in grid units
    float ca, sa, h, nm1;         // cos, sin, grid spacing 1/(n-1) and n-1 (gradient only)
    float inv_sig, ncc_over_var, tbar;  // 1/sigma_T, NCC/sigma_T^2, T_bar at the gradient's parameters
    int n_e, grad;                // request 0: number of parameter sets, gradient wanted
};
#define RIGID_SUMS (3 * REG_MAX_TRIALS + 3)  // 3 energy sums per set, then 3 gradient sums

static inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// Compensated ("double-float") displacement arithmetic.  The accepted steps of
// a level shrink to ~1e-6 grid units while |u| is several units: one float
// cannot take such a step without rounding it by percents, so u is kept as an
// unevaluated sum hi + lo of two floats and updated with an exact two-sum.
// (explicitly rounded adds: the compiler must not contract them into FMAs)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi + lo) + v, renormalised so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ void df_add(float &hi, float &lo, float v)
{
    float s, e;
    two_sum(hi, v, s, e);
    e = __fadd_rn(e, lo);
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

__device__ __forceinline__ float4 df_add2(float4 u, float vx, float vy)
{
    df_add(u.x, u.z, vx);
    df_add(u.y, u.w, vy);
    return u;
}

// floor(x) as an int and as a float without a float-to-int conversion
// instruction (conversions run on the narrow double-precision pipe of this
// GPU): adding 1.5 * 2^23 rounds x to an integer held in the low mantissa
// bits, one correction step turns round-to-nearest into floor.  |x| < 2^22.
__device__ __forceinline__ int floor_i(float x, float &fl)
{
    const float magic = 12582912.0f;  // 1.5 * 2^23
    float t = __fadd_rn(x, magic);
    int i = __float_as_int(t) - 0x4B400000;
    float r = __fsub_rn(t, magic);
    if (r > x) {
        i -= 1;
        r -= 1.f;
    }
    fl = r;
    return i;
}

// Integer part and fraction of hi + lo.  The fraction is rounded to float, the
// integer part is exact: hi - floor(hi) is exact and is either 0 or at least
// ulp(hi) > |lo|, so hi + lo lies below floor(hi) only when that fraction is 0
// and lo < 0.
__device__ __forceinline__ void df_split(float hi, float lo, int &ip, float &fr)
{
    float f;
    int i = floor_i(hi, f);
    float a = (hi - f) + lo;
    if (a < 0.f) {
        i -= 1;
        a += 1.f;
    }
    ip = i;
    fr = a;
}
