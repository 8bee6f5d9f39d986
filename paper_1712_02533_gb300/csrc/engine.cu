// Host side of libreg: series handles, pyramid construction, the batched
// operator loop (a device-resident Armijo state machine stepped by a captured
// CUDA graph), the scan driver and the C-ABI entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/reg.h"
#include "reg_common.cuh"
#include "schedule.h"
#include "cnn_internal.h"

// kernels (kernels.cu)
__global__ void k_embed(const float *, int64_t, int64_t, int, float *, int64_t, int);
__global__ void k_restrict_img(const float *, int64_t, int, int, float *, int64_t, int);
void launch_image_stats(const float *img, int64_t stride, int pitch, int n, int n_img, double *part, double *out,
                        cudaStream_t st);
int image_stats_part_doubles(int n_img);
__global__ void k_normalize(const float *, int64_t, int, int, const double *, void *, int64_t, int, int);
__global__ void k_mass_image(const void *, int64_t, int, int, int, float *, int64_t);
__global__ void k_compose(BatchDev);
__global__ void k_restrict_u(BatchDev, int);
__global__ void k_zero_u(BatchDev);
__global__ void k_init_state(BatchDev, int);
__global__ void k_plan(BatchDev);
__global__ void k_prolong(BatchDev);
void launch_grad(int bf16, int grid, cudaStream_t st, const BatchDev &b);
void launch_trial(int bf16, int J, int grid, cudaStream_t st, const BatchDev &b);
void launch_smooth(int grid, cudaStream_t st, const BatchDev &b);
int step_blocks_per_sm(int which, int J);
__global__ void k_control(BatchDev);
__global__ void k_slot_to_planes(const float2 *, int, int, float *);
__global__ void k_slots_to_planes(const float2 *slots, int64_t slot_elems, int k0, const float2 *slot0, int pitch,
                                  int side, float *out);
__global__ void k_planes_to_slot(const float *, int, float2 *, int);
void launch_rigid(int bf16, int tiles, int n_ops, cudaStream_t st, const RigidLevel *lv, const RigidReq *req,
                  double *part, double *sums);
void launch_rigid_fill(const RigidReq &q, int n, float2 *slot, int pitch, cudaStream_t st);
void launch_average(int bf16, cudaStream_t st, const void *pyr, int64_t frame_block, int64_t img_off, int n,
                    int pitch, const double *fstats, const float2 *const *fields, int slot_pitch, int m, float *out,
                    int opitch);

namespace {

thread_local std::string g_err;

reg_status fail(reg_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(x)                                                                                   \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess) return fail(REG_ECUDA, "%s: %s", #x, cudaGetErrorString(e_));    \
    } while (0)

#define RET(x)                                  \
    do {                                        \
        reg_status r_ = (x);                    \
        if (r_ != REG_OK) return r_;            \
    } while (0)

int round_up(int a, int m) { return (a + m - 1) / m * m; }

struct SlotMeta {
    int start = -1, end = -1;  // end < 0: identity / empty
};

struct SeriesInfo {
    int n_frames = 0, side = 0, L = 0, m0 = 0, nl = 0, frame_base = 0;
    int n_data = 0, n_slots = 0;
    std::vector<int> n, pitch;            // per level index k (0 = coarsest)
    std::vector<size_t> img_off;          // element offset of level k inside a frame's pyramid block
    size_t frame_block = 0;               // elements per frame pyramid
    void *pyr = nullptr;                  // n_frames * frame_block elements (float or bf16)
    float *mr = nullptr;                  // M~ R~ of every frame and level, same layout (float)
    float2 *slots = nullptr;              // n_slots * slot_elems
    size_t slot_elems = 0;
    std::vector<SlotMeta> meta;
    bool pre_from_slots = false;          // next scan: preprocessing starts from the data slots
    // Series averaging: pyramid block n_frames (one past the frames) holds the
    // average frame, slot n_slots (one past the scan's slots) frame 0's
    // deformation to it; fstats: FE mean and sigma of every frame's finest level
    // (n_frames + 1 pairs), to undo the normalisation of the stored pyramid.
    double *fstats = nullptr;
    std::vector<std::array<double, 3>> rigid;  // rigid handles: the slots' parameters (alpha, t0, t1 in Omega units)
    const float2 **d_fields = nullptr;    // per frame: its deformation field (null: identity)
    bool refined = false;                 // slots hold deformations to the average frame
    std::vector<size_t> ws_off;           // per level: offset (bytes) of U0 within an op workspace
    size_t ws_bytes = 0;                  // per op
    size_t rec_bytes(int k) const { return (size_t)n[k] * pitch[k] * sizeof(NodeRec); }
    // op workspace of level k: two node-record fields
    size_t level_ws_bytes(int k) const { return 2 * rec_bytes(k); }
};

struct FamilyStats {
    const char *name;
    int64_t launches = 0;
    double ms = 0.0;
    double bytes_per_unit = 0.0;
};

struct OpReq {
    int series, frame_i, frame_k, init;
    int left, right, dst;  // slot indices (-1 none)
    int skip = 0;          // coarse pyramid levels the operator leaves out
    int judge = 0;         // learned start: measure how far the operator moves it
};

constexpr int GRAPH_STEPS = 8;
constexpr int REG_TILE_LEVELS = 16;

// l with n = 2^l + 1
inline int level_of(int n)
{
    int l = 0;
    while ((1 << l) + 1 < n) l++;
    return l;
}
constexpr int NFAM = 6;  // P, G, T, C, plan, setup
enum { F_P = 0, F_G, F_T, F_C, F_PLAN, F_SETUP };

}  // namespace

struct reg_series {
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
    // host transfers: a copy stream, two staging buffers (HOST_STAGE_BYTES
    // each) and their events, so that copies overlap the kernels that fill or
    // drain the staging buffers
    cudaStream_t copy_stream = nullptr;
    void *host_stage[2] = {nullptr, nullptr};
    cudaEvent_t ev_filled[2] = {nullptr, nullptr}, ev_drained[2] = {nullptr, nullptr};
    reg_params p{};
    int bf16 = 0;
    int nsm = 0;
    int grid_P = 0, grid_G = 0, grid_T = 0;  // resident-block grids of the step kernels
    // strip rows of the gradient and trial tiles per level l (2^l + 1 nodes)
    int tile_hg[REG_TILE_LEVELS] = {0}, tile_ht[REG_TILE_LEVELS] = {0};
    std::vector<SeriesInfo> S;
    std::vector<void *> allocs;
    // batch buffers
    int cap_ops = 0;
    int64_t cap_items = 0;
    size_t cap_ws = 0;
    OpDesc *d_ops = nullptr;
    OpState *d_st = nullptr;
    int *d_lists = nullptr;  // listP, listG, listT, prefP, prefG, prefT
    int *d_ctr = nullptr;
    double *d_partG = nullptr, *d_partT = nullptr;
    unsigned long long *d_work = nullptr;
    char *d_ws = nullptr;
    double *d_scratch = nullptr;
    OpDesc *h_ops = nullptr;
    int *h_ctr = nullptr;
    OpState *h_st = nullptr;
    int h_st_cap = 0;
    // graph of GRAPH_STEPS steps
    cudaGraphExec_t gexec = nullptr;
    int graph_gen = -1, buf_gen = 0;
    // profiling
    cudaEvent_t ev[GRAPH_STEPS][NFAM];
    cudaEvent_t ev_end[GRAPH_STEPS];
    bool ev_ok = false;
    FamilyStats fam[NFAM] = {{"prolong"}, {"grad"}, {"trial"}, {"control"}, {"plan"}, {"setup"}};
    unsigned long long work_prev[16] = {0};
    double *d_trace = nullptr;
    unsigned long long *d_trace_len = nullptr;
    long long trace_cap = 0;
    // lockstep replay (reg_set_lockstep): step sizes for batches of lock_ops ops
    int lock_ops = 0, lock_levels = 0;
    std::vector<int> lock_counts;  // lock_ops x lock_levels, coarsest level first
    std::vector<double> lock_taus;
    double *d_lock = nullptr;
    size_t d_lock_cap = 0;
    // H1-type smoother: Thomas pivots per level l (2^l + 1 nodes), partial sums
    float2 *d_smtab[REG_TILE_LEVELS] = {nullptr};
    double *d_partS = nullptr;
    int sm_rch = 0, sm_cch = 0, grid_S = 0;
    // rigid variant buffers
    RigidLevel *d_rlv = nullptr, *h_rlv = nullptr;
    RigidReq *d_rreq = nullptr, *h_rreq = nullptr;
    double *d_rpart = nullptr, *d_rsums = nullptr, *h_rsums = nullptr;
    int rcap_ops = 0;
    int64_t rcap_part = 0;
    // totals for reports
    int64_t tot_steps = 0, tot_ops = 0, tot_iters = 0, tot_trials = 0, tot_evals = 0;
};

namespace {

reg_status dalloc(reg_series *s, void **ptr, size_t bytes)
{
    *ptr = nullptr;
    if (bytes == 0) return REG_OK;
    if (s->p.allocator.alloc) {
        *ptr = s->p.allocator.alloc(bytes, (void *)s->stream, s->p.allocator.ctx);
        if (!*ptr) return fail(REG_ENOMEM, "allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMallocAsync(ptr, bytes, s->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(REG_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
        }
    }
    return REG_OK;
}

void dfree(reg_series *s, void *ptr, size_t bytes)
{
    if (!ptr) return;
    if (s->p.allocator.alloc) {
        if (s->p.allocator.free) s->p.allocator.free(ptr, bytes, (void *)s->stream, s->p.allocator.ctx);
    } else {
        cudaFreeAsync(ptr, s->stream);
    }
}

}  // namespace

namespace {

reg_status track(reg_series *s, void **ptr, size_t bytes)
{
    RET(dalloc(s, ptr, bytes));
    s->allocs.push_back(*ptr);
    s->allocs.push_back(reinterpret_cast<void *>(bytes));
    return REG_OK;
}

void untrack(reg_series *s, void *ptr)
{
    for (size_t i = 0; i + 1 < s->allocs.size(); i += 2)
        if (s->allocs[i] == ptr) {
            dfree(s, ptr, reinterpret_cast<size_t>(s->allocs[i + 1]));
            s->allocs.erase(s->allocs.begin() + i, s->allocs.begin() + i + 2);
            return;
        }
}

// The copy stream, the two staging buffers and their events of host transfers
// (created once per handle; the buffers are tracked allocations).
constexpr size_t HOST_STAGE_BYTES = 64ull << 20;

reg_status host_transfer_setup(reg_series *s)
{
    if (!s->copy_stream) CK(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; i++) {
        if (!s->ev_filled[i]) CK(cudaEventCreateWithFlags(&s->ev_filled[i], cudaEventDisableTiming));
        if (!s->ev_drained[i]) CK(cudaEventCreateWithFlags(&s->ev_drained[i], cudaEventDisableTiming));
        if (!s->host_stage[i]) RET(track(s, &s->host_stage[i], HOST_STAGE_BYTES));
    }
    return REG_OK;
}

BatchDev make_batch(reg_series *s)
{
    BatchDev b;
    memset(&b, 0, sizeof(b));
    b.ops = s->d_ops;
    b.st = s->d_st;
    int c = s->cap_ops;
    b.listP = s->d_lists;
    b.listG = s->d_lists + c;
    b.listT = s->d_lists + 2 * c;
    b.prefP = s->d_lists + 3 * c;
    b.prefG = s->d_lists + 4 * c + 1;
    b.prefT = s->d_lists + 5 * c + 2;
    b.ctr = s->d_ctr;
    b.partG = s->d_partG;
    b.partT = s->d_partT;
    b.work = s->d_work;
    b.trace = s->d_trace;
    b.trace_len = s->d_trace_len;
    b.trace_cap = s->trace_cap;
    b.lambda = s->p.lambda;
    b.sigma = s->p.armijo_sigma;
    b.tau_init = s->p.tau_init;
    b.tau_max = s->p.tau_max;
    b.tau_min = s->p.tau_min;
    b.eps = s->p.epsilon;
    b.iter_max = s->p.iter_max;
    b.J = s->p.trials_per_pass;
    b.bf16 = s->bf16;
    if (s->p.smooth > 0.0) {
        b.smooth = 1;
        b.partS = s->d_partS;
        b.rch = s->sm_rch;
        b.cch = s->sm_cch;
        const double sg = s->p.smooth;
        b.sm_a = (float)(1.0 / 6.0 - 0.5 * sg * sg);
    }
    return b;
}

// Work items per operator at a level of n nodes per side: the largest of the
// prolongation block tiles and the gradient and trial strip tiles.
int max_tiles(const reg_series *s, int n)
{
    const int l = level_of(n);
    int p = cdiv(n, REG_TX) * cdiv(n, REG_TY);
    int g = cdiv(n, REG_GW) * cdiv(n, s->tile_hg[l]);
    int t = cdiv(n - 1, REG_CW) * cdiv(n - 1, s->tile_ht[l]);
    return std::max(p, std::max(g, t));
}

// The largest max_tiles over the levels of a series (from level index k0).
int max_tiles_series(const reg_series *s, const SeriesInfo &si, int k0 = 0)
{
    int m = 0;
    for (int k = k0; k < si.nl; k++) m = std::max(m, max_tiles(s, si.n[k]));
    return m;
}

void fill_level(const reg_series *s, LevelDesc &L, int n, int pitch)
{
    L.n = n;
    L.pitch = pitch;
    L.hg = s->tile_hg[level_of(n)];
    L.ht = s->tile_ht[level_of(n)];
    const double h = 1.0 / (n - 1);
    L.h2d = h * h;
    L.h2 = (float)L.h2d;
    L.sm_tab = s->d_smtab[level_of(n)];
}

// Batch buffers for n_ops operators with ws_total bytes of workspace and up to
// items_total work items in one step.
reg_status ensure_capacity(reg_series *s, int n_ops, size_t ws_total, int64_t items_total)
{
    bool changed = false;
    if (n_ops > s->cap_ops) {
        int c = std::max(n_ops, 2 * s->cap_ops);
        untrack(s, s->d_ops);
        untrack(s, s->d_st);
        untrack(s, s->d_lists);
        if (s->h_ops) cudaFreeHost(s->h_ops);
        RET(track(s, (void **)&s->d_ops, sizeof(OpDesc) * c));
        RET(track(s, (void **)&s->d_st, sizeof(OpState) * c));
        RET(track(s, (void **)&s->d_lists, sizeof(int) * (6 * c + 3)));
        if (s->p.smooth > 0.0) {
            untrack(s, s->d_partS);
            RET(track(s, (void **)&s->d_partS, sizeof(double) * 2 * (size_t)s->sm_cch * c));
        }
        CK(cudaMallocHost((void **)&s->h_ops, sizeof(OpDesc) * c));
        s->cap_ops = c;
        changed = true;
    }
    const int64_t items = items_total;
    if (items > s->cap_items) {
        int64_t c = std::max(items, (int64_t)(1.25 * s->cap_items));
        untrack(s, s->d_partG);
        untrack(s, s->d_partT);
        RET(track(s, (void **)&s->d_partG, sizeof(double) * PG_STRIDE * c));
        RET(track(s, (void **)&s->d_partT, sizeof(double) * PT_STRIDE * c));
        s->cap_items = c;
        changed = true;
    }
    const size_t ws = ws_total;
    if (ws > s->cap_ws) {
        untrack(s, s->d_ws);
        RET(track(s, (void **)&s->d_ws, ws));
        s->cap_ws = ws;
    }
    if (changed) s->buf_gen++;
    return REG_OK;
}

// Capture GRAPH_STEPS steps [P G T C plan] into one executable graph.
reg_status build_graph(reg_series *s)
{
    if (s->gexec && s->graph_gen == s->buf_gen) return REG_OK;
    if (s->gexec) {
        cudaGraphExecDestroy(s->gexec);
        s->gexec = nullptr;
    }
    BatchDev b = make_batch(s);
    cudaGraph_t g;
    // The caller's stream may be the legacy default stream, which cannot be
    // captured: capture on a private stream, launch on the caller's stream.
    if (!s->cap_stream) CK(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = s->cap_stream;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < GRAPH_STEPS; k++) {
        k_prolong<<<s->grid_P, REG_THREADS, 0, cs>>>(b);
        launch_grad(s->bf16, s->grid_G, cs, b);
        if (b.smooth) launch_smooth(s->grid_S, cs, b);
        launch_trial(s->bf16, s->p.trials_per_pass, s->grid_T, cs, b);
        k_control<<<std::min(s->cap_ops, 2048), 256, 0, cs>>>(b);
        k_plan<<<1, 1024, 0, cs>>>(b);
    }
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) return fail(REG_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&s->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(REG_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    s->graph_gen = s->buf_gen;
    return REG_OK;
}

void collect_profile(reg_series *s)
{
    if (!((s->p.flags & REG_FLAG_PROFILE) && s->ev_ok)) return;
    for (int k = 0; k < GRAPH_STEPS; k++) {
        cudaEvent_t seq[NFAM] = {s->ev[k][F_P], s->ev[k][F_G], s->ev[k][F_T], s->ev[k][F_C], s->ev[k][F_PLAN], s->ev_end[k]};
        for (int f = 0; f < 5; f++) {
            float ms = 0.f;
            cudaError_t e = cudaEventElapsedTime(&ms, seq[f], seq[f + 1]);
            if (e == cudaSuccess) s->fam[f].ms += ms;
            else {
                cudaGetLastError();
                s->ev_ok = false;
            }
        }
    }
}

// Resolve image pointers of frame f (series si) at level index k.
const void *img_ptr(reg_series *s, const SeriesInfo &si, int frame, int k)
{
    size_t esz = s->bf16 ? 2 : 4;
    return (const char *)si.pyr + ((size_t)frame * si.frame_block + si.img_off[k]) * esz;
}

// Run one batch of operator applications.  pre_iter runs on the stream after
// all operands have been read (composition) and before any result is written.
template <class F>
reg_status run_batch_rigid(reg_series *s, const std::vector<OpReq> &ops, F pre_iter, int32_t *status_out,
                           int32_t *iters_out);

template <class F>
reg_status run_batch(reg_series *s, const std::vector<OpReq> &ops, F pre_iter, int32_t *status_out,
                     int32_t *iters_out)
{
    if (s->p.flags & REG_FLAG_RIGID) return run_batch_rigid(s, ops, pre_iter, status_out, iters_out);
    int n = (int)ops.size();
    if (n == 0) return pre_iter();
    // each op's workspace at its own offset (series of different sides share a
    // batch without every op taking the largest one's room); the step's work
    // items are at most the sum of the ops' largest tile counts
    std::vector<size_t> ws_off(n);
    size_t ws = 0;
    int64_t items = 0;
    int nl = 0, nLmax = 0;
    for (int i = 0; i < n; i++) {
        const OpReq &o = ops[i];
        const SeriesInfo &si = s->S[o.series];
        ws_off[i] = ws;
        ws += (si.ws_bytes + 255) / 256 * 256;
        items += max_tiles_series(s, si, o.skip);
        nl = std::max(nl, si.nl);
        nLmax = std::max(nLmax, si.n[si.nl - 1]);
    }
    RET(ensure_capacity(s, n, ws, items));
    for (int i = 0; i < n; i++) {
        const OpReq &o = ops[i];
        const SeriesInfo &si = s->S[o.series];
        OpDesc &d = s->h_ops[i];
        memset(&d, 0, sizeof(d));
        d.nl = si.nl - o.skip;
        d.init = o.init;
        d.left = o.left >= 0 ? si.slots + (size_t)o.left * si.slot_elems : nullptr;
        d.right = o.right >= 0 ? si.slots + (size_t)o.right * si.slot_elems : nullptr;
        d.out = si.slots + (size_t)o.dst * si.slot_elems;
        d.slot_pitch = si.pitch[si.nl - 1];
        d.judge = o.judge;
        char *w = s->d_ws + ws_off[i];
        for (int j = 0; j < d.nl; j++) {
            const int k = o.skip + j;  // level index within the series' pyramid
            LevelDesc &L = d.lv[j];
            fill_level(s, L, si.n[k], si.pitch[k]);
            L.R = img_ptr(s, si, o.frame_i, k);
            L.T = img_ptr(s, si, o.frame_k, k);
            L.MR = si.mr + (size_t)o.frame_i * si.frame_block + si.img_off[k];
            char *base = w + si.ws_off[k];
            L.V[0] = (NodeRec *)base;
            L.V[1] = (NodeRec *)(base + si.rec_bytes(k));
        }
    }
    if (s->lock_ops > 0) {
        // lockstep replay: every op of the batch takes the given step sizes
        if (n != s->lock_ops) return fail(REG_EINVAL, "lockstep set for %d ops, batch has %d", s->lock_ops, n);
        for (int i = 0; i < n; i++)
            if (s->h_ops[i].nl != s->lock_levels)
                return fail(REG_EINVAL, "lockstep set for %d levels, op %d has %d", s->lock_levels, i, s->h_ops[i].nl);
        const size_t nt = std::max<size_t>(1, s->lock_taus.size());
        if (nt > s->d_lock_cap) {
            untrack(s, s->d_lock);
            RET(track(s, (void **)&s->d_lock, nt * sizeof(double)));
            s->d_lock_cap = nt;
        }
        if (!s->lock_taus.empty())
            CK(cudaMemcpyAsync(s->d_lock, s->lock_taus.data(), s->lock_taus.size() * sizeof(double),
                               cudaMemcpyHostToDevice, s->stream));
        int off = 0;
        for (int i = 0; i < n; i++) {
            OpDesc &d = s->h_ops[i];
            d.lock_tau = s->d_lock;
            for (int k = 0; k < d.nl; k++) {
                d.lock_off[k] = off;
                off += s->lock_counts[(size_t)i * s->lock_levels + k];
            }
            d.lock_off[d.nl] = off;
        }
    }
    CK(cudaMemcpyAsync(s->d_ops, s->h_ops, sizeof(OpDesc) * n, cudaMemcpyHostToDevice, s->stream));
    s->h_ctr[0] = n;
    for (int k = 1; k < 16; k++) s->h_ctr[k] = 0;
    CK(cudaMemcpyAsync(s->d_ctr, s->h_ctr, sizeof(int) * 16, cudaMemcpyHostToDevice, s->stream));
    BatchDev b = make_batch(s);
    dim3 blk(32, 8);
    k_compose<<<dim3(cdiv(nLmax, 32), cdiv(nLmax, 8), n), blk, 0, s->stream>>>(b);
    for (int st = 1; st < nl; st++) {
        int nc = 0;
        for (auto &o : ops) {
            const SeriesInfo &si = s->S[o.series];
            int k = si.nl - 1 - st;
            if (k >= 0) nc = std::max(nc, si.n[k]);
        }
        k_restrict_u<<<dim3(cdiv(nc, 32), cdiv(nc, 8), n), blk, 0, s->stream>>>(b, st);
    }
    int n0 = 0;
    for (auto &o : ops) n0 = std::max(n0, s->S[o.series].n[0]);
    k_zero_u<<<dim3(cdiv(n0, 32), cdiv(n0, 8), n), blk, 0, s->stream>>>(b);
    CK(cudaGetLastError());
    RET(pre_iter());
    k_init_state<<<cdiv(n, 256), 256, 0, s->stream>>>(b, n);
    k_plan<<<1, 1024, 0, s->stream>>>(b);
    CK(cudaGetLastError());
    s->fam[F_SETUP].launches += 4 + nl;
    const bool prof = (s->p.flags & REG_FLAG_PROFILE) && s->ev_ok;
    if (!prof) RET(build_graph(s));  // profiling launches the same kernels directly
    int max_steps = s->p.max_steps > 0 ? s->p.max_steps
                                       : nl * (s->p.iter_max * (2 + 48 / std::max(1, s->p.trials_per_pass)) + 4) + 64;
    int steps = 0;
    for (;;) {
        if (prof) {
            // profiling: the same step kernels launched one by one between events
            for (int k = 0; k < GRAPH_STEPS; k++) {
                cudaEventRecord(s->ev[k][F_P], s->stream);
                k_prolong<<<s->grid_P, REG_THREADS, 0, s->stream>>>(b);
                cudaEventRecord(s->ev[k][F_G], s->stream);
                launch_grad(s->bf16, s->grid_G, s->stream, b);
                if (b.smooth) launch_smooth(s->grid_S, s->stream, b);  // timed with the gradient family
                cudaEventRecord(s->ev[k][F_T], s->stream);
                launch_trial(s->bf16, s->p.trials_per_pass, s->grid_T, s->stream, b);
                cudaEventRecord(s->ev[k][F_C], s->stream);
                k_control<<<std::min(s->cap_ops, 2048), 256, 0, s->stream>>>(b);
                cudaEventRecord(s->ev[k][F_PLAN], s->stream);
                k_plan<<<1, 1024, 0, s->stream>>>(b);
                cudaEventRecord(s->ev_end[k], s->stream);
            }
            CK(cudaGetLastError());
        } else {
            CK(cudaGraphLaunch(s->gexec, s->stream));
        }
        CK(cudaMemcpyAsync(s->h_ctr, s->d_ctr, sizeof(int) * 16, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        steps += GRAPH_STEPS;
        collect_profile(s);
        for (int f = 0; f < 5; f++) s->fam[f].launches += GRAPH_STEPS;
        if (s->h_ctr[8]) return fail(REG_EKERNEL, "operator state machine reported an internal error");
        if (s->h_ctr[7] == 0) break;
        if (steps > max_steps) return fail(REG_ETIMEOUT, "batch did not finish within %d steps", max_steps);
    }
    s->tot_steps += steps;
    s->tot_ops += n;
    if (n > s->h_st_cap) {
        if (s->h_st) cudaFreeHost(s->h_st);
        CK(cudaMallocHost((void **)&s->h_st, sizeof(OpState) * n));
        s->h_st_cap = n;
    }
    CK(cudaMemcpyAsync(s->h_st, s->d_st, sizeof(OpState) * n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int i = 0; i < n; i++) {
        const OpState &st = s->h_st[i];
        s->tot_iters += st.iters_total;
        s->tot_trials += st.trials_seq;
        s->tot_evals += st.evals;
        if (status_out) status_out[i] = st.nonfinite_seen ? REG_OP_NONFINITE : st.status;
        if (iters_out) iters_out[i] = st.iters_total;
    }
    return REG_OK;
}

// ---------------------------------------------------------------------------
// Rigid variant (Definition "Rigid transformation"): function A on the three
// parameters theta = (alpha, t0, t1) of phi(x) = R(alpha) x + t, by gradient
// descent (no smoother, Section "Gradient flow") with the Armijo rule with
// widening on every level of the pyramid; theta is carried from level to
// level unchanged (Algorithm "Multilevel gradient flow": a rigid deformation
// is not restricted or prolongated).  The energy is E of the non-rigid
// method at phi; for a rigid map the regulariser is 2 lambda (1 - cos alpha)
// exactly.  All operators of a batch advance level by level together; each
// round evaluates, for every active operator, up to trials_per_pass parameter
// sets (energy sums) or the gradient, in one launch over all their tiles, and
// the FP64 state machine of each operator runs on the host.
// ---------------------------------------------------------------------------
struct RigidState {
    std::array<double, 3> th{}, d{}, btheta{};
    double E = 0, S1 = 0, S2 = 0, S3 = 0, ncc = 0, sig = 0, slope = 0, tau = 1, btau = 0, bE = 0, sh_tau = 0;
    double bS[3] = {0, 0, 0};
    int phase = 0;  // 0 start energy, 1 gradient, 2 trials, 3 level done
    int iter = 0, iters_total = 0, search = 0, ntr = 0, status = OPST_MAXITER, nonfinite = 0;
    double trial_tau[REG_MAX_TRIALS];
};

inline std::array<double, 3> rigid_compose_h(const std::array<double, 3> &a, const std::array<double, 3> &b)
{
    // phi_b o phi_a = R(a0 + b0) x + R(b0) ta + tb (phi_a applied first)
    const double cb = cos(b[0]), sb = sin(b[0]);
    return {a[0] + b[0], cb * a[1] - sb * a[2] + b[1], sb * a[1] + cb * a[2] + b[2]};
}

inline RigidReq rigid_req(const std::array<double, 3> &th, int n)
{
    RigidReq q;
    memset(&q, 0, sizeof(q));
    const double nm1 = n - 1;
    const double sh = sin(0.5 * th[0]);
    q.a = (float)(-2.0 * sh * sh);  // cos(alpha) - 1 without cancellation
    q.b = (float)sin(th[0]);
    q.tx = (float)(th[1] * nm1);
    q.ty = (float)(th[2] * nm1);
    q.ca = (float)cos(th[0]);
    q.sa = q.b;
    q.h = (float)(1.0 / nm1);
    q.nm1 = (float)nm1;
    return q;
}

reg_status rigid_capacity(reg_series *s, int n_ops, int64_t tiles)
{
    if (n_ops > s->rcap_ops) {
        const int c = std::max(n_ops, 2 * s->rcap_ops);
        untrack(s, s->d_rlv);
        untrack(s, s->d_rreq);
        untrack(s, s->d_rsums);
        if (s->h_rlv) cudaFreeHost(s->h_rlv);
        if (s->h_rreq) cudaFreeHost(s->h_rreq);
        if (s->h_rsums) cudaFreeHost(s->h_rsums);
        RET(track(s, (void **)&s->d_rlv, sizeof(RigidLevel) * c));
        RET(track(s, (void **)&s->d_rreq, sizeof(RigidReq) * REG_MAX_TRIALS * c));
        RET(track(s, (void **)&s->d_rsums, sizeof(double) * RIGID_SUMS * c));
        CK(cudaMallocHost((void **)&s->h_rlv, sizeof(RigidLevel) * c));
        CK(cudaMallocHost((void **)&s->h_rreq, sizeof(RigidReq) * REG_MAX_TRIALS * c));
        CK(cudaMallocHost((void **)&s->h_rsums, sizeof(double) * RIGID_SUMS * c));
        s->rcap_ops = c;
    }
    if ((int64_t)n_ops * tiles > s->rcap_part) {
        const int64_t c = std::max<int64_t>((int64_t)n_ops * tiles, 2 * s->rcap_part);
        untrack(s, s->d_rpart);
        RET(track(s, (void **)&s->d_rpart, sizeof(double) * RIGID_SUMS * c));
        s->rcap_part = c;
    }
    return REG_OK;
}

// Trial step sizes of one Armijo search pass, in the order the sequential rule
// would try them (the same order as the non-rigid device state machine).
void rigid_init_trials(RigidState &r, const reg_params &p)
{
    int k = 0;
    r.trial_tau[k++] = r.tau;
    double up = r.tau, dn = r.tau;
    while (k < p.trials_per_pass) {
        if (2.0 * up <= p.tau_max) { up *= 2.0; r.trial_tau[k++] = up; }
        if (k < p.trials_per_pass && 0.5 * dn >= p.tau_min) { dn *= 0.5; r.trial_tau[k++] = dn; }
        if (2.0 * up > p.tau_max && 0.5 * dn < p.tau_min) break;
    }
    r.ntr = k;
    r.search = SEARCH_INIT;
}

double rigid_energy(const reg_params &p, double h2, const double *S, double alpha, double &S1, double &S2, double &S3,
                    double &ncc, double &sig)
{
    S1 = h2 * S[0];
    S2 = h2 * S[1];
    S3 = h2 * S[2];
    const double var = S2 - S1 * S1;
    // A warped template without variance (every sample clamped to one border
    // value: the map moved the frame off the image) has no NCC; the FP32 sums
    // leave a spurious variance at their resolution, which would give a huge
    // NCC.  Such a parameter set has no energy (NaN: a trial is rejected), as
    // the exact 0/0 in FP64.
    if (!(var > 1e-6 * S2)) {
        sig = 0.0;
        ncc = NAN;
        return NAN;
    }
    sig = sqrt(var);
    ncc = S3 / sig;
    return -ncc + 2.0 * p.lambda * (1.0 - cos(alpha));
}

template <class F>
reg_status run_batch_rigid(reg_series *s, const std::vector<OpReq> &ops, F pre_iter, int32_t *status_out,
                           int32_t *iters_out)
{
    const int n = (int)ops.size();
    if (n == 0) return pre_iter();
    const reg_params &p = s->p;
    std::vector<RigidState> st(n);
    int nl = 0;
    int64_t max_tiles = 1;
    for (int i = 0; i < n; i++) {
        const OpReq &o = ops[i];
        const SeriesInfo &si = s->S[o.series];
        nl = std::max(nl, si.nl);
        const int tx = cdiv(si.n[si.nl - 1], 32);
        max_tiles = std::max<int64_t>(max_tiles, (int64_t)tx * tx);
        std::array<double, 3> th{0.0, 0.0, 0.0};
        if (o.init >= 1) th = si.rigid[o.left];
        if (o.init == 2) th = rigid_compose_h(si.rigid[o.left], si.rigid[o.right]);
        st[i].th = th;
    }
    RET(pre_iter());  // operands read: copies may overwrite them now
    RET(rigid_capacity(s, n, max_tiles));
    const int J = std::max(1, std::min(p.trials_per_pass, REG_MAX_TRIALS));
    int64_t rounds = 0;
    for (int lvl = 0; lvl < nl; lvl++) {
        // level descriptors (level index counted from the finest one, so that
        // series of different depths end on their finest levels together)
        std::vector<int> act;
        for (int i = 0; i < n; i++) {
            const SeriesInfo &si = s->S[ops[i].series];
            const int k = si.nl - nl + lvl;
            RigidLevel &L = s->h_rlv[i];
            if (k < 0) { L.n = 0; continue; }
            L.n = si.n[k];
            L.pitch = si.pitch[k];
            L.T = img_ptr(s, si, ops[i].frame_k, k);
            L.MR = si.mr + (size_t)ops[i].frame_i * si.frame_block + si.img_off[k];
            RigidState &r = st[i];
            r.phase = 0;
            r.iter = 0;
            r.tau = p.tau_init;
            act.push_back(i);
        }
        CK(cudaMemcpyAsync(s->d_rlv, s->h_rlv, sizeof(RigidLevel) * n, cudaMemcpyHostToDevice, s->stream));
        int guard = 0;
        while (!act.empty()) {
            if (++guard > 4 * (p.iter_max + 2) * (2 + 48 / J) + 64)
                return fail(REG_ETIMEOUT, "rigid batch did not finish its level");
            // requests of this round
            for (int i = 0; i < n; i++) s->h_rreq[(size_t)i * REG_MAX_TRIALS].n_e = 0;
            for (int i : act) {
                RigidState &r = st[i];
                const int nn = s->h_rlv[i].n;
                RigidReq *q = s->h_rreq + (size_t)i * REG_MAX_TRIALS;
                if (r.phase == 0) {
                    q[0] = rigid_req(r.th, nn);
                    q[0].n_e = 1;
                } else if (r.phase == 1) {
                    q[0] = rigid_req(r.th, nn);
                    q[0].n_e = 1;
                    q[0].grad = 1;
                    q[0].inv_sig = (float)(1.0 / r.sig);
                    q[0].ncc_over_var = (float)(r.ncc / (r.sig * r.sig));
                    q[0].tbar = (float)r.S1;
                } else {
                    for (int j = 0; j < r.ntr; j++) {
                        std::array<double, 3> t;
                        for (int c = 0; c < 3; c++) t[c] = r.th[c] + r.trial_tau[j] * r.d[c];
                        q[j] = rigid_req(t, nn);
                    }
                    q[0].n_e = r.ntr;
                }
            }
            CK(cudaMemcpyAsync(s->d_rreq, s->h_rreq, sizeof(RigidReq) * REG_MAX_TRIALS * n, cudaMemcpyHostToDevice,
                               s->stream));
            int lvl_tiles = 1;
            for (int i : act) lvl_tiles = std::max(lvl_tiles, cdiv(s->h_rlv[i].n, 32) * cdiv(s->h_rlv[i].n, 32));
            launch_rigid(s->bf16, lvl_tiles, n, s->stream, s->d_rlv, s->d_rreq, s->d_rpart, s->d_rsums);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(s->h_rsums, s->d_rsums, sizeof(double) * RIGID_SUMS * n, cudaMemcpyDeviceToHost,
                               s->stream));
            CK(cudaStreamSynchronize(s->stream));
            rounds++;
            std::vector<int> next;
            for (int i : act) {
                RigidState &r = st[i];
                const double *S = s->h_rsums + (size_t)i * RIGID_SUMS;
                const int nn = s->h_rlv[i].n;
                const double h2 = 1.0 / ((double)(nn - 1) * (nn - 1));
                bool done = false;
                auto end_level = [&](int status) {
                    r.status = status;
                    if (status == OPST_NONFINITE) r.nonfinite = 1;
                    done = true;
                };
                if (r.phase == 0) {
                    r.E = rigid_energy(p, h2, S, r.th[0], r.S1, r.S2, r.S3, r.ncc, r.sig);
                    if (!std::isfinite(r.E)) end_level(OPST_NONFINITE);
                    else r.phase = 1;
                } else if (r.phase == 1) {
                    double g[3] = {h2 * S[3 * REG_MAX_TRIALS] + 2.0 * p.lambda * sin(r.th[0]),
                                   h2 * S[3 * REG_MAX_TRIALS + 1], h2 * S[3 * REG_MAX_TRIALS + 2]};
                    r.iter++;
                    r.iters_total++;
                    r.slope = 0.0;
                    for (int c = 0; c < 3; c++) {
                        r.d[c] = -g[c];
                        r.slope += g[c] * r.d[c];
                    }
                    if (!(r.slope < 0.0)) end_level(r.slope == 0.0 ? OPST_ZERO_GRAD : OPST_NONFINITE);
                    else {
                        rigid_init_trials(r, p);
                        r.phase = 2;
                    }
                } else {
                    // walk the sequential Armijo rule with widening over the evaluated steps
                    double Et[REG_MAX_TRIALS];
                    for (int j = 0; j < r.ntr; j++) {
                        double a, b, c2, nc, sg;
                        Et[j] = rigid_energy(p, h2, S + 3 * j, r.th[0] + r.trial_tau[j] * r.d[0], a, b, c2, nc, sg);
                    }
                    for (int guard2 = 0; guard2 < 4 * REG_MAX_TRIALS + 8 && !done; guard2++) {
                        double want = r.search == SEARCH_INIT ? r.tau : (r.search == SEARCH_WIDEN ? 2.0 * r.btau : 0.5 * r.sh_tau);
                        bool finish = false;
                        if (r.search == SEARCH_WIDEN && want > p.tau_max) finish = true;
                        if (r.search == SEARCH_SHRINK && want < p.tau_min) {
                            end_level(OPST_STALLED);
                            break;
                        }
                        if (!finish) {
                            int j = -1;
                            for (int k = 0; k < r.ntr; k++)
                                if (r.trial_tau[k] == want) { j = k; break; }
                            if (j < 0) {
                                // continue the search in another round
                                int k = 0;
                                double t = want;
                                if (r.search == SEARCH_WIDEN) { while (k < J && t <= p.tau_max) { r.trial_tau[k++] = t; t *= 2.0; } }
                                else { while (k < J && t >= p.tau_min) { r.trial_tau[k++] = t; t *= 0.5; } }
                                r.ntr = k;
                                break;
                            }
                            const double dE = Et[j] - r.E;
                            const bool acc = dE <= p.armijo_sigma * want * r.slope;
                            if (acc) {
                                r.bE = Et[j];
                                for (int c = 0; c < 3; c++) r.bS[c] = h2 * S[3 * j + c];
                            }
                            if (r.search == SEARCH_INIT) {
                                if (acc) { r.search = SEARCH_WIDEN; r.btau = want; }
                                else { r.search = SEARCH_SHRINK; r.sh_tau = want; }
                                continue;
                            }
                            if (r.search == SEARCH_WIDEN) {
                                if (acc) { r.btau = want; continue; }
                                finish = true;
                            } else {
                                if (acc) { r.btau = want; finish = true; }
                                else { r.sh_tau = want; continue; }
                            }
                        }
                        if (finish) {
                            const double dec = r.E - r.bE, scale = fabs(r.E) > 1.0 ? fabs(r.E) : 1.0;
                            for (int c = 0; c < 3; c++) r.th[c] += r.btau * r.d[c];
                            r.E = r.bE;
                            r.S1 = r.bS[0];
                            r.S2 = r.bS[1];
                            r.S3 = r.bS[2];
                            const double var = r.S2 - r.S1 * r.S1;
                            r.sig = var > 0.0 ? sqrt(var) : 0.0;
                            r.ncc = r.S3 / r.sig;
                            r.tau = r.btau;
                            if (dec < p.epsilon * scale) end_level(OPST_CONVERGED);
                            else if (r.iter >= p.iter_max) end_level(OPST_MAXITER);
                            else r.phase = 1;
                            break;
                        }
                    }
                }
                if (!done) next.push_back(i);
            }
            act.swap(next);
        }
    }
    // results into the destination slots: parameters and the finest field
    for (int i = 0; i < n; i++) {
        const OpReq &o = ops[i];
        SeriesInfo &si = s->S[o.series];
        si.rigid[o.dst] = st[i].th;
        const int nL = si.n[si.nl - 1];
        launch_rigid_fill(rigid_req(st[i].th, nL), nL, si.slots + (size_t)o.dst * si.slot_elems, si.pitch[si.nl - 1],
                          s->stream);
        if (status_out) status_out[i] = st[i].nonfinite ? REG_OP_NONFINITE : st[i].status;
        if (iters_out) iters_out[i] = st[i].iters_total;
        s->tot_iters += st[i].iters_total;
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    s->tot_ops += n;
    s->tot_steps += rounds;
    return REG_OK;
}

// Resident-block grids of the step kernels (the trial kernel's depends on the
// step sizes per pass).
void set_grids(reg_series *s)
{
    auto grid_of = [&](int which) {
        int occ = step_blocks_per_sm(which, s->p.trials_per_pass);
        return s->nsm * std::max(1, std::min(occ, 32));
    };
    s->grid_P = grid_of(0);
    s->grid_G = grid_of(1);
    s->grid_T = grid_of(2);
}

reg_status validate_params(const reg_params *p)
{
    if (p->iter_max < 1 || p->iter_max > 100000) return fail(REG_EINVAL, "iter_max out of range");
    if (!(p->lambda >= 0.0) || !(p->armijo_sigma > 0.0 && p->armijo_sigma < 1.0))
        return fail(REG_EINVAL, "lambda must be >= 0 and 0 < sigma < 1");
    if (!(p->tau_min > 0.0 && p->tau_init >= p->tau_min && p->tau_max >= p->tau_init))
        return fail(REG_EINVAL, "need 0 < tau_min <= tau_init <= tau_max");
    if (p->trials_per_pass < 1 || p->trials_per_pass > REG_MAX_TRIALS)
        return fail(REG_EINVAL, "trials_per_pass must be in [1, %d]", REG_MAX_TRIALS);
    if (p->storage != REG_STORAGE_F32 && p->storage != REG_STORAGE_BF16) return fail(REG_EINVAL, "bad storage");
    if (p->init_levels < 0 || p->init_levels > p->n_levels)
        return fail(REG_EINVAL, "init_levels must be in [0, n_levels]");
    if (!(p->learned_fallback_px >= 0.0)) return fail(REG_EINVAL, "learned_fallback_px must be >= 0");
    if (p->flags & ~(REG_FLAG_PROFILE | REG_FLAG_RIGID)) return fail(REG_EINVAL, "unknown flag");
    if (!(p->smooth >= 0.0 && p->smooth <= 1e3)) return fail(REG_EINVAL, "smooth must be in [0, 1000]");
    return REG_OK;
}

// Pyramid levels of nf frames from their raw finest levels (rawf: nf blocks of
// frame_block floats, level L filled): the restriction chain (1/16 [1 2 1; 2 4
// 2; 1 2 1], Section "Multilevel"), per level the FE mean and sigma and the
// normalised image (stored as float or bf16) with its M~ R~ image, into pyramid
// blocks f0 .. f0+nf-1.  The finest level's mean and sigma are kept in fstats.
void build_levels(reg_series *s, SeriesInfo &si, float *rawf, int f0, int nf, double *stats)
{
    dim3 blk(32, 8);
    const int kL = si.nl - 1;
    for (int k = kL - 1; k >= 0; k--)
        k_restrict_img<<<dim3(cdiv(si.n[k], 32), cdiv(si.n[k], 8), nf), blk, 0, s->stream>>>(
            rawf + si.img_off[k + 1], (int64_t)si.frame_block, si.pitch[k + 1], si.n[k + 1],
            rawf + si.img_off[k], (int64_t)si.frame_block, si.pitch[k]);
    for (int k = 0; k < si.nl; k++) {
        launch_image_stats(rawf + si.img_off[k], (int64_t)si.frame_block, si.pitch[k], si.n[k], nf, stats + 2 * nf,
                           stats, s->stream);
        size_t esz = s->bf16 ? 2 : 4;
        char *dst = (char *)si.pyr + ((size_t)f0 * si.frame_block + si.img_off[k]) * esz;
        k_normalize<<<dim3(cdiv(si.n[k], 32), cdiv(si.n[k], 8), nf), blk, 0, s->stream>>>(
            rawf + si.img_off[k], (int64_t)si.frame_block, si.pitch[k], si.n[k], (const double *)stats, dst,
            (int64_t)si.frame_block, si.pitch[k], s->bf16);
        k_mass_image<<<dim3(cdiv(si.n[k], 32), cdiv(si.n[k], 8), nf), blk, 0, s->stream>>>(
            dst, (int64_t)si.frame_block, si.pitch[k], si.n[k], s->bf16,
            si.mr + (size_t)f0 * si.frame_block + si.img_off[k], (int64_t)si.frame_block);
    }
    cudaMemcpyAsync(si.fstats + 2 * (size_t)f0, stats, sizeof(double) * 2 * nf, cudaMemcpyDeviceToDevice, s->stream);
}

// Copy a slot field (device) to another slot.
reg_status copy_slot(reg_series *s, SeriesInfo &si, int dst, int src)
{
    si.rigid[dst] = si.rigid[src];
    CK(cudaMemcpyAsync(si.slots + (size_t)dst * si.slot_elems, si.slots + (size_t)src * si.slot_elems,
                       si.slot_elems * sizeof(float2), cudaMemcpyDeviceToDevice, s->stream));
    return REG_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" {

void reg_default_params(reg_params *p)
{
    memset(p, 0, sizeof(*p));
    p->n_levels = 3;
    p->iter_max = 50;
    p->epsilon = 1e-7;
    p->lambda = 10.0;
    p->armijo_sigma = 0.5;
    p->tau_init = 1.0;
    p->tau_max = 1e4;
    p->tau_min = 1e-12;
    p->storage = REG_STORAGE_F32;
    p->trials_per_pass = 4;
    p->learned_fallback_px = 2.0;
    p->max_steps = 0;
    p->flags = 0;
}

const char *reg_status_string(reg_status st)
{
    switch (st) {
    case REG_OK: return "ok";
    case REG_EINVAL: return "invalid argument";
    case REG_ENOMEM: return "out of memory";
    case REG_ECUDA: return "CUDA error";
    case REG_ESTATE: return "invalid state";
    case REG_ETIMEOUT: return "step budget exhausted";
    case REG_EKERNEL: return "kernel reported an error";
    }
    return "unknown status";
}

const char *reg_last_error(void) { return g_err.c_str(); }

reg_status reg_create_series(const float *frames, int32_t n_series, const int32_t *frames_per_series,
                             const int32_t *side_px, int64_t pitch_elems, int32_t frames_on_device,
                             const reg_params *p, void *cuda_stream, reg_series_t *out)
{
    g_err.clear();
    if (!out || !frames || !frames_per_series || !side_px || !p || n_series < 1)
        return fail(REG_EINVAL, "null argument or n_series < 1");
    *out = nullptr;
    RET(validate_params(p));
    int64_t total_frames = 0;
    int maxside = 0;
    for (int i = 0; i < n_series; i++) {
        int sd = side_px[i];
        if (sd < 32 || sd > 4096 || (sd & (sd - 1))) return fail(REG_EINVAL, "side %d is not a power of two in [32, 4096]", sd);
        if (frames_per_series[i] < 2) return fail(REG_EINVAL, "series %d has fewer than 2 frames", i);
        int L = 0;
        while ((1 << L) < sd) L++;
        if (p->n_levels < 1 || p->n_levels > L - 3 || p->n_levels > REG_MAX_LEVELS)
            return fail(REG_EINVAL, "n_levels must be in [1, L-3] (L = %d)", L);
        total_frames += frames_per_series[i];
        maxside = std::max(maxside, sd);
    }
    if (pitch_elems < maxside) return fail(REG_EINVAL, "pitch_elems smaller than the largest side");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    reg_series *s = new reg_series();
    s->stream = (cudaStream_t)cuda_stream;
    s->p = *p;
    s->bf16 = p->storage == REG_STORAGE_BF16;
    cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, dev);
    set_grids(s);
    for (int l = 0; l < REG_TILE_LEVELS; l++) s->tile_hg[l] = s->tile_ht[l] = strip_rows((1 << l) + 1);
    CK(cudaMallocHost((void **)&s->h_ctr, sizeof(int) * 16));
    s->ev_ok = true;
    for (int k = 0; k < GRAPH_STEPS && s->ev_ok; k++) {
        for (int f = 0; f < NFAM; f++)
            if (cudaEventCreate(&s->ev[k][f]) != cudaSuccess) s->ev_ok = false;
        if (cudaEventCreate(&s->ev_end[k]) != cudaSuccess) s->ev_ok = false;
    }
    auto cleanup = [&](reg_status st) {
        reg_destroy_series(s);
        return st;
    };
    reg_status st;
    if ((st = track(s, (void **)&s->d_ctr, sizeof(int) * 16)) != REG_OK) return cleanup(st);
    if ((st = track(s, (void **)&s->d_work, sizeof(unsigned long long) * 16)) != REG_OK) return cleanup(st);
    if (cudaMemsetAsync(s->d_work, 0, sizeof(unsigned long long) * 16, s->stream) != cudaSuccess)
        return cleanup(fail(REG_ECUDA, "memset"));
    // series geometry
    int fb = 0;
    int64_t row_off = 0;  // rows of pitch_elems before the current series
    for (int i = 0; i < n_series; i++) {
        SeriesInfo si;
        si.n_frames = frames_per_series[i];
        si.side = side_px[i];
        while ((1 << si.L) < si.side) si.L++;
        si.nl = p->n_levels;
        si.m0 = si.L - si.nl + 1;
        si.frame_base = fb;
        fb += si.n_frames;
        si.n_data = si.n_frames - 1;
        int aux = 0;
        for (int kind = 0; kind <= regsched::K_BLELLOCH; kind++)
            aux = std::max(aux, regsched::aux_slots(kind, si.n_data, 0, 0));
        // chunked strategies: up to 64 chunks with any global algorithm
        aux = std::max(aux, regsched::aux_slots(regsched::K_CHUNKED, si.n_data, 64, regsched::K_BLELLOCH));
        si.n_slots = si.n_data + aux;
        size_t off = 0, woff = 0;
        for (int k = 0; k < si.nl; k++) {
            int nn = (1 << (si.m0 + k)) + 1;
            si.n.push_back(nn);
            si.pitch.push_back(round_up(nn, 32));
            si.img_off.push_back(off);
            off += (size_t)nn * si.pitch.back();
            si.ws_off.push_back(woff);
            woff += si.level_ws_bytes(k);
        }
        si.frame_block = round_up((int)std::min<size_t>(off, (size_t)1 << 30), 64);
        si.ws_bytes = woff;
        si.slot_elems = (size_t)si.n[si.nl - 1] * si.pitch[si.nl - 1];
        si.meta.assign(si.n_slots, SlotMeta{});
        si.rigid.assign(si.n_slots + 1, {0.0, 0.0, 0.0});
        size_t esz = s->bf16 ? 2 : 4;
        const size_t blocks = (size_t)si.n_frames + 1;  // + the average frame
        if ((st = track(s, &si.pyr, si.frame_block * blocks * esz)) != REG_OK) return cleanup(st);
        if ((st = track(s, (void **)&si.mr, si.frame_block * blocks * sizeof(float))) != REG_OK)
            return cleanup(st);
        if ((st = track(s, (void **)&si.slots, si.slot_elems * (si.n_slots + 1) * sizeof(float2))) != REG_OK)
            return cleanup(st);
        if ((st = track(s, (void **)&si.fstats, sizeof(double) * 2 * blocks)) != REG_OK) return cleanup(st);
        if ((st = track(s, (void **)&si.d_fields, sizeof(void *) * si.n_frames)) != REG_OK) return cleanup(st);
        s->S.push_back(si);
    }
    // H1-type smoother: Thomas pivots (c'_i, m_i) of the dimensionless 1D
    // system T = tridiag(1/6 - s^2/2, 2/3 + s^2, .), 1/3 + s^2/2 at the ends,
    // for every level in use
    if (p->smooth > 0.0) {
        const double sg = p->smooth, a = 1.0 / 6.0 - 0.5 * sg * sg;
        int nmax = 0;
        for (auto &si : s->S)
            for (int k = 0; k < si.nl; k++) {
                const int n = si.n[k], l = level_of(n);
                nmax = std::max(nmax, n);
                if (s->d_smtab[l]) continue;
                std::vector<float2> tab(n);
                double cp = 0.0;
                for (int i = 0; i < n; i++) {
                    const double diag = (i == 0 || i == n - 1) ? 1.0 / 3.0 + 0.5 * sg * sg : 2.0 / 3.0 + sg * sg;
                    const double m = 1.0 / (diag - (i > 0 ? a * cp : 0.0));
                    cp = a * m;
                    tab[i] = make_float2((float)cp, (float)m);
                }
                if ((st = track(s, (void **)&s->d_smtab[l], sizeof(float2) * n)) != REG_OK) return cleanup(st);
                if (cudaMemcpyAsync(s->d_smtab[l], tab.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, s->stream) !=
                    cudaSuccess)
                    return cleanup(fail(REG_ECUDA, "smoother table upload"));
                if (cudaStreamSynchronize(s->stream) != cudaSuccess) return cleanup(fail(REG_ECUDA, "sync"));
            }
        s->sm_rch = cdiv(nmax, 32);
        s->sm_cch = cdiv(nmax, REG_GW);
        s->grid_S = s->nsm * 8;
    }
    // Pyramid construction in chunks of frames: raw level L, restriction chain,
    // per-level FE mean/sigma, normalisation into the stored pyramid.  The
    // staging buffers alternate across the chunks of all series (nc counts
    // them), so that each copy waits for the kernels that last read its buffer.
    int nc = 0;
    for (int i = 0; i < n_series; i++) {
        SeriesInfo &si = s->S[i];
        int nL = si.side + 1;
        int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(si.n_frames, (512ll << 20) / ((int64_t)nL * nL * 4 * 2)));
        const size_t frame_bytes = (size_t)si.side * si.side * 4;
        // host frames: chunks that fit a staging buffer, each copied on the copy
        // stream while the pyramid kernels of the chunk before run
        const bool staged = !frames_on_device && frame_bytes <= HOST_STAGE_BYTES;
        if (!frames_on_device) {
            if ((st = host_transfer_setup(s)) != REG_OK) return cleanup(st);
            if (staged) chunk = (int)std::min<size_t>(chunk, HOST_STAGE_BYTES / frame_bytes);
        }
        void *raw = nullptr, *stage = nullptr, *stats = nullptr;
        size_t raw_bytes = (size_t)chunk * si.frame_block * 4;
        if ((st = dalloc(s, &raw, raw_bytes)) != REG_OK) return cleanup(st);
        if ((st = dalloc(s, &stats, sizeof(double) * (2 * chunk + image_stats_part_doubles(chunk)))) != REG_OK)
            return cleanup(st);
        size_t stage_bytes = (size_t)chunk * frame_bytes;
        if (!frames_on_device && !staged && (st = dalloc(s, &stage, stage_bytes)) != REG_OK) return cleanup(st);
        for (int f0 = 0; f0 < si.n_frames; f0 += chunk, nc++) {
            int nf = std::min(chunk, si.n_frames - f0);
            const int b = nc & 1;
            // series i starts after all rows of the series before it (side_j rows of
            // pitch_elems per frame); frame f0 of it after f0 * side rows of its own
            const float *src = frames + (row_off + (int64_t)f0 * si.side) * pitch_elems;
            int64_t fstride = (int64_t)si.side * pitch_elems, pitch = pitch_elems;
            if (!frames_on_device) {
                void *dst = staged ? s->host_stage[b] : stage;
                cudaStream_t cst = staged ? s->copy_stream : s->stream;
                cudaError_t e = cudaSuccess;
                // the kernels that read this staging buffer two chunks ago are done
                if (staged && nc >= 2) e = cudaStreamWaitEvent(cst, s->ev_drained[b], 0);
                if (e == cudaSuccess)
                    e = cudaMemcpy2DAsync(dst, si.side * 4, src, pitch_elems * 4, si.side * 4, (size_t)si.side * nf,
                                          cudaMemcpyHostToDevice, cst);
                if (e == cudaSuccess && staged) e = cudaEventRecord(s->ev_filled[b], cst);
                if (e == cudaSuccess && staged) e = cudaStreamWaitEvent(s->stream, s->ev_filled[b], 0);
                if (e != cudaSuccess) return cleanup(fail(REG_ECUDA, "frame upload: %s", cudaGetErrorString(e)));
                src = (const float *)dst;
                fstride = (int64_t)si.side * si.side;
                pitch = si.side;
            }
            int kL = si.nl - 1;
            float *rawf = (float *)raw;
            dim3 blk(32, 8);
            k_embed<<<dim3(cdiv(nL, 32), cdiv(nL, 8), nf), blk, 0, s->stream>>>(
                src, fstride, pitch, si.side, rawf + si.img_off[kL], (int64_t)si.frame_block, si.pitch[kL]);
            build_levels(s, si, rawf, f0, nf, (double *)stats);
            if (staged) cudaEventRecord(s->ev_drained[b], s->stream);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cleanup(fail(REG_ECUDA, "pyramid kernels: %s", cudaGetErrorString(e)));
        }
        dfree(s, raw, raw_bytes);
        dfree(s, stats, 0);
        dfree(s, stage, stage_bytes);
        row_off += (int64_t)si.n_frames * si.side;
    }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return cleanup(fail(REG_ECUDA, "pyramid sync"));
    *out = s;
    return REG_OK;
}

reg_status reg_destroy_series(reg_series_t s)
{
    if (!s) return REG_OK;
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    for (int i = 0; i < 2; i++) {
        if (s->ev_filled[i]) cudaEventDestroy(s->ev_filled[i]);
        if (s->ev_drained[i]) cudaEventDestroy(s->ev_drained[i]);
    }
    for (size_t i = 0; i + 1 < s->allocs.size(); i += 2) dfree(s, s->allocs[i], reinterpret_cast<size_t>(s->allocs[i + 1]));
    cudaStreamSynchronize(s->stream);
    if (s->h_ops) cudaFreeHost(s->h_ops);
    if (s->h_ctr) cudaFreeHost(s->h_ctr);
    if (s->h_st) cudaFreeHost(s->h_st);
    for (int k = 0; k < GRAPH_STEPS; k++) {
        for (int f = 0; f < NFAM; f++)
            if (s->ev[k][f]) cudaEventDestroy(s->ev[k][f]);
        if (s->ev_end[k]) cudaEventDestroy(s->ev_end[k]);
    }
    delete s;
    return REG_OK;
}

static reg_status check_op(reg_series *s, const reg_op_desc &o, OpReq &r)
{
    if (o.series < 0 || o.series >= (int)s->S.size()) return fail(REG_EINVAL, "series index out of range");
    const SeriesInfo &si = s->S[o.series];
    if (o.frame_i < 0 || o.frame_i >= si.n_frames || o.frame_k < 0 || o.frame_k >= si.n_frames)
        return fail(REG_EINVAL, "frame index out of range");
    if (o.dst_slot < 0 || o.dst_slot >= si.n_slots) return fail(REG_EINVAL, "dst slot out of range");
    auto slot_ok = [&](int k) { return k < 0 || k < si.n_slots; };
    if (!slot_ok(o.left_slot) || !slot_ok(o.right_slot)) return fail(REG_EINVAL, "slot out of range");
    if (o.right_slot >= 0 && o.left_slot < 0) return fail(REG_EINVAL, "right operand without left operand");
    r.series = o.series;
    r.frame_i = si.frame_base + o.frame_i;
    r.frame_k = si.frame_base + o.frame_k;
    // frame indices inside the series pyramid are local
    r.frame_i = o.frame_i;
    r.frame_k = o.frame_k;
    r.left = o.left_slot;
    r.right = o.right_slot;
    r.dst = o.dst_slot;
    r.init = o.left_slot < 0 ? 0 : (o.right_slot < 0 ? 1 : 2);
    if (r.init >= 1) {
        const SlotMeta &a = si.meta[o.left_slot];
        if (a.end < 0) return fail(REG_EINVAL, "left slot %d holds no deformation", o.left_slot);
        if (r.init == 1 && (a.start != o.frame_i || a.end != o.frame_k))
            return fail(REG_EINVAL, "left slot holds phi_{%d,%d}, op registers (%d,%d)", a.start, a.end, o.frame_i, o.frame_k);
        if (r.init == 2) {
            const SlotMeta &b = si.meta[o.right_slot];
            if (b.end < 0) return fail(REG_EINVAL, "right slot %d holds no deformation", o.right_slot);
            if (a.end != b.start) return fail(REG_EINVAL, "chain mismatch: phi_{%d,%d} then phi_{%d,%d}", a.start, a.end, b.start, b.end);
            if (a.start != o.frame_i || b.end != o.frame_k)
                return fail(REG_EINVAL, "operands span (%d,%d), op registers (%d,%d)", a.start, b.end, o.frame_i, o.frame_k);
        }
    }
    return REG_OK;
}

reg_status reg_apply_operator_batch(reg_series_t s, int32_t n_ops, const reg_op_desc *ops, int32_t *op_status_out,
                                    int32_t *iters_out)
{
    g_err.clear();
    if (!s || n_ops < 0 || (n_ops > 0 && !ops)) return fail(REG_EINVAL, "null handle or ops");
    std::vector<OpReq> req(n_ops);
    for (int i = 0; i < n_ops; i++) RET(check_op(s, ops[i], req[i]));
    for (int i = 0; i < n_ops; i++)
        for (int j = i + 1; j < n_ops; j++)
            if (ops[i].series == ops[j].series && ops[i].dst_slot == ops[j].dst_slot)
                return fail(REG_EINVAL, "two ops write slot %d", ops[i].dst_slot);
    RET(run_batch(s, req, [] { return REG_OK; }, op_status_out, iters_out));
    for (int i = 0; i < n_ops; i++) {
        SlotMeta &m = s->S[ops[i].series].meta[ops[i].dst_slot];
        m.start = ops[i].frame_i;
        m.end = ops[i].frame_k;
    }
    return REG_OK;
}

reg_status reg_prefix_scan(reg_series_t s, reg_scan_kind kind, int32_t chunks, reg_scan_kind global_kind,
                           char *report, size_t buf_len)
{
    g_err.clear();
    if (!s) return fail(REG_EINVAL, "null handle");
    if (kind < REG_SCAN_SERIAL || kind > REG_SCAN_LADNER_FISCHER) return fail(REG_EINVAL, "unknown scan kind");
    if (kind == REG_SCAN_HAN_CARLSON && (chunks < 1 || chunks > 30)) return fail(REG_EINVAL, "Han-Carlson needs 1 <= k <= 30");
    if (kind == REG_SCAN_LADNER_FISCHER && (chunks < 0 || chunks > 30))
        return fail(REG_EINVAL, "Ladner-Fischer needs 0 <= k <= 30");
    if ((kind == REG_SCAN_CHUNKED || kind == REG_SCAN_CHUNKED_ALT) &&
        (chunks < 1 || chunks > 64 || global_kind < REG_SCAN_SERIAL || global_kind > REG_SCAN_BLELLOCH))
        return fail(REG_EINVAL, "chunked scans need 1 <= chunks <= 64 and a non-chunked global kind");
    auto t0 = std::chrono::steady_clock::now();
    int64_t ops0 = s->tot_ops, it0 = s->tot_iters, tr0 = s->tot_trials, st0 = s->tot_steps, ev0 = s->tot_evals;
    // preprocessing: A(f_e, f_{e+1}, I) -> slot e, all series in one batch
    std::vector<OpReq> pre;
    for (int si = 0; si < (int)s->S.size(); si++) {
        SeriesInfo &S = s->S[si];
        for (auto &m : S.meta) m = SlotMeta{};
        S.refined = false;
        // identity start, or (after reg_cnn_init_series) the slot's initial guess
        for (int e = 0; e < S.n_data; e++)
            pre.push_back(S.pre_from_slots
                              ? OpReq{si, e, e + 1, 1, e, -1, e, s->p.init_levels ? S.nl - s->p.init_levels : 0,
                                      s->p.init_levels && s->p.init_levels < S.nl}
                              : OpReq{si, e, e + 1, 0, -1, -1, e});
        S.pre_from_slots = false;
    }
    std::vector<int32_t> stat(pre.size());
    RET(run_batch(s, pre, [] { return REG_OK; }, stat.data(), nullptr));  // returns after a sync
    // A learned start that skips coarse levels is judged by the plain method:
    // the mean move of the operator away from it over the finest nodes (px).
    // An operator that had to move it by more than learned_fallback_px started
    // outside the basin its fine levels can reach: it is run again from the
    // identity on every level.  (A learned start on every level needs no
    // fallback: its coarse levels already had their say.)
    int n_judged = 0, n_fallback = 0;
    double corr_sum = 0.0, corr_max = 0.0;
    {
        std::vector<OpReq> again;
        std::vector<size_t> again_idx;
        for (size_t i = 0; i < pre.size(); i++) {
            if (!pre[i].judge) continue;
            const SeriesInfo &S = s->S[pre[i].series];
            const double nn = (double)S.n[S.nl - 1] * S.n[S.nl - 1];
            const double c = s->h_st[i].corr / nn;
            n_judged++;
            corr_sum += c;
            corr_max = std::max(corr_max, c);
            if (s->p.learned_fallback_px > 0.0 && !(c <= s->p.learned_fallback_px)) {
                const OpReq &o = pre[i];
                again.push_back(OpReq{o.series, o.frame_i, o.frame_k, 0, -1, -1, o.dst});
                again_idx.push_back(i);
            }
        }
        if (!again.empty()) {
            std::vector<int32_t> st2(again.size());
            RET(run_batch(s, again, [] { return REG_OK; }, st2.data(), nullptr));
            for (size_t j = 0; j < again.size(); j++) stat[again_idx[j]] = st2[j];
            n_fallback = (int)again.size();
        }
    }
    const double pre_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    const int64_t pre_iters = s->tot_iters - it0;
    int counts[5] = {0, 0, 0, 0, 0};
    for (auto v : stat) counts[std::min(std::max(v, 0), 4)]++;
    for (auto &o : pre) s->S[o.series].meta[o.dst] = SlotMeta{o.frame_i, o.frame_k};
    std::vector<regsched::Schedule> sch(s->S.size());
    size_t nlev = 0;
    for (size_t si = 0; si < s->S.size(); si++) {
        if (!regsched::make_schedule((int)kind, s->S[si].n_data, chunks, (int)global_kind, sch[si]))
            return fail(REG_EINVAL, "schedule generation failed");
        nlev = std::max(nlev, sch[si].levels.size());
    }
    int batches = 0, scan_ops = 0;
    for (size_t t = 0; t < nlev; t++) {
        std::vector<OpReq> reg;
        struct Copy { int series, dst, src; };
        std::vector<Copy> copies;
        std::vector<std::pair<int, std::pair<int, SlotMeta>>> writes;  // series, (slot, meta)
        for (size_t si = 0; si < s->S.size(); si++) {
            if (t >= sch[si].levels.size()) continue;
            SeriesInfo &S = s->S[si];
            for (auto &o : sch[si].levels[t]) {
                if (o.kind == regsched::OP_IDENTITY) {
                    writes.push_back({(int)si, {o.dst, SlotMeta{}}});
                } else if (o.kind == regsched::OP_COPY) {
                    const SlotMeta &m = S.meta[o.a];
                    if (m.end >= 0) copies.push_back({(int)si, o.dst, o.a});
                    writes.push_back({(int)si, {o.dst, m}});
                } else {
                    const SlotMeta &a = S.meta[o.a], &b = S.meta[o.b];
                    if (a.end < 0) {
                        if (b.end >= 0) copies.push_back({(int)si, o.dst, o.b});
                        writes.push_back({(int)si, {o.dst, b}});
                    } else if (b.end < 0) {
                        copies.push_back({(int)si, o.dst, o.a});
                        writes.push_back({(int)si, {o.dst, a}});
                    } else {
                        if (a.end != b.start) return fail(REG_EKERNEL, "schedule chain mismatch");
                        reg.push_back(OpReq{(int)si, a.start, b.end, 2, o.a, o.b, o.dst});
                        writes.push_back({(int)si, {o.dst, SlotMeta{a.start, b.end}}});
                    }
                }
            }
        }
        // copies whose source is also a destination of this level must read first:
        // they run after composition and before any result is written.
        auto do_copies = [&]() -> reg_status {
            for (auto &c : copies)
                if (c.dst != c.src) RET(copy_slot(s, s->S[c.series], c.dst, c.src));
            return REG_OK;
        };
        std::vector<int32_t> st2(reg.size());
        RET(run_batch(s, reg, do_copies, st2.data(), nullptr));
        for (auto v : st2) counts[std::min(std::max(v, 0), 4)]++;
        if (!reg.empty()) batches++;
        scan_ops += (int)reg.size();
        for (auto &w : writes) s->S[w.first].meta[w.second.first] = w.second.second;
    }
    CK(cudaStreamSynchronize(s->stream));
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (auto &S : s->S)
        for (int e = 0; e < S.n_data; e++)
            if (S.meta[e].start != 0 || S.meta[e].end != e + 1) return fail(REG_EKERNEL, "scan did not produce phi_{0,%d}", e + 1);
    if (report && buf_len > 0) {
        snprintf(report, buf_len,
                 "{\"kind\": %d, \"preprocessing_ops\": %zu, \"preprocessing_ms\": %.3f, "
                 "\"preprocessing_iters\": %lld, \"learned\": {\"ops\": %d, \"mean_correction_px\": %.5f, "
                 "\"max_correction_px\": %.5f, \"fallbacks\": %d}, \"scan_ops\": %d, \"scan_batches\": %d, "
                 "\"ops\": %lld, \"iters\": %lld, \"trials\": %lld, \"evals\": %lld, \"steps\": %lld, \"ms\": %.3f, "
                 "\"grids\": [%d, %d, %d], "
                 "\"status\": {\"converged\": %d, \"maxiter\": %d, \"stalled\": %d, \"nonfinite\": %d, \"zero_gradient\": %d}}",
                 (int)kind, pre.size(), pre_ms, (long long)pre_iters, n_judged,
                 n_judged ? corr_sum / n_judged : 0.0, corr_max, n_fallback, scan_ops, batches, (long long)(s->tot_ops - ops0),
                 (long long)(s->tot_iters - it0), (long long)(s->tot_trials - tr0), (long long)(s->tot_evals - ev0),
                 (long long)(s->tot_steps - st0), ms, s->grid_P, s->grid_G, s->grid_T, counts[0], counts[1], counts[2],
                 counts[3], counts[4]);
    }
    return REG_OK;
}

reg_status reg_average_series(reg_series_t s, int32_t series, int32_t iterations, float *avg_out,
                              int32_t out_on_device)
{
    g_err.clear();
    if (!s || series < 0 || series >= (int)s->S.size()) return fail(REG_EINVAL, "bad handle or series");
    if (iterations < 0 || iterations > 1000) return fail(REG_EINVAL, "iterations must be in [0, 1000]");
    SeriesInfo &si = s->S[series];
    for (int e = 0; e < si.n_data; e++)
        if (si.meta[e].start != 0 || si.meta[e].end != e + 1)
            return fail(REG_ESTATE, "phi_{0,%d} not available (run reg_prefix_scan first)", e + 1);
    const int kL = si.nl - 1, nL = si.n[kL];
    void *raw = nullptr, *stats = nullptr;
    RET(dalloc(s, &raw, si.frame_block * sizeof(float)));
    reg_status st = dalloc(s, &stats, sizeof(double) * (2 + image_stats_part_doubles(1)));
    if (st != REG_OK) {
        dfree(s, raw, 0);
        return st;
    }
    float *rawf = (float *)raw;
    std::vector<const float2 *> fields(si.n_frames);
    auto average = [&]() -> reg_status {
        // frame 0: the identity, or its deformation to the last average; frame
        // e + 1: the field in data slot e
        fields[0] = si.refined ? si.slots + (size_t)si.n_slots * si.slot_elems : nullptr;
        for (int e = 0; e < si.n_data; e++) fields[e + 1] = si.slots + (size_t)e * si.slot_elems;
        CK(cudaMemcpyAsync(si.d_fields, fields.data(), sizeof(void *) * si.n_frames, cudaMemcpyHostToDevice,
                           s->stream));
        launch_average(s->bf16, s->stream, si.pyr, (int64_t)si.frame_block, (int64_t)si.img_off[kL], nL, si.pitch[kL],
                       si.fstats, si.d_fields, si.pitch[kL], si.n_frames, rawf + si.img_off[kL], si.pitch[kL]);
        CK(cudaGetLastError());
        return REG_OK;
    };
    auto body = [&]() -> reg_status {
        RET(average());
        for (int it = 0; it < iterations; it++) {
            // the average becomes the reference frame (pyramid block n_frames);
            // every frame is registered to it by function A, started from its
            // current deformation (frame 0 from the identity at first)
            build_levels(s, si, rawf, si.n_frames, 1, (double *)stats);
            CK(cudaGetLastError());
            std::vector<OpReq> ops;
            for (int k = 0; k < si.n_frames; k++) {
                const int slot = k == 0 ? si.n_slots : k - 1;
                const int init = (k == 0 && !si.refined) ? 0 : 1;
                ops.push_back(OpReq{series, si.n_frames, k, init, init ? slot : -1, -1, slot});
            }
            RET(run_batch(s, ops, [] { return REG_OK; }, nullptr, nullptr));
            si.refined = true;
            RET(average());
        }
        if (avg_out)
            CK(cudaMemcpy2DAsync(avg_out, (size_t)si.side * sizeof(float), rawf + si.img_off[kL],
                                 (size_t)si.pitch[kL] * sizeof(float), (size_t)si.side * sizeof(float), si.side,
                                 out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        return REG_OK;
    };
    st = body();
    dfree(s, raw, 0);
    dfree(s, stats, 0);
    return st;
}

reg_status reg_get_slot(reg_series_t s, int32_t series, int32_t slot, float *out, int32_t out_on_device,
                        int32_t *start_end)
{
    g_err.clear();
    if (!s || series < 0 || series >= (int)s->S.size()) return fail(REG_EINVAL, "bad handle or series");
    SeriesInfo &si = s->S[series];
    if (slot < 0 || slot >= si.n_slots) return fail(REG_EINVAL, "slot out of range");
    if (start_end) {
        start_end[0] = si.meta[slot].start;
        start_end[1] = si.meta[slot].end;
    }
    if (!out) return REG_OK;
    int n = si.side + 1;
    size_t bytes = (size_t)2 * n * n * sizeof(float);
    float *dst = out;
    void *tmp = nullptr;
    if (!out_on_device) {
        RET(dalloc(s, &tmp, bytes));
        dst = (float *)tmp;
    }
    const float2 *src = si.meta[slot].end >= 0 ? si.slots + (size_t)slot * si.slot_elems : nullptr;
    k_slot_to_planes<<<dim3(cdiv(n, 32), cdiv(n, 8)), dim3(32, 8), 0, s->stream>>>(src, si.pitch[si.nl - 1], n, dst);
    CK(cudaGetLastError());
    if (!out_on_device) {
        CK(cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, s->stream));
        dfree(s, tmp, bytes);
    }
    CK(cudaStreamSynchronize(s->stream));
    return REG_OK;
}

reg_status reg_set_slot(reg_series_t s, int32_t series, int32_t slot, const float *field, int32_t on_device,
                        int32_t start, int32_t end)
{
    g_err.clear();
    if (!s || series < 0 || series >= (int)s->S.size()) return fail(REG_EINVAL, "bad handle or series");
    SeriesInfo &si = s->S[series];
    if (slot < 0 || slot >= si.n_slots) return fail(REG_EINVAL, "slot out of range");
    if (end < 0) {
        si.meta[slot] = SlotMeta{};
        return REG_OK;
    }
    if (!field || start < 0 || start >= si.n_frames || end >= si.n_frames) return fail(REG_EINVAL, "bad field or frames");
    int n = si.side + 1;
    size_t bytes = (size_t)2 * n * n * sizeof(float);
    const float *src = field;
    void *tmp = nullptr;
    if (!on_device) {
        RET(dalloc(s, &tmp, bytes));
        CK(cudaMemcpyAsync(tmp, field, bytes, cudaMemcpyHostToDevice, s->stream));
        src = (const float *)tmp;
    }
    k_planes_to_slot<<<dim3(cdiv(n, 32), cdiv(n, 8)), dim3(32, 8), 0, s->stream>>>(
        src, n, si.slots + (size_t)slot * si.slot_elems, si.pitch[si.nl - 1]);
    CK(cudaGetLastError());
    if (tmp) dfree(s, tmp, bytes);
    CK(cudaStreamSynchronize(s->stream));
    si.meta[slot] = SlotMeta{start, end};
    return REG_OK;
}

reg_status reg_get_rigid(reg_series_t s, int32_t series, int32_t slot, double *theta, int32_t *start_end)
{
    g_err.clear();
    if (!s || series < 0 || series >= (int)s->S.size() || !theta) return fail(REG_EINVAL, "bad argument");
    if (!(s->p.flags & REG_FLAG_RIGID)) return fail(REG_ESTATE, "not a rigid handle");
    SeriesInfo &si = s->S[series];
    if (slot < 0 || slot >= si.n_slots) return fail(REG_EINVAL, "slot out of range");
    for (int c = 0; c < 3; c++) theta[c] = si.meta[slot].end >= 0 ? si.rigid[slot][c] : 0.0;
    if (start_end) {
        start_end[0] = si.meta[slot].start;
        start_end[1] = si.meta[slot].end;
    }
    return REG_OK;
}

reg_status reg_set_rigid(reg_series_t s, int32_t series, int32_t slot, const double *theta, int32_t start,
                         int32_t end)
{
    g_err.clear();
    if (!s || series < 0 || series >= (int)s->S.size()) return fail(REG_EINVAL, "bad argument");
    if (!(s->p.flags & REG_FLAG_RIGID)) return fail(REG_ESTATE, "not a rigid handle");
    SeriesInfo &si = s->S[series];
    if (slot < 0 || slot >= si.n_slots) return fail(REG_EINVAL, "slot out of range");
    if (end < 0) {
        si.meta[slot] = SlotMeta{};
        return REG_OK;
    }
    if (!theta || start < 0 || start >= si.n_frames || end >= si.n_frames) return fail(REG_EINVAL, "bad parameters or frames");
    for (int c = 0; c < 3; c++)
        if (!std::isfinite(theta[c])) return fail(REG_EINVAL, "parameters must be finite");
    si.rigid[slot] = {theta[0], theta[1], theta[2]};
    const int nL = si.n[si.nl - 1];
    launch_rigid_fill(rigid_req(si.rigid[slot], nL), nL, si.slots + (size_t)slot * si.slot_elems, si.pitch[si.nl - 1],
                      s->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    si.meta[slot] = SlotMeta{start, end};
    return REG_OK;
}

reg_status reg_num_slots(reg_series_t s, int32_t series, int32_t *n_slots)
{
    if (!s || !n_slots || series < 0 || series >= (int)s->S.size()) return fail(REG_EINVAL, "bad argument");
    *n_slots = s->S[series].n_slots;
    return REG_OK;
}

reg_status reg_get_deformations(reg_series_t s, int32_t series, int32_t first, int32_t count, float *out,
                                int32_t out_on_device)
{
    g_err.clear();
    if (!s || !out || series < 0 || series >= (int)s->S.size()) return fail(REG_EINVAL, "bad argument");
    SeriesInfo &si = s->S[series];
    if (first < 0 || count < 0 || first + count > si.n_frames) return fail(REG_EINVAL, "frame range out of range");
    size_t per = (size_t)2 * si.side * si.side;
    for (int k = std::max(first, 1); k < first + count; k++) {
        const SlotMeta &m = si.meta[k - 1];
        if (m.start != 0 || m.end != k) return fail(REG_ESTATE, "phi_{0,%d} not available (run reg_prefix_scan first)", k);
    }
    const float2 *slot0 = si.refined ? si.slots + (size_t)si.n_slots * si.slot_elems : nullptr;
    const dim3 blk(32, 8), grd(cdiv(si.side, 32), cdiv(si.side, 8));
    auto convert = [&](int k0, int nk, float *dst) {
        k_slots_to_planes<<<dim3(grd.x, grd.y, nk), blk, 0, s->stream>>>(si.slots, (int64_t)si.slot_elems, k0, slot0,
                                                                         si.pitch[si.nl - 1], si.side, dst);
    };
    if (out_on_device || count == 0) {
        for (int k0 = first; k0 < first + count; k0 += 65535) convert(k0, std::min(65535, first + count - k0), out + (size_t)(k0 - first) * per);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s->stream));
        return REG_OK;
    }
    // host output: chunks of frames converted into the two staging buffers on
    // the handle's stream and copied out on the copy stream, each copy
    // overlapping the next chunk's conversion
    RET(host_transfer_setup(s));
    const int fc = (int)std::max<size_t>(1, std::min<size_t>(65535, HOST_STAGE_BYTES / (per * sizeof(float))));
    if (per * sizeof(float) > HOST_STAGE_BYTES) {
        // frames larger than a staging buffer: one temporary buffer
        void *tmp = nullptr;
        RET(dalloc(s, &tmp, per * sizeof(float) * count));
        convert(first, count, (float *)tmp);
        CK(cudaMemcpyAsync(out, tmp, per * count * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
        dfree(s, tmp, 0);
        CK(cudaStreamSynchronize(s->stream));
        return REG_OK;
    }
    int c = 0;
    for (int k0 = first; k0 < first + count; k0 += fc, c++) {
        const int nk = std::min(fc, first + count - k0), b = c & 1;
        if (c >= 2) CK(cudaStreamWaitEvent(s->stream, s->ev_drained[b], 0));  // its last copy is done
        convert(k0, nk, (float *)s->host_stage[b]);
        CK(cudaEventRecord(s->ev_filled[b], s->stream));
        CK(cudaStreamWaitEvent(s->copy_stream, s->ev_filled[b], 0));
        CK(cudaMemcpyAsync(out + (size_t)(k0 - first) * per, s->host_stage[b], per * nk * sizeof(float),
                           cudaMemcpyDeviceToHost, s->copy_stream));
        CK(cudaEventRecord(s->ev_drained[b], s->copy_stream));
    }
    CK(cudaGetLastError());
    // the handle's stream waits for the last copies (so that later work on it
    // may reuse the buffers), then the host for both streams
    for (int b = 0; b < 2 && b < c; b++) CK(cudaStreamWaitEvent(s->stream, s->ev_drained[b], 0));
    CK(cudaStreamSynchronize(s->copy_stream));
    CK(cudaStreamSynchronize(s->stream));
    return REG_OK;
}

// Diagnostics: one START step (energy) and optionally one G pass (direction)
// of a single op at a single level, through the same kernels as the batches.
static reg_status diag_setup(reg_series *s, int series, int fi, int fk, int level, const float *u_grid, int &k)
{
    if (!s || series < 0 || series >= (int)s->S.size()) return fail(REG_EINVAL, "bad handle or series");
    SeriesInfo &si = s->S[series];
    if (fi < 0 || fi >= si.n_frames || fk < 0 || fk >= si.n_frames) return fail(REG_EINVAL, "frame out of range");
    k = level - si.m0;
    if (k < 0 || k >= si.nl) return fail(REG_EINVAL, "level outside the pyramid");
    if (!u_grid) return fail(REG_EINVAL, "null displacement");
    std::vector<OpReq> one{OpReq{series, fi, fk, 0, -1, -1, 0}};
    RET(ensure_capacity(s, 1, si.ws_bytes, max_tiles_series(s, si)));
    OpDesc &d = s->h_ops[0];
    memset(&d, 0, sizeof(d));
    d.nl = si.nl;
    d.init = 0;
    d.out = nullptr;
    for (int q = 0; q < si.nl; q++) {
        LevelDesc &L = d.lv[q];
        fill_level(s, L, si.n[q], si.pitch[q]);
        L.R = img_ptr(s, si, fi, q);
        L.T = img_ptr(s, si, fk, q);
        L.MR = si.mr + (size_t)fi * si.frame_block + si.img_off[q];
        char *base = s->d_ws + si.ws_off[q];
        L.V[0] = (NodeRec *)base;
        L.V[1] = (NodeRec *)(base + si.rec_bytes(q));
    }
    CK(cudaMemcpyAsync(s->d_ops, s->h_ops, sizeof(OpDesc), cudaMemcpyHostToDevice, s->stream));
    // u planes (2 x n x n) -> float2 field U0 of level k
    int n = si.n[k];
    std::vector<NodeRec> tmp((size_t)n * si.pitch[k]);
    memset(tmp.data(), 0, tmp.size() * sizeof(NodeRec));
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++)
            tmp[(size_t)r * si.pitch[k] + c].u =
                make_float4(u_grid[(size_t)r * n + c], u_grid[(size_t)n * n + (size_t)r * n + c], 0.f, 0.f);
    CK(cudaMemcpyAsync(d.lv[k].V[0], tmp.data(), tmp.size() * sizeof(NodeRec), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));  // tmp is pageable and goes out of scope
    s->h_ctr[0] = 1;
    for (int q = 1; q < 16; q++) s->h_ctr[q] = 0;
    CK(cudaMemcpyAsync(s->d_ctr, s->h_ctr, sizeof(int) * 16, cudaMemcpyHostToDevice, s->stream));
    BatchDev b = make_batch(s);
    k_init_state<<<1, 32, 0, s->stream>>>(b, 1);
    OpState st;
    memset(&st, 0, sizeof(st));
    st.phase = PH_START;
    st.lvl = k;
    st.tau = s->p.tau_init;
    CK(cudaMemcpyAsync(s->d_st, &st, sizeof(OpState), cudaMemcpyHostToDevice, s->stream));
    // START: plan, T, C
    k_plan<<<1, 1024, 0, s->stream>>>(b);
    launch_trial(s->bf16, s->p.trials_per_pass, s->grid_T, s->stream, b);
    k_control<<<1, 256, 0, s->stream>>>(b);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    return REG_OK;
}

reg_status reg_eval_energy(reg_series_t s, int32_t series, int32_t frame_i, int32_t frame_k, int32_t level,
                           const float *u_grid, double *parts)
{
    g_err.clear();
    int k;
    RET(diag_setup(s, series, frame_i, frame_k, level, u_grid, k));
    OpState st;
    CK(cudaMemcpy(&st, s->d_st, sizeof(OpState), cudaMemcpyDeviceToHost));
    if (parts) {
        parts[0] = st.E;
        parts[1] = st.ncc;
        parts[2] = st.E + st.ncc;
        parts[3] = st.Tbar;
        parts[4] = st.sigT;
    }
    return REG_OK;
}

__global__ void k_sum_range(const double *v, int stride, int b, int e, double *out)
{
    double s = 0.0;
    for (int i = b + threadIdx.x; i < e; i += 32) s += v[(int64_t)i * stride];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
}

reg_status reg_eval_direction(reg_series_t s, int32_t series, int32_t frame_i, int32_t frame_k, int32_t level,
                              const float *u_grid, float *d_out, double *slope)
{
    g_err.clear();
    int k;
    RET(diag_setup(s, series, frame_i, frame_k, level, u_grid, k));
    BatchDev b = make_batch(s);
    // state is now PH_GRAD with src = 0, cur = 1 (no pending step)
    k_plan<<<1, 1024, 0, s->stream>>>(b);
    launch_grad(s->bf16, s->grid_G, s->stream, b);
    CK(cudaGetLastError());
    OpState st;
    CK(cudaMemcpyAsync(&st, s->d_st, sizeof(OpState), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (st.phase != PH_GRAD) return fail(REG_ESTATE, "energy at the given displacement is not finite");
    if (!s->d_scratch) RET(track(s, (void **)&s->d_scratch, sizeof(double) * 16));
    k_sum_range<<<1, 32, 0, s->stream>>>(s->d_partG, PG_STRIDE, st.g_begin, st.g_end, s->d_scratch);
    double sl = 0.0;
    CK(cudaMemcpyAsync(&sl, s->d_scratch, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    const SeriesInfo &si = s->S[series];
    int n = si.n[k];
    std::vector<NodeRec> tmp((size_t)n * si.pitch[k]);
    OpDesc d;
    CK(cudaMemcpyAsync(&d, s->d_ops, sizeof(OpDesc), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaMemcpy(tmp.data(), d.lv[k].V[st.cur], tmp.size() * sizeof(NodeRec), cudaMemcpyDeviceToHost));
    if (slope) *slope = sl;
    if (d_out)
        for (int r = 0; r < n; r++)
            for (int c = 0; c < n; c++) {
                d_out[(size_t)r * n + c] = tmp[(size_t)r * si.pitch[k] + c].d.x;
                d_out[(size_t)n * n + (size_t)r * n + c] = tmp[(size_t)r * si.pitch[k] + c].d.y;
            }
    return REG_OK;
}

reg_status reg_eval_trials(reg_series_t s, int32_t series, int32_t frame_i, int32_t frame_k, int32_t level,
                           const float *u_grid, int32_t n_tau, const double *taus, float *d_out, double *dE_out)
{
    g_err.clear();
    if (!s || !taus || !dE_out) return fail(REG_EINVAL, "bad argument");
    if (n_tau < 1 || n_tau > s->p.trials_per_pass)
        return fail(REG_EINVAL, "n_tau must be in [1, trials_per_pass = %d]", s->p.trials_per_pass);
    int k;
    RET(diag_setup(s, series, frame_i, frame_k, level, u_grid, k));
    BatchDev b = make_batch(s);
    // gradient pass at u (state PH_GRAD, no pending step), then one trial pass
    // over the given step sizes (still PH_GRAD, so that it also forms d^T K d)
    k_plan<<<1, 1024, 0, s->stream>>>(b);
    launch_grad(s->bf16, s->grid_G, s->stream, b);
    CK(cudaGetLastError());
    OpState st;
    CK(cudaMemcpyAsync(&st, s->d_st, sizeof(OpState), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (st.phase != PH_GRAD) return fail(REG_ESTATE, "energy at the given displacement is not finite");
    st.ntr = n_tau;
    for (int j = 0; j < REG_MAX_TRIALS; j++) st.trial_tau[j] = j < n_tau ? taus[j] : 0.0;
    CK(cudaMemcpyAsync(s->d_st, &st, sizeof(OpState), cudaMemcpyHostToDevice, s->stream));
    launch_trial(s->bf16, s->p.trials_per_pass, s->grid_T, s->stream, b);
    CK(cudaGetLastError());
    std::vector<double> pt((size_t)(st.t_end - st.t_begin) * PT_STRIDE), pg((size_t)(st.g_end - st.g_begin) * PG_STRIDE);
    CK(cudaMemcpyAsync(pt.data(), s->d_partT + (size_t)st.t_begin * PT_STRIDE, pt.size() * sizeof(double),
                       cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(pg.data(), s->d_partG + (size_t)st.g_begin * PG_STRIDE, pg.size() * sizeof(double),
                       cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    double S[PT_STRIDE] = {0.0}, qud = 0.0;
    for (size_t i = 0; i < pt.size(); i++) S[i % PT_STRIDE] += pt[i];
    for (size_t i = 1; i < pg.size(); i += PG_STRIDE) qud += pg[i];
    // the energy change of each step size, as the operator state machine forms it
    const SeriesInfo &si = s->S[series];
    const double hh = 1.0 / (si.n[k] - 1), h2 = hh * hh, qdd = S[3 * REG_MAX_TRIALS + 2];
    for (int j = 0; j < n_tau; j++) {
        double S1 = st.S1 + h2 * S[3 * j], S2 = st.S2 + h2 * S[3 * j + 1], S3 = st.S3 + h2 * S[3 * j + 2];
        double var = S2 - S1 * S1;
        double nc = S3 / (var > 0.0 ? std::sqrt(var) : 0.0);
        dE_out[j] = -(nc - st.ncc) + 0.5 * s->p.lambda * h2 * (2.0 * taus[j] * qud + taus[j] * taus[j] * qdd);
    }
    if (d_out) {
        int n = si.n[k];
        std::vector<NodeRec> tmp((size_t)n * si.pitch[k]);
        OpDesc d;
        CK(cudaMemcpy(&d, s->d_ops, sizeof(OpDesc), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(tmp.data(), d.lv[k].V[st.cur], tmp.size() * sizeof(NodeRec), cudaMemcpyDeviceToHost));
        for (int r = 0; r < n; r++)
            for (int c = 0; c < n; c++) {
                d_out[(size_t)r * n + c] = tmp[(size_t)r * si.pitch[k] + c].d.x;
                d_out[(size_t)n * n + (size_t)r * n + c] = tmp[(size_t)r * si.pitch[k] + c].d.y;
            }
    }
    return REG_OK;
}

reg_status reg_schedule(reg_scan_kind kind, int32_t n, int32_t chunks, reg_scan_kind global_kind,
                        reg_schedule_op *buf, int64_t buf_len, int64_t *n_out, int32_t *n_aux)
{
    g_err.clear();
    if (n < 0 || !n_out) return fail(REG_EINVAL, "bad argument");
    regsched::Schedule sch;
    if (!regsched::make_schedule((int)kind, n, chunks, (int)global_kind, sch)) return fail(REG_EINVAL, "unknown schedule");
    int64_t cnt = 0;
    for (size_t l = 0; l < sch.levels.size(); l++)
        for (auto &o : sch.levels[l]) {
            if (buf && cnt < buf_len) buf[cnt] = reg_schedule_op{(int32_t)l, o.kind, o.dst, o.a, o.b};
            cnt++;
        }
    *n_out = cnt;
    if (n_aux) *n_aux = regsched::aux_slots((int)kind, n, chunks, (int)global_kind);
    return REG_OK;
}

reg_status reg_get_kernel_stats(reg_series_t s, reg_kernel_stats *buf, int32_t buf_len, int32_t *n_out)
{
    if (!s || !n_out) return fail(REG_EINVAL, "bad argument");
    unsigned long long w[16];
    CK(cudaMemcpyAsync(w, s->d_work, sizeof(w), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    // node counters beside the families: trial-pass nodes that took the exact
    // path (largest move leaves the cell); nodes x sequential Armijo trials (the
    // trials the one-at-a-time rule would evaluate); level-start energy nodes
    const struct { const char *name; int k; } extra[3] = {
        {"trial_exact_nodes", KW_TEXACT}, {"trial_seq_nodes", KW_TSEQ}, {"trial_start_nodes", KW_TSTART}};
    *n_out = NFAM + 3;
    for (int j = 0; j < 3 && NFAM + j < buf_len; j++) {
        memset(&buf[NFAM + j], 0, sizeof(reg_kernel_stats));
        snprintf(buf[NFAM + j].name, sizeof(buf[NFAM + j].name), "%s", extra[j].name);
        buf[NFAM + j].items = (int64_t)w[extra[j].k];
    }
    for (int f = 0; f < NFAM && f < buf_len; f++) {
        reg_kernel_stats &k = buf[f];
        memset(&k, 0, sizeof(k));
        snprintf(k.name, sizeof(k.name), "%s", s->fam[f].name);
        k.launches = s->fam[f].launches;
        k.ms = s->fam[f].ms;
        // algorithmic bytes per node (float storage; bf16 images save 2 B per image read)
        double img = s->bf16 ? 2.0 : 4.0;
        // per node: u 16 B (float pair per component), d 8 B, R and T one image value each
        if (f == F_G) {
            k.items = (int64_t)w[KW_G];
            // needed fields: reads u, d, M~R~, the template; writes u, d, 36 M~That
            k.bytes = w[KW_G] * (16.0 + 8.0 + 4.0 + img + 16.0 + 8.0 + 4.0);
        } else if (f == F_T) {
            k.items = (int64_t)(w[KW_T] + w[KW_TSTART]);
            // trial: reads u, d, M~That, M~R~, the template; start: u, M~R~, the template
            k.bytes = w[KW_T] * (16.0 + 8.0 + 4.0 + 4.0 + img) + w[KW_TSTART] * (16.0 + 4.0 + img);
        } else if (f == F_P) {
            k.items = (int64_t)(w[KW_PPROL] + w[KW_PFIN]);
            k.bytes = w[KW_PPROL] * (16.0 + 6.0) + w[KW_PFIN] * (16.0 + 8.0 + 8.0);
        }
    }
    return REG_OK;
}

reg_status reg_set_trace(reg_series_t s, int64_t capacity)
{
    g_err.clear();
    if (!s || capacity < 0) return fail(REG_EINVAL, "bad argument");
    if (s->d_trace) {
        untrack(s, s->d_trace);
        untrack(s, s->d_trace_len);
        s->d_trace = nullptr;
        s->d_trace_len = nullptr;
    }
    s->trace_cap = capacity;
    if (capacity > 0) {
        RET(track(s, (void **)&s->d_trace, sizeof(double) * 7 * capacity));
        RET(track(s, (void **)&s->d_trace_len, sizeof(unsigned long long)));
        CK(cudaMemsetAsync(s->d_trace_len, 0, sizeof(unsigned long long), s->stream));
    }
    s->buf_gen++;  // the captured step graph holds the old pointers
    CK(cudaStreamSynchronize(s->stream));
    return REG_OK;
}

reg_status reg_set_flags(reg_series_t s, int32_t flags)
{
    g_err.clear();
    if (!s || (flags & ~REG_FLAG_PROFILE)) return fail(REG_EINVAL, "bad handle or unknown flag");
    flags |= s->p.flags & REG_FLAG_RIGID;  // the operator of a handle is fixed at creation
    s->p.flags = flags;
    return REG_OK;
}

reg_status reg_set_lockstep(reg_series_t s, int32_t n_ops, int32_t n_levels, const int32_t *counts,
                            const double *taus)
{
    g_err.clear();
    if (!s || n_ops < 0) return fail(REG_EINVAL, "bad argument");
    if (n_ops == 0) {
        s->lock_ops = 0;
        s->lock_levels = 0;
        s->lock_counts.clear();
        s->lock_taus.clear();
        return REG_OK;
    }
    if (n_levels < 1 || n_levels > REG_MAX_LEVELS || !counts) return fail(REG_EINVAL, "bad level count or counts");
    int64_t total = 0;
    for (int64_t i = 0; i < (int64_t)n_ops * n_levels; i++) {
        if (counts[i] < 0 || counts[i] > 100000) return fail(REG_EINVAL, "step count %d out of range", counts[i]);
        total += counts[i];
    }
    if (total > (1ll << 30)) return fail(REG_EINVAL, "too many step sizes");
    if (total > 0 && !taus) return fail(REG_EINVAL, "null step sizes");
    for (int64_t i = 0; i < total; i++)
        if (!(taus[i] > 0.0) || !std::isfinite(taus[i])) return fail(REG_EINVAL, "step size %lld is not positive", (long long)i);
    s->lock_ops = n_ops;
    s->lock_levels = n_levels;
    s->lock_counts.assign(counts, counts + (size_t)n_ops * n_levels);
    s->lock_taus.assign(taus, taus + total);
    return REG_OK;
}

reg_status reg_get_trace(reg_series_t s, double *out, int64_t cap, int64_t *n_out)
{
    g_err.clear();
    if (!s || !n_out) return fail(REG_EINVAL, "bad argument");
    *n_out = 0;
    if (!s->d_trace) return REG_OK;
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, s->d_trace_len, sizeof(n), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    long long m = std::min<long long>((long long)n, s->trace_cap);
    *n_out = m;
    if (out && cap > 0) {
        CK(cudaMemcpyAsync(out, s->d_trace, sizeof(double) * 7 * std::min<long long>(m, cap), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    return REG_OK;
}

reg_status reg_reset_kernel_stats(reg_series_t s)
{
    if (!s) return fail(REG_EINVAL, "null handle");
    for (auto &f : s->fam) {
        f.launches = 0;
        f.ms = 0.0;
    }
    CK(cudaMemsetAsync(s->d_work, 0, sizeof(unsigned long long) * 16, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return REG_OK;
}

reg_status reg_set_tile_rows(reg_series_t s, int32_t level, int32_t grad_rows, int32_t trial_rows)
{
    g_err.clear();
    if (!s || level < 1 || level >= REG_TILE_LEVELS) return fail(REG_EINVAL, "bad handle or level");
    auto ok = [](int r) { return r == 4 || r == 8 || r == 16 || r == 32 || r == 64; };
    if (!ok(grad_rows) || !ok(trial_rows)) return fail(REG_EINVAL, "tile rows must be 4, 8, 16, 32 or 64");
    s->tile_hg[level] = grad_rows;
    s->tile_ht[level] = trial_rows;
    return REG_OK;
}

reg_status reg_get_tile_rows(reg_series_t s, int32_t level, int32_t *grad_rows, int32_t *trial_rows)
{
    g_err.clear();
    if (!s || level < 1 || level >= REG_TILE_LEVELS || !grad_rows || !trial_rows)
        return fail(REG_EINVAL, "bad argument");
    *grad_rows = s->tile_hg[level];
    *trial_rows = s->tile_ht[level];
    return REG_OK;
}

reg_status reg_autotune(reg_series_t s, int32_t series, int32_t n_pairs, int32_t repeats, char *report,
                        size_t buf_len)
{
    g_err.clear();
    if (!s || series < 0 || series >= (int)s->S.size()) return fail(REG_EINVAL, "bad handle or series");
    SeriesInfo &si = s->S[series];
    if (n_pairs < 1 || n_pairs > si.n_data || repeats < 1) return fail(REG_EINVAL, "need 1 <= n_pairs <= frames - 1");
    std::vector<OpReq> ops;
    for (int e = 0; e < n_pairs; e++) ops.push_back(OpReq{series, e, e + 1, 0, -1, -1, e});
    int runs = 0;
    // best of `repeats` runs of the sample batch: wall time per device step
    // (tile shapes change the per-step cost; the step count follows the Armijo
    // decisions) and in total (step sizes per pass change the step count)
    auto measure = [&](double &per_step, double &total) -> reg_status {
        per_step = total = 1e300;
        for (int r = 0; r < repeats; r++) {
            const int64_t st0 = s->tot_steps;
            const auto t0 = std::chrono::steady_clock::now();
            RET(run_batch(s, ops, [] { return REG_OK; }, nullptr, nullptr));  // returns after a sync
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            total = std::min(total, ms);
            per_step = std::min(per_step, ms / (double)std::max<int64_t>(1, s->tot_steps - st0));
            runs++;
        }
        return REG_OK;
    };
    double ps, tot, ps0, tot0;
    RET(run_batch(s, ops, [] { return REG_OK; }, nullptr, nullptr));  // warm-up: buffers, graph
    RET(measure(ps0, tot0));
    // coordinate descent, finest level first; a change must gain 2%
    const int cand[] = {8, 16, 32, 64};
    for (int k = si.nl - 1; k >= 0; k--) {
        if (si.n[k] < 129) continue;  // launch-bound levels: the defaults
        const int l = level_of(si.n[k]);
        for (int which = 0; which < 2; which++) {
            int *tab = which ? s->tile_ht : s->tile_hg;
            const int keep0 = tab[l];
            RET(measure(ps, tot));
            double best = ps;
            int keep = keep0;
            for (int c : cand) {
                if (c == keep0 || c > si.n[k]) continue;
                tab[l] = c;
                RET(measure(ps, tot));
                if (ps < 0.98 * best) { best = ps; keep = c; }
            }
            tab[l] = keep;
        }
    }
    // step sizes per Armijo pass
    {
        const int keep0 = s->p.trials_per_pass;
        RET(measure(ps, tot));
        double best = tot;
        int keep = keep0;
        for (int J : {2, 3, 4, 8}) {
            if (J == keep0) continue;
            s->p.trials_per_pass = J;
            set_grids(s);
            s->buf_gen++;  // the captured graph launches the trial kernel for J
            RET(measure(ps, tot));
            if (tot < 0.98 * best) { best = tot; keep = J; }
        }
        s->p.trials_per_pass = keep;
        set_grids(s);
        s->buf_gen++;
    }
    double ps1, tot1;
    RET(measure(ps1, tot1));
    // the sample overwrote these data slots
    for (int e = 0; e < n_pairs; e++) si.meta[e] = SlotMeta{};
    si.pre_from_slots = false;
    if (report && buf_len > 0) {
        std::string js = "{\"levels\": [";
        for (int k = 0; k < si.nl; k++) {
            const int l = level_of(si.n[k]);
            char b[128];
            snprintf(b, sizeof b, "%s{\"level\": %d, \"n\": %d, \"grad_rows\": %d, \"trial_rows\": %d}", k ? ", " : "",
                     l, si.n[k], s->tile_hg[l], s->tile_ht[l]);
            js += b;
        }
        char b[256];
        snprintf(b, sizeof b,
                 "], \"trials_per_pass\": %d, \"sample_ops\": %d, \"runs\": %d, \"ms_before\": %.3f, "
                 "\"ms_after\": %.3f}",
                 s->p.trials_per_pass, n_pairs, runs, tot0, tot1);
        js += b;
        snprintf(report, buf_len, "%s", js.c_str());
    }
    return REG_OK;
}

}  // extern "C"

reg_status reg_internal_fail(reg_status st, const char *msg) { return fail(st, "%s", msg); }

// ---------------------------------------------------------------------------
// The learned initialiser on a series: input pairs from the pyramid level of
// 257^2 nodes (256^2 of them: the last row and column dropped), predictions
// upsampled onto the finest vertex grid (pixels) in the data slots.
// ---------------------------------------------------------------------------
namespace {

__global__ void k_cnn_pairs(const void *pyr, int64_t frame_block, int64_t img_off, int pitch, int bf16, int first,
                            int side, float *x)
{
    const int p = blockIdx.z, ch = blockIdx.y;  // pair p of the chunk, channel (0 reference, 1 template)
    const int frame = first + p + ch;
    const int64_t base = (int64_t)frame * frame_block + img_off;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < side * side; i += gridDim.x * blockDim.x) {
        const int r = i / side, c = i % side;
        const int64_t o = base + (int64_t)r * pitch + c;
        const float v = bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(pyr)[o])
                             : reinterpret_cast<const float *>(pyr)[o];
        x[((int64_t)p * 2 + ch) * side * side + i] = v;
    }
}

// Output (2 x q x q, input pixels at input pixels 4i, 4j) -> displacement in
// frame pixels on the (side+1)^2 grid of the slot: bilinear in the output grid,
// clamped at its border, scaled by k = side / (4 q) frame pixels per input pixel.
__global__ void k_cnn_to_slot(const float *y, int q, int side, float2 *slot, int pitch)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r > side || c > side) return;
    const float k = (float)side / (4.f * q);
    auto coord = [&](int i, int &i0, float &f) {
        const float t = (float)i / (4.f * k);
        i0 = min(max((int)floorf(t), 0), q - 2);
        f = fminf(fmaxf(t - i0, 0.f), 1.f);
    };
    int r0, c0;
    float fr, fc;
    coord(r, r0, fr);
    coord(c, c0, fc);
    float2 o;
    for (int ch = 0; ch < 2; ch++) {
        const float *m = y + (int64_t)ch * q * q;
        const float top = (1.f - fc) * m[r0 * q + c0] + fc * m[r0 * q + c0 + 1];
        const float bot = (1.f - fc) * m[(r0 + 1) * q + c0] + fc * m[(r0 + 1) * q + c0 + 1];
        const float v = k * ((1.f - fr) * top + fr * bot);
        if (ch == 0) o.x = v; else o.y = v;
    }
    slot[(int64_t)r * pitch + c] = o;
}

// Index of the pyramid level with 257^2 nodes, or -1.
int cnn_level(const SeriesInfo &si)
{
    for (int k = 0; k < si.nl; k++)
        if (si.n[k] == 257) return k;
    return -1;
}

}  // namespace

reg_status reg_cnn_pairs(reg_series_t s, int32_t series, int32_t first_pair, int32_t count, float *x)
{
    g_err.clear();
    if (!s || series < 0 || series >= (int)s->S.size() || !x || count < 1) return fail(REG_EINVAL, "bad argument");
    const SeriesInfo &si = s->S[series];
    if (first_pair < 0 || first_pair + count > si.n_data) return fail(REG_EINVAL, "pair range outside the series");
    const int k = cnn_level(si);
    if (k < 0) return fail(REG_EINVAL, "the pyramid has no level of 257^2 nodes");
    k_cnn_pairs<<<dim3(64, 2, count), 256, 0, s->stream>>>(si.pyr, (int64_t)si.frame_block, (int64_t)si.img_off[k],
                                                            si.pitch[k], s->bf16, first_pair, 256, x);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    return REG_OK;
}

reg_status reg_cnn_init_series(reg_series_t s, int32_t series, reg_cnn_t h, int32_t tensor_cores)
{
    g_err.clear();
    if (!s || !h || series < 0 || series >= (int)s->S.size()) return fail(REG_EINVAL, "bad argument");
    SeriesInfo &si = s->S[series];
    if (cnn_input_side(h) != 256) return fail(REG_EINVAL, "the network must take 256^2 inputs");
    const int k = cnn_level(si);
    if (k < 0) return fail(REG_EINVAL, "the pyramid has no level of 257^2 nodes");
    const int B = cnn_max_batch(h), q = (int)cnn_output_side(h), nL = si.n[si.nl - 1];
    float *x = nullptr, *y = nullptr;
    RET(dalloc(s, (void **)&x, sizeof(float) * (size_t)B * 2 * 256 * 256));
    reg_status st = dalloc(s, (void **)&y, sizeof(float) * (size_t)B * 2 * q * q);
    for (int p0 = 0; st == REG_OK && p0 < si.n_data; p0 += B) {
        const int cnt = std::min(B, si.n_data - p0);
        k_cnn_pairs<<<dim3(64, 2, cnt), 256, 0, s->stream>>>(si.pyr, (int64_t)si.frame_block,
                                                              (int64_t)si.img_off[k], si.pitch[k], s->bf16, p0, 256, x);
        st = cnn_forward(h, x, cnt, y, s->stream, tensor_cores != 0);
        for (int e = 0; st == REG_OK && e < cnt; e++) {
            k_cnn_to_slot<<<dim3(cdiv(nL, 32), cdiv(nL, 8)), dim3(32, 8), 0, s->stream>>>(
                y + (size_t)e * 2 * q * q, q, nL - 1, si.slots + (size_t)(p0 + e) * si.slot_elems, si.pitch[si.nl - 1]);
            si.meta[p0 + e] = SlotMeta{p0 + e, p0 + e + 1};  // an initial guess of phi_{e,e+1}
        }
        if (st == REG_OK && cudaGetLastError() != cudaSuccess) st = fail(REG_ECUDA, "learned initialiser kernels");
    }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess && st == REG_OK) st = fail(REG_ECUDA, "sync");
    if (st == REG_OK) st = cnn_check_device_error(h);
    dfree(s, x, 0);
    dfree(s, y, 0);
    if (st == REG_OK) si.pre_from_slots = true;
    return st;
}
