// lbm_capi.cu -- C ABI of the library (include/lbm.h): solver object, upload of
// the tiled grid, the recursive level scheduler (Sec 2.1: each finer level takes
// two sub-steps per parent step) captured into CUDA graphs, and host queries.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <omp.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include <nvtx3/nvToolsExt.h>
#include "device.cuh"
#include "grid.hpp"

using lbmdev::LevelView;
using lbmdev::LoadsView;
using lbmdev::RecView;
using lbmdev::StepConsts;

namespace {

const int CXh[9] = LBM_CX_INIT;
const int CYh[9] = LBM_CY_INIT;
const double WQh[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

// shifted equilibrium g_q = f_q^eq - w_q as the product of two one-dimensional
// three-velocity equilibria (equal to the fourth-order Hermite form of eq 4)
void feq_shifted(double rho, double ux, double uy, float *g)
{
    auto h = [](int c, double u) { return c == 0 ? 2.0 / 3.0 - u * u : 0.5 * (u * u + 1.0 / 3.0 + c * u); };
    for (int q = 0; q < 9; q++) g[q] = (float)(rho * h(CXh[q], ux) * h(CYh[q], uy) - WQh[q]);
}

// bytes of one stored population: FP32, FP16 or BF16
size_t pop_bytes(int store) { return store == 0 ? 4 : 2; }

// Step 1 of Sec 2.3 as fixed linear combinations of the stencil values, from the static
// geometry of a wall record: rho_R = sum wr_m rho_m with inverse-distance weights 1/d^2
// (normalised), u_R = sum wu_m u_m with wu the intercept row of the unweighted linear
// least-squares fit a + b dx + c dy, or the IDW weights when fewer than 3 points or a
// near-singular normal matrix leave the fit undefined.  Computed in FP64.
void stencil_weights(const lbmgrid::Record &R, double wr[16], double wu[16])
{
    double sw = 0.0, A[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double dx[16], dy[16];
    for (int m = 0; m < R.ns; m++) {
        dx[m] = R.si[m] + 0.5 - R.r[0];
        dy[m] = R.sj[m] + 0.5 - R.r[1];
        const double d2 = dx[m] * dx[m] + dy[m] * dy[m];
        wr[m] = 1.0 / (d2 > 1e-20 ? d2 : 1e-20);
        sw += wr[m];
        const double phi[3] = {1.0, dx[m], dy[m]};
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) A[3 * a + b] += phi[a] * phi[b];
    }
    for (int m = 0; m < R.ns; m++) { wr[m] /= sw; wu[m] = wr[m]; }
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (R.ns >= 3 && det > 1e-9 * A[0] * A[4] * A[8]) {
        // first column of A^-1 (A is symmetric) by cofactors
        const double x0 = (A[4] * A[8] - A[5] * A[7]) / det;
        const double x1 = -(A[3] * A[8] - A[5] * A[6]) / det;
        const double x2 = (A[3] * A[7] - A[4] * A[6]) / det;
        for (int m = 0; m < R.ns; m++) wu[m] = x0 + x1 * dx[m] + x2 * dy[m];
    }
}

struct HostLevelDev {
    LevelView v;
    std::vector<uint32_t> flags;   // host copy
    std::vector<int> band_ij;      // global cell indices of the band cells, in band-index order
    std::vector<int> work_tiles;   // host copies of the level kernel's work lists (cost order)
    std::vector<int> work_warps;
};

}  // namespace

struct lbm_solver {
    lbm_config cfg;
    std::string err;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    int device = 0;
    int L = 0;
    double U = 0;
    bool geometry = false;         // device state built (steps, fields, loads)
    bool grid_ready = false;       // host grid tables built (also on host-only handles)
    lbmgrid::Grid g;
    HostLevelDev lv[LBM_MAXL];
    RecView rec;
    LoadsView segs;
    StepConsts k;
    int parity[LBM_MAXL];
    int min_blocks[LBM_MAXL];     // register budget of each level's kernel (lbm_autotune)
    // prolongations of consecutive levels that read nothing the other writes go out as one
    // launch: prolong_indep[l] holds when no band cell of level l has a ghost of level l in
    // its 3 x 3 neighbourhood (prolongation l - 1 writes those ghosts, prolongation l reads
    // the band cells' neighbourhoods)
    bool prolong_indep[LBM_MAXL];
    int prolong_merge = 1;          // lbm_set_prolong_merge
    lbmdev::ProlongBatchArgs pend;  // prolongations waiting for the next level-step launch
    // launch timeline (lbm_set_timeline): 3 clock readings per block of every launch of the
    // step graphs, records [tl_meta base, base + blocks) of a launch; meta 5 ints per launch
    // load history (lbm_set_load_history): ring of hist_cap records of 6 doubles, one every
    // hist_every coarse steps of lbm_step / lbm_step_async; hist_count records taken
    double *d_hist = nullptr;
    int hist_every = 0, hist_cap = 0, hist_alloc = 0;
    long long hist_count = 0;
    unsigned long long *d_tl = nullptr;
    long long tl_cap = 0, tl_next = 0;
    int tl_on = 0, tl_graph = -1;
    std::vector<int> tl_meta;         // graph, level, kind (0 even, 1 odd, 2 prolongation), base, blocks
    unsigned pend_grid = 0;
    int pend_level = 0;
    int sched[LBM_MAXL];          // grid schedule (LBM_SCHED_*) of each level's kernel (lbm_autotune)
    int shape[LBM_MAXL];          // work shape of a warp for each level's kernel (lbm_autotune)
    int pdl = 1;                  // programmatic dependent launch (lbm_autotune)
    bool off_schedule = false;    // single launches (lbm_step_launch) left the level schedule
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::vector<void *> allocs;
    double device_bytes = 0;
    int *d_status = nullptr;
    double *d_acc = nullptr;
    float *d_slip = nullptr;
    long long step = 0;
    double last_cl = 0;
    bool have_cl = false;
    long long kernels_per_step = 0;
    int n_loops = 0;
    // memory plan (lbm_plan_geometry): allocations are counted, not made
    bool planning = false;
    size_t plan_cursor = 1 << 20;
    // eager timing (lbm_time_kernels)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_marks;   // (class, event index pair start)
    std::vector<long long> ev_cells;
    std::vector<int> ev_level;
    int ev_used = 0;
};

static lbm_status fail(lbm_solver *s, lbm_status code, const std::string &m)
{
    if (s) s->err = m;
    return code;
}

static lbm_status cuda_fail(lbm_solver *s, cudaError_t e, const char *where)
{
    return fail(s, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return cuda_fail(s, _e, #call);       \
    } while (0)

// NVTX range over a scope: the library's calls and, outside graph capture, each launch of
// the level schedule show up by name in a profiler's timeline (no-ops without a tool)
struct NvtxRange {
    explicit NvtxRange(const char *m) { nvtxRangePushA(m); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

static void *dalloc(lbm_solver *s, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (s->planning) {
        // memory plan only: count the bytes (rounded as cudaMalloc aligns them), hand back
        // a distinct placeholder that is never dereferenced
        bytes = (bytes + 255) & ~(size_t)255;
        s->device_bytes += (double)bytes;
        s->plan_cursor += bytes;
        return (void *)(uintptr_t)s->plan_cursor;
    }
    void *p = nullptr;
    if (s->cfg.dev_alloc) {
        p = s->cfg.dev_alloc(bytes, (void *)s->stream, s->cfg.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    if (p && ((uintptr_t)p & 255u)) {
        // every tile plane (1 KB in FP32) starts on a 256-byte boundary only if its array
        // does, which keeps each warp's row segments in whole sectors (cudaMalloc gives
        // 256-byte alignment); refuse anything less
        if (s->cfg.dev_free) s->cfg.dev_free(p, (void *)s->stream, s->cfg.alloc_ctx);
        return nullptr;
    }
    if (p) { s->allocs.push_back(p); s->device_bytes += (double)((bytes + 255) & ~(size_t)255); }
    return p;
}

// device scratch of a host utility (queries, set_fields): through the caller's allocator
// when given, freed before the call returns
static void *tmp_alloc(lbm_solver *s, size_t bytes)
{
    void *p = nullptr;
    if (s->cfg.dev_alloc) p = s->cfg.dev_alloc(bytes, (void *)s->stream, s->cfg.alloc_ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    return p;
}

static void tmp_free(lbm_solver *s, void *p)
{
    if (!p) return;
    cudaStreamSynchronize(s->stream);
    if (s->cfg.dev_free) s->cfg.dev_free(p, (void *)s->stream, s->cfg.alloc_ctx);
    else cudaFree(p);
}

static void free_all(lbm_solver *s)
{
    if (s->planning) {
        s->device_bytes = 0;
        s->plan_cursor = 1 << 20;
        return;
    }
    for (int b = 0; b < 2; b++)
        if (s->graph[b]) { cudaGraphExecDestroy(s->graph[b]); s->graph[b] = nullptr; }
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (void *p : s->allocs) {
        if (s->cfg.dev_free) s->cfg.dev_free(p, (void *)s->stream, s->cfg.alloc_ctx);
        else cudaFree(p);
    }
    s->allocs.clear();
    s->device_bytes = 0;
    s->geometry = false;
    s->d_tl = nullptr;
    s->d_hist = nullptr;
    s->hist_every = s->hist_cap = s->hist_alloc = 0;
    s->hist_count = 0;
    s->tl_cap = s->tl_next = 0;
    s->tl_on = 0;
    s->tl_meta.clear();
    for (auto &e : s->ev_pool) cudaEventDestroy(e);
    s->ev_pool.clear();
}

template <class T>
static T *upload(lbm_solver *s, const std::vector<T> &h, bool &ok)
{
    T *d = (T *)dalloc(s, h.size() * sizeof(T));
    if (!d) { ok = false; return nullptr; }
    if (!s->planning && !h.empty() && cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        ok = false;
    return d;
}

// ---------------------------------------------------------------- scheduler
// Kernel classes for lbm_time_kernels.
enum { KC_LEVEL_FINEST = 0, KC_LEVEL_COARSE = 1, KC_PROLONG = 2, KC_N = 3 };
static const char *KC_NAME[KC_N] = {"level_step_finest", "level_step_coarse", "prolong"};

static void mark_begin(lbm_solver *s)
{
    if (!s->timing) return;
    if (s->ev_used + 2 > (int)s->ev_pool.size()) {
        for (int i = 0; i < 256; i++) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            s->ev_pool.push_back(e);
        }
    }
    cudaEventRecord(s->ev_pool[s->ev_used], s->stream);
}

static void mark_end(lbm_solver *s, int cls, long long cells, int level)
{
    if (!s->timing) return;
    cudaEventRecord(s->ev_pool[s->ev_used + 1], s->stream);
    s->ev_marks.push_back({cls, s->ev_used});
    s->ev_cells.push_back(cells);
    s->ev_level.push_back(level);
    s->ev_used += 2;
}

// Records for one launch of the graph being captured, when the timeline is on: the first
// record, or -1 (no timeline, or no room; the launch then records nothing).
static int tl_reserve(lbm_solver *s, int level, int kind, int blocks)
{
    if (!s->tl_on || s->tl_graph < 0 || !s->d_tl || s->tl_next + blocks > s->tl_cap) return -1;
    const int base = (int)s->tl_next;
    s->tl_meta.insert(s->tl_meta.end(), {s->tl_graph, level, kind, base, blocks});
    s->tl_next += blocks;
    return base;
}

// Launch the pending prolongations (one kernel for all of them).
static void flush_prolong(lbm_solver *s, cudaStream_t st, long long &nk)
{
    if (s->pend.n == 0) return;
    char nm[48];
    snprintf(nm, sizeof nm, "prolong level %d (+%d)", s->pend_level, s->pend.n - 1);
    NvtxRange range(s->tl_graph < 0 ? nm : "capture");
    mark_begin(s);
    const int base = tl_reserve(s, s->pend_level, 2, (int)s->pend_grid);
    unsigned long long *tl = base >= 0 ? s->d_tl : nullptr;
    if (s->pend.n == 1) {
        lbmdev::launch_prolong(st, s->pend.d[0].P, s->pend.d[0].F, s->pend.d[0].p, s->pdl, tl, base);
    } else {
        s->pend.tl = tl;
        s->pend.tl_base = base;
        lbmdev::launch_prolong_batch(st, s->pend, s->pend_grid, s->pdl);
    }
    mark_end(s, KC_PROLONG, (long long)s->pend_grid * LBM_TILE, s->pend_level);
    nk++;
    s->pend.n = 0;
    s->pend_grid = 0;
}

// One level-l step (Sec 2.1 recursive sub-cycling): the ghost fields of level l+1 are
// reconstructed from level l at time t, level l+1 takes two sub-steps (the second one
// restricts its new fields into the covered cells of level l), then one fused launch
// advances level l itself (wall function on the finest level, SA-neg, stream with
// coalescence and cut links, collide, explode).
static void advance(lbm_solver *s, cudaStream_t st, int l, int restrict_up, long long &nk)
{
    const int L = s->L;
    LevelView &P = s->lv[l].v;
    const LevelView *F = (l < L - 1) ? &s->lv[l + 1].v : nullptr;
    const LevelView *C = (l > 0) ? &s->lv[l - 1].v : nullptr;
    if (F) {
        // the prolongation joins the pending ones when it reads nothing they write (it
        // follows the prolongation of level l - 1 in the descent); the next level step
        // launches them
        if (P.n_band_tiles > 0) {
            if (s->pend.n > 0 && !(s->prolong_merge && s->prolong_indep[l] && s->pend_level + s->pend.n == l))
                flush_prolong(s, st, nk);
            if (s->pend.n == 0) s->pend_level = l;
            lbmdev::ProlongDesc &d = s->pend.d[s->pend.n++];
            d.P = P; d.F = *F; d.p = s->parity[l]; d.first_block = (int)s->pend_grid;
            s->pend_grid += (unsigned)P.n_band_tiles;
        }
        advance(s, st, l + 1, 0, nk);
        advance(s, st, l + 1, 1, nk);
    }
    flush_prolong(s, st, nk);
    lbmdev::LevelStep ls{};
    ls.p = s->parity[l];
    ls.has_child = F != nullptr;
    ls.is_level0 = l == 0;
    ls.wall = (l == L - 1) && s->rec.n > 0;
    ls.restrict_up = restrict_up && C != nullptr;
    ls.pp = C ? s->parity[l - 1] : 0;
    ls.shape = s->shape[l];
    ls.status = s->d_status;
    char nm[48];
    snprintf(nm, sizeof nm, "level %d %s step", l, ls.p ? "odd" : "even");
    NvtxRange range(s->tl_graph < 0 ? nm : "capture");
    {
        const int base = tl_reserve(s, l, ls.p, std::max(P.n_work_tiles, (P.n_work_warps + 1) / 2));
        ls.tl = base >= 0 ? s->d_tl : nullptr;
        ls.tl_base = base;
    }
    mark_begin(s);
    const lbmdev::LevelTune tu{s->min_blocks[l], s->pdl, s->sched[l], s->shape[l]};
    lbmdev::launch_level(st, P, F, C, s->rec, s->k, ls, tu);
    mark_end(s, l == L - 1 ? KC_LEVEL_FINEST : KC_LEVEL_COARSE, P.ns, l);
    nk++;
    s->parity[l] ^= 1;
}

// one graph per level-0 parity; the graph of the current parity is captured first, and
// the two captures leave every level's parity as it was
static lbm_status capture_graphs(lbm_solver *s)
{
    s->tl_next = 0;
    s->tl_meta.clear();
    for (int b = 0; b < 2; b++)
        if (s->graph[b]) { cudaGraphExecDestroy(s->graph[b]); s->graph[b] = nullptr; }
    const int b0 = s->parity[0];
    for (int bi = 0; bi < 2; bi++) {
        const int b = b0 ^ bi;
        if (s->parity[0] != b) return fail(s, LBM_ERR_CUDA, "internal: parity mismatch at capture");
        cudaGraph_t gr;
        long long nk = 0;
        CK(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
        s->tl_graph = b;
        advance(s, s->cap_stream, 0, 0, nk);
        s->tl_graph = -1;
        CK(cudaStreamEndCapture(s->cap_stream, &gr));
        CK(cudaGraphInstantiate(&s->graph[b], gr, 0));
        cudaGraphDestroy(gr);
        s->kernels_per_step = nk;
    }
    return LBM_OK;
}

static lbm_status enqueue_mass(lbm_solver *s);
static void enqueue_history(lbm_solver *s);

static lbm_status enqueue_steps(lbm_solver *s, int n)
{
    for (int it = 0; it < n; it++) {
        CK(cudaGraphLaunch(s->graph[s->parity[0]], s->stream));
        s->parity[0] ^= 1;
        s->step++;
        if (s->hist_every > 0 && s->step % s->hist_every == 0) enqueue_history(s);
    }
    return LBM_OK;
}

// non-finite check and FP64 mass into d_acc[4]
static lbm_status enqueue_mass(lbm_solver *s)
{
    CK(cudaMemsetAsync(s->d_acc + 4, 0, sizeof(double), s->stream));
    for (int l = 0; l < s->L; l++) {
        double area = (double)(1LL << (s->L - 1 - l));
        lbmdev::launch_mass(s->stream, s->lv[l].v, s->parity[l], area * area, s->d_acc + 4, s->d_status);
    }
    return LBM_OK;
}

// the loads of lbm_get_loads (wall state query, eq 29-30 sums, FP64 mass) into the next
// slot of the load history, on the solver stream
static void enqueue_history(lbm_solver *s)
{
    lbmdev::launch_wallfn(s->stream, s->lv[s->L - 1].v, s->parity[s->L - 1], s->rec, s->k);
    cudaMemsetAsync(s->d_acc, 0, 4 * sizeof(double), s->stream);
    lbmdev::launch_loads(s->stream, s->segs, s->rec, (float)s->U, s->d_acc);
    enqueue_mass(s);
    const double chord = s->cfg.chord / (s->cfg.h0 / (double)(1LL << (s->L - 1)));
    lbmdev::launch_hist_push(s->stream, s->d_acc, s->d_hist, (int)(s->hist_count % s->hist_cap), s->step, chord);
    s->hist_count++;
}

static lbm_status check_status(lbm_solver *s)
{
    int st = 0;
    CK(cudaMemcpyAsync(&st, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (st & LBM_STATUS_TIMEOUT) return fail(s, LBM_ERR_TIMEOUT, "a device wait reached its limit");
    if (st & LBM_STATUS_BOUNDS)
        return fail(s, LBM_ERR_CUDA, "a device index left its buffer (caught by the bounds-checked build)");
    if (st & LBM_STATUS_NONFINITE) return fail(s, LBM_ERR_DIVERGED, "diverged (non-finite field)");
    if (st) return fail(s, LBM_ERR_CUDA, "device status word set");
    return LBM_OK;
}

// the grid builder's specification from a solver configuration
static lbmgrid::Spec grid_spec(const lbm_config &c)
{
    return lbmgrid::Spec{c.levels, c.nx0, c.ny0, c.layers, c.x0, c.y0, c.h0, c.d_wr, c.d_wv,
                         c.periodic, c.solid_walls, c.wall_model};
}

// 64-bit FNV-1a over raw bytes (grid digest)
namespace {
struct Fnv {
    unsigned long long h = 1469598103934665603ull;
    void bytes(const void *p, size_t n)
    {
        const unsigned char *c = (const unsigned char *)p;
        for (size_t i = 0; i < n; i++) { h ^= c[i]; h *= 1099511628211ull; }
    }
    template <class T> void val(const T &v) { bytes(&v, sizeof v); }
    template <class V> void vec(const V &v)
    {
        const size_t n = v.size();
        val(n);
        if (n) bytes(v.data(), n * sizeof(v[0]));
    }
};
}  // namespace

// ---------------------------------------------------------------- API
extern "C" {

static bool config_ok(const lbm_config *cfg)
{
    return !(cfg->levels < 1 || cfg->levels > LBM_MAXL || cfg->nx0 < 4 || cfg->ny0 < 4 || !(cfg->h0 > 0) ||
        cfg->layers < 3 || !(cfg->Re > 0) || !(cfg->Ma > 0) || !(cfg->chord > 0) || cfg->store < 0 || cfg->store > 2 ||
        (cfg->periodic && (cfg->nx0 % LBM_TX || cfg->ny0 % LBM_TY)) || (!cfg->periodic && (cfg->nx0 < 8)) ||
        cfg->wall_model < 0 || cfg->wall_model > 3 || cfg->sa_convection < 0 || cfg->sa_convection > 1 ||
        cfg->outlet < 0 || cfg->outlet > 1 ||
        (!cfg->dev_alloc != !cfg->dev_free));
}

lbm_status lbm_create(const lbm_config *cfg, lbm_solver **out)
{
    if (!cfg || !out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!config_ok(cfg)) return LBM_ERR_INVALID_ARG;
    lbm_solver *s = new (std::nothrow) lbm_solver();
    if (!s) return LBM_ERR_OOM;
    s->cfg = *cfg;
    s->L = cfg->levels;
    s->U = cfg->Ma * std::sqrt(1.0 / 3.0);
    for (int l = 0; l < LBM_MAXL; l++) {
        s->parity[l] = 0; s->min_blocks[l] = 5; s->sched[l] = LBM_SCHED_TILE; s->shape[l] = 0;
        s->prolong_indep[l] = false;
    }
    s->pend.n = 0;
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return LBM_ERR_CUDA; }
    if (cfg->cuda_stream) {
        s->stream = (cudaStream_t)cfg->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) { delete s; return LBM_ERR_CUDA; }
        s->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return LBM_ERR_CUDA;
    }
    *out = s;
    return LBM_OK;
}

lbm_status lbm_create_host(const lbm_config *cfg, lbm_solver **out)
{
    if (!cfg || !out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!config_ok(cfg)) return LBM_ERR_INVALID_ARG;
    lbm_solver *s = new (std::nothrow) lbm_solver();
    if (!s) return LBM_ERR_OOM;
    s->cfg = *cfg;
    s->cfg.cuda_stream = nullptr;
    s->cfg.dev_alloc = nullptr;
    s->cfg.dev_free = nullptr;
    s->L = cfg->levels;
    s->U = cfg->Ma * std::sqrt(1.0 / 3.0);
    s->planning = true;
    *out = s;
    return LBM_OK;
}

void lbm_destroy(lbm_solver *s)
{
    if (!s) return;
    free_all(s);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

const char *lbm_last_error(const lbm_solver *s) { return s ? s->err.c_str() : "null handle"; }

lbm_status lbm_set_geometry(lbm_solver *s, const double *xy, const int *loop_off, int n_loops)
{
    NvtxRange range("lbm_set_geometry");
    if (!s || n_loops < 0 || (n_loops > 0 && (!xy || !loop_off))) return fail(s, LBM_ERR_INVALID_ARG, "bad geometry arguments");
    free_all(s);
    s->grid_ready = false;
    const lbm_config &c = s->cfg;
    std::string msg;
    int rc = lbmgrid::build(grid_spec(c), xy, loop_off, n_loops, s->g, msg);
    if (rc != 0) return fail(s, (lbm_status)rc, msg);
    const int L = s->L;
    bool ok = true;
    // band indices (the explosion and coalescence buffers of each level with a finer one):
    // band cells in row-major order of the level's box
    std::vector<std::vector<int>> bidx(L);
    std::vector<int> n_band(L, 0);
    for (int l = 0; l + 1 < L; l++) {
        const lbmgrid::Level &G = s->g.lv[l];
        bidx[l].assign(G.kind.size(), -1);
        std::vector<int> row(G.bny + 1, 0);
#pragma omp parallel for schedule(static)
        for (int r = 0; r < G.bny; r++) {
            int n = 0;
            for (int q = 0; q < G.bnx; q++) n += G.band[(size_t)r * G.bnx + q] != 0;
            row[r + 1] = n;
        }
        for (int r = 0; r < G.bny; r++) row[r + 1] += row[r];
#pragma omp parallel for schedule(static)
        for (int r = 0; r < G.bny; r++) {
            int n = row[r];
            for (int q = 0; q < G.bnx; q++)
                if (G.band[(size_t)r * G.bnx + q]) bidx[l][(size_t)r * G.bnx + q] = n++;
        }
        n_band[l] = row[G.bny];
        std::vector<int> &bij = s->lv[l].band_ij;
        bij.assign(2 * (size_t)n_band[l], 0);
#pragma omp parallel for schedule(static)
        for (int r = 0; r < G.bny; r++)
            for (int q = 0; q < G.bnx; q++) {
                const int b = bidx[l][(size_t)r * G.bnx + q];
                if (b >= 0) { bij[2 * (size_t)b] = G.bi0 + q; bij[2 * (size_t)b + 1] = G.bj0 + r; }
            }
    }
    s->lv[L - 1].band_ij.clear();
    // per-level flag words and device arrays
    for (int l = 0; l < L; l++) {
        lbmgrid::Level &G = s->g.lv[l];
        HostLevelDev &H = s->lv[l];
        const long long ns = (long long)G.ntiles * LBM_TILE;
        if (9 * ns >= (1LL << 31)) { free_all(s); return fail(s, LBM_ERR_INVALID_ARG, "level too large for 32-bit slot indices"); }
        H.flags.assign(ns, 0);
        std::vector<float> inv_d2(ns, 0.f);
        std::vector<int> aux(ns, -1);
        const lbmgrid::Level *Gc = l > 0 ? &s->g.lv[l - 1] : nullptr;
        const lbmgrid::Level *Gf = l + 1 < L ? &s->g.lv[l + 1] : nullptr;
        // every slot is written by the thread of its tile
#pragma omp parallel for schedule(static)
        for (int t = 0; t < G.ntiles; t++)
            for (int c2 = 0; c2 < LBM_TILE; c2++) {
                long long i = (long long)G.tile_x[t] * LBM_TX + (c2 & 31), j = (long long)G.tile_y[t] * LBM_TY + (c2 >> 5);
                long b = G.idx(i, j);
                if (b < 0 || G.kind[b] == KIND_ABSENT) continue;
                long long sl = (long long)t * LBM_TILE + c2;
                uint32_t f = G.kind[b];
                if (G.solid[b]) f |= FL_SOLID;
                if (G.band[b]) f |= FL_BAND;
                if (G.bnode[b]) f |= FL_BNODE;
                for (int d = 1; d < 9; d++)
                    if (G.coal[b] >> d & 1) f |= 1u << (FL_COAL_SHIFT + d - 1);
                if (G.kind[b] == KIND_GHOST) {
                    // the ghost keeps its own value along d where the upstream cell is not an
                    // active or ghost fluid cell; aux: the parent's band index and the child index
                    for (int d = 1; d < 9; d++) {
                        const long u = G.idx(i - CXh[d], j - CYh[d]);
                        const bool flows = u >= 0 && !G.solid[u] && (G.kind[u] == KIND_ACTIVE || G.kind[u] == KIND_GHOST);
                        if (!flows) f |= 1u << (FL_KEEP_SHIFT + d - 1);
                    }
                    const long pc = Gc->idx(i >> 1, j >> 1);
                    aux[sl] = 4 * bidx[l - 1][pc] + (int)(((j & 1) << 1) | (i & 1));
                } else {
                    for (int d = 1; d < 9; d++)
                        if (G.cut[b] >> d & 1) f |= 1u << (FL_CUT_SHIFT + d - 1);
                }
                if (G.band[b] && Gf) {
                    // band cell: its index, and which children are solid or have no tile
                    aux[sl] = bidx[l][b];
                    for (int m = 0; m < 4; m++) {
                        const long long fi = 2 * i + (m & 1), fj = 2 * j + (m >> 1);
                        const long fc = Gf->idx(fi, fj);
                        if (Gf->slot(fi, fj) < 0 || fc < 0 || Gf->solid[fc]) f |= 1u << (FL_SCH_SHIFT + m);
                    }
                }
                if (l == L - 1 && G.bnode[b]) aux[sl] = G.rec[b];
                if (l == 0 && !c.periodic) {
                    if (i == 0) f |= FL_INLET;
                    if (i == c.nx0 - 1) f |= FL_OUTLET;
                    if (i == c.nx0 - 2) f |= FL_OUTLET2;
                    if (j == 0) f |= FL_BOTTOM;
                    if (j == c.ny0 - 1) f |= FL_TOP;
                }
                H.flags[sl] = f;
                // SA-neg sees d >= 1/2 (level units): a fluid node closer to the wall than that
                // lies beside a wall sliver thinner than the lattice (a sharp trailing edge
                // between nodes), where d -> 0 makes the explicit destruction term unstable
                const double dsa = G.dist[b] > 0.5 ? (double)G.dist[b] : 0.5;
                inv_d2[sl] = (float)(1.0 / (dsa * dsa));
            }
        // every index the kernels follow from aux stays inside its buffer
        {
            const int nr = (int)s->g.recs.size();
            bool bad = false;
#pragma omp parallel for schedule(static) reduction(|| : bad)
            for (long long sl = 0; sl < ns; sl++) {
                const uint32_t f = H.flags[sl];
                const uint32_t kd = f & FL_KIND_MASK;
                const int a = aux[sl];
                if (kd == KIND_GHOST && !(f & FL_SOLID)) bad = bad || a < 0 || l == 0 || (a >> 2) >= n_band[l - 1];
                if ((f & FL_BAND) && l + 1 < L) bad = bad || a < 0 || a >= n_band[l];
                if ((f & FL_BNODE) && l == L - 1) bad = bad || a < 0 || a >= nr;
            }
            if (bad) { free_all(s); return fail(s, LBM_ERR_GEOMETRY, "internal: inconsistent band or record index"); }
        }
        LevelView &v = H.v;
        v.ntiles = G.ntiles;
        v.ns = (int)ns;
        v.n_wall_tiles = G.n_wall_tiles;
        v.tile_x = upload(s, G.tile_x, ok);
        v.tile_y = upload(s, G.tile_y, ok);
        v.nbr = upload(s, G.nbr, ok);
        v.child = upload(s, G.child, ok);
        v.parent = upload(s, G.parent, ok);
        v.band_tiles = upload(s, G.band_tiles, ok);
        v.n_band_tiles = (int)G.band_tiles.size();
        {
            // work tiles in the same cost order as the warps below (a block's warps start
            // together, so the expensive tiles go first and the last blocks are cheap)
            const long nwt = (long)G.work_tiles.size();
            std::vector<uint8_t> tcls(nwt, 0);
#pragma omp parallel for schedule(static)
            for (long m = 0; m < nwt; m++) {
                const int t = G.work_tiles[m];
                int cls = 0;
                for (int c = 0; c < LBM_TILE; c++) {
                    const uint32_t f = H.flags[(size_t)t * LBM_TILE + c];
                    if ((f & FL_SOLID) || (f & FL_KIND_MASK) != KIND_ACTIVE) continue;
                    int k = 1;
                    if (f & (FL_BAND | (0xFFu << FL_COAL_SHIFT))) k = 2;
                    if ((f & FL_BNODE) && l == L - 1) k = 3;
                    cls = std::max(cls, k);
                }
                tcls[m] = (uint8_t)cls;
            }
            std::vector<int> wt;
            wt.reserve(nwt);
            for (int k = 3; k >= 0; k--)
                for (long m = 0; m < nwt; m++)
                    if (tcls[m] == k) wt.push_back(G.work_tiles[m]);
            v.work_tiles = upload(s, wt, ok);
            v.n_work_tiles = (int)wt.size();
            H.work_tiles = wt;
        }
        {
            // warps (work shape 0: 16 x 2 cells) of the work tiles that hold an active or ghost
            // fluid cell, the expensive ones first so that the last blocks to start are cheap:
            // warps with a boundary node (wall function), then with a band or coalescing cell
            // (explosion, coalescence), then with another active cell, then ghosts only (a
            // relay); tile order within each class
            const long nwt8 = 8 * (long)G.work_tiles.size();
            std::vector<int8_t> wcls(nwt8, -1);
#pragma omp parallel for schedule(static)
            for (long mw = 0; mw < nwt8; mw++) {
                const int t = G.work_tiles[mw >> 3], w = (int)(mw & 7);
                int cls = -1;
                for (int c = 0; c < 32; c++) {
                    const int lx = (w & 1) * 16 + (c & 15), ly = (w >> 1) * 2 + (c >> 4);
                    const uint32_t f = H.flags[(size_t)t * LBM_TILE + ly * LBM_TX + lx];
                    const uint32_t kd = f & FL_KIND_MASK;
                    if (f & FL_SOLID) continue;
                    if (kd == KIND_GHOST) cls = std::max(cls, 0);
                    if (kd != KIND_ACTIVE) continue;
                    int k = 1;
                    if (f & (FL_BAND | (0xFFu << FL_COAL_SHIFT))) k = 2;
                    if ((f & FL_BNODE) && l == L - 1) k = 3;
                    cls = std::max(cls, k);
                }
                wcls[mw] = (int8_t)cls;
            }
            std::vector<int> ww;
            for (int k = 3; k >= 0; k--)
                for (long mw = 0; mw < nwt8; mw++)
                    if (wcls[mw] == k) ww.push_back(G.work_tiles[mw >> 3] * 8 + (int)(mw & 7));
            v.work_warps = upload(s, ww, ok);
            v.n_work_warps = (int)ww.size();
            H.work_warps = ww;
        }
        v.flags = upload(s, H.flags, ok);
        v.inv_d2 = upload(s, inv_d2, ok);
        v.aux = upload(s, aux, ok);
        v.f = dalloc(s, 9 * ns * pop_bytes(c.store));
        ok = ok && v.f;
        for (int b = 0; b < 2; b++) {
            v.chi[b] = (float *)dalloc(s, ns * sizeof(float));
            v.drho[b] = (float *)dalloc(s, ns * sizeof(float));
            v.ux[b] = (float *)dalloc(s, ns * sizeof(float));
            v.uy[b] = (float *)dalloc(s, ns * sizeof(float));
            ok = ok && v.chi[b] && v.drho[b] && v.ux[b] && v.uy[b];
        }
        v.n_band = n_band[l];
        v.ebuf = (float *)dalloc(s, 9 * (size_t)std::max(n_band[l], 1) * sizeof(float));
        v.gbuf = (float *)dalloc(s, 36 * (size_t)std::max(n_band[l], 1) * sizeof(float));
        ok = ok && v.ebuf && v.gbuf;
        v.nu = (float)(s->U * (c.chord / c.h0) * (double)(1LL << l) / c.Re);
        v.store = c.store;
        if (!ok) { free_all(s); return fail(s, LBM_ERR_OOM, "device allocation failed"); }
    }
    // wall records
    const int nr = (int)s->g.recs.size();
    {
        const lbmgrid::Level &G = s->g.lv[L - 1];
        std::vector<int> bslot(nr), nsv(nr), st_slot((size_t)nr * 16, -1), loop(nr);
        std::vector<float> st_wr((size_t)nr * 16, 0.f), st_wu((size_t)nr * 16, 0.f), nx(nr), ny(nr), dwb(nr), q((size_t)nr * 9, 0.f);
        std::vector<float> yc((size_t)nr * 18, 0.f);
        for (int r = 0; r < nr; r++) {
            const lbmgrid::Record &R = s->g.recs[r];
            bslot[r] = (int)G.slot(R.i, R.j);
            nsv[r] = R.ns;
            double wr[16], wu[16];
            stencil_weights(R, wr, wu);
            for (int m = 0; m < 16; m++) {
                // unused entries point at the boundary node itself with zero weight
                st_slot[(size_t)r * 16 + m] = m < R.ns ? (int)G.slot(R.si[m], R.sj[m]) : bslot[r];
                st_wr[(size_t)r * 16 + m] = m < R.ns ? (float)wr[m] : 0.f;
                st_wu[(size_t)r * 16 + m] = m < R.ns ? (float)wu[m] : 0.f;
            }
            nx[r] = (float)R.n[0]; ny[r] = (float)R.n[1]; dwb[r] = (float)R.dwb;
            for (int d = 0; d < 9; d++) {
                q[(size_t)r * 9 + d] = (float)R.q[d];
                yc[(size_t)r * 18 + 2 * d] = (float)(1.0 / (1.0 + R.q[d]));
                yc[(size_t)r * 18 + 2 * d + 1] = (float)(R.q[d] / (1.0 + R.q[d]));
            }
            loop[r] = R.loop;
        }
        // per record, the directions q whose node B + c_q is active fluid: its tile is present
        // (through the tile neighbour table, as the level kernel finds it) and the cell is
        // active and not solid
        std::vector<uint32_t> nfluid(nr, 0u);
        {
            static const int CX[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1}, CY[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
            auto dir_of = [](int dx, int dy) {
                for (int d = 0; d < 9; d++)
                    if (CX[d] == dx && CY[d] == dy) return d;
                return 0;
            };
            const std::vector<uint32_t> &fl = s->lv[L - 1].flags;
#pragma omp parallel for schedule(static)
            for (int r = 0; r < nr; r++) {
                const int t = bslot[r] / LBM_TILE, lx = bslot[r] % LBM_TX, ly = (bslot[r] % LBM_TILE) / LBM_TX;
                for (int d = 1; d < 9; d++) {
                    const int ax = lx + CX[d], ay = ly + CY[d];
                    const int sx = ax < 0 ? -1 : (ax >= LBM_TX ? 1 : 0), sy = ay < 0 ? -1 : (ay >= LBM_TY ? 1 : 0);
                    const int tt = (sx == 0 && sy == 0) ? t : G.nbr[(size_t)t * 9 + dir_of(sx, sy)];
                    if (tt < 0) continue;
                    const uint32_t f = fl[(size_t)tt * LBM_TILE + (ay & (LBM_TY - 1)) * LBM_TX + (ax & (LBM_TX - 1))];
                    if ((f & FL_KIND_MASK) == KIND_ACTIVE && !(f & FL_SOLID)) nfluid[r] |= 1u << d;
                }
            }
        }
        RecView &v = s->rec;
        v.n = nr;
        v.bslot = upload(s, bslot, ok);
        v.ns = upload(s, nsv, ok);
        v.st_slot = upload(s, st_slot, ok);
        v.st_wr = upload(s, st_wr, ok);
        v.st_wu = upload(s, st_wu, ok);
        v.nx = upload(s, nx, ok);
        v.ny = upload(s, ny, ok);
        v.dwb = upload(s, dwb, ok);
        v.q = upload(s, q, ok);
        v.loop = upload(s, loop, ok);
        v.nfluid = upload(s, nfluid, ok);
        v.yc = upload(s, yc, ok);
        s->d_slip = (float *)dalloc(s, 2 * (size_t)std::max(n_loops, 1) * sizeof(float));
        v.slip = s->d_slip;
        float **outs[9] = {&v.drhoW, &v.uWx, &v.uWy, &v.utau, &v.chiB, &v.tx, &v.ty, &v.ut, &v.utau_start};
        for (auto o : outs) { *o = (float *)dalloc(s, (size_t)std::max(nr, 1) * sizeof(float)); ok = ok && *o; }
        v.fpost = (float *)dalloc(s, 9 * (size_t)std::max(nr, 1) * sizeof(float));
        s->k.obuf = (float *)dalloc(s, 12 * (size_t)c.ny0 * sizeof(float));
        if (!ok || !s->d_slip || !v.fpost || !s->k.obuf) { free_all(s); return fail(s, LBM_ERR_OOM, "device allocation failed"); }
        if (!s->planning) {
            CK(cudaMemsetAsync(s->d_slip, 0, 2 * (size_t)std::max(n_loops, 1) * sizeof(float), s->stream));
            for (auto o : outs) CK(cudaMemsetAsync(*o, 0, (size_t)std::max(nr, 1) * sizeof(float), s->stream));
        }
    }
    // which prolongations may share a launch with the one of the level above
    for (int l = 0; l < L; l++) {
        bool indep = l >= 1 && l + 1 < L;
        const lbmgrid::Level &G = s->g.lv[l];
        const std::vector<uint32_t> &fl = s->lv[l].flags;
        static const int CX[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1}, CY[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
        // (levels without a parent or a child are never grouped: no scan; each thread's copy
        // of indep starts true and the reduction ands them into the outer value)
        if (indep) {
#pragma omp parallel for schedule(static) reduction(&& : indep)
        for (int t = 0; t < G.ntiles; t++)
            for (int c = 0; indep && c < LBM_TILE; c++) {
                if (!(fl[(size_t)t * LBM_TILE + c] & FL_BAND)) continue;
                const int lx = c % LBM_TX, ly = c / LBM_TX;
                for (int d = 1; d < 9 && indep; d++) {
                    const int ax = lx + CX[d], ay = ly + CY[d];
                    const int sx = ax < 0 ? -1 : (ax >= LBM_TX ? 1 : 0), sy = ay < 0 ? -1 : (ay >= LBM_TY ? 1 : 0);
                    int dd = 0;
                    for (int e = 0; e < 9; e++)
                        if (CX[e] == sx && CY[e] == sy) dd = e;
                    const int tt = dd == 0 ? t : G.nbr[(size_t)t * 9 + dd];
                    if (tt < 0) continue;
                    const uint32_t f = fl[(size_t)tt * LBM_TILE + (ay & (LBM_TY - 1)) * LBM_TX + (ax & (LBM_TX - 1))];
                    if ((f & FL_KIND_MASK) == KIND_GHOST) indep = false;
                }
            }
        }
        s->prolong_indep[l] = indep;
    }
    // surface segments for the loads
    {
        const size_t n = s->g.sa.size();
        std::vector<double> tx(n), ty(n), nxv(n), nyv(n), ds(n);
        for (size_t k2 = 0; k2 < n; k2++) {
            double ax = (double)s->g.v[s->g.sa[k2]].x / 4096.0, ay = (double)s->g.v[s->g.sa[k2]].y / 4096.0;
            double bx = (double)s->g.v[s->g.sb[k2]].x / 4096.0, by = (double)s->g.v[s->g.sb[k2]].y / 4096.0;
            double len = std::sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
            tx[k2] = (bx - ax) / len; ty[k2] = (by - ay) / len; ds[k2] = len;
            bool ccw = s->g.loop_ccw[s->g.sloop[k2]];
            nxv[k2] = ccw ? ty[k2] : -ty[k2];
            nyv[k2] = ccw ? -tx[k2] : tx[k2];
        }
        LoadsView &v = s->segs;
        v.nseg = c.solid_walls ? (int)n : 0;
        v.b1 = upload(s, s->g.seg_b1, ok);
        v.b2 = upload(s, s->g.seg_b2, ok);
        v.w1 = upload(s, s->g.seg_w1, ok);
        v.w2 = upload(s, s->g.seg_w2, ok);
        v.tx = upload(s, tx, ok);
        v.ty = upload(s, ty, ok);
        v.nx = upload(s, nxv, ok);
        v.ny = upload(s, nyv, ok);
        v.ds = upload(s, ds, ok);
        v.cp = (double *)dalloc(s, std::max<size_t>(n, 1) * sizeof(double));
        v.cf = (double *)dalloc(s, std::max<size_t>(n, 1) * sizeof(double));
        if (!ok || !v.cp || !v.cf) { free_all(s); return fail(s, LBM_ERR_OOM, "device allocation failed"); }
    }
    s->d_status = (int *)dalloc(s, 16);
    s->d_acc = (double *)dalloc(s, 8 * sizeof(double));
    if (!s->d_status || !s->d_acc) { free_all(s); return fail(s, LBM_ERR_OOM, "device allocation failed"); }
    if (s->planning) { s->grid_ready = true; return LBM_OK; }
    CK(cudaMemsetAsync(s->d_status, 0, 16, s->stream));
    // constants and initial state: equilibrium of rho = 1, u = (U, 0), chi = chi_inf
    s->k.level0_edges = !c.periodic;
    s->k.nx0 = c.nx0; s->k.ny0 = c.ny0; s->k.ntx0 = s->g.lv[0].ntx;
    s->k.turbulence = c.turbulence; s->k.wall_model = c.wall_model; s->k.sa_convection = c.sa_convection;
    s->k.outlet = c.outlet;
    s->k.U = (float)s->U; s->k.chi_inf = (float)c.chi_inf;
    s->k.d_wr = (float)c.d_wr; s->k.d_wv = (float)c.d_wv;
    {
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
        s->k.sms = sms;
    }
    float g9[9];
    feq_shifted(1.0, s->U, 0.0, g9);
    for (int q = 0; q < 9; q++) s->k.pshift[q] = c.store != 0 ? g9[q] : 0.0f;
    float st9[9];
    for (int q = 0; q < 9; q++) st9[q] = g9[q] - s->k.pshift[q];
    for (int l = 0; l < L; l++) {
        lbmdev::launch_init_feq(s->stream, s->lv[l].v, st9, (float)s->U, (float)c.chi_inf);
        lbmdev::launch_fill9(s->stream, s->lv[l].v.ebuf, s->lv[l].v.n_band, g9);
        lbmdev::launch_fill9(s->stream, s->lv[l].v.gbuf, 4LL * s->lv[l].v.n_band, g9);
    }
    lbmdev::launch_fill9(s->stream, s->rec.fpost, s->rec.n, g9);
    {
        // outlet buffer at rest: [parity][column][direction 2, 6, 8][row]
        std::vector<float> ob(12 * (size_t)c.ny0);
        for (int b = 0; b < 4; b++)
            for (int m = 0; m < 3; m++)
                for (int j = 0; j < c.ny0; j++) ob[((size_t)b * 3 + m) * c.ny0 + j] = g9[m == 0 ? 2 : (m == 1 ? 6 : 8)];
        CK(cudaMemcpyAsync(s->k.obuf, ob.data(), ob.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    for (int l = 0; l < LBM_MAXL; l++) s->parity[l] = 0;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    lbm_status st = capture_graphs(s);
    if (st != LBM_OK) { free_all(s); return st; }
    s->step = 0;
    s->have_cl = false;
    s->n_loops = n_loops;
    s->geometry = true;
    s->grid_ready = true;
    return LBM_OK;
}

lbm_status lbm_plan_geometry(const lbm_config *cfg, const double *xy, const int *loop_offsets, int n_loops,
                             lbm_plan *out)
{
    if (!cfg || !out) return LBM_ERR_INVALID_ARG;
    if (!config_ok(cfg)) return LBM_ERR_INVALID_ARG;
    lbm_solver *s = new (std::nothrow) lbm_solver();
    if (!s) return LBM_ERR_OOM;
    s->cfg = *cfg;
    s->L = cfg->levels;
    s->U = cfg->Ma * std::sqrt(1.0 / 3.0);
    s->planning = true;
    lbm_status st = lbm_set_geometry(s, xy, loop_offsets, n_loops);
    std::memset(out, 0, sizeof *out);
    if (st != LBM_OK) std::snprintf(out->reason, sizeof out->reason, "%s", s->err.c_str());
    if (st == LBM_OK) {
        out->levels = s->L;
        out->device_bytes = s->device_bytes;
        long long nu = 0;
        for (int l = 0; l < s->L; l++) {
            const lbmgrid::Level &G = s->g.lv[l];
            long long act = 0;
#pragma omp parallel for schedule(static) reduction(+ : act)
            for (long b = 0; b < (long)G.kind.size(); b++)
                if (G.kind[b] == KIND_ACTIVE && !G.solid[b]) act++;
            out->cells_active[l] = act;
            nu += act << l;
        }
        out->node_updates_per_step = nu;
        out->wall_records = (long long)s->g.recs.size();
    }
    delete s;
    return st;
}

void lbm_set_host_threads(int n)
{
    static const int process_default = omp_get_max_threads();   // read before the first change
    omp_set_num_threads(n > 0 ? n : process_default);
}

lbm_status lbm_grid_digest(const lbm_config *cfg, const double *xy, const int *loop_offsets, int n_loops,
                           unsigned long long *digest)
{
    if (!digest) return LBM_ERR_INVALID_ARG;
    *digest = 0;
    if (!cfg || !config_ok(cfg) || n_loops < 0 || (n_loops > 0 && (!xy || !loop_offsets))) return LBM_ERR_INVALID_ARG;
    lbmgrid::Grid g;
    std::string msg;
    const int rc = lbmgrid::build(grid_spec(*cfg), xy, loop_offsets, n_loops, g, msg);
    if (rc != 0) return (lbm_status)rc;
    Fnv f;
    for (const lbmgrid::Level &G : g.lv) {
        const int box[15] = {G.l, G.bi0, G.bj0, G.bnx, G.bny, G.pi0, G.pj0, G.pnx, G.pny,
                             G.tx0, G.ty0, G.ntx, G.nty, G.ntiles, G.n_wall_tiles};
        f.bytes(box, sizeof box);
        f.val(G.scale);
        f.vec(G.kind); f.vec(G.solid); f.vec(G.band); f.vec(G.bnode); f.vec(G.coal); f.vec(G.cut);
        f.vec(G.dist); f.vec(G.rec);
        f.vec(G.tile_of); f.vec(G.tile_x); f.vec(G.tile_y); f.vec(G.nbr); f.vec(G.child); f.vec(G.parent);
        f.vec(G.band_tiles); f.vec(G.work_tiles);
    }
    for (const lbmgrid::Record &r : g.recs) {
        f.val(r.i); f.val(r.j); f.val(r.seg); f.val(r.loop);
        f.bytes(r.iw, sizeof r.iw); f.bytes(r.n, sizeof r.n); f.val(r.dwb); f.bytes(r.r, sizeof r.r);
        f.val(r.ns); f.bytes(r.si, sizeof(int) * r.ns); f.bytes(r.sj, sizeof(int) * r.ns); f.bytes(r.q, sizeof r.q);
    }
    f.vec(g.seg_b1); f.vec(g.seg_b2); f.vec(g.seg_w1); f.vec(g.seg_w2); f.val(g.n_cut);
    f.vec(g.sa); f.vec(g.sb); f.vec(g.sloop); f.vec(g.loop_ccw);
    *digest = f.h;
    return LBM_OK;
}

lbm_status lbm_set_wall_slip(lbm_solver *s, const double *uw, int n_loops)
{
    if (!s || !uw) return fail(s, LBM_ERR_INVALID_ARG, "null argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    if (n_loops != s->n_loops) return fail(s, LBM_ERR_INVALID_ARG, "slip count differs from the loop count");
    std::vector<float> h(2 * (size_t)n_loops);
    for (int i = 0; i < 2 * n_loops; i++) h[i] = (float)uw[i];
    CK(cudaMemcpyAsync(s->d_slip, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

lbm_status lbm_step_async(lbm_solver *s, int n)
{
    NvtxRange range("lbm_step_async");
    if (!s) return LBM_ERR_INVALID_ARG;
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    if (s->off_schedule)
        return fail(s, LBM_ERR_INVALID_ARG, "single launches left the level schedule (restore a checkpoint first)");
    if (n < 0) return fail(s, LBM_ERR_INVALID_ARG, "negative step count");
    return enqueue_steps(s, n);
}

lbm_status lbm_synchronize(lbm_solver *s)
{
    if (!s) return LBM_ERR_INVALID_ARG;
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    lbm_status st = enqueue_mass(s);
    if (st != LBM_OK) return st;
    CK(cudaGetLastError());
    return check_status(s);
}

lbm_status lbm_step_launch(lbm_solver *s, int level, int kind)
{
    if (!s) return LBM_ERR_INVALID_ARG;
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    if (level < 0 || level >= s->L || kind < 0 || kind > 2 || (kind == 2 && level == s->L - 1))
        return fail(s, LBM_ERR_INVALID_ARG, "bad level or launch kind");
    const int L = s->L, l = level;
    LevelView &P = s->lv[l].v;
    if (kind == 2) {
        lbmdev::launch_prolong(s->stream, P, s->lv[l + 1].v, s->parity[l], 0);
    } else {
        const LevelView *F = (l < L - 1) ? &s->lv[l + 1].v : nullptr;
        const LevelView *C = (l > 0) ? &s->lv[l - 1].v : nullptr;
        lbmdev::LevelStep ls{};
        ls.p = s->parity[l];
        ls.has_child = F != nullptr;
        ls.is_level0 = l == 0;
        ls.wall = (l == L - 1) && s->rec.n > 0;
        ls.restrict_up = kind == 1 && C != nullptr;
        ls.pp = C ? s->parity[l - 1] : 0;
        ls.shape = s->shape[l];
        ls.status = s->d_status;
        const lbmdev::LevelTune tu{s->min_blocks[l], 0, s->sched[l], s->shape[l]};
        lbmdev::launch_level(s->stream, P, F, C, s->rec, s->k, ls, tu);
        s->parity[l] ^= 1;
    }
    s->off_schedule = true;
    CK(cudaGetLastError());
    return check_status(s);
}

lbm_status lbm_get_ghost_relay(lbm_solver *s, int level, int *ij, double *vals, int cap, int *n)
{
    if (!s || !n) return fail(s, LBM_ERR_INVALID_ARG, "null argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    if (level < 0 || level >= s->L - 1) return fail(s, LBM_ERR_INVALID_ARG, "level has no finer level");
    const LevelView &v = s->lv[level].v;
    *n = v.n_band;
    if (!ij) return LBM_OK;
    if (v.n_band > cap || !vals) return fail(s, LBM_ERR_INVALID_ARG, "capacity too small");
    std::vector<float> h(36 * (size_t)v.n_band);
    if (!h.empty()) {
        CK(cudaMemcpyAsync(h.data(), v.gbuf, h.size() * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    for (int b = 0; b < v.n_band; b++) {
        ij[2 * b] = s->lv[level].band_ij[2 * (size_t)b];
        ij[2 * b + 1] = s->lv[level].band_ij[2 * (size_t)b + 1];
        for (int m = 0; m < 36; m++) vals[36 * (size_t)b + m] = (double)h[36 * (size_t)b + m] + WQh[m % 9];
    }
    return LBM_OK;
}

lbm_status lbm_step(lbm_solver *s, int n)
{
    NvtxRange range("lbm_step");
    lbm_status st = lbm_step_async(s, n);
    if (st != LBM_OK) return st;
    return lbm_synchronize(s);
}

lbm_status lbm_get_level_box(lbm_solver *s, int level, int *i0, int *j0, int *nx, int *ny)
{
    if (!s || !i0 || !j0 || !nx || !ny) return fail(s, LBM_ERR_INVALID_ARG, "null argument");
    if (!s->grid_ready) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    if (level < 0 || level >= s->L) return fail(s, LBM_ERR_INVALID_ARG, "level out of range");
    const lbmgrid::Level &G = s->g.lv[level];
    *i0 = G.pi0; *j0 = G.pj0; *nx = G.pnx; *ny = G.pny;
    return LBM_OK;
}

static lbm_status download_level(lbm_solver *s, int l, std::vector<float> &dr, std::vector<float> &ux,
                                 std::vector<float> &uy, std::vector<float> &chi)
{
    const LevelView &v = s->lv[l].v;
    const int p = s->parity[l];
    const size_t nb = (size_t)v.ns * sizeof(float);
    dr.resize(v.ns); ux.resize(v.ns); uy.resize(v.ns); chi.resize(v.ns);
    CK(cudaMemcpyAsync(dr.data(), v.drho[p], nb, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(ux.data(), v.ux[p], nb, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(uy.data(), v.uy[p], nb, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(chi.data(), v.chi[p], nb, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

// mask code of a cell from the host copy of the grid (solid-only tiles have no slots)
static unsigned char mask_of(const lbmgrid::Level &G, long b)
{
    if (b < 0 || G.kind[b] == KIND_ABSENT) return 0;
    if (G.solid[b]) return 5;
    if (G.kind[b] == KIND_COVERED) return 3;
    if (G.kind[b] == KIND_GHOST) return 4;
    return G.bnode[b] ? 2 : 1;
}

lbm_status lbm_get_fields(lbm_solver *s, int level, double *rho, double *ux, double *uy, double *chi,
                          unsigned char *mask, int cap)
{
    int i0, j0, nx, ny;
    lbm_status st = lbm_get_level_box(s, level, &i0, &j0, &nx, &ny);
    if (st != LBM_OK) return st;
    if ((long long)nx * ny > cap) return fail(s, LBM_ERR_INVALID_ARG, "capacity too small");
    const bool fields = rho || ux || uy || chi;
    if (fields && !s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no device state (host-only handle): only the mask");
    std::vector<float> dr, u, v, c2;
    if (fields) {
        st = download_level(s, level, dr, u, v, c2);
        if (st != LBM_OK) return st;
    }
    const lbmgrid::Level &G = s->g.lv[level];
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long sl = G.slot(i0 + i, j0 + j);
            long long o = (long long)j * nx + i;
            unsigned char m = mask_of(G, G.idx(i0 + i, j0 + j));
            if (mask) mask[o] = m;
            bool has = m >= 1 && m <= 4 && sl >= 0;
            if (rho) rho[o] = has ? 1.0 + (double)dr[sl] : NAN;
            if (ux) ux[o] = has ? (double)u[sl] : NAN;
            if (uy) uy[o] = has ? (double)v[sl] : NAN;
            if (chi) chi[o] = has ? (double)c2[sl] : NAN;
        }
    return LBM_OK;
}

// logical post-collision populations f - w of a level's cells, [q * ns + slot] on the host
static lbm_status gather_post(lbm_solver *s, int l, std::vector<float> &out)
{
    const LevelView &v = s->lv[l].v;
    const size_t n = 9 * (size_t)v.ns;
    float *d = (float *)tmp_alloc(s, n * sizeof(float));
    if (!d) return fail(s, LBM_ERR_OOM, "device allocation failed (query scratch)");
    lbmdev::launch_gather_post(s->stream, v, l > 0 ? &s->lv[l - 1].v : nullptr, s->rec, s->k, s->parity[l], l == 0, d);
    out.resize(n);
    cudaError_t e = cudaMemcpyAsync(out.data(), d, n * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    tmp_free(s, d);
    if (e != cudaSuccess) return cuda_fail(s, e, "gather_post");
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_solver *s, int level, double *pop, long long cap)
{
    if (s && !s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    int i0, j0, nx, ny;
    lbm_status st = lbm_get_level_box(s, level, &i0, &j0, &nx, &ny);
    if (st != LBM_OK) return st;
    const long long ncell = (long long)nx * ny;
    if (!pop || 9 * ncell > cap) return fail(s, LBM_ERR_INVALID_ARG, "capacity too small");
    const LevelView &v = s->lv[level].v;
    std::vector<float> f;
    if ((st = gather_post(s, level, f)) != LBM_OK) return st;
    const lbmgrid::Level &G = s->g.lv[level];
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const long b = G.idx(i0 + i, j0 + j);
            const long sl = G.slot(i0 + i, j0 + j);
            const unsigned char m = mask_of(G, b);
            const bool has = sl >= 0 && (m == 1 || m == 2 || m == 4);
            for (int q = 0; q < 9; q++)
                pop[q * ncell + (long long)j * nx + i] = has ? (double)f[(size_t)q * v.ns + sl] + WQh[q] : NAN;
        }
    return LBM_OK;
}

lbm_status lbm_get_flags(lbm_solver *s, int level, unsigned int *flags, int cap)
{
    int i0, j0, nx, ny;
    lbm_status st = lbm_get_level_box(s, level, &i0, &j0, &nx, &ny);
    if (st != LBM_OK) return st;
    if (!flags || (long long)nx * ny > cap) return fail(s, LBM_ERR_INVALID_ARG, "capacity too small");
    const lbmgrid::Level &G = s->g.lv[level];
    const std::vector<uint32_t> &fl = s->lv[level].flags;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const long sl = G.slot(i0 + i, j0 + j);
            flags[(long long)j * nx + i] = sl >= 0 ? fl[sl] : 0u;
        }
    return LBM_OK;
}

lbm_status lbm_get_prolong_independence(lbm_solver *s, int *indep, int cap)
{
    if (!s || !indep || cap < s->L) return fail(s, LBM_ERR_INVALID_ARG, "bad argument");
    if (!s->grid_ready) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    for (int l = 0; l < s->L; l++) indep[l] = s->prolong_indep[l] ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_get_work_list(lbm_solver *s, int level, int warps, int *out, int cap, int *n)
{
    if (!s || !n || (warps != 0 && warps != 1) || (cap > 0 && !out)) return fail(s, LBM_ERR_INVALID_ARG, "bad argument");
    if (!s->grid_ready) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    if (level < 0 || level >= s->L) return fail(s, LBM_ERR_INVALID_ARG, "level out of range");
    const lbmgrid::Level &G = s->g.lv[level];
    const std::vector<int> &w = warps ? s->lv[level].work_warps : s->lv[level].work_tiles;
    *n = (int)w.size();
    if (cap <= 0) return LBM_OK;
    if ((int)w.size() > cap) return fail(s, LBM_ERR_INVALID_ARG, "capacity too small");
    for (size_t k = 0; k < w.size(); k++) {
        const int t = warps ? w[k] >> 3 : w[k];
        out[3 * k] = G.tile_x[t] * LBM_TX;
        out[3 * k + 1] = G.tile_y[t] * LBM_TY;
        out[3 * k + 2] = warps ? (w[k] & 7) : -1;
    }
    return LBM_OK;
}

lbm_status lbm_get_wall_distance(lbm_solver *s, int level, double *d, int cap)
{
    int i0, j0, nx, ny;
    lbm_status st = lbm_get_level_box(s, level, &i0, &j0, &nx, &ny);
    if (st != LBM_OK) return st;
    if (!d || (long long)nx * ny > cap) return fail(s, LBM_ERR_INVALID_ARG, "capacity too small");
    const lbmgrid::Level &G = s->g.lv[level];
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long b = G.idx(i0 + i, j0 + j);
            bool act = b >= 0 && G.kind[b] == KIND_ACTIVE && !G.solid[b];
            d[(long long)j * nx + i] = act ? (double)G.dist[b] : NAN;
        }
    return LBM_OK;
}

lbm_status lbm_set_fields(lbm_solver *s, int level, const double *rho, const double *ux, const double *uy,
                          const double *chi)
{
    if (s && !s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    int i0, j0, nx, ny;
    lbm_status st = lbm_get_level_box(s, level, &i0, &j0, &nx, &ny);
    if (st != LBM_OK) return st;
    const LevelView &v = s->lv[level].v;
    const int p = s->parity[level];
    std::vector<float> dr, u, w, c2, c3(v.ns), post;
    st = download_level(s, level, dr, u, w, c2);
    if (st != LBM_OK) return st;
    CK(cudaMemcpyAsync(c3.data(), v.chi[p ^ 1], v.ns * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    if ((st = gather_post(s, level, post)) != LBM_OK) return st;
    const lbmgrid::Level &G = s->g.lv[level];
    const std::vector<uint32_t> &fl = s->lv[level].flags;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long sl = G.slot(i0 + i, j0 + j);
            if (sl < 0) continue;
            uint32_t fw = fl[sl];
            if ((fw & FL_KIND_MASK) != KIND_ACTIVE || (fw & FL_SOLID)) continue;
            long long o = (long long)j * nx + i;
            double r = rho ? rho[o] : 1.0 + (double)dr[sl];
            double a = ux ? ux[o] : (double)u[sl];
            double b = uy ? uy[o] : (double)w[sl];
            dr[sl] = (float)(r - 1.0); u[sl] = (float)a; w[sl] = (float)b;
            if (chi) { c2[sl] = (float)chi[o]; c3[sl] = (float)chi[o]; }
            float g9[9];
            feq_shifted(r, a, b, g9);
            for (int q = 0; q < 9; q++) post[(size_t)q * v.ns + sl] = g9[q];
        }
    CK(cudaMemcpyAsync(v.drho[p], dr.data(), v.ns * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(v.ux[p], u.data(), v.ns * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(v.uy[p], w.data(), v.ns * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(v.chi[p], c2.data(), v.ns * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(v.chi[p ^ 1], c3.data(), v.ns * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    size_t ns_max = 0;
    for (int l = 0; l < s->L; l++) ns_max = std::max(ns_max, (size_t)s->lv[l].v.ns);
    float *d = (float *)tmp_alloc(s, 9 * ns_max * sizeof(float));
    if (!d) return fail(s, LBM_ERR_OOM, "device allocation failed (set_fields scratch)");
    cudaError_t e = cudaMemcpyAsync(d, post.data(), post.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) {
        lbmdev::launch_store_post(s->stream, v, s->rec, s->k, p, level == 0, d);
        // re-synchronise the interfaces: restriction bottom-up, then explosion and ghost
        // reconstruction top-down
        for (int l = s->L - 2; l >= 0; l--)
            lbmdev::launch_restrict(s->stream, s->lv[l].v, s->lv[l + 1].v, s->parity[l], s->parity[l + 1]);
        for (int l = 0; l < s->L - 1; l++) {
            lbmdev::launch_gather_post(s->stream, s->lv[l].v, l > 0 ? &s->lv[l - 1].v : nullptr, s->rec, s->k, s->parity[l],
                                       l == 0, d);
            lbmdev::launch_explode(s->stream, s->lv[l].v, s->lv[l + 1].v, s->rec, s->k, d);
            lbmdev::launch_prolong(s->stream, s->lv[l].v, s->lv[l + 1].v, s->parity[l], 0);
        }
        e = cudaGetLastError();
    }
    tmp_free(s, d);
    if (e != cudaSuccess) return cuda_fail(s, e, "set_fields");
    CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

lbm_status lbm_get_loads(lbm_solver *s, lbm_loads *out, double *cp_seg, double *cf_seg, int cap, int *n_seg)
{
    NvtxRange range("lbm_get_loads");
    if (!s || !out) return fail(s, LBM_ERR_INVALID_ARG, "null argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    const int nseg = s->segs.nseg;
    if (n_seg) *n_seg = nseg;
    lbmdev::launch_wallfn(s->stream, s->lv[s->L - 1].v, s->parity[s->L - 1], s->rec, s->k);
    CK(cudaMemsetAsync(s->d_acc, 0, 4 * sizeof(double), s->stream));
    lbmdev::launch_loads(s->stream, s->segs, s->rec, (float)s->U, s->d_acc);
    lbm_status st = enqueue_mass(s);
    if (st != LBM_OK) return st;
    double acc[5];
    CK(cudaMemcpyAsync(acc, s->d_acc, 5 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    if (cp_seg && cap > 0) CK(cudaMemcpyAsync(cp_seg, s->segs.cp, std::min(cap, nseg) * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    if (cf_seg && cap > 0) CK(cudaMemcpyAsync(cf_seg, s->segs.cf, std::min(cap, nseg) * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaGetLastError());
    st = check_status(s);
    if (st != LBM_OK) return st;
    const double chord = s->cfg.chord / (s->cfg.h0 / (double)(1LL << (s->L - 1)));
    out->CDf = acc[0] / chord;
    out->CDp = acc[2] / chord;
    out->CD = out->CDf + out->CDp;
    out->CL = acc[3] / chord;
    out->mass = acc[4];
    out->dCL = s->have_cl ? out->CL - s->last_cl : 0.0;
    s->last_cl = out->CL;
    s->have_cl = true;
    out->step = s->step;
    return LBM_OK;
}

lbm_status lbm_get_cut_links(lbm_solver *s, int *ijd, double *q, int cap, int *n)
{
    if (!s || !n) return fail(s, LBM_ERR_INVALID_ARG, "null argument");
    if (!s->grid_ready) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    const lbmgrid::Level &G = s->g.lv[s->L - 1];
    int cnt = 0;
    for (const auto &R : s->g.recs) {
        uint16_t m = G.cut[G.idx(R.i, R.j)];
        for (int d = 1; d < 9; d++) {
            if (!(m >> d & 1)) continue;
            if (ijd && q && cnt < cap) { ijd[3 * cnt] = R.i; ijd[3 * cnt + 1] = R.j; ijd[3 * cnt + 2] = d; q[cnt] = R.q[d]; }
            cnt++;
        }
    }
    *n = cnt;
    return (ijd && cnt > cap) ? fail(s, LBM_ERR_INVALID_ARG, "capacity too small") : LBM_OK;
}

lbm_status lbm_get_wall_records(lbm_solver *s, int *ij, double *geo, int *nst, int cap, int *n)
{
    if (!s || !n) return fail(s, LBM_ERR_INVALID_ARG, "null argument");
    if (!s->grid_ready) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    const int nr = (int)s->g.recs.size();
    *n = nr;
    if (!ij) return LBM_OK;
    if (nr > cap || !geo || !nst) return fail(s, LBM_ERR_INVALID_ARG, "capacity too small");
    for (int r = 0; r < nr; r++) {
        const lbmgrid::Record &R = s->g.recs[r];
        ij[2 * r] = R.i; ij[2 * r + 1] = R.j;
        double *gg = geo + 9 * r;
        gg[0] = R.iw[0]; gg[1] = R.iw[1]; gg[2] = R.n[0]; gg[3] = R.n[1]; gg[4] = R.dwb;
        gg[5] = R.r[0]; gg[6] = R.r[1]; gg[7] = R.loop; gg[8] = R.seg;
        nst[r] = R.ns;
    }
    return LBM_OK;
}

lbm_status lbm_get_wall_stencils(lbm_solver *s, int *sij, double *wr, double *wu, int cap, int *n)
{
    if (!s || !n) return fail(s, LBM_ERR_INVALID_ARG, "null argument");
    if (!s->grid_ready) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    const int nr = (int)s->g.recs.size();
    *n = nr;
    if (!sij) return LBM_OK;
    if (nr > cap || !wr || !wu) return fail(s, LBM_ERR_INVALID_ARG, "capacity too small");
    for (int r = 0; r < nr; r++) {
        const lbmgrid::Record &R = s->g.recs[r];
        double a[16], b[16];
        stencil_weights(R, a, b);
        for (int m = 0; m < 16; m++) {
            const bool in = m < R.ns;
            sij[32 * r + 2 * m] = in ? R.si[m] : -1;
            sij[32 * r + 2 * m + 1] = in ? R.sj[m] : -1;
            wr[16 * r + m] = in ? a[m] : 0.0;
            wu[16 * r + m] = in ? b[m] : 0.0;
        }
    }
    return LBM_OK;
}

lbm_status lbm_get_segment_map(lbm_solver *s, double *mid, int *b12, double *w12, int cap, int *n)
{
    if (!s || !n) return fail(s, LBM_ERR_INVALID_ARG, "null argument");
    if (!s->grid_ready) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    const int ns = (int)s->g.sa.size();
    *n = ns;
    if (!b12) return LBM_OK;
    if (ns > cap || !mid || !w12) return fail(s, LBM_ERR_INVALID_ARG, "capacity too small");
    for (int k = 0; k < ns; k++) {
        const lbmgrid::IPt a = s->g.v[s->g.sa[k]], b = s->g.v[s->g.sb[k]];
        mid[2 * k] = 0.5 * (double)(a.x + b.x) / 4096.0;
        mid[2 * k + 1] = 0.5 * (double)(a.y + b.y) / 4096.0;
        b12[2 * k] = s->g.seg_b1[k]; b12[2 * k + 1] = s->g.seg_b2[k];
        w12[2 * k] = s->g.seg_w1[k]; w12[2 * k + 1] = s->g.seg_w2[k];
    }
    return LBM_OK;
}

lbm_status lbm_get_wall_state(lbm_solver *s, double *st8, int cap, int *n)
{
    if (!s || !n) return fail(s, LBM_ERR_INVALID_ARG, "null argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    const int nr = s->rec.n;
    *n = nr;
    if (!st8) return LBM_OK;
    if (nr > cap) return fail(s, LBM_ERR_INVALID_ARG, "capacity too small");
    if (nr == 0) return LBM_OK;
    lbmdev::launch_wallfn(s->stream, s->lv[s->L - 1].v, s->parity[s->L - 1], s->rec, s->k);
    std::vector<float> a[8];
    float *src[8] = {s->rec.drhoW, s->rec.uWx, s->rec.uWy, s->rec.utau, s->rec.chiB, s->rec.tx, s->rec.ty, s->rec.ut};
    for (int m = 0; m < 8; m++) {
        a[m].resize(nr);
        CK(cudaMemcpyAsync(a[m].data(), src[m], nr * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    }
    CK(cudaStreamSynchronize(s->stream));
    for (int r = 0; r < nr; r++) {
        st8[8 * r] = 1.0 + (double)a[0][r];
        for (int m = 1; m < 8; m++) st8[8 * r + m] = a[m][r];
    }
    return LBM_OK;
}

lbm_status lbm_get_info(lbm_solver *s, lbm_info *out)
{
    if (!s || !out) return fail(s, LBM_ERR_INVALID_ARG, "null argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    std::memset(out, 0, sizeof *out);
    out->levels = s->L;
    long long nu = 0;
    for (int l = 0; l < s->L; l++) {
        const lbmgrid::Level &G = s->g.lv[l];
        long long act = 0, pres = 0;
        for (size_t b = 0; b < G.kind.size(); b++) {
            if (G.kind[b] != KIND_ABSENT) pres++;
            if (G.kind[b] == KIND_ACTIVE && !G.solid[b]) act++;
        }
        out->cells_active[l] = act;
        out->cells_present[l] = pres;
        out->slots[l] = (long long)G.ntiles * LBM_TILE;
        out->work_tiles[l] = s->lv[l].v.n_work_tiles;
        out->work_warps[l] = s->lv[l].v.n_work_warps;
        nu += act << l;
    }
    out->node_updates_per_step = nu;
    out->wall_records = (long long)s->g.recs.size();
    out->cut_links = s->g.n_cut;
    out->surface_segments = s->segs.nseg;
    out->kernels_per_step = s->kernels_per_step;
    // fused level step, per node update: 9 populations read and 9 written, the flag word and
    // chi read, rho - 1 and u written; with SA-neg also chi written, u read for the stencil
    // (its neighbours' values come through the caches) and 1/d^2 read
    out->bytes_per_node_update = 18.0 * (double)pop_bytes(s->cfg.store) + 12.0 + 4.0 + 4.0 +
                                 (s->cfg.turbulence ? 4.0 + 8.0 + 4.0 : 0.0);
    out->device_bytes = s->device_bytes;
    return LBM_OK;
}

lbm_status lbm_time_kernels(lbm_solver *s, int n, lbm_kernel_times *out)
{
    NvtxRange range("lbm_time_kernels");
    if (!s || !out || n < 0) return fail(s, LBM_ERR_INVALID_ARG, "bad argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    std::memset(out, 0, sizeof *out);
    out->n_classes = KC_N;
    for (int c2 = 0; c2 < KC_N; c2++) std::snprintf(out->name[c2], 32, "%s", KC_NAME[c2]);
    for (int it = 0; it < n; it++) {
        s->timing = true;
        s->ev_used = 0;
        s->ev_marks.clear();
        s->ev_cells.clear();
        s->ev_level.clear();
        long long nk = 0;
        advance(s, s->stream, 0, 0, nk);
        s->timing = false;
        s->step++;
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s->stream));
        for (size_t m = 0; m < s->ev_marks.size(); m++) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, s->ev_pool[s->ev_marks[m].second], s->ev_pool[s->ev_marks[m].second + 1]));
            int cls = s->ev_marks[m].first;
            out->total_ms[cls] += ms;
            out->launches[cls]++;
            out->cells[cls] += s->ev_cells[m];
        }
    }
    return check_status(s);
}

// mean per-launch time (us) of each level's fused kernel over n eager coarse steps
static lbm_status level_launch_times(lbm_solver *s, int n, double *us)
{
    double tot[LBM_MAXL] = {0};
    long long cnt[LBM_MAXL] = {0};
    for (int it = 0; it < n; it++) {
        s->timing = true;
        s->ev_used = 0;
        s->ev_marks.clear();
        s->ev_cells.clear();
        s->ev_level.clear();
        long long nk = 0;
        advance(s, s->stream, 0, 0, nk);
        s->timing = false;
        s->step++;
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s->stream));
        for (size_t m = 0; m < s->ev_marks.size(); m++) {
            const int cls = s->ev_marks[m].first;
            if (cls != KC_LEVEL_FINEST && cls != KC_LEVEL_COARSE) continue;
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, s->ev_pool[s->ev_marks[m].second], s->ev_pool[s->ev_marks[m].second + 1]));
            tot[s->ev_level[m]] += 1e3 * ms;
            cnt[s->ev_level[m]]++;
        }
    }
    for (int l = 0; l < s->L; l++) us[l] = cnt[l] ? tot[l] / (double)cnt[l] : 0.0;
    return LBM_OK;
}

// mean time (us) of one coarse step through the captured graphs, over n steps
static lbm_status graph_step_time(lbm_solver *s, int n, double *us)
{
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return fail(s, LBM_ERR_CUDA, "cudaEventCreate"); }
    cudaEventRecord(a, s->stream);
    lbm_status st = enqueue_steps(s, n);
    cudaEventRecord(b, s->stream);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != LBM_OK) return st;
    if (e != cudaSuccess) return cuda_fail(s, e, "graph step timing");
    *us = 1e3 * ms / (double)n;
    return LBM_OK;
}

static int no_persist(int sched) { return sched == LBM_SCHED_PERSIST ? LBM_SCHED_TILE : sched; }

lbm_status lbm_autotune(lbm_solver *s, int steps, lbm_tune_report *out)
{
    NvtxRange range("lbm_autotune");
    if (!s || !out || steps < 1) return fail(s, LBM_ERR_INVALID_ARG, "bad argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    static const int CAND_MB[LBM_TUNE_CANDIDATES] = {5, 6, 5, 6, 5, 6, 5, 6, 5, 6, 5, 6};
    static const int CAND_PE[LBM_TUNE_CANDIDATES] = {0, 0, 1, 1, 0, 0, 1, 1, 2, 2, 3, 3};
    static const int CAND_SH[LBM_TUNE_CANDIDATES] = {0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0};
    std::memset(out, 0, sizeof *out);
    const int L = s->L;
    out->levels = L;
    lbm_status st;
    if ((st = graph_step_time(s, steps, &out->default_step_us)) != LBM_OK) return st;
    int keep_mb[LBM_MAXL], keep_pe[LBM_MAXL], keep_sh[LBM_MAXL];
    for (int l = 0; l < L; l++) { keep_mb[l] = s->min_blocks[l]; keep_pe[l] = s->sched[l]; keep_sh[l] = s->shape[l]; }
    // 1: register budget and grid schedule per level, from per-launch event timings of
    //    every candidate
    for (int c = 0; c < LBM_TUNE_CANDIDATES; c++) {
        for (int l = 0; l < L; l++) { s->min_blocks[l] = CAND_MB[c]; s->sched[l] = CAND_PE[c]; s->shape[l] = CAND_SH[c]; }
        out->candidate_min_blocks[c] = CAND_MB[c];
        out->candidate_sched[c] = CAND_PE[c];
        out->candidate_shape[c] = CAND_SH[c];
        if ((st = level_launch_times(s, steps, out->level_us[c])) != LBM_OK) {
            for (int l = 0; l < L; l++) { s->min_blocks[l] = keep_mb[l]; s->sched[l] = keep_pe[l]; s->shape[l] = keep_sh[l]; }
            return st;
        }
    }
    for (int l = 0; l < L; l++) {
        int best = 0;
        for (int c = 1; c < LBM_TUNE_CANDIDATES; c++)
            if (out->level_us[c][l] < out->level_us[best][l]) best = c;
        s->min_blocks[l] = CAND_MB[best];
        s->sched[l] = CAND_PE[best];
        s->shape[l] = CAND_SH[best];
        out->min_blocks[l] = CAND_MB[best];
        out->sched[l] = CAND_PE[best];
        out->shape[l] = CAND_SH[best];
    }
    // 1b: per-launch timings miss how launches overlap inside the graph (a persistent grid
    //     occupies every SM while the next launch would start): keep the per-level choice
    //     only if whole graph steps confirm it, against the same choice with one block per
    //     tile where it took a persistent grid, against the default form, and against each
    //     candidate on every level
    {
        int pick_mb[LBM_MAXL], pick_pe[LBM_MAXL], pick_sh[LBM_MAXL];
        for (int l = 0; l < L; l++) { pick_mb[l] = s->min_blocks[l]; pick_pe[l] = s->sched[l]; pick_sh[l] = s->shape[l]; }
        auto form = [&](int v, int l, int &mb, int &pe, int &sh) {
            if (v >= 3) { mb = CAND_MB[v - 3]; pe = CAND_PE[v - 3]; sh = CAND_SH[v - 3]; return; }
            mb = v == 2 ? keep_mb[l] : pick_mb[l];
            pe = v == 0 ? pick_pe[l] : (v == 1 ? no_persist(pick_pe[l]) : keep_pe[l]);
            sh = v == 2 ? keep_sh[l] : pick_sh[l];
        };
        double best_us = 0.0;
        int best = 0;
        for (int v = 0; v < 3 + LBM_TUNE_CANDIDATES; v++) {
            for (int l = 0; l < L; l++) form(v, l, s->min_blocks[l], s->sched[l], s->shape[l]);
            double us = 0.0;
            if ((st = capture_graphs(s)) != LBM_OK) return st;
            if ((st = graph_step_time(s, steps, &us)) != LBM_OK) return st;
            out->step_us_confirm[v] = us;
            if (v == 0 || us < best_us) { best_us = us; best = v; }
        }
        for (int l = 0; l < L; l++) {
            form(best, l, s->min_blocks[l], s->sched[l], s->shape[l]);
            out->min_blocks[l] = s->min_blocks[l];
            out->sched[l] = s->sched[l];
            out->shape[l] = s->shape[l];
        }
        out->confirm_choice = best;
    }
    // 2: programmatic dependent launch on or off, from whole graph steps
    for (int pdl = 0; pdl < 2; pdl++) {
        s->pdl = pdl;
        if ((st = capture_graphs(s)) != LBM_OK) return st;
        if ((st = graph_step_time(s, steps, &out->step_us[pdl])) != LBM_OK) return st;
    }
    s->pdl = out->step_us[1] <= out->step_us[0] ? 1 : 0;
    out->pdl = s->pdl;
    if ((st = capture_graphs(s)) != LBM_OK) return st;
    out->steps_taken = (long long)steps * (6 + 2 * LBM_TUNE_CANDIDATES);
    return check_status(s);
}

// ---------------------------------------------------------------- batched solves
// One batch steps several resident solves in lockstep: every node of the recursive level
// schedule (Sec 2.1) is one launch over all member solves that have that level.  Level l
// takes 2^l sub-steps per coarse step in every solve, so the recursion of the deepest member
// drives all of them; a member without level l has no blocks in that node's launch.
struct lbm_batch {
    std::vector<lbm_solver *> m;
    std::vector<int> parity0;          // each member's level-0 parity the next graph expects
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int phase = 0;
    int Lmax = 0, store = 0;
    cudaEvent_t done = nullptr;
    std::vector<cudaEvent_t> ready;
    long long kernels_per_step = 0;
    std::string err;
};

static lbm_status bfail(lbm_batch *b, lbm_status code, const std::string &msg)
{
    if (b) b->err = msg;
    return code;
}

static void batch_advance(lbm_batch *b, cudaStream_t st, int l, int restrict_up, long long &nk)
{
    // prolongation of level l into the ghosts of l + 1, for the members that have l + 1
    {
        lbmdev::ProlongBatchArgs a;
        a.n = 0;
        a.tl = nullptr;
        a.tl_base = 0;
        unsigned grid = 0;
        for (lbm_solver *s : b->m) {
            if (l + 1 >= s->L || s->lv[l].v.n_band_tiles <= 0) continue;
            lbmdev::ProlongDesc &d = a.d[a.n++];
            d.P = s->lv[l].v; d.F = s->lv[l + 1].v; d.p = s->parity[l]; d.first_block = (int)grid;
            grid += (unsigned)s->lv[l].v.n_band_tiles;
        }
        if (grid) { lbmdev::launch_prolong_batch(st, a, grid, 1); nk++; }
    }
    if (l + 1 < b->Lmax) {
        batch_advance(b, st, l + 1, 0, nk);
        batch_advance(b, st, l + 1, 1, nk);
    }
    lbmdev::BatchArgs a;
    a.n = 0;
    unsigned grid = 0;
    for (lbm_solver *s : b->m) {
        if (l >= s->L) continue;
        const int L = s->L;
        lbmdev::SolveDesc &d = a.d[a.n++];
        d.P = s->lv[l].v;
        d.F = l + 1 < L ? s->lv[l + 1].v : d.P;
        d.C = l > 0 ? s->lv[l - 1].v : d.P;
        d.R = s->rec;
        d.k = s->k;
        d.ls.p = s->parity[l];
        d.ls.has_child = l + 1 < L;
        d.ls.is_level0 = l == 0;
        d.ls.wall = (l == L - 1) && s->rec.n > 0;
        d.ls.restrict_up = restrict_up && l > 0;
        d.ls.pp = l > 0 ? s->parity[l - 1] : 0;
        d.ls.shape = 0;
        d.ls.status = s->d_status;
        d.ls.tl = nullptr;
        d.ls.tl_base = 0;
        d.kind = d.ls.wall ? 2 : (d.ls.has_child ? 1 : 0);
        d.first_block = (int)grid;
        grid += (unsigned)std::max(d.P.n_work_tiles, 0);
        s->parity[l] ^= 1;
    }
    if (grid) { lbmdev::launch_level_batch(st, a, b->store, grid, 1); nk++; }
}

static lbm_status batch_capture(lbm_batch *b)
{
    for (int g = 0; g < 2; g++) {
        cudaGraph_t gr;
        long long nk = 0;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return bfail(b, LBM_ERR_CUDA, "batch capture begin");
        batch_advance(b, b->stream, 0, 0, nk);
        if (cudaStreamEndCapture(b->stream, &gr) != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "batch capture end");
        const cudaError_t e = cudaGraphInstantiate(&b->graph[g], gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
        b->kernels_per_step = nk;
    }
    // the two captures advanced every member's parities by two coarse steps: as they were
    return LBM_OK;
}

extern "C" {

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (int g = 0; g < 2; g++)
        if (b->graph[g]) cudaGraphExecDestroy(b->graph[g]);
    for (cudaEvent_t e : b->ready) cudaEventDestroy(e);
    if (b->done) cudaEventDestroy(b->done);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

lbm_status lbm_batch_create(lbm_solver *const *solvers, int n, lbm_batch **out)
{
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    static_assert(LBM_BATCH_MAX == LBM_BATCH_MAX_SOLVES, "batch sizes of the ABI and the kernels");
    if (!solvers || n < 1 || n > LBM_BATCH_MAX) return LBM_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
    for (int i = 0; i < n; i++) {
        const lbm_solver *s = solvers[i];
        if (!s || !s->geometry || s->off_schedule || s->device != dev || s->cfg.store != solvers[0]->cfg.store)
            return LBM_ERR_INVALID_ARG;
        for (int j = 0; j < i; j++)
            if (solvers[j] == s) return LBM_ERR_INVALID_ARG;
    }
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    b->m.assign(solvers, solvers + n);
    b->store = solvers[0]->cfg.store;
    for (lbm_solver *s : b->m) {
        b->Lmax = std::max(b->Lmax, s->L);
        b->parity0.push_back(s->parity[0]);
    }
    bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < n; i++) {
        cudaEvent_t e;
        ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (ok) b->ready.push_back(e);
    }
    if (!ok) { lbm_batch_destroy(b); return LBM_ERR_CUDA; }
    if (batch_capture(b) != LBM_OK) { lbm_batch_destroy(b); return LBM_ERR_CUDA; }
    *out = b;
    return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->err.c_str() : "null handle"; }

lbm_status lbm_batch_step(lbm_batch *b, int n)
{
    if (!b || n < 0) return bfail(b, LBM_ERR_INVALID_ARG, "bad argument");
    for (size_t i = 0; i < b->m.size(); i++)
        if (b->m[i]->off_schedule || b->m[i]->parity[0] != (b->parity0[i] ^ b->phase))
            return bfail(b, LBM_ERR_INVALID_ARG, "a member stepped outside the batch (create a new batch)");
    // the batch stream follows everything enqueued on the members' own streams ...
    for (size_t i = 0; i < b->m.size(); i++) {
        if (cudaEventRecord(b->ready[i], b->m[i]->stream) != cudaSuccess ||
            cudaStreamWaitEvent(b->stream, b->ready[i], 0) != cudaSuccess)
            return bfail(b, LBM_ERR_CUDA, "batch stream ordering");
    }
    for (int it = 0; it < n; it++) {
        if (cudaGraphLaunch(b->graph[b->phase], b->stream) != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "batch graph launch");
        b->phase ^= 1;
        for (lbm_solver *s : b->m) { s->parity[0] ^= 1; s->step++; }
    }
    // ... and the members' streams follow the batch (queries see the stepped state)
    if (cudaEventRecord(b->done, b->stream) != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "batch event");
    for (lbm_solver *s : b->m)
        if (cudaStreamWaitEvent(s->stream, b->done, 0) != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "batch stream ordering");
    return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_batch *b, int *members, int *levels, long long *kernels_per_step)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (members) *members = (int)b->m.size();
    if (levels) *levels = b->Lmax;
    if (kernels_per_step) *kernels_per_step = b->kernels_per_step;
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- checkpoint / resume
struct StateHeader {
    char magic[8];                 // "LBMSTAT3"
    int levels, store, turbulence, have_cl;
    int parity0, pad;              // level-0 parity of the in-place layout (finer levels are at 0)
    long long step, nrec;
    double last_cl;
    long long ns[LBM_MAXL];
    unsigned long long grid_hash;  // FNV-1a of every level's flag words and wall distances and of the wall records
    unsigned long long cfg_hash;   // FNV-1a of the configuration's physical and model parameters
};

static unsigned long long grid_hash(const lbm_solver *s)
{
    Fnv f;
    for (int l = 0; l < s->L; l++) {
        f.vec(s->lv[l].flags);
        f.vec(s->g.lv[l].dist);
    }
    for (const lbmgrid::Record &r : s->g.recs) {
        f.val(r.i); f.val(r.j); f.val(r.loop);
        f.bytes(r.n, sizeof r.n); f.val(r.dwb); f.bytes(r.r, sizeof r.r); f.bytes(r.q, sizeof r.q);
        f.val(r.ns); f.bytes(r.si, sizeof(int) * r.ns); f.bytes(r.sj, sizeof(int) * r.ns);
    }
    return f.h;
}

// every configuration value that changes the arithmetic of a step (not the stream or the
// allocator hooks)
static unsigned long long cfg_hash(const lbm_solver *s)
{
    const lbm_config &c = s->cfg;
    Fnv f;
    const int iv[14] = {c.levels, c.nx0, c.ny0, c.layers, c.turbulence, c.wall_model, c.periodic, c.solid_walls,
                        c.store, c.sa_convection, c.outlet, 0, 0, 0};
    const double dv[9] = {c.x0, c.y0, c.h0, c.chord, c.Re, c.Ma, c.chi_inf, c.d_wr, c.d_wv};
    f.bytes(iv, sizeof iv);
    f.bytes(dv, sizeof dv);
    return f.h;
}

// the raw device arrays of a checkpoint, in blob order: per level the lattice, the fields of
// the current time level and the explosion / coalescence buffers; then the wall records'
// Newton starts and post-collision buffers and the outlet buffer
static void state_arrays(lbm_solver *s, std::vector<std::pair<void *, size_t>> &a)
{
    const size_t pb = pop_bytes(s->cfg.store);
    for (int l = 0; l < s->L; l++) {
        LevelView &v = s->lv[l].v;
        const int p = s->parity[l];
        const size_t nm = (size_t)v.ns * sizeof(float);
        a.push_back({v.f, 9 * (size_t)v.ns * pb});
        a.push_back({v.drho[p], nm}); a.push_back({v.ux[p], nm}); a.push_back({v.uy[p], nm}); a.push_back({v.chi[p], nm});
        a.push_back({v.ebuf, 9 * (size_t)v.n_band * sizeof(float)});
        a.push_back({v.gbuf, 36 * (size_t)v.n_band * sizeof(float)});
    }
    a.push_back({s->rec.utau_start, (size_t)s->rec.n * sizeof(float)});
    a.push_back({s->rec.fpost, 9 * (size_t)s->rec.n * sizeof(float)});
    a.push_back({s->k.obuf, 12 * (size_t)s->cfg.ny0 * sizeof(float)});
}

static size_t state_bytes(lbm_solver *s)
{
    std::vector<std::pair<void *, size_t>> a;
    state_arrays(s, a);
    size_t n = sizeof(StateHeader);
    for (auto &x : a) n += x.second;
    return n;
}

lbm_status lbm_get_state(lbm_solver *s, void *buf, size_t cap, size_t *size)
{
    if (!s || !size) return fail(s, LBM_ERR_INVALID_ARG, "null argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    *size = state_bytes(s);
    if (!buf) return LBM_OK;
    if (cap < *size) return fail(s, LBM_ERR_INVALID_ARG, "state buffer too small");
    CK(cudaStreamSynchronize(s->stream));
    StateHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "LBMSTAT3", 8);
    h.levels = s->L; h.store = s->cfg.store; h.turbulence = s->cfg.turbulence; h.have_cl = s->have_cl;
    h.parity0 = s->parity[0];
    h.step = s->step; h.nrec = s->rec.n; h.last_cl = s->last_cl;
    for (int l = 0; l < s->L; l++) h.ns[l] = s->lv[l].v.ns;
    h.grid_hash = grid_hash(s);
    h.cfg_hash = cfg_hash(s);
    unsigned char *o = (unsigned char *)buf;
    std::memcpy(o, &h, sizeof h);
    o += sizeof h;
    std::vector<std::pair<void *, size_t>> a;
    state_arrays(s, a);
    for (auto &x : a) {
        if (x.second) CK(cudaMemcpyAsync(o, x.first, x.second, cudaMemcpyDeviceToHost, s->stream));
        o += x.second;
    }
    CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_solver *s, const void *buf, size_t size)
{
    if (!s || !buf) return fail(s, LBM_ERR_INVALID_ARG, "null argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    StateHeader h;
    if (size < sizeof h) return fail(s, LBM_ERR_INVALID_ARG, "state blob too short");
    std::memcpy(&h, buf, sizeof h);
    if (std::memcmp(h.magic, "LBMSTAT3", 8) != 0) return fail(s, LBM_ERR_INVALID_ARG, "not a state blob");
    bool same = h.levels == s->L && h.store == s->cfg.store && h.turbulence == s->cfg.turbulence && h.nrec == s->rec.n &&
                (h.parity0 == 0 || h.parity0 == 1);
    for (int l = 0; same && l < s->L; l++) same = h.ns[l] == s->lv[l].v.ns;
    if (!same || h.grid_hash != grid_hash(s)) return fail(s, LBM_ERR_INVALID_ARG, "state blob from another configuration or grid");
    if (h.cfg_hash != cfg_hash(s))
        return fail(s, LBM_ERR_INVALID_ARG, "state blob from a solve with other physical or model parameters");
    if (size != state_bytes(s)) return fail(s, LBM_ERR_INVALID_ARG, "state blob size differs");
    CK(cudaStreamSynchronize(s->stream));
    // the blob's level-0 parity becomes the solver's (the step graphs exist for both parities);
    // finer levels are at parity 0 at every coarse step
    s->parity[0] = h.parity0;
    for (int l = 1; l < s->L; l++) s->parity[l] = 0;
    s->off_schedule = false;
    const unsigned char *o = (const unsigned char *)buf + sizeof h;
    std::vector<std::pair<void *, size_t>> a;
    state_arrays(s, a);
    for (auto &x : a) {
        if (x.second) CK(cudaMemcpyAsync(x.first, o, x.second, cudaMemcpyHostToDevice, s->stream));
        o += x.second;
    }
    CK(cudaMemsetAsync(s->d_status, 0, sizeof(int), s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->step = h.step;
    s->have_cl = h.have_cl != 0;
    s->last_cl = h.last_cl;
    return LBM_OK;
}

lbm_status lbm_set_load_history(lbm_solver *s, int every, int capacity)
{
    if (!s || every < 0 || (every > 0 && capacity < 1)) return fail(s, LBM_ERR_INVALID_ARG, "bad argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    if (s->planning) return fail(s, LBM_ERR_NO_GEOMETRY, "host-only handle");
    if (every > 0 && capacity > s->hist_alloc) {
        s->d_hist = (double *)dalloc(s, (size_t)capacity * 6 * sizeof(double));
        if (!s->d_hist) { s->hist_alloc = 0; s->hist_every = 0; return fail(s, LBM_ERR_OOM, "load history"); }
        s->hist_alloc = capacity;
    }
    if (every > 0) s->hist_cap = capacity;
    s->hist_every = every;
    s->hist_count = 0;
    return LBM_OK;
}

lbm_status lbm_get_load_history(lbm_solver *s, lbm_load_record *out, int cap, int *n)
{
    if (!s || !n || (cap > 0 && !out)) return fail(s, LBM_ERR_INVALID_ARG, "bad argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    const long long kept = s->d_hist ? std::min<long long>(s->hist_count, s->hist_cap) : 0;
    *n = (int)kept;
    if (kept == 0 || cap <= 0) return LBM_OK;
    if (kept > cap) return fail(s, LBM_ERR_INVALID_ARG, "capacity too small");
    std::vector<double> h((size_t)s->hist_cap * 6);
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaMemcpy(h.data(), s->d_hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    const long long first = s->hist_count - kept;                    // oldest kept record
    for (long long i = 0; i < kept; i++) {
        const double *r = &h[(size_t)((first + i) % s->hist_cap) * 6];
        lbm_load_record &o = out[i];
        o.step = (long long)r[0];
        o.CL = r[1]; o.CD = r[2]; o.CDp = r[3]; o.CDf = r[4]; o.mass = r[5];
    }
    return check_status(s);
}

lbm_status lbm_set_timeline(lbm_solver *s, int on)
{
    if (!s || (on != 0 && on != 1)) return fail(s, LBM_ERR_INVALID_ARG, "bad argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    if (s->planning) return fail(s, LBM_ERR_NO_GEOMETRY, "host-only handle");
    if (on && !s->d_tl) {
        // every launch of both step graphs: level l takes 2^l steps, each at most its tile
        // count or half its work warps in blocks, and a prolongation launch its band tiles
        long long need = 0;
        for (int l = 0; l < s->L; l++) {
            const lbmdev::LevelView &v = s->lv[l].v;
            need += (1LL << l) * (std::max(v.n_work_tiles, (v.n_work_warps + 1) / 2) + v.n_band_tiles);
        }
        need *= 2;
        s->d_tl = (unsigned long long *)dalloc(s, (size_t)need * 3 * sizeof(unsigned long long));
        if (!s->d_tl) return fail(s, LBM_ERR_OOM, "timeline buffer");
        s->tl_cap = need;
        CK(cudaMemsetAsync(s->d_tl, 0, (size_t)need * 3 * sizeof(unsigned long long), s->stream));
    }
    s->tl_on = on;
    return capture_graphs(s);
}

lbm_status lbm_get_timeline(lbm_solver *s, lbm_launch_time *out, int cap, int *n)
{
    if (!s || !n || (cap > 0 && !out)) return fail(s, LBM_ERR_INVALID_ARG, "bad argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    const int nl = (int)s->tl_meta.size() / 5;
    *n = s->tl_on ? nl : 0;
    if (!s->tl_on || nl == 0 || cap <= 0) return LBM_OK;
    if (nl > cap) return fail(s, LBM_ERR_INVALID_ARG, "capacity too small");
    std::vector<unsigned long long> h((size_t)s->tl_next * 3);
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaMemcpy(h.data(), s->d_tl, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    unsigned long long t0[2] = {~0ull, ~0ull};
    std::vector<unsigned long long> wmin(nl, ~0ull), emax(nl, 0ull);
    std::vector<int> ran(nl, 0);
    for (int i = 0; i < nl; i++) {
        const int *m = &s->tl_meta[(size_t)i * 5];
        for (int b = 0; b < m[4]; b++) {
            const unsigned long long *r = &h[3 * ((size_t)m[3] + b)];
            if (r[2] == 0) continue;                      // block not run since the capture
            ran[i]++;
            wmin[i] = std::min(wmin[i], r[1]);
            emax[i] = std::max(emax[i], r[2]);
        }
        if (ran[i]) t0[m[0] & 1] = std::min(t0[m[0] & 1], wmin[i]);
    }
    for (int i = 0; i < nl; i++) {
        const int *m = &s->tl_meta[(size_t)i * 5];
        lbm_launch_time &o = out[i];
        o.graph = m[0];
        o.level = m[1];
        o.kind = m[2];
        o.blocks = ran[i];
        const unsigned long long g0 = t0[m[0] & 1];
        o.t_wait_us = ran[i] ? 1e-3 * (double)(wmin[i] - g0) : 0.0;
        o.t_end_us = ran[i] ? 1e-3 * (double)(emax[i] - g0) : 0.0;
    }
    return LBM_OK;
}

lbm_status lbm_set_prolong_merge(lbm_solver *s, int on, int *merged_levels)
{
    if (!s || (on != 0 && on != 1)) return fail(s, LBM_ERR_INVALID_ARG, "bad argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    s->prolong_merge = on;
    if (merged_levels) {
        int n = 0;
        for (int l = 0; l < s->L; l++) n += s->prolong_indep[l] ? 1 : 0;
        *merged_levels = n;
    }
    return capture_graphs(s);
}

lbm_status lbm_set_launch_variant(lbm_solver *s, const int *min_blocks, const int *sched, const int *shape,
                                  int pdl)
{
    if (!s || !min_blocks || !sched || (pdl != 0 && pdl != 1)) return fail(s, LBM_ERR_INVALID_ARG, "bad argument");
    if (!s->geometry) return fail(s, LBM_ERR_NO_GEOMETRY, "no geometry");
    for (int l = 0; l < s->L; l++) {
        const int sh = shape ? shape[l] : 0;
        if ((min_blocks[l] != 5 && min_blocks[l] != 6) || sched[l] < LBM_SCHED_TILE || sched[l] > LBM_SCHED_WARPS4 ||
            (sh != 0 && sh != 1) || (sched[l] >= LBM_SCHED_WARPS && sh != 0))
            return fail(s, LBM_ERR_INVALID_ARG,
                        "launch variant: min_blocks must be 5 or 6, sched one of LBM_SCHED_*, shape 0 or 1 (0 with "
                        "the warp-list schedules)");
    }
    for (int l = 0; l < s->L; l++) {
        s->min_blocks[l] = min_blocks[l];
        s->sched[l] = sched[l];
        s->shape[l] = shape ? shape[l] : 0;
    }
    s->pdl = pdl;
    return capture_graphs(s);
}

}  // extern "C"
