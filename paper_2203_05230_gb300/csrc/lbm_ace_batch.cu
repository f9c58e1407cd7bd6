// lbm_ace_batch.cu -- many independent single-vortex lattices advanced together.
//
// A batch holds N lattices of possibly different sizes and parameters (each a
// single-vortex problem of Section 3 / Eq. 14, FP32 populations). One time step of the
// batch is one launch of a persistent kernel: a grid of (SMs x resident CTAs) CTAs whose
// warps (when every nx is a multiple of 4) or CTAs (otherwise) pull work items from an
// atomic counter -- a 128-column strip or a 256-column tile of one row band of one
// lattice -- and run the single-lattice kernels' code on each (quad32_strip of the FP32
// quad kernel, or pair_tile of the column-pair kernel), so small lattices that could
// never fill the GPU alone share it.
// The step counter t lives on the device; each lattice's phase cos(pi t / T) is
// computed there, so a captured graph of {step, advance} replays any number of steps
// without host work. Tile heights and the persistent grid's CTAs per SM come from
// lbm_ace_batch_autotune (coordinate descent, timed with CUDA events on the batch's
// stream).
//
// Uneven runs: each lattice may have its own end step (its period T, Section 3, whose
// shape at t = T is the benchmark's measure); it advances while t < end and then keeps
// its state. The work list orders the lattices by end, latest first, so the tiles still
// active at any t are a prefix of the list; the small per-step kernel that advances the
// phases also computes that prefix's length for the next step, and the persistent
// kernel stops pulling work there. Retired lattices cost nothing, in the graph too.
#include "lbm_ace.h"
#include "ace_kernels.cuh"
#include "ace_reduce.cuh"
#include "ace_step_pair.cuh"
#include "ace_step_quad.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <new>
#include <string>
#include <vector>

using namespace lbmace;

namespace {

constexpr double kPiB = 3.14159265358979323846;
constexpr int kMinRows = 8; // smallest tile height the batch is sized for

struct BatchInst {
    long long end;        // the lattice advances while t < end (LLONG_MAX: no end)
    float* f[2];          // population ping-pong buffers; f[t & 1] holds f*(t - 1)
    float* phi;           // phi(t - 1)
    const float* sx2; const float* s2x; const float* sy2; const float* s2y; // Eq. 14 tables
    double* mass_part;    // one partial per tile
    int nx, ny, rows, tiles_x, tiles_y, tile0;
    float omega, fpref, eps, inv_eps, inv4eps, delta, inv1p2d, amp;
    double T_period;
};

struct BatchCtl {
    int next;        // work-item counter of the step in flight
    int t;           // time of the next step (every active lattice advances together)
    int active;      // tiles of the lattices still active at time t: a prefix of the work list
    int active_next; // the same for time t + 1, filled in by ace_batch_phase
};

// Step arguments of lattice I at time t (tiles `rows` tall) and its velocity at the
// phase ph = (cos(pi t / T), cos(pi (t - 1) / T)).
__device__ __forceinline__ StepArgs<float> batch_args(const BatchInst& I, int t, int rows)
{
    StepArgs<float> a;
    a.fin = I.f[t & 1];
    a.fout = I.f[(t & 1) ^ 1];
    a.phi = I.phi;
    a.mass_part = I.mass_part;
    a.nx = I.nx; a.ny = I.ny;
    a.plane = (long long)I.nx * I.ny;
    a.rows = rows;
    a.first = t == 0;
    a.tdir = t & 1;
    a.omega = I.omega; a.fpref = I.fpref;
    a.eps = I.eps; a.inv_eps = I.inv_eps; a.inv4eps = I.inv4eps;
    a.delta = I.delta; a.inv1p2d = I.inv1p2d;
    return a;
}

__device__ __forceinline__ VelVortex<float> batch_vel(const BatchInst& I, float2 ph)
{
    VelVortex<float> vel;
    vel.sx2 = I.sx2; vel.s2x = I.s2x; vel.sy2 = I.sy2; vel.s2y = I.s2y;
    vel.amp = I.amp;
    vel.ct = ph.x;
    vel.ctm1 = ph.y;
    return vel;
}

// Tile (bx, by) of lattice I at time t with tiles `rows` tall; the tile's mass partial
// goes to *mass_out. pair_tile marches its default direction (down).
template <int MODEL>
__device__ __forceinline__ void batch_tile_at(const BatchInst& I, float2 ph, int bx, int by, int rows, int t,
                                              float (*chi_s)[PAIR_COLS + 4], double* red_s, double* mass_out)
{
    pair_tile<float, MODEL>(batch_args(I, t, rows), batch_vel(I, ph), bx * PAIR_COLS, by * rows, chi_s, red_s,
                            mass_out);
}

// Work item lt (row-major over the lattice's tiles of the batch's height I.rows).
template <int MODEL>
__device__ __forceinline__ void batch_tile(const BatchInst& I, float2 ph, int lt, int t, float (*chi_s)[PAIR_COLS + 4],
                                           double* red_s)
{
    batch_tile_at<MODEL>(I, ph, lt % I.tiles_x, lt / I.tiles_x, I.rows, t, chi_s, red_s, &I.mass_part[lt]);
}

template <int MODEL>
__global__ void __launch_bounds__(PAIR_THREADS, 5)
ace_batch_step(const BatchInst* __restrict__ inst, const float2* __restrict__ phase, const int* __restrict__ tile_inst,
               BatchCtl* ctl)
{
    __shared__ __align__(16) float chi_s[4][PAIR_COLS + 4];
    __shared__ double red_s[PAIR_THREADS / 32];
    __shared__ int tile_s;
    const int t = ctl->t;
    const int ntiles = ctl->active;
    for (;;) {
        if (threadIdx.x == 0) tile_s = atomicAdd(&ctl->next, 1);
        __syncthreads();
        const int tile = tile_s;
        __syncthreads();
        if (tile >= ntiles) break;
        const int i = tile_inst[tile];
        batch_tile<MODEL>(inst[i], phase[i], tile - inst[i].tile0, t, chi_s, red_s);
    }
}

// One launch per lattice (the per-lattice baseline): a grid over lattice i in the launch
// shape the single-lattice library picks (tiles `rows` tall), with the same tile code
// and device-side phases as the persistent kernel; mass partials go to a scratch array.
template <int MODEL>
__global__ void __launch_bounds__(PAIR_THREADS, 5)
ace_batch_one(const BatchInst* __restrict__ inst, const float2* __restrict__ phase, int i, int rows,
              const BatchCtl* ctl, double* part)
{
    __shared__ __align__(16) float chi_s[4][PAIR_COLS + 4];
    __shared__ double red_s[PAIR_THREADS / 32];
    const int t = ctl->t;
    if (t < inst[i].end)
        batch_tile_at<MODEL>(inst[i], phase[i], blockIdx.x, blockIdx.y, rows, t, chi_s, red_s,
                             &part[blockIdx.y * gridDim.x + blockIdx.x]);
}

// The persistent kernel on four-column strips (every lattice's nx a multiple of 4): each
// warp pulls its own work item -- one 128-column strip of one row band of one lattice --
// and runs the single-lattice kernel's strip code (quad32_strip) on it, bands marching
// up or down by band and step parity as in that kernel; the warp's mass sum is the
// item's partial. Warps of a CTA share nothing but the CTA's shared-memory layout, so a
// lattice narrower than a CTA's four strips leaves no warp idle.
template <int MODEL>
__global__ void __launch_bounds__(Q32_THREADS, Q32_MIN_CTAS)
ace_batch_step_q(const BatchInst* __restrict__ inst, const float2* __restrict__ phase,
                 const int* __restrict__ tile_inst, BatchCtl* ctl)
{
    extern __shared__ __align__(16) unsigned char bq_smem[];
    Quad32Smem& sm = *reinterpret_cast<Quad32Smem*>(bq_smem);
    const int tx = threadIdx.x, lane = tx & 31, wid = tx >> 5;
    const int t = ctl->t;
    const int ntiles = ctl->active;
    for (;;) {
        int tile = 0;
        if (lane == 0) tile = atomicAdd(&ctl->next, 1);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= ntiles) break;
        const int i = tile_inst[tile];
        const BatchInst& I = inst[i];
        const int lt = tile - I.tile0;
        const int sx = lt % I.tiles_x, by = lt / I.tiles_x;
        const StepArgs<float> a = batch_args(I, t, I.rows);
        const VelVortex<float> vel = batch_vel(I, phase[i]);
        const int y0 = by * I.rows, y1 = min(y0 + I.rows, I.ny);
        double m;
        if (march_up((unsigned)by, a.tdir))
            m = quad32_strip<MODEL, VelVortex<float>, true>(a, vel, sx * Q32_STRIP, y0, y1, sm.chi[wid], sm.park, tx);
        else
            m = quad32_strip<MODEL, VelVortex<float>, false>(a, vel, sx * Q32_STRIP, y0, y1, sm.chi[wid], sm.park, tx);
        if (lane == 0) I.mass_part[lt] = m;
    }
}

// The per-lattice baseline on four-column strips: lattice i alone, in the launch shape of
// the single-lattice library's quad kernel (CTAs of four strips, bands `rows` tall).
template <int MODEL>
__global__ void __launch_bounds__(Q32_THREADS, Q32_MIN_CTAS)
ace_batch_one_q(const BatchInst* __restrict__ inst, const float2* __restrict__ phase, int i, int rows,
                const BatchCtl* ctl, double* part)
{
    extern __shared__ __align__(16) unsigned char bq_smem[];
    Quad32Smem& sm = *reinterpret_cast<Quad32Smem*>(bq_smem);
    const int t = ctl->t;
    if (t >= inst[i].end) return;
    StepArgs<float> a = batch_args(inst[i], t, rows);
    a.mass_part = part;
    const VelVortex<float> vel = batch_vel(inst[i], phase[i]);
    if (march_up(blockIdx.y, a.tdir))
        quad32_tile<MODEL, VelVortex<float>, true>(a, vel, sm);
    else
        quad32_tile<MODEL, VelVortex<float>, false>(a, vel, sm);
}

// For the next step, t + 1: the phase of Eq. 14, (cos(pi (t+1) / T), cos(pi t / T)), per
// lattice, and the length of the active prefix of the work list. end_sorted holds the
// lattices' ends in work-list order (non-increasing), prefix[j] the tiles of positions
// 0 .. j; the position j with end_sorted[j] > t + 1 >= end_sorted[j + 1] is the last
// active one.
__global__ void ace_batch_phase(BatchCtl* __restrict__ ctl, const BatchInst* __restrict__ inst, int n,
                                const long long* __restrict__ end_sorted, const int* __restrict__ prefix,
                                float2* __restrict__ phase)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const long long tn = (long long)ctl->t + 1;
        const double t = (double)tn;
        phase[i] = make_float2((float)cos(kPiB * t / inst[i].T_period), (float)cos(kPiB * (t - 1.0) / inst[i].T_period));
        if (end_sorted[i] > tn && (i == n - 1 || end_sorted[i + 1] <= tn)) ctl->active_next = prefix[i];
        if (i == 0 && end_sorted[0] <= tn) ctl->active_next = 0;
    }
}

__global__ void ace_batch_tick(BatchCtl* ctl)
{
    ctl->next = 0;
    ctl->t += 1;
    ctl->active = ctl->active_next;
}

} // namespace

struct lbm_ace_batch {
    int n = 0;
    int model = 0;
    int dev = 0, sms = 0;
    cudaStream_t stream = nullptr;
    std::vector<lbm_ace_params> p;
    std::vector<BatchInst> inst;  // host copy
    BatchInst* d_inst = nullptr;
    std::vector<int> tile_inst;
    int* d_tile_inst = nullptr;
    int ntiles = 0, max_tiles = 0;
    BatchCtl* ctl = nullptr;
    float2* phase = nullptr; // (cos(pi t / T), cos(pi (t-1) / T)) per lattice for the next step
    std::vector<int> order;  // lattices in work-list order (end descending, then index)
    long long* d_end_sorted = nullptr; // ends in work-list order
    int* d_prefix = nullptr;           // tiles of work-list positions 0 .. j
    std::vector<int> prefix;           // host copy
    bool per_lattice_graph = false;    // the graph replays the per-lattice baseline
    float* pool = nullptr; size_t pool_elems = 0;
    float* tabs = nullptr;
    double* mass_pool = nullptr;
    double* seq_part = nullptr; // mass partials of the one-launch-per-lattice baseline
    std::vector<int> seq_rows;  // its one-wave tile heights
    double* red_part = nullptr; int n_red = 0;
    double* result = nullptr;
    double* scratch = nullptr; size_t scratch_elems = 0;
    int grid = 0, grid_max = 0; // persistent CTAs (tuned), and SMs x resident CTAs
    bool quad = false;          // every nx a multiple of 4: work items are four-column strips
    int cols = PAIR_COLS;       // columns of a work item (Q32_STRIP when quad)
    bool own_stream = false;
    long long t = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_berr;

int bfail(lbm_ace_batch* b, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf; else g_berr = buf;
    return code;
}

#define BK(b, call)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? LBM_ACE_ENOMEM : LBM_ACE_ECUDA,   \
                         "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);   \
    } while (0)

void drop_graph(lbm_ace_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Lay out the work list for the current tile heights and upload it (no device work in
// flight may use the old list).
int build_tiles(lbm_ace_batch* b)
{
    b->tile_inst.clear();
    b->order.resize(b->n);
    for (int i = 0; i < b->n; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return b->inst[x].end > b->inst[y].end; });
    b->prefix.assign(b->n, 0);
    std::vector<long long> ends(b->n);
    for (int j = 0; j < b->n; ++j) {
        const int i = b->order[j];
        BatchInst& I = b->inst[i];
        // heights below kMinRows would need more mass partials than were allocated; strips
        // take at most 4095 rows (the exact integer part of their mass sums)
        I.rows = std::max(std::min(kMinRows, I.ny), std::min(I.rows, I.ny));
        if (b->quad) I.rows = std::min(I.rows, 4095);
        I.tiles_x = (I.nx + b->cols - 1) / b->cols;
        I.tiles_y = (I.ny + I.rows - 1) / I.rows;
        I.tile0 = (int)b->tile_inst.size();
        for (int k = 0; k < I.tiles_x * I.tiles_y; ++k) b->tile_inst.push_back(i);
        b->prefix[j] = (int)b->tile_inst.size();
        ends[j] = I.end;
    }
    b->ntiles = (int)b->tile_inst.size();
    if (b->ntiles > b->max_tiles) return bfail(b, LBM_ACE_EINVAL, "work list larger than allocated");
    BK(b, cudaMemcpyAsync(b->d_inst, b->inst.data(), b->n * sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream));
    BK(b, cudaMemcpyAsync(b->d_tile_inst, b->tile_inst.data(), b->ntiles * sizeof(int), cudaMemcpyHostToDevice,
                          b->stream));
    BK(b, cudaMemcpyAsync(b->d_end_sorted, ends.data(), b->n * sizeof(long long), cudaMemcpyHostToDevice, b->stream));
    BK(b, cudaMemcpyAsync(b->d_prefix, b->prefix.data(), b->n * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BK(b, cudaStreamSynchronize(b->stream));
    drop_graph(b);
    return LBM_ACE_OK;
}

void launch_batch_step(lbm_ace_batch* b)
{
    const size_t qs = sizeof(Quad32Smem);
    if (b->quad && b->model == LBM_ACE_MODEL_MODIFIED)
        ace_batch_step_q<MODEL_MODIFIED><<<b->grid, Q32_THREADS, qs, b->stream>>>(b->d_inst, b->phase,
                                                                                 b->d_tile_inst, b->ctl);
    else if (b->quad)
        ace_batch_step_q<MODEL_CONSERVATIVE><<<b->grid, Q32_THREADS, qs, b->stream>>>(b->d_inst, b->phase,
                                                                                     b->d_tile_inst, b->ctl);
    else if (b->model == LBM_ACE_MODEL_MODIFIED)
        ace_batch_step<MODEL_MODIFIED><<<b->grid, PAIR_THREADS, 0, b->stream>>>(b->d_inst, b->phase, b->d_tile_inst,
                                                                              b->ctl);
    else
        ace_batch_step<MODEL_CONSERVATIVE><<<b->grid, PAIR_THREADS, 0, b->stream>>>(b->d_inst, b->phase, b->d_tile_inst,
                                                                                  b->ctl);
    ace_batch_phase<<<(b->n + 255) / 256, 256, 0, b->stream>>>(b->ctl, b->d_inst, b->n, b->d_end_sorted, b->d_prefix,
                                                              b->phase);
    ace_batch_tick<<<1, 1, 0, b->stream>>>(b->ctl);
}

// The per-lattice baseline: one launch per lattice in the single-lattice library's launch
// shape, then the same phase and tick kernels. A lattice past its end still launches,
// and its CTAs return at once.
void launch_per_lattice_step(lbm_ace_batch* b)
{
    for (int i = 0; i < b->n; ++i) {
        const BatchInst& I = b->inst[i];
        const int rows = b->seq_rows[i];
        if (b->quad) {
            const dim3 grid((I.nx + Q32_COLS - 1) / Q32_COLS, (I.ny + rows - 1) / rows);
            const size_t qs = sizeof(Quad32Smem);
            if (b->model == LBM_ACE_MODEL_MODIFIED)
                ace_batch_one_q<MODEL_MODIFIED><<<grid, Q32_THREADS, qs, b->stream>>>(b->d_inst, b->phase, i, rows,
                                                                                    b->ctl, b->seq_part);
            else
                ace_batch_one_q<MODEL_CONSERVATIVE><<<grid, Q32_THREADS, qs, b->stream>>>(b->d_inst, b->phase, i,
                                                                                        rows, b->ctl, b->seq_part);
            continue;
        }
        const dim3 grid(I.tiles_x, (I.ny + rows - 1) / rows);
        if (b->model == LBM_ACE_MODEL_MODIFIED)
            ace_batch_one<MODEL_MODIFIED><<<grid, PAIR_THREADS, 0, b->stream>>>(b->d_inst, b->phase, i, rows, b->ctl,
                                                                             b->seq_part);
        else
            ace_batch_one<MODEL_CONSERVATIVE><<<grid, PAIR_THREADS, 0, b->stream>>>(b->d_inst, b->phase, i, rows,
                                                                                 b->ctl, b->seq_part);
    }
    ace_batch_phase<<<(b->n + 255) / 256, 256, 0, b->stream>>>(b->ctl, b->d_inst, b->n, b->d_end_sorted, b->d_prefix,
                                                              b->phase);
    ace_batch_tick<<<1, 1, 0, b->stream>>>(b->ctl);
}

// Host-side reset of the device time and phases to the batch's time b->t.
int active_tiles(const lbm_ace_batch* b, long long t)
{
    int a = 0;
    for (int j = 0; j < b->n; ++j)
        if (b->inst[b->order[j]].end > t) a = b->prefix[j];
    return a;
}

int set_time(lbm_ace_batch* b)
{
    std::vector<float2> ph(b->n);
    for (int i = 0; i < b->n; ++i)
        ph[i] = make_float2(float(std::cos(kPiB * (double)b->t / b->inst[i].T_period)),
                            float(std::cos(kPiB * ((double)b->t - 1.0) / b->inst[i].T_period)));
    const int act = active_tiles(b, b->t);
    BatchCtl c{0, (int)b->t, act, act};
    BK(b, cudaMemcpyAsync(b->ctl, &c, sizeof c, cudaMemcpyHostToDevice, b->stream));
    BK(b, cudaMemcpyAsync(b->phase, ph.data(), b->n * sizeof(float2), cudaMemcpyHostToDevice, b->stream));
    BK(b, cudaStreamSynchronize(b->stream));
    return LBM_ACE_OK;
}

int ensure_graph(lbm_ace_batch* b, bool per_lattice = false)
{
    if (b->exec && b->per_lattice_graph == per_lattice) return LBM_ACE_OK;
    drop_graph(b);
    b->per_lattice_graph = per_lattice;
    BK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    if (per_lattice) launch_per_lattice_step(b);
    else launch_batch_step(b);
    cudaGraph_t g = nullptr;
    BK(b, cudaStreamEndCapture(b->stream, &g));
    b->graph = g;
    BK(b, cudaGraphInstantiate(&b->exec, b->graph, 0));
    return LBM_ACE_OK;
}

int check_inst(lbm_ace_batch* b, int i)
{
    if (!b) return bfail(nullptr, LBM_ACE_EINVAL, "batch is NULL");
    if (i < 0 || i >= b->n) return bfail(b, LBM_ACE_EINVAL, "instance %d out of range [0, %d)", i, b->n);
    return LBM_ACE_OK;
}

int ensure_bscratch(lbm_ace_batch* b, size_t elems)
{
    if (b->scratch_elems >= elems) return LBM_ACE_OK;
    if (b->scratch) cudaFree(b->scratch);
    b->scratch = nullptr;
    b->scratch_elems = 0;
    BK(b, cudaMalloc(&b->scratch, elems * sizeof(double)));
    b->scratch_elems = elems;
    return LBM_ACE_OK;
}

// Time `steps` graph steps (after one warm-up step); the lattices' states move on.
int time_steps(lbm_ace_batch* b, int steps, float* ms)
{
    int rc = ensure_graph(b);
    if (rc) return rc;
    BK(b, cudaGraphLaunch(b->exec, b->stream));
    cudaEvent_t e0, e1;
    BK(b, cudaEventCreate(&e0));
    BK(b, cudaEventCreate(&e1));
    BK(b, cudaEventRecord(e0, b->stream));
    for (int s = 0; s < steps; ++s) BK(b, cudaGraphLaunch(b->exec, b->stream));
    BK(b, cudaEventRecord(e1, b->stream));
    BK(b, cudaEventSynchronize(e1));
    BK(b, cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->t += steps + 1;
    return LBM_ACE_OK;
}

} // namespace

extern "C" {

int lbm_ace_batch_init(const lbm_ace_params* params, int count, lbm_ace_batch** out)
{
    if (!out) return bfail(nullptr, LBM_ACE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || count < 1) return bfail(nullptr, LBM_ACE_EINVAL, "need at least one lattice");
    for (int i = 0; i < count; ++i) {
        const lbm_ace_params& q = params[i];
        if (q.nx < 3 || q.ny < 3 || q.nx % 2 || (long long)q.nx * q.ny > (1LL << 31) / 9)
            return bfail(nullptr, LBM_ACE_EINVAL, "lattice %d: %d x %d (need an even nx >= 4, ny >= 3)", i, q.nx, q.ny);
        if (q.precision != LBM_ACE_F32) return bfail(nullptr, LBM_ACE_EINVAL, "lattice %d: batches use LBM_ACE_F32", i);
        if (q.velocity_kind != LBM_ACE_VEL_SINGLE_VORTEX)
            return bfail(nullptr, LBM_ACE_EINVAL, "lattice %d: batches use the single-vortex velocity", i);
        if (q.model != params[0].model) return bfail(nullptr, LBM_ACE_EINVAL, "lattice %d: all lattices need one model", i);
        if (!(q.tau > 0.5) || !(q.eps > 0.0) || !(q.T_period > 0.0) || !std::isfinite(q.U0) ||
            !std::isfinite(q.vortex_sign) || q.reg_delta < 0.0)
            return bfail(nullptr, LBM_ACE_EINVAL, "lattice %d: need tau > 0.5, eps > 0, T_period > 0", i);
        if (q.M >= 0.0 && std::fabs(q.M - (q.tau - 0.5) / 3.0) > 1e-12 * (q.tau - 0.5) / 3.0)
            return bfail(nullptr, LBM_ACE_EINVAL, "lattice %d: M differs from c_s^2 (tau - 0.5)", i);
        if (q.phi0) return bfail(nullptr, LBM_ACE_EINVAL, "lattice %d: batches build the disk (phi0 must be NULL)", i);
        if (q.rows_per_cta < 0) return bfail(nullptr, LBM_ACE_EINVAL, "lattice %d: rows_per_cta must be >= 0", i);
    }
    lbm_ace_batch* b = new (std::nothrow) lbm_ace_batch;
    if (!b) return bfail(nullptr, LBM_ACE_ENOMEM, "host allocation failed");
    b->n = count;
    b->p.assign(params, params + count);
    b->model = params[0].model;
    b->dev = params[0].device;
    b->stream = (cudaStream_t)params[0].stream;
    auto cleanup = [&](int rc) {
        g_berr = b->err;
        lbm_ace_batch_destroy(b);
        return rc;
    };
#define BI(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            bfail(b, e_ == cudaErrorMemoryAllocation ? LBM_ACE_ENOMEM : LBM_ACE_ECUDA, "%s: %s", #call, \
                  cudaGetErrorString(e_));                                                       \
            return cleanup(e_ == cudaErrorMemoryAllocation ? LBM_ACE_ENOMEM : LBM_ACE_ECUDA);     \
        }                                                                                        \
    } while (0)
    BI(cudaSetDevice(b->dev));
    BI(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev));
    if (!b->stream) { // graphs cannot be captured on the legacy default stream
        BI(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }

    // work items: four-column strips of 128 columns when every nx allows them (the
    // single-lattice library's FP32 kernel), else column-pair tiles of 256 columns
    b->quad = true;
    for (const auto& q : b->p) b->quad = b->quad && q.nx % 4 == 0;
    b->cols = b->quad ? Q32_STRIP : PAIR_COLS;
    // memory: populations x2 and phi per lattice in one pool; tables; mass partials
    size_t elems = 0, tab = 0;
    long long max_tiles = 0;
    for (const auto& q : b->p) {
        const size_t n = (size_t)q.nx * q.ny;
        elems += 19 * n + 3 * 64; // 2 x 9 planes + phi, each buffer padded to a 256-byte boundary
        tab += 2 * (size_t)(q.nx + q.ny) + 64;
        max_tiles += (long long)((q.nx + b->cols - 1) / b->cols) * ((q.ny + kMinRows - 1) / kMinRows);
    }
    b->max_tiles = (int)max_tiles;
    b->pool_elems = elems;
    BI(cudaMalloc(&b->pool, elems * sizeof(float)));
    BI(cudaMalloc(&b->tabs, tab * sizeof(float)));
    BI(cudaMalloc(&b->mass_pool, (size_t)max_tiles * sizeof(double)));
    BI(cudaMalloc(&b->d_inst, count * sizeof(BatchInst)));
    BI(cudaMalloc(&b->d_tile_inst, (size_t)max_tiles * sizeof(int)));
    BI(cudaMalloc(&b->ctl, sizeof(BatchCtl)));
    BI(cudaMalloc(&b->phase, count * sizeof(float2)));
    BI(cudaMalloc(&b->d_end_sorted, count * sizeof(long long)));
    BI(cudaMalloc(&b->d_prefix, count * sizeof(int)));
    // the mass and the flag slot of write_result, a spare, the reduction's ticket counter
    BI(cudaMalloc(&b->result, 4 * sizeof(double)));
    BI(cudaMemset(b->result, 0, 4 * sizeof(double)));
    long long maxn = 0;
    for (const auto& q : b->p) maxn = std::max(maxn, (long long)q.nx * q.ny);
    int rocc = 0;
    BI(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rocc, ace_sum_partials_f32, RED_THREADS, 0));
    b->n_red = mass_reduction_grid(b->sms, std::min(rocc, 4), 9 * maxn); // as the single-lattice library
    BI(cudaMalloc(&b->red_part, b->n_red * sizeof(double)));

    b->inst.resize(count);
    float* fp = b->pool;
    float* tp = b->tabs;
    double* mp = b->mass_pool;
    auto align64 = [](float* q) { return (float*)(((uintptr_t)q + 255) & ~(uintptr_t)255); };
    std::vector<float> h;
    std::vector<double> hphi;
    for (int i = 0; i < count; ++i) {
        const lbm_ace_params& q = b->p[i];
        BatchInst& I = b->inst[i];
        const size_t n = (size_t)q.nx * q.ny;
        fp = align64(fp); I.f[0] = fp; fp += 9 * n;
        fp = align64(fp); I.f[1] = fp; fp += 9 * n;
        fp = align64(fp); I.phi = fp; fp += n;
        const double delta = q.reg_delta == 0.0 ? std::exp(-20.0) : q.reg_delta;
        I.nx = q.nx; I.ny = q.ny;
        I.rows = q.rows_per_cta > 0 ? q.rows_per_cta : 64;
        I.omega = float(1.0 / q.tau); I.fpref = float(1.0 - 0.5 / q.tau);
        I.eps = float(q.eps); I.inv_eps = float(1.0 / q.eps); I.inv4eps = float(0.25 / q.eps);
        I.delta = float(delta); I.inv1p2d = float(1.0 / (1.0 + 2.0 * delta));
        I.amp = float(q.vortex_sign * q.U0);
        I.T_period = q.T_period;
        I.end = LLONG_MAX;
        I.mass_part = mp;
        mp += (size_t)((q.nx + b->cols - 1) / b->cols) * ((q.ny + kMinRows - 1) / kMinRows);
        // Eq. 14 tables, as in the single-lattice library
        h.assign(2 * (q.nx + q.ny), 0.0f);
        for (int x = 0; x < q.nx; ++x) {
            const double s = std::sin(kPiB * x / q.nx);
            h[x] = float(s * s);
            h[q.nx + x] = float(std::sin(2.0 * kPiB * x / q.nx));
        }
        for (int y = 0; y < q.ny; ++y) {
            const double s = std::sin(kPiB * y / q.ny);
            h[2 * q.nx + y] = float(s * s);
            h[2 * q.nx + q.ny + y] = float(std::sin(2.0 * kPiB * y / q.ny));
        }
        tp = align64(tp);
        I.sx2 = tp; I.s2x = tp + q.nx; I.sy2 = tp + 2 * q.nx; I.s2y = tp + 2 * q.nx + q.ny;
        BI(cudaMemcpy(tp, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
        tp += h.size();
        // initial state: the disk of each lattice, f = f^eq(phi0, u(x, 0))
        hphi.resize(n);
        for (int y = 0; y < q.ny; ++y)
            for (int x = 0; x < q.nx; ++x) {
                const double r = std::sqrt((x - q.xc) * (x - q.xc) + (y - q.yc) * (y - q.yc));
                hphi[(size_t)y * q.nx + x] = 0.5 * (1.0 + std::tanh((q.R - r) / (2.0 * q.eps)));
            }
        size_t need = n;
        if (b->scratch_elems < need) {
            if (b->scratch) cudaFree(b->scratch);
            b->scratch = nullptr;
            BI(cudaMalloc(&b->scratch, need * sizeof(double)));
            b->scratch_elems = need;
        }
        BI(cudaMemcpy(b->scratch, hphi.data(), n * sizeof(double), cudaMemcpyHostToDevice));
        VelVortex<float> v;
        v.sx2 = I.sx2; v.s2x = I.s2x; v.sy2 = I.sy2; v.s2y = I.s2y;
        v.amp = I.amp; v.ct = 1.0f; v.ctm1 = float(std::cos(-kPiB / q.T_period));
        const int g = (int)std::min<long long>(((long long)n + 255) / 256, (long long)b->sms * 8);
        ace_init<float><<<g, 256, 0, b->stream>>>(b->scratch, I.f[0], I.phi, q.nx, q.ny, v);
        BI(cudaGetLastError());
        BI(cudaStreamSynchronize(b->stream));
    }
    int occ = 0;
    const int qs = (int)sizeof(Quad32Smem);
    if (b->quad) {
        BI(cudaFuncSetAttribute(ace_batch_step_q<MODEL_MODIFIED>, cudaFuncAttributeMaxDynamicSharedMemorySize, qs));
        BI(cudaFuncSetAttribute(ace_batch_step_q<MODEL_CONSERVATIVE>, cudaFuncAttributeMaxDynamicSharedMemorySize, qs));
        BI(cudaFuncSetAttribute(ace_batch_one_q<MODEL_MODIFIED>, cudaFuncAttributeMaxDynamicSharedMemorySize, qs));
        BI(cudaFuncSetAttribute(ace_batch_one_q<MODEL_CONSERVATIVE>, cudaFuncAttributeMaxDynamicSharedMemorySize, qs));
        BI(cudaFuncSetAttribute(ace_step_quad<MODEL_MODIFIED, VelVortex<float>>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, qs));
        BI(cudaFuncSetAttribute(ace_step_quad<MODEL_CONSERVATIVE, VelVortex<float>>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, qs));
        BI(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ace_batch_step_q<MODEL_MODIFIED>, Q32_THREADS, qs));
    } else if (b->model == LBM_ACE_MODEL_MODIFIED) {
        BI(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ace_batch_step<MODEL_MODIFIED>, PAIR_THREADS, 0));
    } else {
        BI(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ace_batch_step<MODEL_CONSERVATIVE>, PAIR_THREADS, 0));
    }
    b->grid = b->sms * std::max(1, occ);
    // the baseline launches each lattice as the single-lattice library would: rows per
    // CTA for one wave of resident CTAs of the same kernel form (CTAs of four strips, or
    // column-pair CTAs)
    {
        int pocc = 0;
        if (b->quad)
            BI(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pocc, ace_batch_one_q<MODEL_MODIFIED>, Q32_THREADS, qs));
        else if (b->model == LBM_ACE_MODEL_MODIFIED)
            BI(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pocc, ace_step_pair<float, MODEL_MODIFIED, VelVortex<float>>,
                                                             PAIR_THREADS, 0));
        else
            BI(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &pocc, ace_step_pair<float, MODEL_CONSERVATIVE, VelVortex<float>>, PAIR_THREADS, 0));
        const long long slots = (long long)b->sms * std::max(1, pocc);
        const int cta_cols = b->quad ? Q32_COLS : PAIR_COLS;
        long long maxp = 1;
        b->seq_rows.resize(count);
        for (int i = 0; i < count; ++i) {
            const int gx = (b->inst[i].nx + cta_cols - 1) / cta_cols;
            const long long bands = std::max(1LL, slots / gx);
            long long r = std::max(4LL, std::min<long long>(b->inst[i].ny, (b->inst[i].ny + bands - 1) / bands));
            if (b->quad) r = std::min(r, 4095LL);
            b->seq_rows[i] = (int)r;
            maxp = std::max(maxp, (long long)gx * ((b->inst[i].ny + r - 1) / r));
        }
        BI(cudaMalloc(&b->seq_part, maxp * sizeof(double)));
    }
    int rc = build_tiles(b);
    if (rc == LBM_ACE_OK) rc = set_time(b);
    if (rc) return cleanup(rc);
    b->grid_max = b->grid;
#undef BI
    *out = b;
    return LBM_ACE_OK;
}

int lbm_ace_batch_step(lbm_ace_batch* b, long long n)
{
    if (!b) return bfail(nullptr, LBM_ACE_EINVAL, "batch is NULL");
    if (n < 0) return bfail(b, LBM_ACE_EINVAL, "n must be >= 0");
    int rc = ensure_graph(b);
    if (rc) return rc;
    for (long long s = 0; s < n; ++s) BK(b, cudaGraphLaunch(b->exec, b->stream));
    b->t += n;
    return LBM_ACE_OK;
}

int lbm_ace_batch_step_sequential(lbm_ace_batch* b, long long n)
{
    if (!b) return bfail(nullptr, LBM_ACE_EINVAL, "batch is NULL");
    if (n < 0) return bfail(b, LBM_ACE_EINVAL, "n must be >= 0");
    for (long long s = 0; s < n; ++s) {
        const long long t = b->t + s;
        for (int i = 0; i < b->n; ++i) {
            const BatchInst& I = b->inst[i];
            if (t >= I.end) continue; // retired
            StepArgs<float> a;
            a.fin = I.f[t & 1];
            a.fout = I.f[(t & 1) ^ 1];
            a.phi = I.phi;
            a.mass_part = b->seq_part;
            a.nx = I.nx; a.ny = I.ny;
            a.plane = (long long)I.nx * I.ny;
            a.rows = b->seq_rows[i];
            a.first = t == 0;
            a.tdir = (int)(t & 1);
            a.omega = I.omega; a.fpref = I.fpref; a.eps = I.eps; a.inv_eps = I.inv_eps; a.inv4eps = I.inv4eps;
            a.delta = I.delta; a.inv1p2d = I.inv1p2d;
            VelVortex<float> v;
            v.sx2 = I.sx2; v.s2x = I.s2x; v.sy2 = I.sy2; v.s2y = I.s2y;
            v.amp = I.amp;
            v.ct = float(std::cos(kPiB * (double)t / I.T_period));
            v.ctm1 = float(std::cos(kPiB * ((double)t - 1.0) / I.T_period));
            if (b->quad) { // the single-lattice library's kernel for this lattice
                const dim3 grid((I.nx + Q32_COLS - 1) / Q32_COLS, (I.ny + a.rows - 1) / a.rows);
                if (b->model == LBM_ACE_MODEL_MODIFIED)
                    ace_step_quad<MODEL_MODIFIED, VelVortex<float>><<<grid, Q32_THREADS, sizeof(Quad32Smem), b->stream>>>(
                        a, v);
                else
                    ace_step_quad<MODEL_CONSERVATIVE, VelVortex<float>>
                        <<<grid, Q32_THREADS, sizeof(Quad32Smem), b->stream>>>(a, v);
                continue;
            }
            dim3 grid(I.tiles_x, (I.ny + a.rows - 1) / a.rows);
            if (b->model == LBM_ACE_MODEL_MODIFIED)
                ace_step_pair<float, MODEL_MODIFIED, VelVortex<float>><<<grid, PAIR_THREADS, 0, b->stream>>>(a, v);
            else
                ace_step_pair<float, MODEL_CONSERVATIVE, VelVortex<float>><<<grid, PAIR_THREADS, 0, b->stream>>>(a, v);
        }
        BK(b, cudaGetLastError());
    }
    b->t += n;
    return set_time(b);
}

int lbm_ace_batch_autotune(lbm_ace_batch* b, int steps_per_trial, int* rows_out)
{
    if (!b) return bfail(nullptr, LBM_ACE_EINVAL, "batch is NULL");
    if (steps_per_trial < 1) return bfail(b, LBM_ACE_EINVAL, "steps_per_trial must be >= 1");
    // keep the state: trials run real steps on a copy that is restored afterwards
    float* backup = nullptr;
    BK(b, cudaMalloc(&backup, b->pool_elems * sizeof(float)));
    BK(b, cudaMemcpyAsync(backup, b->pool, b->pool_elems * sizeof(float), cudaMemcpyDeviceToDevice, b->stream));
    const long long t_saved = b->t;
    std::map<int, std::vector<int>> by_size; // lattice width -> lattices
    for (int i = 0; i < b->n; ++i) by_size[b->inst[i].nx].push_back(i);
    const int cand[] = {8, 16, 32, 64, 128, 256};
    auto set_rows = [&](int nx, int rows) {
        for (int i : by_size[nx]) b->inst[i].rows = rows;
    };
    auto trial = [&](float* ms) {
        int rc = build_tiles(b);
        if (rc == LBM_ACE_OK) rc = set_time(b);
        if (rc) return rc;
        return time_steps(b, steps_per_trial, ms);
    };
    float best = 0.0f;
    int rc = trial(&best);
    for (int pass = 0; pass < 2 && rc == LBM_ACE_OK; ++pass) {
        for (auto& kv : by_size) {
            const int nx = kv.first;
            const int cur = b->inst[kv.second[0]].rows;
            int best_rows = cur;
            for (int r : cand) {
                if (r == cur || r > b->inst[kv.second[0]].ny) continue;
                set_rows(nx, r);
                float ms = 0.0f;
                rc = trial(&ms);
                if (rc) break;
                if (ms < best) { best = ms; best_rows = r; }
            }
            set_rows(nx, best_rows);
            if (rc) break;
        }
        // CTAs per SM of the persistent grid, with the tile heights chosen so far
        const int occ = std::max(1, b->grid_max / std::max(1, b->sms));
        const int cur_grid = b->grid;
        int best_grid = cur_grid;
        for (int c = 1; c <= occ && rc == LBM_ACE_OK; ++c) {
            const int gsz = c * b->sms;
            if (gsz == cur_grid) continue;
            b->grid = gsz;
            float ms = 0.0f;
            rc = trial(&ms);
            if (rc == LBM_ACE_OK && ms < best) { best = ms; best_grid = gsz; }
        }
        b->grid = best_grid;
    }
    // restore the state and time, keep the chosen tiles
    cudaMemcpyAsync(b->pool, backup, b->pool_elems * sizeof(float), cudaMemcpyDeviceToDevice, b->stream);
    b->t = t_saved;
    const int rc_t = set_time(b);
    cudaFree(backup);
    if (rc) return rc;
    if (rc_t) return rc_t;
    rc = build_tiles(b);
    if (rc == LBM_ACE_OK) rc = set_time(b);
    if (rc) return rc;
    if (rows_out)
        for (int i = 0; i < b->n; ++i) rows_out[i] = b->inst[i].rows;
    return LBM_ACE_OK;
}

int lbm_ace_batch_set_ends(lbm_ace_batch* b, const long long* end_steps)
{
    if (!b) return bfail(nullptr, LBM_ACE_EINVAL, "batch is NULL");
    std::vector<long long> e(b->n);
    for (int i = 0; i < b->n; ++i) {
        long long v = end_steps ? end_steps[i] : (long long)std::llround(b->inst[i].T_period);
        if (v < 0) v = LLONG_MAX;
        if (v < b->t) return bfail(b, LBM_ACE_EINVAL, "lattice %d: end %lld is before the batch's time %lld", i, v, b->t);
        e[i] = v;
    }
    BK(b, cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; ++i) b->inst[i].end = e[i];
    const int rc = build_tiles(b);
    return rc ? rc : set_time(b);
}

long long lbm_ace_batch_lattice_steps(const lbm_ace_batch* b, int i)
{
    if (!b || i < 0 || i >= b->n) return -1;
    return std::min(b->t, b->inst[i].end);
}

int lbm_ace_batch_active(const lbm_ace_batch* b, int* lattices, int* tiles)
{
    if (!b) return bfail(nullptr, LBM_ACE_EINVAL, "batch is NULL");
    int n = 0;
    for (int i = 0; i < b->n; ++i) n += b->inst[i].end > b->t;
    if (lattices) *lattices = n;
    if (tiles) *tiles = active_tiles(b, b->t);
    return LBM_ACE_OK;
}

int lbm_ace_batch_step_per_lattice(lbm_ace_batch* b, long long n)
{
    if (!b) return bfail(nullptr, LBM_ACE_EINVAL, "batch is NULL");
    if (n < 0) return bfail(b, LBM_ACE_EINVAL, "n must be >= 0");
    int rc = ensure_graph(b, true);
    if (rc) return rc;
    for (long long s = 0; s < n; ++s) BK(b, cudaGraphLaunch(b->exec, b->stream));
    b->t += n;
    return LBM_ACE_OK;
}

int lbm_ace_batch_get_phi(lbm_ace_batch* b, int i, double* out, size_t count)
{
    int rc = check_inst(b, i);
    if (rc) return rc;
    const BatchInst& I = b->inst[i];
    const size_t n = (size_t)I.nx * I.ny;
    if (!out || count != n) return bfail(b, LBM_ACE_EINVAL, "out must hold nx*ny = %zu values", n);
    rc = ensure_bscratch(b, n);
    if (rc) return rc;
    const int g = (int)std::min<long long>(((long long)n + 255) / 256, (long long)b->sms * 8);
    ace_moment<float><<<g, 256, 0, b->stream>>>(I.f[std::min(b->t, I.end) & 1], b->scratch, I.nx, I.ny);
    BK(b, cudaGetLastError());
    BK(b, cudaMemcpyAsync(out, b->scratch, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BK(b, cudaStreamSynchronize(b->stream));
    return LBM_ACE_OK;
}

int lbm_ace_batch_mass(lbm_ace_batch* b, int i, double* out)
{
    int rc = check_inst(b, i);
    if (rc) return rc;
    if (!out) return bfail(b, LBM_ACE_EINVAL, "out is NULL");
    const BatchInst& I = b->inst[i];
    const long long n9 = 9LL * I.nx * I.ny;
    ace_sum_partials_f32<<<b->n_red, RED_THREADS, 0, b->stream>>>(I.f[std::min(b->t, I.end) & 1], n9, b->red_part,
                                                                  reinterpret_cast<unsigned*>(b->result + 3), b->result,
                                                                  nullptr);
    BK(b, cudaGetLastError());
    BK(b, cudaMemcpyAsync(out, b->result, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BK(b, cudaStreamSynchronize(b->stream));
    if (!std::isfinite(*out)) return bfail(b, LBM_ACE_ENUMERIC, "mass of lattice %d is not finite", i);
    return LBM_ACE_OK;
}

int lbm_ace_batch_info(const lbm_ace_batch* b, int i, int* rows, int* tiles, int* grid, long long* nodes)
{
    if (!b) return bfail(nullptr, LBM_ACE_EINVAL, "batch is NULL");
    if (i < 0 || i >= b->n) return bfail(nullptr, LBM_ACE_EINVAL, "instance %d out of range", i);
    if (rows) *rows = b->inst[i].rows;
    if (tiles) *tiles = b->ntiles;
    if (grid) *grid = b->grid;
    if (nodes) {
        long long s = 0;
        for (const auto& I : b->inst) s += (long long)I.nx * I.ny;
        *nodes = s;
    }
    return LBM_ACE_OK;
}

long long lbm_ace_batch_steps_done(const lbm_ace_batch* b) { return b ? b->t : -1; }

int lbm_ace_batch_synchronize(lbm_ace_batch* b)
{
    if (!b) return bfail(nullptr, LBM_ACE_EINVAL, "batch is NULL");
    BK(b, cudaStreamSynchronize(b->stream));
    return LBM_ACE_OK;
}

const char* lbm_ace_batch_last_error(const lbm_ace_batch* b) { return b ? b->err.c_str() : g_berr.c_str(); }

void lbm_ace_batch_destroy(lbm_ace_batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream); else cudaDeviceSynchronize();
    drop_graph(b);
    void* bufs[] = {b->pool, b->tabs, b->mass_pool, b->seq_part, b->d_inst, b->d_tile_inst, b->ctl, b->phase,
                    b->result, b->red_part, b->scratch, b->d_end_sorted, b->d_prefix};
    for (void* q : bufs) if (q) cudaFree(q);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

} // extern "C"
