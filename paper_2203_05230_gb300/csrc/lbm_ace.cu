// lbm_ace.cu -- host side of the C ABI declared in include/lbm_ace.h.
//
// Owns the device state of one lattice (two ping-pong population buffers, the phi
// plane, velocity tables or planes, reduction partials), validates parameters,
// and issues one fused step kernel per time step on the caller's stream.
#include "lbm_ace.h"
#include "ctx_id.h"
#include "ace_kernels.cuh"
#include "ace_reduce.cuh"
#include "ace_step_bulk.cuh"
#include "ace_step_warp.cuh"
#include "ace_step_pair.cuh"
#include "ace_step_dev.cuh"
#include "ace_step_dev4.cuh"
#include "ace_step_quad.cuh"
#include "ace_step_tb2.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>

using namespace lbmace;

namespace {

thread_local std::string g_err; // errors raised before a context exists

constexpr double kPi = 3.14159265358979323846;
// phi0 fields up to this many values are checked for non-finite entries on the host
// before any device work; larger ones right after their upload, on the device (a host
// pass over a 2048^2 field costs milliseconds)
constexpr size_t kHostCheckMax = 1u << 16;

// --- memory of the contexts ----------------------------------------------------------
// Device buffers come from one stream-ordered memory pool per device that keeps the
// blocks a destroyed context frees (no release threshold), so a lattice created after
// another one was destroyed reuses that memory. Measured on GB300: the six buffers of a
// 2048^2 FP32 lattice cost 225 us through cudaMalloc, 7 us from the pool.
// lbm_ace_release_cached_memory hands the unused blocks back to the driver. A pool lives
// as long as the device's context: after cudaDeviceReset (a new context id) a new one
// is made. The calls below run with `dev` current.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};
unsigned long long g_pool_ctx[kMaxDevices] = {};

cudaError_t device_pool(int dev, cudaMemPool_t* out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned long long id = 0;
    if (!current_ctx_id(&id)) return cudaErrorDeviceUninitialized;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev] || g_pool_ctx[dev] != id) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        unsigned long long keep = ~0ULL;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pools[dev] = pool;
        g_pool_ctx[dev] = id;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

// A second stream per device (non-blocking), on which lattice creation uploads phi0 in row
// chunks while the context's stream initialises the chunks already there; like the pool
// it is made again when the device's context changes.
cudaStream_t g_aux[kMaxDevices] = {};
unsigned long long g_aux_ctx[kMaxDevices] = {};

cudaError_t aux_stream(int dev, cudaStream_t* out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned long long id = 0;
    if (!current_ctx_id(&id)) return cudaErrorDeviceUninitialized;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_aux[dev] || g_aux_ctx[dev] != id) {
        cudaStream_t st;
        const cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        g_aux[dev] = st;
        g_aux_ctx[dev] = id;
    }
    *out = g_aux[dev];
    return cudaSuccess;
}

// Mapped pinned host memory for the contexts' result blocks, in 128-byte slots (one
// cache line each) cut from 4 KiB pages that are never freed: a cudaHostAlloc costs
// about 80 us, more than a whole mass call. A page belongs to the CUDA context that was
// current when it was allocated and dies with it (cudaDeviceReset), so every slot
// carries that context's id and is handed out only while the same context is current.
struct PinnedSlot { double* host; double* dev; unsigned long long ctx; };
std::mutex g_slot_mu;
std::vector<PinnedSlot> g_free_slots;
constexpr size_t kSlotBytes = 128, kSlotPage = 4096;

cudaError_t acquire_slot(PinnedSlot* out)
{
    unsigned long long id = 0;
    if (!current_ctx_id(&id)) return cudaErrorDeviceUninitialized;
    std::lock_guard<std::mutex> lock(g_slot_mu);
    for (size_t k = g_free_slots.size(); k-- > 0;)
        if (g_free_slots[k].ctx == id) {
            *out = g_free_slots[k];
            g_free_slots.erase(g_free_slots.begin() + (long)k);
            std::memset(out->host, 0, kSlotBytes);
            return cudaSuccess;
        }
    void* page = nullptr;
    cudaError_t e = cudaHostAlloc(&page, kSlotPage, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) return e;
    void* dpage = nullptr;
    e = cudaHostGetDevicePointer(&dpage, page, 0);
    if (e != cudaSuccess) {
        cudaFreeHost(page);
        return e;
    }
    for (size_t off = kSlotBytes; off < kSlotPage; off += kSlotBytes) // slot 0 is handed out now
        g_free_slots.push_back({reinterpret_cast<double*>(static_cast<char*>(page) + off),
                                reinterpret_cast<double*>(static_cast<char*>(dpage) + off), id});
    *out = {static_cast<double*>(page), static_cast<double*>(dpage), id};
    std::memset(out->host, 0, kSlotBytes);
    return cudaSuccess;
}

void release_slot(const PinnedSlot& s)
{
    std::lock_guard<std::mutex> lock(g_slot_mu);
    g_free_slots.push_back(s);
}

struct VelState {
    // single vortex tables, in the storage precision of the arithmetic (T)
    void* sx2 = nullptr; void* s2x = nullptr; void* sy2 = nullptr; void* s2y = nullptr;
    // FP64 planes for field / callback velocities: pair 0 and pair 1
    double* pu[2] = {nullptr, nullptr};
    double* pv[2] = {nullptr, nullptr};
    int cur = 0; // pair holding u(t)
    std::vector<double> hu, hv; // host buffers for the callback
};

} // namespace

struct lbm_ace_ctx {
    lbm_ace_params p{};
    cudaStream_t stream = nullptr;
    int dev = 0;
    int sms = 0;
    size_t elem = 0;        // bytes per stored value
    void* f[2] = {nullptr, nullptr};
    int cur = 0;            // buffer holding f*(t-1)
    void* phi = nullptr;    // phi(t-1) plane (deviation storage: phi2[pcur])
    void* phi_alt = nullptr; // second FP32 phi plane of the two-step kernel (variant 6)
    float* phi2[2] = {nullptr, nullptr}; // deviation storage: ping-pong FP32 phi planes
    int pcur = 0;
    double* step_part = nullptr; int n_step_part = 0;
    double* red_part = nullptr; int n_red_part = 0;
    double* result = nullptr;
    PinnedSlot slot{nullptr, nullptr, 0}; // mapped pinned result block (acquire_slot)
    double* hres = nullptr;     // its host address: the finishing kernels write results to hres[0..1];
                                // hres[4] takes the index the init's check of phi0 found
    double* hres_dev = nullptr; // its device address
    void* arena = nullptr;  // the one pool allocation every fixed buffer above and in vel is cut from
    double* scratch = nullptr; size_t scratch_elems = 0; // FP64 staging for state/phi copies (own allocation)
    VelState vel;
    long long t = 0;
    bool stepped = false;
    bool fresh = true;      // next step is the first after init or a restart: d_t(phi u) = 0
    int rows = 0, grid_x = 0, grid_y = 0;
    int variant = 1;        // 1: ace_step (direct loads), 2: ace_step_bulk
    int dev4_ctas = 3;      // resident CTAs per SM the 16-bit quad kernel is compiled for
    int l2_keep = 0;        // L2 priority bits of the stores (StepArgs::l2_keep)
    cudaStream_t upload = nullptr; // the second stream while it may still copy into scratch (creation)
    int tile_x = TILE_X;
    size_t smem = 0;        // dynamic shared memory of the chosen step kernel
    int* dev_err = nullptr; // set by a kernel whose bounded wait gave up (inside the result block)
    std::string err;
};

namespace {

int fail(lbm_ace_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_err = buf;
    return code;
}

#define CK(ctx, call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? LBM_ACE_ENOMEM : LBM_ACE_ECUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);  \
    } while (0)

// A device buffer of the context from the device's pool (device_pool), ordered on the
// context's stream. Every use of a context's buffers (kernels, copies, memsets) is issued
// on that stream, so none needs a synchronisation here; a block that another context freed
// on another stream is reused after that free, by the dependencies the pool's default
// reuse policies give the allocation.
template <typename P>
int pool_alloc(lbm_ace_ctx* c, P** ptr, size_t bytes)
{
    cudaMemPool_t pool;
    CK(c, device_pool(c->dev, &pool));
    void* q = nullptr;
    CK(c, cudaMallocFromPoolAsync(&q, bytes, pool, c->stream));
    *ptr = static_cast<P*>(q);
    return LBM_ACE_OK;
}
#define PA(ctx, ptr, bytes)                              \
    do {                                                 \
        const int rc_ = pool_alloc((ctx), (ptr), (bytes)); \
        if (rc_) return rc_;                             \
    } while (0)

int grid_for(long long n, int sms) // grid of a grid-stride elementwise kernel
{
    long long g = (n + 255) / 256;
    long long cap = (long long)sms * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// --- typed dispatch -----------------------------------------------------------

template <typename T>
StepArgs<T> make_args(lbm_ace_ctx* c)
{
    StepArgs<T> a;
    a.fin = (const T*)c->f[c->cur];
    a.fout = (T*)c->f[1 - c->cur];
    a.phi = (T*)c->phi;
    a.mass_part = c->step_part;
    a.nx = c->p.nx; a.ny = c->p.ny;
    a.plane = (long long)c->p.nx * c->p.ny;
    a.rows = c->rows;
    a.first = c->fresh;
    a.tdir = (int)(c->t & 1);
    a.l2_keep = c->l2_keep;
    a.omega = T(1.0 / c->p.tau);
    a.fpref = T(1.0 - 0.5 / c->p.tau);
    a.eps = T(c->p.eps);
    a.inv_eps = T(1.0 / c->p.eps);
    a.inv4eps = T(0.25 / c->p.eps);
    a.delta = T(c->p.reg_delta);
    a.inv1p2d = T(1.0 / (1.0 + 2.0 * c->p.reg_delta));
    return a;
}

template <typename T>
VelVortex<T> vortex(lbm_ace_ctx* c, double t)
{
    VelVortex<T> v;
    v.sx2 = (const T*)c->vel.sx2; v.s2x = (const T*)c->vel.s2x;
    v.sy2 = (const T*)c->vel.sy2; v.s2y = (const T*)c->vel.s2y;
    v.amp = T(c->p.vortex_sign * c->p.U0);
    v.ct = T(std::cos(kPi * t / c->p.T_period));
    v.ctm1 = T(std::cos(kPi * (t - 1.0) / c->p.T_period));
    return v;
}

template <typename T>
VelPlanes<T> planes(lbm_ace_ctx* c)
{
    VelPlanes<T> v;
    const int cu = c->vel.cur;
    // FIELD: one static pair; CALLBACK: u(t) in pair `cur`, u(t-1) in the other
    const int pv = c->p.velocity_kind == LBM_ACE_VEL_CALLBACK && c->t > 0 ? 1 - cu : cu;
    v.u = c->vel.pu[cu]; v.v = c->vel.pv[cu];
    v.up = c->vel.pu[pv]; v.vp = c->vel.pv[pv];
    v.nx = c->p.nx;
    return v;
}

constexpr int BULK_TX = 128;
constexpr int BULK_STAGES = 6;

// Launch with programmatic stream serialisation: the kernel may start while the previous
// kernel in the stream drains; it waits (griddepcontrol.wait) before reading the state.
template <typename... KArgs, typename... Args>
void launch_pdl_smem(void (*kernel)(KArgs...), dim3 grid, int threads, size_t smem, cudaStream_t stream,
                     Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, int threads, cudaStream_t stream, Args&&... args)
{
    launch_pdl_smem(kernel, grid, threads, 0, stream, std::forward<Args>(args)...);
}

template <typename T, int MODEL, class Vel>
void launch_step_k(lbm_ace_ctx* c, const Vel& vel)
{
    dim3 grid(c->grid_x, c->grid_y);
    if (c->variant == 2)
        ace_step_bulk<T, MODEL, Vel, BULK_TX, BULK_STAGES>
            <<<grid, BULK_TX, c->smem, c->stream>>>(make_args<T>(c), vel, c->dev_err);
    else if (c->variant == 3)
        ace_step_warp<T, MODEL, Vel><<<grid, TILE_X, 0, c->stream>>>(make_args<T>(c), vel);
    else if (c->variant == 4 || c->variant == 6) // variant 6: a lone step (odd count) is one pair step
        launch_pdl(ace_step_pair<T, MODEL, Vel>, grid, PAIR_THREADS, c->stream, make_args<T>(c), vel);
    else if (c->variant == 8) {
        if constexpr (sizeof(T) == 4)
            launch_pdl_smem(ace_step_quad<MODEL, Vel>, grid, Q32_THREADS, c->smem, c->stream, make_args<T>(c), vel);
    }
    else
        ace_step<T, MODEL, Vel><<<grid, TILE_X, 0, c->stream>>>(make_args<T>(c), vel);
}

template <typename T, int MODEL>
void launch_step_m(lbm_ace_ctx* c)
{
    switch (c->p.velocity_kind) {
    case LBM_ACE_VEL_SINGLE_VORTEX: launch_step_k<T, MODEL>(c, vortex<T>(c, (double)c->t)); break;
    case LBM_ACE_VEL_UNIFORM: {
        VelUniform<T> v; v.ux = T(c->p.ux); v.uy = T(c->p.uy);
        launch_step_k<T, MODEL>(c, v);
        break;
    }
    default: launch_step_k<T, MODEL>(c, planes<T>(c)); break;
    }
}

template <typename T>
void launch_step_t(lbm_ace_ctx* c)
{
    if (c->p.model == LBM_ACE_MODEL_MODIFIED) launch_step_m<T, MODEL_MODIFIED>(c);
    else launch_step_m<T, MODEL_CONSERVATIVE>(c);
}

template <typename S>
DevArgs<S> make_dev(lbm_ace_ctx* c)
{
    DevArgs<S> d;
    d.gin = (const unsigned short*)c->f[c->cur];
    d.gout = (unsigned short*)c->f[1 - c->cur];
    d.phin = c->phi2[c->pcur];
    d.phout = c->phi2[1 - c->pcur];
    return d;
}

template <typename S, int MODEL, class Vel>
void launch_dev_k(lbm_ace_ctx* c, const Vel& vel)
{
    dim3 grid(c->grid_x, c->grid_y);
    StepArgs<float> a = make_args<float>(c);
    if constexpr (Vel::row_uniform) { // the 4-CTA instantiation exists for these velocities only
        if (c->variant == 7 && c->dev4_ctas == 4) {
            launch_pdl_smem(ace_step_dev4<S, MODEL, Vel, 4>, grid, QUAD_THREADS, c->smem, c->stream, make_dev<S>(c), a,
                            vel);
            return;
        }
    }
    if (c->variant == 7)
        launch_pdl_smem(ace_step_dev4<S, MODEL, Vel, 3>, grid, QUAD_THREADS, c->smem, c->stream, make_dev<S>(c), a, vel);
    else
        launch_pdl(ace_step_dev<S, MODEL, Vel>, grid, PAIR_THREADS, c->stream, make_dev<S>(c), a, vel);
}

template <typename S, int MODEL>
void launch_dev_m(lbm_ace_ctx* c)
{
    switch (c->p.velocity_kind) {
    case LBM_ACE_VEL_SINGLE_VORTEX: launch_dev_k<S, MODEL>(c, vortex<float>(c, (double)c->t)); break;
    case LBM_ACE_VEL_UNIFORM: {
        VelUniform<float> v; v.ux = float(c->p.ux); v.uy = float(c->p.uy);
        launch_dev_k<S, MODEL>(c, v);
        break;
    }
    default: launch_dev_k<S, MODEL>(c, planes<float>(c)); break;
    }
}

template <typename S>
void launch_dev_s(lbm_ace_ctx* c)
{
    if (c->p.model == LBM_ACE_MODEL_MODIFIED) launch_dev_m<S, MODEL_MODIFIED>(c);
    else launch_dev_m<S, MODEL_CONSERVATIVE>(c);
}

// Two steps t -> t + 2 in one launch (variant 6, FP32): reads f[cur] and phi, writes
// f[1 - cur] and phi_alt.
template <int MODEL, class Vel>
void launch_tb2_k(lbm_ace_ctx* c, const Vel& va, const Vel& vb)
{
    StepArgs<float> a = make_args<float>(c);
    StepArgs<float> b = a;
    b.phi = (float*)c->phi_alt;
    b.first = 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c->grid_x, c->grid_y);
    cfg.blockDim = dim3(TB_THREADS);
    cfg.dynamicSmemBytes = c->smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, ace_step_tb2<MODEL, Vel>, a, b, va, vb);
}

template <int MODEL>
void launch_tb2_m(lbm_ace_ctx* c)
{
    switch (c->p.velocity_kind) {
    case LBM_ACE_VEL_SINGLE_VORTEX:
        launch_tb2_k<MODEL>(c, vortex<float>(c, (double)c->t), vortex<float>(c, (double)c->t + 1.0));
        break;
    case LBM_ACE_VEL_UNIFORM: {
        VelUniform<float> v; v.ux = float(c->p.ux); v.uy = float(c->p.uy);
        launch_tb2_k<MODEL>(c, v, v);
        break;
    }
    default: launch_tb2_k<MODEL>(c, planes<float>(c), planes<float>(c)); break;
    }
}

void launch_tb2_any(lbm_ace_ctx* c)
{
    if (c->p.model == LBM_ACE_MODEL_MODIFIED) launch_tb2_m<MODEL_MODIFIED>(c);
    else launch_tb2_m<MODEL_CONSERVATIVE>(c);
}

void launch_step_any(lbm_ace_ctx* c)
{
    switch (c->p.precision) {
    case LBM_ACE_F64: launch_step_t<double>(c); break;
    case LBM_ACE_F32: launch_step_t<float>(c); break;
    case LBM_ACE_F16DEV: launch_dev_s<__half>(c); break;
    default: launch_dev_s<__nv_bfloat16>(c); break;
    }
}

template <typename S>
void launch_init_dev(lbm_ace_ctx* c, const double* dphi0, double t0)
{
    const long long n = (long long)c->p.nx * c->p.ny;
    const int g = grid_for(n, c->sms);
    unsigned short* gs = (unsigned short*)c->f[c->cur];
    float* phi = c->phi2[c->pcur];
    switch (c->p.velocity_kind) {
    case LBM_ACE_VEL_SINGLE_VORTEX:
        ace_init_dev<S><<<g, 256, 0, c->stream>>>(dphi0, gs, phi, c->p.nx, c->p.ny, vortex<float>(c, t0));
        break;
    case LBM_ACE_VEL_UNIFORM: {
        VelUniform<float> v; v.ux = float(c->p.ux); v.uy = float(c->p.uy);
        ace_init_dev<S><<<g, 256, 0, c->stream>>>(dphi0, gs, phi, c->p.nx, c->p.ny, v);
        break;
    }
    default:
        ace_init_dev<S><<<g, 256, 0, c->stream>>>(dphi0, gs, phi, c->p.nx, c->p.ny, planes<float>(c));
        break;
    }
}

// The initial state of rows [y0, y1): the push of ace_init (f*_i(x - c_i) = f_i^eq(phi0(x),
// u(x, 0)), phi plane = phi0) on those rows, the same arithmetic node for node, plus the
// smallest index whose phi is not finite in the storage precision into *first_bad.
// Rows are independent, so the upload of phi0 can be cut into row chunks that this
// kernel initialises while the next chunk is still on its way.
template <typename T, class Vel>
__global__ void ace_init_rows(const double* __restrict__ phi0, T* __restrict__ fst, T* __restrict__ phi, int nx,
                              int ny, int y0, int y1, Vel vel, unsigned long long* first_bad)
{
    const long long plane = (long long)nx * ny;
    const long long k1 = (long long)y1 * nx;
    for (long long k = (long long)y0 * nx + blockIdx.x * (long long)blockDim.x + threadIdx.x; k < k1;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        const T ph = T(phi0[k]);
        if (!isfinite(ph)) atomicMin(first_bad, (unsigned long long)k);
        T u, v, up, vp, feq[9];
        const typename Vel::Col cl = vel.col(x);
        vel.at(cl, vel.rowv(cl, x, y), u, v, up, vp);
        equilibrium(ph, u, v, feq);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            fst[i * plane + (long long)wrap_idx(y - cy_of(i), ny) * nx + wrap_idx(x - cx_of(i), nx)] = feq[i];
        phi[k] = ph;
    }
}

template <typename T>
void launch_init_rows(lbm_ace_ctx* c, const double* dphi0, int y0, int y1, unsigned long long* first_bad)
{
    const int g = grid_for((long long)(y1 - y0) * c->p.nx, c->sms);
    T* fst = (T*)c->f[c->cur];
    T* phi = (T*)c->phi;
    const int nx = c->p.nx, ny = c->p.ny;
    switch (c->p.velocity_kind) {
    case LBM_ACE_VEL_SINGLE_VORTEX:
        ace_init_rows<T><<<g, 256, 0, c->stream>>>(dphi0, fst, phi, nx, ny, y0, y1, vortex<T>(c, 0.0), first_bad);
        break;
    case LBM_ACE_VEL_UNIFORM: {
        VelUniform<T> v; v.ux = T(c->p.ux); v.uy = T(c->p.uy);
        ace_init_rows<T><<<g, 256, 0, c->stream>>>(dphi0, fst, phi, nx, ny, y0, y1, v, first_bad);
        break;
    }
    default:
        ace_init_rows<T><<<g, 256, 0, c->stream>>>(dphi0, fst, phi, nx, ny, y0, y1, planes<T>(c), first_bad);
        break;
    }
}

template <typename T>
void launch_init_t(lbm_ace_ctx* c, const double* dphi0, double t0)
{
    const long long n = (long long)c->p.nx * c->p.ny;
    const int g = grid_for(n, c->sms);
    T* fst = (T*)c->f[c->cur];
    T* phi = (T*)c->phi;
    switch (c->p.velocity_kind) {
    case LBM_ACE_VEL_SINGLE_VORTEX:
        ace_init<T><<<g, 256, 0, c->stream>>>(dphi0, fst, phi, c->p.nx, c->p.ny, vortex<T>(c, t0));
        break;
    case LBM_ACE_VEL_UNIFORM: {
        VelUniform<T> v; v.ux = T(c->p.ux); v.uy = T(c->p.uy);
        ace_init<T><<<g, 256, 0, c->stream>>>(dphi0, fst, phi, c->p.nx, c->p.ny, v);
        break;
    }
    default:
        ace_init<T><<<g, 256, 0, c->stream>>>(dphi0, fst, phi, c->p.nx, c->p.ny, planes<T>(c));
        break;
    }
}

// The four single-vortex tables (sx2, s2x over x; sy2, s2y over y) sit back to back in one
// block of the context's allocation, each padded to 256 bytes.
size_t pad256(size_t b) { return (b + 255) & ~size_t(255); }
size_t vortex_table_bytes(int nx, int ny, size_t elem) { return 2 * pad256(nx * elem) + 2 * pad256(ny * elem); }

// Fill the tables at c->vel.sx2 (a block of vortex_table_bytes) with one copy from the host.
template <typename T>
int fill_vortex_tables(lbm_ace_ctx* c)
{
    const int nx = c->p.nx, ny = c->p.ny;
    const size_t ox = pad256(nx * sizeof(T)) / sizeof(T), oy = pad256(ny * sizeof(T)) / sizeof(T);
    std::vector<T> h(vortex_table_bytes(nx, ny, sizeof(T)) / sizeof(T), T(0));
    T* sx2 = h.data(); T* s2x = sx2 + ox; T* sy2 = s2x + ox; T* s2y = sy2 + oy;
    for (int x = 0; x < nx; ++x) {
        const double s = std::sin(kPi * x / nx);
        sx2[x] = T(s * s);
        s2x[x] = T(std::sin(2.0 * kPi * x / nx));
    }
    if (ny == nx) { // the same expressions of the same arguments
        std::copy(sx2, sx2 + nx, sy2);
        std::copy(s2x, s2x + nx, s2y);
    } else {
        for (int y = 0; y < ny; ++y) {
            const double s = std::sin(kPi * y / ny);
            sy2[y] = T(s * s);
            s2y[y] = T(std::sin(2.0 * kPi * y / ny));
        }
    }
    T* d = static_cast<T*>(c->vel.sx2);
    c->vel.s2x = d + ox;
    c->vel.sy2 = d + 2 * ox;
    c->vel.s2y = d + 2 * ox + oy;
    // pageable source: the copy has staged its bytes when it returns
    CK(c, cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return LBM_ACE_OK;
}

// Offsets of a context's fixed buffers inside its one pool allocation, each 256-byte
// aligned: one cudaMallocFromPoolAsync costs about 7 us of host time on GB300, and
// creating a lattice took ten of them.
struct Carve {
    std::vector<std::function<void(char*)>> set;
    size_t total = 0;
    template <typename P>
    void add(P** ptr, size_t bytes)
    {
        const size_t off = total;
        set.push_back([ptr, off](char* base) { *ptr = reinterpret_cast<P*>(base + off); });
        total += pad256(bytes);
    }
    void assign(void* base) const
    {
        for (const auto& f : set) f(static_cast<char*>(base));
    }
};

// Occupancy (resident CTAs per SM) of the chosen step kernel; opts the bulk kernel
// into its dynamic shared memory.
template <typename T, int MODEL, class Vel>
int occupancy_k(lbm_ace_ctx* c, int* blocks)
{
    if (c->variant == 2) {
        auto k = ace_step_bulk<T, MODEL, Vel, BULK_TX, BULK_STAGES>;
        c->smem = sizeof(BulkSmem<T, BULK_TX, BULK_STAGES>);
        c->tile_x = BULK_TX;
        CK(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem));
        CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, BULK_TX, c->smem));
    } else if (c->variant == 3) {
        c->smem = 0;
        c->tile_x = TILE_X;
        CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, ace_step_warp<T, MODEL, Vel>, TILE_X, 0));
    } else if (c->variant == 4) {
        c->smem = 0;
        c->tile_x = PAIR_COLS;
        CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, ace_step_pair<T, MODEL, Vel>, PAIR_THREADS, 0));
    } else if (c->variant == 8) {
        if constexpr (sizeof(T) == 4) {
            auto k = ace_step_quad<MODEL, Vel>;
            c->smem = sizeof(Quad32Smem);
            c->tile_x = Q32_COLS;
            CK(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem));
            CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, Q32_THREADS, c->smem));
        } else {
            return fail(c, LBM_ACE_EINVAL, "kernel_variant 8 is FP32 only");
        }
    } else if (c->variant == 6) {
        if constexpr (sizeof(T) == 4) {
            auto k = ace_step_tb2<MODEL, Vel>;
            c->smem = sizeof(TbSmem);
            c->tile_x = TB_COLS;
            CK(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem));
            CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, TB_THREADS, c->smem));
        } else {
            return fail(c, LBM_ACE_EINVAL, "kernel_variant 6 is FP32 only");
        }
    } else {
        c->smem = 0;
        c->tile_x = TILE_X;
        CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, ace_step<T, MODEL, Vel>, TILE_X, 0));
    }
    return LBM_ACE_OK;
}

template <typename T, int MODEL>
int occupancy_m(lbm_ace_ctx* c, int* blocks)
{
    switch (c->p.velocity_kind) {
    case LBM_ACE_VEL_SINGLE_VORTEX: return occupancy_k<T, MODEL, VelVortex<T>>(c, blocks);
    case LBM_ACE_VEL_UNIFORM: return occupancy_k<T, MODEL, VelUniform<T>>(c, blocks);
    default: return occupancy_k<T, MODEL, VelPlanes<T>>(c, blocks);
    }
}

template <typename S, int MODEL, class Vel>
int occupancy_dev_k(lbm_ace_ctx* c, int* blocks)
{
    if (c->variant == 7) {
        // 4 CTAs/SM above 2^23 nodes (measured faster at 4096^2), 3 below (faster at 2048^2);
        // velocity planes (per-node loads) always 3: at the 128-register cap of 4 CTAs/SM
        // that instantiation spills
        c->dev4_ctas = Vel::row_uniform && (long long)c->p.nx * c->p.ny > (1LL << 23) ? 4 : 3;
        auto k = ace_step_dev4<S, MODEL, Vel, 3>;
        if constexpr (Vel::row_uniform)
            if (c->dev4_ctas == 4) k = ace_step_dev4<S, MODEL, Vel, 4>;
        c->smem = sizeof(QuadSmem);
        c->tile_x = QUAD_COLS;
        CK(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem));
        CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, QUAD_THREADS, c->smem));
        return LBM_ACE_OK;
    }
    c->smem = 0;
    c->tile_x = PAIR_COLS;
    CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, ace_step_dev<S, MODEL, Vel>, PAIR_THREADS, 0));
    return LBM_ACE_OK;
}

template <typename S, int MODEL>
int occupancy_dev_m(lbm_ace_ctx* c, int* blocks)
{
    switch (c->p.velocity_kind) {
    case LBM_ACE_VEL_SINGLE_VORTEX: return occupancy_dev_k<S, MODEL, VelVortex<float>>(c, blocks);
    case LBM_ACE_VEL_UNIFORM: return occupancy_dev_k<S, MODEL, VelUniform<float>>(c, blocks);
    default: return occupancy_dev_k<S, MODEL, VelPlanes<float>>(c, blocks);
    }
}

template <typename S>
int occupancy_dev(lbm_ace_ctx* c, int* blocks)
{
    return c->p.model == LBM_ACE_MODEL_MODIFIED ? occupancy_dev_m<S, MODEL_MODIFIED>(c, blocks)
                                                : occupancy_dev_m<S, MODEL_CONSERVATIVE>(c, blocks);
}

template <typename T>
int occupancy_t(lbm_ace_ctx* c, int* blocks)
{
    return c->p.model == LBM_ACE_MODEL_MODIFIED ? occupancy_m<T, MODEL_MODIFIED>(c, blocks)
                                                : occupancy_m<T, MODEL_CONSERVATIVE>(c, blocks);
}

bool is_f64(const lbm_ace_ctx* c) { return c->p.precision == LBM_ACE_F64; }
bool is_dev(const lbm_ace_ctx* c) { return c->p.precision == LBM_ACE_F16DEV || c->p.precision == LBM_ACE_BF16DEV; }

int ensure_scratch(lbm_ace_ctx* c, size_t elems)
{
    if (c->scratch_elems >= elems) return LBM_ACE_OK;
    if (c->scratch) cudaFreeAsync(c->scratch, c->stream);
    c->scratch = nullptr;
    c->scratch_elems = 0;
    PA(c, &c->scratch, elems * sizeof(double));
    c->scratch_elems = elems;
    return LBM_ACE_OK;
}

// Velocity planes for time t from the host callback into pair `pair`.
int callback_upload(lbm_ace_ctx* c, double t, int pair)
{
    const size_t n = (size_t)c->p.nx * c->p.ny;
    const int rc = c->p.vel_fn(t, c->p.nx, c->p.ny, c->vel.hu.data(), c->vel.hv.data(), c->p.vel_user);
    if (rc != 0) return fail(c, LBM_ACE_ECALLBACK, "velocity callback returned %d at t = %g", rc, t);
    CK(c, cudaMemcpyAsync(c->vel.pu[pair], c->vel.hu.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->vel.pv[pair], c->vel.hv.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    // the pageable source is staged before return, but keep the host buffer stable
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_ACE_OK;
}

int check_device_error(lbm_ace_ctx* c);

// The device address of the host range [p, p + bytes) when the range is page-locked host
// memory (cudaHostAlloc, cudaMallocHost or cudaHostRegister; with unified addressing such
// memory is mapped for every device), checked at its first and last byte; nullptr for
// pageable or device memory, which the callers copy through cudaMemcpyAsync instead.
const void* mapped_host(const void* p, size_t bytes)
{
    if (!p || bytes == 0) return nullptr;
    const char* q = static_cast<const char*>(p);
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, q) != cudaSuccess || cudaPointerGetAttributes(&b, q + bytes - 1) != cudaSuccess) {
        (void)cudaGetLastError(); // clear the query's own error
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    if (static_cast<const char*>(b.devicePointer) - static_cast<const char*>(a.devicePointer) != (ptrdiff_t)(bytes - 1))
        return nullptr;
    return a.devicePointer;
}

// The sum and the wait-failure flag, which the finishing kernel wrote to the mapped host
// block (write_result): no copy, only the stream synchronisation.
int fetch_result(lbm_ace_ctx* c, double* out)
{
    CK(c, cudaGetLastError());
    CK(c, cudaStreamSynchronize(c->stream));
    const double* back = c->hres;
    if (back[1] != 0.0) {
        CK(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        return fail(c, LBM_ACE_ETIMEOUT, "a bounded wait in the step kernel gave up; the state is not valid");
    }
    *out = back[0];
    return LBM_ACE_OK;
}

int finalize_sum(lbm_ace_ctx* c, const double* part, int n, double* out)
{
    ace_finalize<<<1, RED_THREADS, 0, c->stream>>>(part, n, c->hres_dev, c->dev_err);
    return fetch_result(c, out);
}

// After a stream synchronisation: report (and clear) a bounded wait that gave up.
int check_device_error(lbm_ace_ctx* c)
{
    int e = 0;
    CK(c, cudaMemcpyAsync(&e, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (e) {
        CK(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        return fail(c, LBM_ACE_ETIMEOUT, "a bounded wait in the step kernel gave up; the state is not valid");
    }
    return LBM_ACE_OK;
}

// One CTA waits, with the step kernels' bounded wait, for an mbarrier nobody arrives on;
// when the wait gives up it sets *err as a step kernel would (1), otherwise 0 is kept.
__global__ void ace_wait_selftest(long long limit_cycles, int* err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit_cycles)) atomicExch(err, 1);
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) { if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d); else prev = -1; }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

// phi(x, t) of the current state as FP64 into dst (device memory, or the mapped address
// of page-locked host memory), on the context's stream.
int phi_to(lbm_ace_ctx* c, double* dst)
{
    const size_t n = (size_t)c->p.nx * c->p.ny;
    const int gr = grid_for((long long)n, c->sms);
    const unsigned short* gs = (const unsigned short*)c->f[c->cur];
    switch (c->p.precision) {
    case LBM_ACE_F64: ace_moment<double><<<gr, 256, 0, c->stream>>>((const double*)c->f[c->cur], dst, c->p.nx, c->p.ny); break;
    case LBM_ACE_F32: ace_moment<float><<<gr, 256, 0, c->stream>>>((const float*)c->f[c->cur], dst, c->p.nx, c->p.ny); break;
    case LBM_ACE_F16DEV:
        ace_pull_state_dev<__half><<<gr, 256, 0, c->stream>>>(gs, c->phi2[c->pcur], nullptr, dst, nullptr, c->p.nx, c->p.ny);
        break;
    default:
        ace_pull_state_dev<__nv_bfloat16><<<gr, 256, 0, c->stream>>>(gs, c->phi2[c->pcur], nullptr, dst, nullptr,
                                                                     c->p.nx, c->p.ny);
        break;
    }
    CK(c, cudaGetLastError());
    return LBM_ACE_OK;
}

// phi(x, t) into c->scratch (FP64).
int phi_to_scratch(lbm_ace_ctx* c)
{
    const int rc = ensure_scratch(c, (size_t)c->p.nx * c->p.ny);
    return rc ? rc : phi_to(c, c->scratch);
}

// Smallest index k with v[k] not finite, into *first (which starts at ULLONG_MAX).
template <typename T>
__global__ void ace_first_nonfinite(const T* __restrict__ v, long long n, unsigned long long* first)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        if (!isfinite(v[k])) atomicMin(first, (unsigned long long)k);
}

__global__ void ace_narrow(const double* __restrict__ in, float* __restrict__ out, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        out[k] = (float)in[k];
}

__global__ void ace_widen(const float* __restrict__ in, double* __restrict__ out, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        out[k] = (double)in[k];
}

// u(x, t), v(x, t) of a velocity source, rounded to FP32.
template <typename T, class Vel>
__global__ void ace_velocity(Vel vel, int nx, int ny, float* __restrict__ u_out, float* __restrict__ v_out)
{
    // launched with programmatic stream serialisation (its launch and ramp overlap the
    // previous kernel); it writes only after that kernel has finished
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    const long long plane = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < plane;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        T u, v, up, vp;
        const typename Vel::Col cl = vel.col(x);
        vel.at(cl, vel.rowv(cl, x, y), u, v, up, vp);
        u_out[k] = (float)u;
        v_out[k] = (float)v;
    }
}

} // namespace

extern "C" {

int lbm_ace_params_default(lbm_ace_params* p)
{
    if (!p) return fail(nullptr, LBM_ACE_EINVAL, "params is NULL");
    std::memset(p, 0, sizeof *p);
    p->nx = p->ny = 64;
    p->tau = 0.8;
    p->M = -1.0;
    p->eps = 1.0;
    p->reg_delta = 0.0;
    p->precision = LBM_ACE_F64;
    p->model = LBM_ACE_MODEL_MODIFIED;
    p->velocity_kind = LBM_ACE_VEL_SINGLE_VORTEX;
    p->U0 = 0.04;
    p->T_period = 2000.0;
    p->vortex_sign = -1.0;
    p->xc = 32.0; p->yc = 48.0; p->R = 9.6;
    return LBM_ACE_OK;
}

const char* lbm_ace_status_string(int s)
{
    switch (s) {
    case LBM_ACE_OK: return "ok";
    case LBM_ACE_EINVAL: return "invalid argument";
    case LBM_ACE_ENOMEM: return "out of memory";
    case LBM_ACE_ECUDA: return "CUDA error";
    case LBM_ACE_ENUMERIC: return "non-finite values";
    case LBM_ACE_ETIMEOUT: return "device wait timed out";
    case LBM_ACE_ECALLBACK: return "velocity callback failed";
    default: return "unknown status";
    }
}

const char* lbm_ace_last_error(const lbm_ace_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

long long lbm_ace_steps_done(const lbm_ace_ctx* c) { return c ? c->t : -1; }

void lbm_ace_destroy(lbm_ace_ctx* c)
{
    if (!c) return;
    DeviceGuard g(c->dev);
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    if (c->upload) cudaStreamSynchronize(c->upload); // a creation that failed half-way
    for (void* b : {c->arena, static_cast<void*>(c->scratch)})
        if (b) cudaFreeAsync(b, c->stream); // back to the device's pool
    if (c->slot.host) release_slot(c->slot);
    delete c;
}

static int init_impl(lbm_ace_ctx* c, const lbm_ace_params* p)
{
    c->p = *p;
    if (c->p.reg_delta == 0.0) c->p.reg_delta = std::exp(-20.0);
    c->dev = p->device;
    c->stream = (cudaStream_t)p->stream;
    CK(c, cudaSetDevice(c->dev));
    CK(c, cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev));
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny;
    c->elem = is_f64(c) ? sizeof(double) : (is_dev(c) ? 2 : sizeof(float));

    // kernel variant, automatic choice measured on GB300 (FP32): four columns per thread in warp strips
    // up to 2^23 nodes (1024^2: 71k against 67k MLUPS for column pairs; 2048^2: 80k against
    // 79k), column pairs above (4096^2: 82k against 80k), direct loads for odd nx; FP64:
    // column pairs for even nx
    if (p->kernel_variant != 0)
        c->variant = p->kernel_variant;
    else if (p->precision == LBM_ACE_F32 && nx % 4 == 0 && (long long)nx * ny <= (1LL << 23))
        c->variant = 8;
    else
        c->variant = nx % 2 == 0 ? 4 : 1;
    // the deviation-storage kernels: four columns per thread when nx allows, else pairs
    if (is_dev(c)) c->variant = p->kernel_variant != 0 ? p->kernel_variant : (nx % 4 == 0 ? 7 : 5);
    // L2 priority of the stores (StepArgs::l2_keep, ace_kernels.cuh): the FP32 and 16-bit
    // kernels keep the phi plane they store when it takes at most 0.6 of the L2 (measured
    // on GB300, us per step: FP32 quads at 2048^2 51.7 -> 47.8, FP32 column pairs at 4096^2
    // 204.5 -> 200.0, 16-bit quads 151.3 -> 150.0 at 4096^2 and 42.6 -> 41.9 at 2048^2).
    // L2_KEEP_F (a quarter of the f* lines) is not set: alone it helped from 1536^2 to
    // 2560^2, but beside the kept phi plane it competes for the same lines and was slower
    // (2048^2: 49.9 against 47.8 us; 2560^2: 80.2 against 74.3).
    {
        int l2 = 0;
        CK(c, cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->dev));
        c->l2_keep = 0;
        if (!is_f64(c) && l2 > 0 && 4.0 * (double)n <= 0.6 * l2) c->l2_keep |= L2_KEEP_PHI;
    }

    // launch shape of the fused step: one wave of resident CTAs when possible
    int occ = 0;
    int rc;
    switch (p->precision) {
    case LBM_ACE_F64: rc = occupancy_t<double>(c, &occ); break;
    case LBM_ACE_F32: rc = occupancy_t<float>(c, &occ); break;
    case LBM_ACE_F16DEV: rc = occupancy_dev<__half>(c, &occ); break;
    default: rc = occupancy_dev<__nv_bfloat16>(c, &occ); break;
    }
    if (rc) return rc;
    if (occ < 1) occ = 1;
    c->grid_x = (nx + c->tile_x - 1) / c->tile_x;
    int rows = p->rows_per_cta;
    if (rows <= 0) {
        // one wave: at most `slots` resident CTAs, so at most slots / grid_x row bands
        const long long slots = (long long)c->sms * occ;
        long long bands = slots / c->grid_x;
        if (bands < 1) bands = 1;
        long long r = (ny + bands - 1) / bands;
        if (r < 4) r = 4;
        rows = (int)r;
    }
    if (rows > ny) rows = ny;
    // the integer part of the quad kernels' mass partials is exact for bands of at most
    // 4095 rows (four values below 2 per thread and row)
    const int max_rows = (c->variant == 7 || c->variant == 8) ? 4095 : ny;
    if (rows > max_rows) {
        if (p->rows_per_cta > 0)
            return fail(c, LBM_ACE_EINVAL, "rows_per_cta %d: kernel variant %d takes at most %d rows per CTA",
                        p->rows_per_cta, c->variant, max_rows);
        rows = max_rows;
    }
    c->rows = rows;
    c->grid_y = (ny + rows - 1) / rows;
    c->n_step_part = c->grid_x * c->grid_y;
    // global mass: FP64 states by the compensated grid-stride kernel, the others by the
    // fused kernels sized to one wave of resident CTAs (FP32: 4 CTAs/SM of the 6 that
    // fit, measured 35.0 against 36.9 us at 2048^2; 16-bit: all that fit)
    {
        int rocc = 0;
        if (p->precision == LBM_ACE_F32) {
            CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rocc, ace_sum_partials_f32, RED_THREADS, 0));
            rocc = std::min(rocc, 4);
        }
        else if (p->precision == LBM_ACE_F16DEV)
            CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rocc, ace_sum_partials_dev<__half>, RED_THREADS, 0));
        else if (p->precision == LBM_ACE_BF16DEV)
            CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rocc, ace_sum_partials_dev<__nv_bfloat16>, RED_THREADS, 0));
        c->n_red_part = p->precision == LBM_ACE_F64 ? grid_for(9 * (long long)n, c->sms)
                                                    : mass_reduction_grid(c->sms, rocc, 10 * (long long)n);
    }

    // every fixed buffer of the context in one allocation from the device's pool
    const int pairs = p->velocity_kind == LBM_ACE_VEL_CALLBACK ? 2 : p->velocity_kind == LBM_ACE_VEL_FIELD ? 1 : 0;
    {
        Carve cv;
        cv.add(&c->f[0], 9 * n * c->elem);
        cv.add(&c->f[1], 9 * n * c->elem);
        if (is_dev(c)) {
            cv.add(&c->phi2[0], n * sizeof(float));
            cv.add(&c->phi2[1], n * sizeof(float));
        } else {
            cv.add(&c->phi, n * c->elem);
        }
        if (c->variant == 6) cv.add(&c->phi_alt, n * sizeof(float));
        // result block: the reduced sum, a spare double, the device wait-failure flag, and
        // the ticket counter of the mass reductions that finish in their last CTA
        cv.add(&c->result, 4 * sizeof(double));
        cv.add(&c->step_part, c->n_step_part * sizeof(double));
        cv.add(&c->red_part, c->n_red_part * sizeof(double));
        if (p->velocity_kind == LBM_ACE_VEL_SINGLE_VORTEX) // FP32 tables for 16-bit storage
            cv.add(&c->vel.sx2, vortex_table_bytes(nx, ny, is_f64(c) ? sizeof(double) : sizeof(float)));
        for (int k = 0; k < pairs; ++k) {
            cv.add(&c->vel.pu[k], n * sizeof(double));
            cv.add(&c->vel.pv[k], n * sizeof(double));
        }
        PA(c, &c->arena, cv.total);
        cv.assign(c->arena);
    }
    c->dev_err = reinterpret_cast<int*>(c->result + 2);
    CK(c, cudaMemsetAsync(c->result, 0, 4 * sizeof(double), c->stream));
    CK(c, acquire_slot(&c->slot));
    c->hres = c->slot.host;
    c->hres_dev = c->slot.dev;

    // initial phi first: its upload (asynchronous from page-locked memory) runs while the
    // host computes the velocity tables below. For a large FP64 or FP32 lattice it goes in
    // kChunks row chunks on a second stream, each followed by an event on which the
    // context's stream waits before it initialises that chunk, so the init kernel works
    // under the upload of the next chunk (the 16-bit init reads phi0 around each node and
    // takes it whole).
    rc = ensure_scratch(c, n);
    if (rc) return rc;
    constexpr int kChunks = 4;
    const bool chunked = p->phi0 && !is_dev(c) && n >= (size_t(1) << 20) && ny >= kChunks;
    struct Events { // released on every return
        cudaEvent_t e[kChunks + 1] = {};
        ~Events() { for (cudaEvent_t x : e) if (x) cudaEventDestroy(x); }
    } ev;
    auto chunk_row = [&](int k) { return (int)((long long)ny * k / kChunks); };
    if (chunked) {
        cudaStream_t aux;
        CK(c, aux_stream(c->dev, &aux));
        for (cudaEvent_t& x : ev.e) CK(c, cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
        CK(c, cudaEventRecord(ev.e[0], c->stream)); // the scratch buffer is allocated on c->stream
        CK(c, cudaStreamWaitEvent(aux, ev.e[0], 0));
        c->upload = aux;
        for (int k = 0; k < kChunks; ++k) {
            const size_t o = (size_t)chunk_row(k) * nx, m = (size_t)(chunk_row(k + 1) - chunk_row(k)) * nx;
            CK(c, cudaMemcpyAsync(c->scratch + o, p->phi0 + o, m * sizeof(double), cudaMemcpyHostToDevice, aux));
            CK(c, cudaEventRecord(ev.e[k + 1], aux));
        }
    } else if (p->phi0) {
        CK(c, cudaMemcpyAsync(c->scratch, p->phi0, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    }

    // velocity
    if (p->velocity_kind == LBM_ACE_VEL_SINGLE_VORTEX) {
        rc = is_f64(c) ? fill_vortex_tables<double>(c) : fill_vortex_tables<float>(c);
        if (rc) return rc;
    } else if (pairs > 0) {
        if (pairs == 1) {
            // the caller's arrays are read by the time init returns (it ends synchronised)
            CK(c, cudaMemcpyAsync(c->vel.pu[0], p->u_field, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            CK(c, cudaMemcpyAsync(c->vel.pv[0], p->v_field, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        } else {
            c->vel.hu.assign(n, 0.0);
            c->vel.hv.assign(n, 0.0);
            c->vel.cur = 0;
            rc = callback_upload(c, 0.0, 0);
            if (rc) return rc;
        }
    }

    // without phi0: the disk, built on the host
    const double* src = c->scratch;
    if (!p->phi0) {
        std::vector<double> h(n);
        auto disk_rows = [&](int ya, int yb) {
            for (int y = ya; y < yb; ++y)
                for (int x = 0; x < nx; ++x) {
                    const double r = std::sqrt((x - p->xc) * (x - p->xc) + (y - p->yc) * (y - p->yc));
                    h[(size_t)y * nx + x] = 0.5 * (1.0 + std::tanh((p->R - r) / (2.0 * p->eps)));
                }
        };
        // row bands on host threads for large lattices (one Grace core takes 26 ms for
        // 2048^2); every value is the same expression whichever thread computes it
        const unsigned hw = std::thread::hardware_concurrency();
        const int nt = n >= (size_t(1) << 18) ? (int)std::min(16u, std::max(1u, hw)) : 1;
        std::vector<std::thread> pool;
        const int own = (int)((long long)ny / nt); // rows [0, own) are this thread's
        int start = own;                           // the first row no thread has taken
        try {
            for (int k = 1; k < nt; ++k) {
                const int yb = (int)((long long)ny * (k + 1) / nt);
                pool.emplace_back(disk_rows, start, yb);
                start = yb;
            }
        } catch (...) { // no further thread to be had: the rest on this one
        }
        disk_rows(0, own);
        disk_rows(start, ny); // empty when every band got its thread
        for (auto& t : pool) t.join();
        CK(c, cudaMemcpyAsync(c->scratch, h.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    c->cur = 0;
    c->t = 0;
    c->pcur = 0;
    if (chunked) { // each chunk once its rows are on the device; phi0 checked on the way
        unsigned long long* first_bad = reinterpret_cast<unsigned long long*>(c->result + 1);
        CK(c, cudaMemsetAsync(first_bad, 0xff, sizeof(unsigned long long), c->stream));
        for (int k = 0; k < kChunks; ++k) {
            CK(c, cudaStreamWaitEvent(c->stream, ev.e[k + 1], 0));
            if (is_f64(c)) launch_init_rows<double>(c, src, chunk_row(k), chunk_row(k + 1), first_bad);
            else launch_init_rows<float>(c, src, chunk_row(k), chunk_row(k + 1), first_bad);
        }
        c->fresh = true;
        CK(c, cudaGetLastError());
        unsigned long long* hbad = reinterpret_cast<unsigned long long*>(c->hres + 4);
        CK(c, cudaMemcpyAsync(hbad, first_bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaMemsetAsync(first_bad, 0, sizeof(unsigned long long), c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        c->upload = nullptr; // the stream waited for every chunk's copy
        const unsigned long long bad = *hbad;
        if (bad != ~0ULL)
            return fail(c, LBM_ACE_EINVAL, is_f64(c) ? "phi0[%llu] is not finite" : "phi0[%llu] is not finite as FP32", bad);
        return LBM_ACE_OK;
    }
    switch (p->precision) {
    case LBM_ACE_F64: launch_init_t<double>(c, src, 0.0); break;
    case LBM_ACE_F32: launch_init_t<float>(c, src, 0.0); break;
    case LBM_ACE_F16DEV: launch_init_dev<__half>(c, src, 0.0); break;
    default: launch_init_dev<__nv_bfloat16>(c, src, 0.0); break;
    }
    c->fresh = true;
    CK(c, cudaGetLastError());
    // a large phi0 is checked where it now is, in the phi plane the init wrote in the
    // storage precision (smaller ones were checked on the host before any device work)
    if (p->phi0 && n > kHostCheckMax) {
        unsigned long long* first_bad = reinterpret_cast<unsigned long long*>(c->result + 1);
        CK(c, cudaMemsetAsync(first_bad, 0xff, sizeof(unsigned long long), c->stream));
        const int gr = grid_for((long long)n, c->sms);
        if (is_f64(c))
            ace_first_nonfinite<double><<<gr, 256, 0, c->stream>>>((const double*)c->phi, (long long)n, first_bad);
        else
            ace_first_nonfinite<float><<<gr, 256, 0, c->stream>>>(is_dev(c) ? c->phi2[c->pcur] : (const float*)c->phi,
                                                                (long long)n, first_bad);
        CK(c, cudaGetLastError());
        // read back into the context's page-locked result slot (an asynchronous copy; a
        // pageable destination would add a synchronisation of its own)
        unsigned long long* hbad = reinterpret_cast<unsigned long long*>(c->hres + 4);
        CK(c, cudaMemcpyAsync(hbad, first_bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaMemsetAsync(first_bad, 0, sizeof(unsigned long long), c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        const unsigned long long bad = *hbad;
        if (bad != ~0ULL)
            return fail(c, LBM_ACE_EINVAL, is_f64(c) ? "phi0[%llu] is not finite" : "phi0[%llu] is not finite as FP32", bad);
        return LBM_ACE_OK;
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_ACE_OK;
}

int lbm_ace_init(const lbm_ace_params* p, lbm_ace_ctx** out)
{
    if (!out) return fail(nullptr, LBM_ACE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, LBM_ACE_EINVAL, "params is NULL");
    if (p->nx < 3 || p->ny < 3) return fail(nullptr, LBM_ACE_EINVAL, "lattice %d x %d: each side must be >= 3", p->nx, p->ny);
    if ((long long)p->nx * p->ny > (1LL << 31) / 9) return fail(nullptr, LBM_ACE_EINVAL, "lattice %d x %d too large", p->nx, p->ny);
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return fail(nullptr, LBM_ACE_EINVAL, "tau = %g: must be > 0.5", p->tau);
    if (!(p->eps > 0.0) || !std::isfinite(p->eps)) return fail(nullptr, LBM_ACE_EINVAL, "eps = %g: must be > 0", p->eps);
    if (p->reg_delta < 0.0 || !std::isfinite(p->reg_delta)) return fail(nullptr, LBM_ACE_EINVAL, "reg_delta = %g: must be >= 0", p->reg_delta);
    if (p->M >= 0.0) {
        const double m = (p->tau - 0.5) / 3.0;
        if (std::fabs(p->M - m) > 1e-12 * m)
            return fail(nullptr, LBM_ACE_EINVAL, "M = %.17g differs from c_s^2 (tau - 0.5) = %.17g", p->M, m);
    }
    if (p->precision < LBM_ACE_F64 || p->precision > LBM_ACE_BF16DEV)
        return fail(nullptr, LBM_ACE_EINVAL, "precision %d unknown", p->precision);
    if ((p->precision == LBM_ACE_F16DEV || p->precision == LBM_ACE_BF16DEV) && p->nx % 2 != 0)
        return fail(nullptr, LBM_ACE_EINVAL, "16-bit deviation storage needs an even nx (nx = %d)", p->nx);
    const bool dev16 = p->precision == LBM_ACE_F16DEV || p->precision == LBM_ACE_BF16DEV;
    if (dev16 && p->kernel_variant != 0 && p->kernel_variant != 5 && p->kernel_variant != 7)
        return fail(nullptr, LBM_ACE_EINVAL, "16-bit deviation storage takes kernel_variant 0, 5 or 7 (got %d)",
                    p->kernel_variant);
    if (dev16 && p->kernel_variant == 7 && p->nx % 4 != 0)
        return fail(nullptr, LBM_ACE_EINVAL, "kernel_variant 7 needs nx a multiple of 4 (nx = %d)", p->nx);
    if (!dev16 && (p->kernel_variant == 5 || p->kernel_variant == 7))
        return fail(nullptr, LBM_ACE_EINVAL, "kernel_variant %d is for the 16-bit deviation storage", p->kernel_variant);
    if (p->model != LBM_ACE_MODEL_MODIFIED && p->model != LBM_ACE_MODEL_CONSERVATIVE)
        return fail(nullptr, LBM_ACE_EINVAL, "model %d unknown", p->model);
    switch (p->velocity_kind) {
    case LBM_ACE_VEL_SINGLE_VORTEX:
        if (!(p->T_period > 0.0) || !std::isfinite(p->U0) || !std::isfinite(p->vortex_sign))
            return fail(nullptr, LBM_ACE_EINVAL, "single vortex needs T_period > 0 and finite U0, vortex_sign");
        break;
    case LBM_ACE_VEL_UNIFORM:
        if (!std::isfinite(p->ux) || !std::isfinite(p->uy)) return fail(nullptr, LBM_ACE_EINVAL, "uniform velocity not finite");
        break;
    case LBM_ACE_VEL_FIELD:
        if (!p->u_field || !p->v_field) return fail(nullptr, LBM_ACE_EINVAL, "velocity field arrays are NULL");
        break;
    case LBM_ACE_VEL_CALLBACK:
        if (!p->vel_fn) return fail(nullptr, LBM_ACE_EINVAL, "velocity callback is NULL");
        break;
    default: return fail(nullptr, LBM_ACE_EINVAL, "velocity kind %d unknown", p->velocity_kind);
    }
    if (p->phi0 && (size_t)p->nx * p->ny <= kHostCheckMax) { // larger fields are checked on the device
        const size_t n = (size_t)p->nx * p->ny;
        // the FP32-based forms keep phi in FP32: a value must also round to a finite FP32
        // (magnitude below 2^128 - 2^103; round to nearest takes the midpoint up to infinity)
        const bool f64 = p->precision == LBM_ACE_F64;
        for (size_t k = 0; k < n; ++k) {
            if (!std::isfinite(p->phi0[k]))
                return fail(nullptr, LBM_ACE_EINVAL, "phi0[%zu] is not finite", k);
            if (!f64 && !(std::fabs(p->phi0[k]) < 0x1p128 - 0x1p103))
                return fail(nullptr, LBM_ACE_EINVAL, "phi0[%zu] is not finite as FP32", k);
        }
    } else if (!p->phi0 && (!std::isfinite(p->xc) || !std::isfinite(p->yc) || !std::isfinite(p->R))) {
        return fail(nullptr, LBM_ACE_EINVAL, "disk centre/radius not finite");
    }
    if (p->rows_per_cta < 0) return fail(nullptr, LBM_ACE_EINVAL, "rows_per_cta must be >= 0");
    if (p->kernel_variant < 0 || p->kernel_variant > 8)
        return fail(nullptr, LBM_ACE_EINVAL, "kernel_variant %d unknown", p->kernel_variant);
    if (p->kernel_variant == 8 && (p->precision != LBM_ACE_F32 || p->nx % 4 != 0))
        return fail(nullptr, LBM_ACE_EINVAL, "kernel_variant 8 needs FP32 and nx a multiple of 4 (nx = %d)", p->nx);
    if (p->kernel_variant == 6 && (p->precision != LBM_ACE_F32 || p->nx % 2 != 0 ||
                                   p->velocity_kind == LBM_ACE_VEL_CALLBACK))
        return fail(nullptr, LBM_ACE_EINVAL,
                    "kernel_variant 6 needs FP32, an even nx and a vortex, uniform or field velocity");
    if (p->kernel_variant == 4 && p->nx % 2 != 0)
        return fail(nullptr, LBM_ACE_EINVAL, "kernel_variant 4 needs an even nx (nx = %d)", p->nx);
    if (p->kernel_variant == 2) {
        const size_t elem = p->precision == LBM_ACE_F64 ? 8 : 4;
        if (((size_t)p->nx * elem) % 16 != 0)
            return fail(nullptr, LBM_ACE_EINVAL, "kernel_variant 2 needs nx * %zu bytes to be a multiple of 16 (nx = %d)",
                        elem, p->nx);
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || p->device < 0 || p->device >= ndev)
        return fail(nullptr, LBM_ACE_ECUDA, "CUDA device %d unavailable (%s)", p->device,
                    e == cudaSuccess ? "ordinal out of range" : cudaGetErrorString(e));

    lbm_ace_ctx* c = new (std::nothrow) lbm_ace_ctx;
    if (!c) return fail(nullptr, LBM_ACE_ENOMEM, "host allocation failed");
    DeviceGuard g(p->device);
    const int rc = init_impl(c, p);
    if (rc != LBM_ACE_OK) {
        g_err = c->err;
        lbm_ace_destroy(c);
        return rc;
    }
    *out = c;
    return LBM_ACE_OK;
}

int lbm_ace_step(lbm_ace_ctx* c, long long n)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    if (n < 0) return fail(c, LBM_ACE_EINVAL, "n = %lld: must be >= 0", n);
    DeviceGuard g(c->dev);
    for (long long s = 0; s < n; ++s) {
        if (c->variant == 6 && n - s >= 2) { // two steps in one launch
            launch_tb2_any(c);
            CK(c, cudaGetLastError());
            c->cur = 1 - c->cur;
            std::swap(c->phi, c->phi_alt);
            c->t += 2;
            c->stepped = true;
            c->fresh = false;
            ++s;
            continue;
        }
        if (c->p.velocity_kind == LBM_ACE_VEL_CALLBACK && c->t > 0) {
            // u(t) into the pair that held u(t-2); the pair with u(t-1) becomes "previous"
            const int next = 1 - c->vel.cur;
            const int rc = callback_upload(c, (double)c->t, next);
            if (rc) return rc;
            c->vel.cur = next;
        }
        launch_step_any(c);
        CK(c, cudaGetLastError());
        c->cur = 1 - c->cur;
        if (is_dev(c)) c->pcur = 1 - c->pcur;
        c->t += 1;
        c->stepped = true;
        c->fresh = false;
    }
    return LBM_ACE_OK;
}

int lbm_ace_get_phi(lbm_ace_ctx* c, double* out, size_t count)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    const size_t n = (size_t)c->p.nx * c->p.ny;
    if (!out || count != n) return fail(c, LBM_ACE_EINVAL, "out must hold nx*ny = %zu values (got %zu)", n, count);
    DeviceGuard g(c->dev);
    // page-locked out: the moment kernel writes it through its mapped address (one pass
    // over the host link, no device staging); else staged in c->scratch and copied
    double* mapped = static_cast<double*>(const_cast<void*>(mapped_host(out, n * sizeof(double))));
    const int rc = mapped ? phi_to(c, mapped) : phi_to_scratch(c);
    if (rc) return rc;
    if (!mapped) CK(c, cudaMemcpyAsync(out, c->scratch, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

int lbm_ace_get_phi_device(lbm_ace_ctx* c, float* phi_out)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    if (!phi_out) return fail(c, LBM_ACE_EINVAL, "phi_out is NULL");
    DeviceGuard g(c->dev);
    const int rc = phi_to_scratch(c);
    if (rc) return rc;
    const long long n = (long long)c->p.nx * c->p.ny;
    ace_narrow<<<grid_for(n, c->sms), 256, 0, c->stream>>>(c->scratch, phi_out, n);
    CK(c, cudaGetLastError());
    return LBM_ACE_OK;
}

int lbm_ace_velocity_device(lbm_ace_ctx* c, double t, float* u_out, float* v_out)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    if (!u_out || !v_out) return fail(c, LBM_ACE_EINVAL, "u_out or v_out is NULL");
    if (!std::isfinite(t)) return fail(c, LBM_ACE_EINVAL, "t is not finite");
    if (c->p.velocity_kind == LBM_ACE_VEL_CALLBACK)
        return fail(c, LBM_ACE_EINVAL, "velocity_device is not available with a velocity callback");
    DeviceGuard g(c->dev);
    const long long n = (long long)c->p.nx * c->p.ny;
    const int gr = grid_for(n, c->sms);
    const int nx = c->p.nx, ny = c->p.ny;
    switch (c->p.velocity_kind) {
    case LBM_ACE_VEL_SINGLE_VORTEX:
        if (is_f64(c)) launch_pdl(ace_velocity<double, VelVortex<double>>, dim3(gr), 256, c->stream, vortex<double>(c, t), nx, ny, u_out, v_out);
        else launch_pdl(ace_velocity<float, VelVortex<float>>, dim3(gr), 256, c->stream, vortex<float>(c, t), nx, ny, u_out, v_out);
        break;
    case LBM_ACE_VEL_UNIFORM: {
        VelUniform<double> v; v.ux = c->p.ux; v.uy = c->p.uy;
        launch_pdl(ace_velocity<double, VelUniform<double>>, dim3(gr), 256, c->stream, v, nx, ny, u_out, v_out);
        break;
    }
    default:
        launch_pdl(ace_velocity<double, VelPlanes<double>>, dim3(gr), 256, c->stream, planes<double>(c), nx, ny, u_out, v_out);
        break;
    }
    CK(c, cudaGetLastError());
    return LBM_ACE_OK;
}

int lbm_ace_reset_device(lbm_ace_ctx* c, const float* phi, long long t)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    if (!phi) return fail(c, LBM_ACE_EINVAL, "phi is NULL");
    if (t < 0) return fail(c, LBM_ACE_EINVAL, "t = %lld: must be >= 0", t);
    if (c->p.velocity_kind == LBM_ACE_VEL_CALLBACK)
        return fail(c, LBM_ACE_EINVAL, "reset_device is not available with a velocity callback");
    DeviceGuard g(c->dev);
    const long long n = (long long)c->p.nx * c->p.ny;
    int rc = ensure_scratch(c, (size_t)n);
    if (rc) return rc;
    ace_widen<<<grid_for(n, c->sms), 256, 0, c->stream>>>(phi, c->scratch, n);
    CK(c, cudaGetLastError());
    switch (c->p.precision) {
    case LBM_ACE_F64: launch_init_t<double>(c, c->scratch, (double)t); break;
    case LBM_ACE_F32: launch_init_t<float>(c, c->scratch, (double)t); break;
    case LBM_ACE_F16DEV: launch_init_dev<__half>(c, c->scratch, (double)t); break;
    default: launch_init_dev<__nv_bfloat16>(c, c->scratch, (double)t); break;
    }
    CK(c, cudaGetLastError());
    c->t = t;
    c->stepped = false;
    c->fresh = true;
    return LBM_ACE_OK;
}

void* lbm_ace_get_stream(const lbm_ace_ctx* c) { return c ? (void*)c->stream : nullptr; }

int lbm_ace_release_cached_memory(int device)
{
    if (device < 0 || device >= kMaxDevices) return fail(nullptr, LBM_ACE_EINVAL, "device %d out of range", device);
    DeviceGuard g(device);
    unsigned long long id = 0;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (current_ctx_id(&id) && g_pool_ctx[device] == id) pool = g_pools[device];
    }
    if (!pool) return LBM_ACE_OK; // nothing allocated in the device's current context
    // the frees of destroyed contexts are ordered on their streams: let them land first
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
    if (e != cudaSuccess) return fail(nullptr, LBM_ACE_ECUDA, "releasing cached memory: %s", cudaGetErrorString(e));
    return LBM_ACE_OK;
}

int lbm_ace_get_params(const lbm_ace_ctx* c, lbm_ace_params* out)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    if (!out) return fail(const_cast<lbm_ace_ctx*>(c), LBM_ACE_EINVAL, "out is NULL");
    *out = c->p;
    return LBM_ACE_OK;
}

int lbm_ace_mass(lbm_ace_ctx* c, double* out)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    if (!out) return fail(c, LBM_ACE_EINVAL, "out is NULL");
    DeviceGuard g(c->dev);
    const long long n = (long long)c->p.nx * c->p.ny, n9 = 9 * n;
    const unsigned short* gs = (const unsigned short*)c->f[c->cur];
    unsigned* done = reinterpret_cast<unsigned*>(c->result + 3);
    int rc;
    switch (c->p.precision) {
    case LBM_ACE_F64:
        ace_sum_partials<double><<<c->n_red_part, RED_THREADS, 0, c->stream>>>((const double*)c->f[c->cur], n9, c->red_part);
        rc = finalize_sum(c, c->red_part, c->n_red_part, out);
        break;
    case LBM_ACE_F32:
        ace_sum_partials_f32<<<c->n_red_part, RED_THREADS, 0, c->stream>>>((const float*)c->f[c->cur], n9, c->red_part,
                                                                           done, c->hres_dev, c->dev_err);
        rc = fetch_result(c, out);
        break;
    case LBM_ACE_F16DEV:
        ace_sum_partials_dev<__half><<<c->n_red_part, RED_THREADS, 0, c->stream>>>(gs, c->phi2[c->pcur], n, c->red_part,
                                                                                   done, c->hres_dev, c->dev_err);
        rc = fetch_result(c, out);
        break;
    default:
        ace_sum_partials_dev<__nv_bfloat16><<<c->n_red_part, RED_THREADS, 0, c->stream>>>(gs, c->phi2[c->pcur], n,
                                                                                          c->red_part, done, c->hres_dev,
                                                                                          c->dev_err);
        rc = fetch_result(c, out);
        break;
    }
    if (rc) return rc;
    if (!std::isfinite(*out)) return fail(c, LBM_ACE_ENUMERIC, "global mass is not finite (%g)", *out);
    return LBM_ACE_OK;
}

int lbm_ace_step_mass(lbm_ace_ctx* c, double* out)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    if (!out) return fail(c, LBM_ACE_EINVAL, "out is NULL");
    if (!c->stepped) return fail(c, LBM_ACE_EINVAL, "no step has run yet");
    DeviceGuard g(c->dev);
    const int rc = finalize_sum(c, c->step_part, c->n_step_part, out);
    if (rc) return rc;
    if (!std::isfinite(*out)) return fail(c, LBM_ACE_ENUMERIC, "step mass is not finite (%g)", *out);
    return LBM_ACE_OK;
}

int lbm_ace_get_state(lbm_ace_ctx* c, double* f, double* phi_prev)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    DeviceGuard g(c->dev);
    const size_t n = (size_t)c->p.nx * c->p.ny;
    int rc = ensure_scratch(c, 10 * n);
    if (rc) return rc;
    const int gr = grid_for((long long)n, c->sms);
    const unsigned short* gs = (const unsigned short*)c->f[c->cur];
    switch (c->p.precision) {
    case LBM_ACE_F64:
        ace_pull_state<double><<<gr, 256, 0, c->stream>>>((const double*)c->f[c->cur], (const double*)c->phi,
                                                          c->scratch, c->scratch + 9 * n, c->p.nx, c->p.ny);
        break;
    case LBM_ACE_F32:
        ace_pull_state<float><<<gr, 256, 0, c->stream>>>((const float*)c->f[c->cur], (const float*)c->phi,
                                                         c->scratch, c->scratch + 9 * n, c->p.nx, c->p.ny);
        break;
    case LBM_ACE_F16DEV:
        ace_pull_state_dev<__half><<<gr, 256, 0, c->stream>>>(gs, c->phi2[c->pcur], c->scratch, nullptr,
                                                              c->scratch + 9 * n, c->p.nx, c->p.ny);
        break;
    default:
        ace_pull_state_dev<__nv_bfloat16><<<gr, 256, 0, c->stream>>>(gs, c->phi2[c->pcur], c->scratch, nullptr,
                                                                     c->scratch + 9 * n, c->p.nx, c->p.ny);
        break;
    }
    CK(c, cudaGetLastError());
    if (f) CK(c, cudaMemcpyAsync(f, c->scratch, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (phi_prev) CK(c, cudaMemcpyAsync(phi_prev, c->scratch + 9 * n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

int lbm_ace_set_state(lbm_ace_ctx* c, const double* f, const double* phi_prev, long long t)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    if (!f || !phi_prev) return fail(c, LBM_ACE_EINVAL, "f and phi_prev are required");
    if (t < 0) return fail(c, LBM_ACE_EINVAL, "t = %lld: must be >= 0", t);
    if (c->p.velocity_kind == LBM_ACE_VEL_CALLBACK)
        return fail(c, LBM_ACE_EINVAL, "set_state is not supported with a velocity callback");
    DeviceGuard g(c->dev);
    const size_t n = (size_t)c->p.nx * c->p.ny;
    for (size_t k = 0; k < 9 * n; ++k)
        if (!std::isfinite(f[k])) return fail(c, LBM_ACE_EINVAL, "f[%zu] is not finite", k);
    int rc = ensure_scratch(c, 10 * n);
    if (rc) return rc;
    CK(c, cudaMemcpyAsync(c->scratch, f, 9 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->scratch + 9 * n, phi_prev, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    const int gr = grid_for((long long)n, c->sms);
    unsigned short* gs = (unsigned short*)c->f[c->cur];
    switch (c->p.precision) {
    case LBM_ACE_F64:
        ace_push_state<double><<<gr, 256, 0, c->stream>>>(c->scratch, c->scratch + 9 * n, (double*)c->f[c->cur],
                                                          (double*)c->phi, c->p.nx, c->p.ny);
        break;
    case LBM_ACE_F32:
        ace_push_state<float><<<gr, 256, 0, c->stream>>>(c->scratch, c->scratch + 9 * n, (float*)c->f[c->cur],
                                                         (float*)c->phi, c->p.nx, c->p.ny);
        break;
    case LBM_ACE_F16DEV:
        ace_push_state_dev<__half><<<gr, 256, 0, c->stream>>>(c->scratch, c->scratch + 9 * n, gs, c->phi2[c->pcur],
                                                              c->p.nx, c->p.ny);
        break;
    default:
        ace_push_state_dev<__nv_bfloat16><<<gr, 256, 0, c->stream>>>(c->scratch, c->scratch + 9 * n, gs,
                                                                     c->phi2[c->pcur], c->p.nx, c->p.ny);
        break;
    }
    CK(c, cudaGetLastError());
    CK(c, cudaStreamSynchronize(c->stream));
    c->t = t;
    c->stepped = false;
    c->fresh = t == 0;
    return LBM_ACE_OK;
}

int lbm_ace_launch_shape(const lbm_ace_ctx* c, int* tile_x, int* rows_per_cta, int* grid_x, int* grid_y,
                         int* kernel_variant)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    if (tile_x) *tile_x = c->tile_x;
    if (rows_per_cta) *rows_per_cta = c->rows;
    if (grid_x) *grid_x = c->grid_x;
    if (grid_y) *grid_y = c->grid_y;
    if (kernel_variant) *kernel_variant = c->variant;
    return LBM_ACE_OK;
}

int lbm_ace_wait_selftest(lbm_ace_ctx* c, long long limit_cycles)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    if (limit_cycles < 1 || limit_cycles > kWaitLimitCycles)
        return fail(c, LBM_ACE_EINVAL, "limit_cycles = %lld: must be in [1, %lld]", limit_cycles, kWaitLimitCycles);
    DeviceGuard g(c->dev);
    ace_wait_selftest<<<1, 32, 0, c->stream>>>(limit_cycles, c->dev_err);
    CK(c, cudaGetLastError());
    CK(c, cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

int lbm_ace_synchronize(lbm_ace_ctx* c)
{
    if (!c) return fail(nullptr, LBM_ACE_EINVAL, "ctx is NULL");
    DeviceGuard g(c->dev);
    CK(c, cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

} // extern "C"
