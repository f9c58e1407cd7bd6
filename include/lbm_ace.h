/*
 * lbm_ace.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann solver for the
 * modified conservative Allen-Cahn equation of H. Liang, "An accurate lattice
 * Boltzmann method for interface capturing" (arXiv 2203.05230).
 *
 * The library advances a phase field phi on a periodic nx x ny D2Q9 lattice
 * with the BGK equation plus forcing of Eq. 9, the equilibrium of Eq. 10, the
 * forcing of Eq. 11 and the moment of Eq. 12, computing psi and the unit
 * normal with the regularisation and the phi clip of Eq. 13, so that the
 * scheme recovers Eq. 8 with mobility M = c_s^2 (tau - 1/2). The prescribed
 * velocity is the time-reversed single vortex of Eq. 14 (Section 3), a
 * uniform velocity, a static field, or a host callback.
 *
 * Conventions for every function:
 *  - The return value is a status (LBM_ACE_OK = 0, negative on error). No
 *    function aborts or exits; on error a message is available through
 *    lbm_ace_last_error(ctx) (or lbm_ace_last_error(NULL) when no context
 *    exists yet). Messages are owned by the library and stay valid until the
 *    next call on the same context (or, for NULL, on the same thread).
 *  - Host pointers are owned by the caller and are only read or written
 *    during the call. The context owns its device memory.
 *  - All device work is issued on the stream given at init. lbm_ace_step
 *    returns without waiting; the functions that return values to the host
 *    synchronise that stream first and then report LBM_ACE_ETIMEOUT if a
 *    bounded wait inside a kernel gave up since the last such report.
 *  - Arrays are row-major: a scalar field is [ny][nx] with x fastest; a
 *    population field is [9][ny][nx] in the D2Q9 order c_0 = (0,0),
 *    c_1..c_4 = (1,0), (0,1), (-1,0), (0,-1), c_5..c_8 = (1,1), (-1,1),
 *    (-1,-1), (1,-1). Node (x, y) sits at integer coordinates.
 *
 * Readings of the paper built into the library (where it is silent or
 * inconsistent):
 *  - Interface parameter. Eq. 5's middle form disagrees with Eq. 13 by a
 *    factor 4. The library takes eps as printed in Eq. 13,
 *    psi = eps ln((phi_c + delta) / (1 - phi_c + delta)), so the equilibrium
 *    profile of Eq. 2 is phi = 1/2 + 1/2 tanh(s / (2 eps)) and the sharpening
 *    magnitude of Eqs. 6, 11 is (1/(4 eps)) [1 - tanh^2(psi / (2 eps))]
 *    = phi_c (1 - phi_c) / eps (up to delta). The paper's eps is 4x this one.
 *  - Gradient: the D2Q9 isotropic stencil, grad chi = sum_i w_i c_i chi(x + c_i) / c_s^2.
 *  - Time derivative d_t(phi u) (Section 2.2, "explicit Euler"): the backward
 *    difference phi(t) u(t) - phi(t-1) u(t-1); zero at the first step t = 0.
 *  - Initial populations: f_i = f_i^eq(phi0, u(x, 0)); phi(-1) = phi0.
 */
#ifndef LBM_ACE_H
#define LBM_ACE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    LBM_ACE_OK = 0,
    LBM_ACE_EINVAL = -1,   /* invalid argument or parameter */
    LBM_ACE_ENOMEM = -2,   /* device or host allocation failed */
    LBM_ACE_ECUDA = -3,    /* a CUDA runtime call failed (message has the CUDA error) */
    LBM_ACE_ENUMERIC = -4, /* non-finite values found by a numeric check */
    LBM_ACE_ETIMEOUT = -5, /* a bounded device-side wait gave up */
    LBM_ACE_ECALLBACK = -6 /* the host velocity callback returned non-zero */
};

/* Storage and arithmetic of the populations. */
enum {
    LBM_ACE_F64 = 0,    /* FP64 populations, FP64 arithmetic */
    LBM_ACE_F32 = 1,    /* FP32 populations, FP32 arithmetic, FP64 mass sums */
    LBM_ACE_F16DEV = 2, /* populations stored as FP16 deviations g_i = f*_i - s_i phi, with
                           split weights s = (1820, 455 x4, 114 x4)/4096 (close to the D2Q9
                           weights, summing exactly to 1); phi in FP32, FP32 arithmetic,
                           44 bytes per node update; needs an even nx */
    LBM_ACE_BF16DEV = 3 /* as above with BF16 storage */
};

/* Interface model. */
enum {
    LBM_ACE_MODEL_MODIFIED = 0,    /* the paper's model: Eq. 8 via psi (Eqs. 11, 13) */
    LBM_ACE_MODEL_CONSERVATIVE = 1 /* ablation: conservative ACE of Eq. 1, normal and
                                      sharpening from phi itself (S = phi(1-phi)/eps) */
};

/* Prescribed velocity. */
enum {
    LBM_ACE_VEL_SINGLE_VORTEX = 0, /* Eq. 14, see vortex_sign */
    LBM_ACE_VEL_UNIFORM = 1,       /* (ux, uy) everywhere, all times */
    LBM_ACE_VEL_FIELD = 2,         /* static field u_field, v_field, all times */
    LBM_ACE_VEL_CALLBACK = 3       /* vel_fn called on the host once per step */
};

/* Host velocity callback: fill u and v ([ny][nx], host memory owned by the
 * library, valid during the call) with the velocity at time t (in steps).
 * Return 0 on success; any other value stops lbm_ace_step with
 * LBM_ACE_ECALLBACK. */
typedef int (*lbm_ace_velocity_fn)(double t, int nx, int ny, double* u, double* v, void* user);

typedef struct lbm_ace_params {
    int nx, ny;        /* periodic lattice, each >= 3 (Section 3: L x L) */
    double tau;        /* BGK relaxation time of Eq. 9, > 0.5 */
    double M;          /* mobility; must equal (tau - 0.5)/3 within 1e-12 relative
                          (Section 2.2: M = c_s^2 (tau - 0.5) delta_t), or < 0 to derive it */
    double eps;        /* interface parameter, > 0, convention of the header comment */
    double reg_delta;  /* regulariser of Eq. 13; 0 selects the paper's e^-20 */
    int precision;     /* LBM_ACE_F64 .. LBM_ACE_BF16DEV */
    int model;         /* LBM_ACE_MODEL_* */
    int velocity_kind; /* LBM_ACE_VEL_* */
    /* single vortex (Eq. 14): u = s U0 sin^2(pi x/nx) sin(2 pi y/ny) cos(pi t/T),
       v = -s U0 sin^2(pi y/ny) sin(2 pi x/nx) cos(pi t/T), s = vortex_sign
       (+1: the sign printed in Eq. 14; -1: the mirror image) */
    double U0, T_period, vortex_sign;
    double ux, uy;                 /* LBM_ACE_VEL_UNIFORM */
    const double* u_field;         /* LBM_ACE_VEL_FIELD: host [ny][nx], copied at init */
    const double* v_field;
    lbm_ace_velocity_fn vel_fn;    /* LBM_ACE_VEL_CALLBACK */
    void* vel_user;
    const double* phi0;  /* host [ny][nx] initial phi, read during init only; NULL selects
                            the disk phi0 = 1/2 (1 + tanh((R - r) / (2 eps))) about (xc, yc).
                            Every value must be finite and, for all precisions but
                            LBM_ACE_F64 (whose phi is FP32), round to a finite FP32. Its
                            upload runs while the host prepares the velocity, without
                            waiting when phi0 is page-locked (cudaHostAlloc, cudaMallocHost,
                            cudaHostRegister); from 2^20 nodes, FP64 and FP32 lattices
                            upload it in row chunks on a second stream of the library's
                            and initialise each chunk as it lands */
    double xc, yc, R;
    int device;          /* CUDA device ordinal */
    void* stream;        /* cudaStream_t for all device work; NULL = the legacy default stream */
    int rows_per_cta;    /* launch shape of the fused step: rows each CTA marches over;
                            0 selects a default for the lattice size and the device;
                            at most 4095 with kernel variants 7 and 8 (else
                            LBM_ACE_EINVAL) */
    int kernel_variant;  /* fused step kernel: 0 = automatic (FP32 with nx a multiple of 4 and at
                            most 2^23 nodes: 8; else 4 for even nx, else 1), 1 = direct global
                            loads with a CTA-wide row barrier, 2 = rows staged in shared
                            memory by bulk copies (needs nx * element size a multiple of
                            16 bytes), 3 = independent 32-column warps with loads issued a
                            row ahead, 4 = two columns per thread with paired loads and
                            stores (needs an even nx), 6 = two steps per launch with the
                            intermediate populations in shared memory (FP32, even nx, no
                            velocity callback; an odd step count ends with one variant-4
                            step; keeps a second phi plane), 8 = four columns per thread in
                            independent 128-column warp strips (FP32, nx a multiple of 4).
                            All give bit-identical results.
                            The 16-bit deviation storage has two kernels of its own, also
                            bit-identical: 5 = two columns per thread (even nx), 7 = four
                            columns per thread (nx a multiple of 4); 0 picks 7 when it
                            applies, else 5. The FP32 and 16-bit kernels give their
                            stores L2 eviction priorities chosen from the lattice's size
                            and the device's L2 size; they change timing, not results. */
} lbm_ace_params;

typedef struct lbm_ace_ctx lbm_ace_ctx; /* opaque; owns its device buffers */

/* Fill *p with defaults: 64 x 64, tau 0.8, M derived, eps 1, delta e^-20, FP64,
 * the paper's model, single vortex with U0 0.04, T 2000, sign -1, disk R 9.6 at
 * (32, 48), device 0, default stream. */
int lbm_ace_params_default(lbm_ace_params* p);

/* Validate *p, allocate device state and initialise it (f_i = f_i^eq(phi0,
 * u(x, 0)), t = 0). Checks: nx, ny >= 3; tau > 0.5; eps > 0; M consistent; phi0
 * finite (in FP32 for the FP32-based precisions: fields of up to 65,536 values on the
 * host before any device work, larger ones on the device right after the init kernel,
 * with the smallest bad index in the message); the velocity source present. On success
 * *out owns the context. */
int lbm_ace_init(const lbm_ace_params* p, lbm_ace_ctx** out);

/* Advance n >= 0 steps (Eq. 9, one fused kernel per step). Asynchronous on the
 * context's stream, except that the callback velocity mode calls the host
 * function each step. */
int lbm_ace_step(lbm_ace_ctx* c, long long n);

/* phi(x, t) = sum_i f_i(x, t) (Eq. 12) at the current time t, written to the
 * host array out[count], count == nx*ny. Synchronous. A page-locked out (cudaHostAlloc,
 * cudaMallocHost, cudaHostRegister; checked at its first and last byte) is written by
 * the moment kernel itself through its mapped address; other memory through a device
 * buffer and a copy. The values are the same either way. */
int lbm_ace_get_phi(lbm_ace_ctx* c, double* out, size_t count);

/* Device memory. A context's device buffers come from a stream-ordered memory pool
 * that the library keeps per device; lbm_ace_destroy returns them to that pool, and
 * contexts created later on the device reuse them without calling cudaMalloc (225 us
 * for the buffers of a 2048^2 FP32 lattice on GB300, 7 us from the pool). The pool
 * keeps what it caches until this call, which waits for the device to go idle
 * (cudaDeviceSynchronize) and hands every cached block no context uses back to the
 * driver; live contexts keep theirs. LBM_ACE_OK also when the library has allocated
 * nothing on the device; LBM_ACE_EINVAL for an ordinal outside [0, 64). */
int lbm_ace_release_cached_memory(int device);

/* Global mass sum_x sum_i f_i(x, t) of the current state, summed on the device in
 * a fixed order (deterministic). FP64 states: Neumaier-compensated FP64 sums. FP32 and
 * 16-bit states: each value split into a multiple of 2^-16, summed exactly as an
 * integer, and a remainder below 2^-17 summed in FP32 (a thread that meets a value of
 * 2 or more in magnitude sums its values in FP64 instead), per-thread totals combined
 * with a compensated FP64 tree; relative error about 1e-14 (a thread adds a few hundred
 * values at 2048^2; at the limit of 8192 values per thread, about 1e-10). One kernel
 * launch; the result reaches the host through mapped pinned memory. Synchronous.
 * Returns LBM_ACE_ENUMERIC (with *out set) when it is not finite. */
int lbm_ace_mass(lbm_ace_ctx* c, double* out);

/* Global mass sum_x phi(x, t-1) as reduced block by block inside the last
 * fused step (FP64 block partials, compensated final sum; the quad kernels sum a
 * thread's values in split parts whose FP32 remainder sum rounds by about 1e-14 of the
 * total in the default launch shapes and up to about 1e-10 for bands thousands of rows
 * tall). Synchronous. LBM_ACE_EINVAL before the first step. */
int lbm_ace_step_mass(lbm_ace_ctx* c, double* out);

/* Checkpoint: f[9*nx*ny] receives f_i(x, t) (after streaming, as in Eq. 9's
 * left side), phi_prev[nx*ny] receives phi(x, t-1); either may be NULL.
 * Synchronous. FP16/BF16 deviation storage is expanded to FP64. */
int lbm_ace_get_state(lbm_ace_ctx* c, double* f, double* phi_prev);

/* Restore a state written by lbm_ace_get_state (or any state in that layout) at
 * time t >= 0. Values are rounded to the context's storage precision. */
int lbm_ace_set_state(lbm_ace_ctx* c, const double* f, const double* phi_prev, long long t);

/* Current time t (number of steps taken since init, or as set). */
long long lbm_ace_steps_done(const lbm_ace_ctx* c);

/* Launch shape chosen for the fused step: columns and rows per CTA, grid, and the
 * kernel variant (1 to 8, see lbm_ace_params.kernel_variant). Any pointer may be NULL. */
int lbm_ace_launch_shape(const lbm_ace_ctx* c, int* tile_x, int* rows_per_cta, int* grid_x, int* grid_y,
                         int* kernel_variant);

/* Block until all device work of the context has finished. */
int lbm_ace_synchronize(lbm_ace_ctx* c);

/* Failure-detection self-test (no GPU fault). Launches, on the context's stream, one
 * CTA that initialises an mbarrier no thread ever arrives on and waits for it with the
 * bounded wait the step kernels use (mbarrier.try_wait polled against clock64), giving
 * up after `limit_cycles` SM clock cycles (1 .. 4e9; 2e6 is about 1 ms). The CTA then
 * sets the context's device error flag, as a step kernel whose wait gave up does, and
 * returns. The call synchronises the stream and reports through the same path as
 * lbm_ace_synchronize: LBM_ACE_ETIMEOUT when the wait gave up (the expected result; the
 * flag is cleared and the context stays usable), LBM_ACE_OK if the barrier somehow
 * completed, LBM_ACE_EINVAL for a limit out of range, LBM_ACE_ECUDA on a CUDA error.
 * The lattice state is not touched. */
int lbm_ace_wait_selftest(lbm_ace_ctx* c, long long limit_cycles);

/* ---- Device-side access (for a caller that keeps fields on the GPU) ---------------
 * These three calls are asynchronous on the context's stream and take DEVICE pointers
 * (on the context's device) to FP32 [ny][nx] arrays that the caller owns; each must
 * stay valid until the stream has passed the call. A NULL pointer returns
 * LBM_ACE_EINVAL without device work. */

/* phi(x, t) = sum_i f_i(x, t) (Eq. 12) at the current time, rounded to FP32, into
 * phi_out. */
int lbm_ace_get_phi_device(lbm_ace_ctx* c, float* phi_out);

/* The prescribed velocity u(x, t) at time t (in steps; any real t) into u_out and
 * v_out: the single vortex of Eq. 14 (evaluated in FP64, rounded), the uniform
 * velocity or the static field. LBM_ACE_EINVAL for the callback mode. */
int lbm_ace_velocity_device(lbm_ace_ctx* c, double t, float* u_out, float* v_out);

/* Restart the lattice at time t >= 0 from the phase field phi (device, FP32): the
 * populations become f_i^eq(phi, u(x, t)) (Eq. 10) and phi(t-1) = phi, as at
 * initialisation, so d_t(phi u) is zero on the first step after the restart. Used to
 * hand a phase field produced elsewhere (a learned surrogate) back to the lattice
 * Boltzmann scheme. LBM_ACE_EINVAL for the callback mode. */
int lbm_ace_reset_device(lbm_ace_ctx* c, const float* phi, long long t);

/* The CUDA stream (cudaStream_t) the context issues its work on. */
void* lbm_ace_get_stream(const lbm_ace_ctx* c);

/* A copy of the parameters the context was created with (pointers inside refer to the
 * caller's original arrays and must not be dereferenced after init returned). */
int lbm_ace_get_params(const lbm_ace_ctx* c, lbm_ace_params* out);

/* ---- Batches: many independent single-vortex lattices advanced together ----------
 * Each lattice of a batch is a single-vortex problem (Section 3, Eq. 14) with its own
 * size, disk, eps, tau, U0 and period, FP32 populations, and one model for the whole
 * batch. A batch step advances every lattice by one time step with one launch of a
 * persistent kernel (resident CTAs whose warps, or whole CTAs, pull work items of all
 * lattices from a work counter), replayed from a captured CUDA graph; the time t is
 * shared. The
 * batch owns its device memory and works on params[0].stream (or on a stream of its
 * own when that is NULL, since graphs cannot be captured on the legacy stream). */
typedef struct lbm_ace_batch lbm_ace_batch;

/* Build a batch of `count` lattices from params[0..count-1]. Each needs precision
 * LBM_ACE_F32, velocity LBM_ACE_VEL_SINGLE_VORTEX, an even nx, phi0 == NULL (the disk
 * from xc, yc, R is built on the device), the same model; rows_per_cta sets the tile
 * height of that lattice (0: 64; at least 8 is used, and at most 4095 with strips).
 * Work items: when every nx is a multiple of 4, strips of 128 columns, each taken by one
 * warp with the single-lattice library's four-columns-per-thread code (kernel variant 8);
 * otherwise tiles of 256 columns, each taken by a CTA with the column-pair code (variant
 * 4). Device and stream come from params[0]. */
int lbm_ace_batch_init(const lbm_ace_params* params, int count, lbm_ace_batch** out);

/* Advance the batch's clock by n >= 0 steps: n replays of the captured {step, advance}
 * graph. A lattice advances while the clock is below its end step (lbm_ace_batch_set_ends;
 * by default it has none) and then keeps its state; retired lattices' tiles leave the
 * persistent kernel's work list, on the device. Asynchronous on the batch's stream. */
int lbm_ace_batch_step(lbm_ace_batch* b, long long n);

/* The same n steps as one ordinary launch per lattice per step (the single-lattice
 * kernel of the batch's work-item form -- variant 8 or 4 -- in the launch shape the
 * single-lattice library picks, host-side loop, lattices past their end skipped): a
 * baseline a batch is compared with. Synchronous. */
int lbm_ace_batch_step_sequential(lbm_ace_batch* b, long long n);

/* The same n steps as one launch per lattice per step, all launches of a step captured
 * in one CUDA graph with the batch's own tiles and device-side phases: the baseline
 * without host launch overhead, so that a comparison isolates what the persistent
 * kernel's shared work list gains. Asynchronous on the batch's stream. */
int lbm_ace_batch_step_per_lattice(lbm_ace_batch* b, long long n);

/* Per-lattice end steps for uneven runs: lattice i advances while the batch's clock t <
 * end_steps[i] (a negative entry: no end). NULL sets each lattice's end to its period
 * T_period rounded to an integer, the time at which the single-vortex benchmark
 * (Section 3) compares the shape with the initial one. Every end must be >= the current
 * clock. Rebuilds the work list (latest end first) and drops the captured graphs. */
int lbm_ace_batch_set_ends(lbm_ace_batch* b, const long long* end_steps);

/* Steps lattice i has taken: min(clock, its end); -1 for a bad argument. */
long long lbm_ace_batch_lattice_steps(const lbm_ace_batch* b, int i);

/* Lattices and work-list tiles still active at the current clock. */
int lbm_ace_batch_active(const lbm_ace_batch* b, int* lattices, int* tiles);

/* Choose the tile height of each lattice size by coordinate descent over {8, 16, 32,
 * 64, 128, 256}, then the persistent grid's CTAs per SM (1 up to the occupancy limit),
 * timing steps_per_trial batch steps per trial with CUDA events; the lattices' states
 * and time are saved before and restored after the trials. Writes the chosen heights
 * to rows_out[count] when not NULL (the grid is reported by lbm_ace_batch_info).
 * Allocates a copy of the state for the duration of the call. */
int lbm_ace_batch_autotune(lbm_ace_batch* b, int steps_per_trial, int* rows_out);

/* phi(x, t) of lattice i (host out[count], count == nx*ny of that lattice). Synchronous. */
int lbm_ace_batch_get_phi(lbm_ace_batch* b, int i, double* out, size_t count);

/* Global mass of lattice i (compensated FP64 sum on the device). Synchronous. */
int lbm_ace_batch_mass(lbm_ace_batch* b, int i, double* out);

/* Tile height of lattice i, total tiles per step, persistent grid size, total nodes. */
int lbm_ace_batch_info(const lbm_ace_batch* b, int i, int* rows, int* tiles, int* grid, long long* nodes);

long long lbm_ace_batch_steps_done(const lbm_ace_batch* b);
int lbm_ace_batch_synchronize(lbm_ace_batch* b);
const char* lbm_ace_batch_last_error(const lbm_ace_batch* b);
void lbm_ace_batch_destroy(lbm_ace_batch* b); /* NULL-safe */

/* Allocation-free global mass, for callers that cannot allocate device memory (the
 * paper has no counterpart; it is a service of this library). Some callers cannot
 * call cudaMalloc: their device memory is already handed out by their own pool or
 * caching allocator, or their time-critical loop cannot take the implicit device
 * synchronisation that cudaMalloc/cudaFree may bring. They pass their own buffers:
 *   values   device address of `count` values, FP64 (precision LBM_ACE_F64) or FP32
 *            (LBM_ACE_F32), e.g. the 9 population planes of a lattice or a phi field;
 *   out      device address of one double that receives the sum (0 for count == 0):
 *            a Neumaier-compensated FP64 sum of the values in a fixed order (for FP64
 *            values the algorithm of lbm_ace_mass, in a different order; FP32 states
 *            lbm_ace_mass sums in exact split parts), so the two agree to about 1e-14
 *            relative, not bitwise;
 *   stream   cudaStream_t of the current device (NULL: legacy default stream).
 * The work is asynchronous on `stream` and runs on the current CUDA device. Both
 * pointers must be device memory of the current device (or managed memory); a host
 * pointer (pageable or pinned), another device's buffer, or a range whose last byte
 * is not such memory returns LBM_ACE_EINVAL before any launch.
 * Scratch: the per-chunk partial sums live in a fixed array of static device memory
 * inside the library, LBM_ACE_NOALLOC_MAX_PARTIALS doubles (32 KiB), present on every
 * GPU that loads the library until the process exits. Each call overwrites the slots
 * it uses, so nothing carries over between calls. Because every call shares that one
 * array, calls whose work can overlap on the GPU (other streams, other threads)
 * race and may return wrong sums: order them on one stream or synchronise.
 * The first call on a device looks up the array's device address for that device
 * (cudaGetSymbolAddress); make that first call before any stream capture. The lookup
 * is repeated when the device's context has changed (after cudaDeviceReset), so make
 * the first call after a reset before any capture too.
 * Limits: count <= LBM_ACE_NOALLOC_MAX_COUNT (268,435,456 values); a larger count,
 * a NULL pointer or another precision returns LBM_ACE_EINVAL without device work.
 * Calls no cudaMalloc, cudaFree or other allocating routine. Returns LBM_ACE_ECUDA,
 * without launching, when a CUDA error from earlier work is already pending (the error
 * is left pending for its owner), and when a launch or the address lookup fails. */
#define LBM_ACE_NOALLOC_CHUNK 65536
#define LBM_ACE_NOALLOC_MAX_PARTIALS 4096
#define LBM_ACE_NOALLOC_MAX_COUNT (65536LL * 4096LL)
int lbm_ace_mass_noalloc(const void* values, int precision, long long count, double* out, void* stream);

const char* lbm_ace_last_error(const lbm_ace_ctx* c);
const char* lbm_ace_status_string(int status);

/* Free the context: waits for its stream, then returns its device buffers to the
 * device's pool in stream order on that stream (so the stream it was created with must
 * still exist) and its result slot to the library. NULL is accepted. */
void lbm_ace_destroy(lbm_ace_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* LBM_ACE_H */
