// lbm_ace_surrogate.cu -- the learned surrogate declared in include/lbm_ace_surrogate.h:
// a 5-layer periodic 3x3 convolutional network (3 -> 32 -> 32 -> 32 -> 32 -> 1, GELU,
// residual with the image mean of the output removed), its training kernels
// (loss, back-propagation, Adam) and the hybrid advance with the lattice Boltzmann
// fallback.
//
// Kernels (all hand-written):
//   surr_in_fwd      layer 1 on FP32 units: 27 inputs -> 32 outputs per node
//   surr_conv_umma   layers 2-5 forward and the input gradients of layers 2-4: implicit
//                    GEMM on the fifth-generation tensor cores (tcgen05.mma, BF16
//                    operands from shared memory, FP32 accumulators in tensor memory),
//                    4 x 128 output tiles, persistent CTAs
//   surr_wgrad_mma   layers 2-4 weight gradients: per-tap GEMM over the pixels on the
//                    tensor cores (mma.sync m16n8k16, ldmatrix.trans operands), per-CTA partials
//   surr_residual    mean removal of z_5 and the residual add
//   surr_loss_part / surr_gz5      loss and dL/dz_5 through the mean removal
//   surr_out_bwd     layer 5 weight gradient and dL/dz_4
//   surr_in_wgrad    layer 1 weight gradient
//   surr_reduce      deterministic FP64 sum of the per-CTA gradient partials
//   surr_adam, surr_pack, surr_metrics
//
// Activations are NHWC BF16 ([image][y][x][32]); in shared memory a pixel's 32 channels
// take 80 bytes (64 + 16 padding) so that the eight 16-byte rows an ldmatrix reads from
// eight consecutive pixels fall in distinct bank groups.
#include "lbm_ace_surrogate.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

namespace surr {

typedef __nv_bfloat16 bf16;

constexpr int C = 32;                 // hidden width
constexpr int TH = 16, TW = 16;       // output tile
constexpr int HH = TH + 2, HWD = TW + 2;
constexpr int HPX = HH * HWD;         // halo pixels (324)
constexpr int PS = 40;                // shared-memory pixel stride in bf16 (80 bytes)
constexpr int NPARAM = LBM_ACE_NET_PARAMS;
constexpr int OFF_W1 = 0, OFF_W2 = 896, OFF_W3 = 10144, OFF_W4 = 19392, OFF_W5 = 28640;
constexpr int L1_N = 896;             // W1 (864) + b1 (32)
constexpr int LH_N = 9248;            // W (9216) + b (32) of a hidden layer
constexpr int L5_N = 289;             // W5 (288) + b5 (1)
constexpr float U_SCALE = 20.0f;      // velocity input scale (1 / 0.05)
constexpr int WG_THREADS = 288;       // 9 warps, one per tap
constexpr int RED_BLOCKS = 64;        // blocks per image for per-image reductions
constexpr int MET_BLOCKS = 256;       // blocks of surr_metrics (one field; all SMs at 256^2)

static_assert(OFF_W2 == OFF_W1 + L1_N && OFF_W3 == OFF_W2 + LH_N && OFF_W4 == OFF_W3 + LH_N &&
              OFF_W5 == OFF_W4 + LH_N && OFF_W5 + L5_N == NPARAM, "parameter layout");

struct Geo {
    int B, H, W;
    int tx, ty;           // tiles per image along x and y
    long long ntiles;
};

__host__ __device__ inline Geo make_geo(int B, int H, int W)
{
    Geo g;
    g.B = B; g.H = H; g.W = W;
    g.tx = (W + TW - 1) / TW;
    g.ty = (H + TH - 1) / TH;
    g.ntiles = (long long)B * g.tx * g.ty;
    return g;
}

// v in [-1, 2n): one conditional add or subtract (a neighbour of a node inside the image)
__device__ __forceinline__ int wrap1(int v, int n)
{
    v = v < 0 ? v + n : v;
    return v >= n ? v - n : v;
}

// v >= -1 (a halo row or column of a tile that starts inside the image); images narrower
// than a tile can wrap more than once
__device__ __forceinline__ int wrap_halo(int v, int n)
{
    if (v < 0) v += n;
    if (v >= n) {
        v -= n;
        if (v >= n) v %= n;
    }
    return v;
}

__device__ __forceinline__ void tile_origin(const Geo& g, long long t, int& b, int& y0, int& x0)
{
    const long long per = (long long)g.tx * g.ty;
    b = (int)(t / per);
    const int r = (int)(t - (long long)b * per);
    y0 = (r / g.tx) * TH;
    x0 = (r % g.tx) * TW;
}

// erfc(x) by the Chebyshev-fitted form of Numerical Recipes (Press et al., 2nd ed.,
// Section 6.2): erfc(x) = t exp(-x^2 + P(t)), t = 1 / (1 + |x| / 2), P of degree 9, for
// x >= 0 (fractional error below 1.2e-7 in exact arithmetic, ~1e-7 in FP32 where GELU
// needs it), and 2 - erfc(-x) for x < 0. One reciprocal, one exponential, nine FMAs.
__device__ __forceinline__ float erfc_nr(float x)
{
    const float ax = fabsf(x);
    const float t = __fdividef(1.0f, fmaf(0.5f, ax, 1.0f));
    float p = 0.17087277f;
    p = fmaf(p, t, -0.82215223f);
    p = fmaf(p, t, 1.48851587f);
    p = fmaf(p, t, -1.13520398f);
    p = fmaf(p, t, 0.27886807f);
    p = fmaf(p, t, -0.18628806f);
    p = fmaf(p, t, 0.09678418f);
    p = fmaf(p, t, 0.37409196f);
    p = fmaf(p, t, 1.00002368f);
    p = fmaf(p, t, -1.26551223f);
    const float y = t * __expf(fmaf(-ax, ax, p));
    return x >= 0.0f ? y : 2.0f - y;
}

// GELU(z) = z Phi(z) = z erfc(-z / sqrt 2) / 2, and its derivative Phi(z) + z phi(z).
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * erfc_nr(-0.70710678118654752f * z); }

__device__ __forceinline__ float gelu_grad_f(float z)
{
    return fmaf(z * 0.39894228040143268f, __expf(-0.5f * z * z), 0.5f * erfc_nr(-0.70710678118654752f * z));
}

// The same functions on two values at once with the packed FP32x2 instructions of
// sm_100+ (each lane rounds as the scalar operation does, so the results are
// bit-identical to gelu_f / gelu_grad_f).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

__device__ __forceinline__ float2 erfc_nr2(float2 x)
{
    const float2 ax = make_float2(fabsf(x.x), fabsf(x.y));
    const float2 d = __ffma2_rn(f2(0.5f), ax, f2(1.0f));
    const float2 t = make_float2(__fdividef(1.0f, d.x), __fdividef(1.0f, d.y));
    float2 p = f2(0.17087277f);
    p = __ffma2_rn(p, t, f2(-0.82215223f));
    p = __ffma2_rn(p, t, f2(1.48851587f));
    p = __ffma2_rn(p, t, f2(-1.13520398f));
    p = __ffma2_rn(p, t, f2(0.27886807f));
    p = __ffma2_rn(p, t, f2(-0.18628806f));
    p = __ffma2_rn(p, t, f2(0.09678418f));
    p = __ffma2_rn(p, t, f2(0.37409196f));
    p = __ffma2_rn(p, t, f2(1.00002368f));
    p = __ffma2_rn(p, t, f2(-1.26551223f));
    const float2 a = __ffma2_rn(make_float2(-ax.x, -ax.y), ax, p);
    const float2 y = __fmul2_rn(t, make_float2(__expf(a.x), __expf(a.y)));
    return make_float2(x.x >= 0.0f ? y.x : 2.0f - y.x, x.y >= 0.0f ? y.y : 2.0f - y.y);
}

__device__ __forceinline__ float2 gelu2(float2 z)
{
    return __fmul2_rn(__fmul2_rn(f2(0.5f), z), erfc_nr2(__fmul2_rn(f2(-0.70710678118654752f), z)));
}

__device__ __forceinline__ float2 gelu_grad2(float2 z)
{
    const float2 e = make_float2(__expf(-0.5f * z.x * z.x), __expf(-0.5f * z.y * z.y));
    return __ffma2_rn(__fmul2_rn(z, f2(0.39894228040143268f)), e,
                      __fmul2_rn(f2(0.5f), erfc_nr2(__fmul2_rn(f2(-0.70710678118654752f), z))));
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Programmatic dependent launch: let the next kernel of the forward chain be scheduled
// early, then wait until the previous one has finished and its writes are visible.
// Both are no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() { pdl_trigger(); pdl_wait(); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

// D += A B for one m16n8k16 tile (A row-major 16x16 BF16, B column-major 16x8 BF16, FP32 D).
__device__ __forceinline__ void mma_bf16(float* d, const unsigned* a, unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned*>(&v);
}

__device__ __forceinline__ float2 unpack_bf16(unsigned w)
{
    __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&w);
    return __bfloat1622float2(v);
}

// Stage the 18 x 18 halo of a 16 x 16 tile of an NHWC BF16 tensor (32 channels),
// wrapping periodically, into hs[pixel * PS + channel] with 16-byte cp.async copies.
__device__ __forceinline__ void load_halo(bf16* hs, const bf16* __restrict__ in, const Geo& g, long long tile,
                                          int tid, int nthreads)
{
    int b, y0, x0;
    tile_origin(g, tile, b, y0, x0);
    for (int k = tid; k < HPX * 4; k += nthreads) {
        const int q = k >> 2, part = k & 3;
        const int hy = q / HWD, hx = q - hy * HWD;
        const int y = wrap_halo(y0 + hy - 1, g.H), x = wrap_halo(x0 + hx - 1, g.W);
        const bf16* src = in + ((((size_t)b * g.H + y) * g.W + x) * C + part * 8);
        cp_async16(hs + q * PS + part * 8, src);
    }
}

// ---------------------------------------------------------------------------------
// Layer 1 (FP32 units): z_1 = conv3x3((phi, 20u, 20v), W_1) + b_1, a_1 = GELU(z_1).
// Two pixels per thread; the weights sit transposed in shared memory (wt[k][co]) so one
// 16-byte load feeds eight FMAs (four channels of two pixels).
// (pixel indices fit in 32 bits: batch * ny * nx * 32 < 2^31 is checked on the host)
__device__ __forceinline__ void gather27(const float* __restrict__ phi, const float* __restrict__ u,
                                         const float* __restrict__ v, int p, int H, int W, float* in)
{
    const int r = p / W, x = p - r * W;
    const int b = r / H, y = r - b * H;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int row = (b * H + wrap1(y + j - 1, H)) * W;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int q = row + wrap1(x + i - 1, W);
            in[j * 3 + i] = phi[q];
            in[9 + j * 3 + i] = u[q] * U_SCALE;
            in[18 + j * 3 + i] = v[q] * U_SCALE;
        }
    }
}

__global__ void __launch_bounds__(256) surr_in_fwd(const float* __restrict__ phi, const float* __restrict__ u,
                                                   const float* __restrict__ v, const float* __restrict__ params,
                                                   bf16* __restrict__ z1, bf16* __restrict__ a1, int B, int H, int W)
{
    __shared__ __align__(16) float wt[27][C];
    __shared__ __align__(16) float bs[C];
    pdl_enter();
    for (int k = threadIdx.x; k < 864; k += blockDim.x) wt[k % 27][k / 27] = params[OFF_W1 + k];
    if (threadIdx.x < C) bs[threadIdx.x] = params[OFF_W1 + 864 + threadIdx.x];
    __syncthreads();
    // one pixel per thread; the packed FP32x2 FMAs take two output channels at once
    // (each channel summed over the 27 taps in the same order as before)
    const int P = B * H * W;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        float in[27];
        gather27(phi, u, v, p, H, W, in);
#pragma unroll 1
        for (int cb = 0; cb < 4; ++cb) { // eight output channels per 16-byte store
            float2 s2[4];                // channels (cb * 8 + 2 h, cb * 8 + 2 h + 1)
#pragma unroll
            for (int h = 0; h < 4; ++h) s2[h] = make_float2(bs[cb * 8 + 2 * h], bs[cb * 8 + 2 * h + 1]);
#pragma unroll
            for (int k = 0; k < 27; ++k) {
                const float4 wa = *reinterpret_cast<const float4*>(&wt[k][cb * 8]);
                const float4 wb = *reinterpret_cast<const float4*>(&wt[k][cb * 8 + 4]);
                const float2 x = f2(in[k]);
                s2[0] = __ffma2_rn(make_float2(wa.x, wa.y), x, s2[0]);
                s2[1] = __ffma2_rn(make_float2(wa.z, wa.w), x, s2[1]);
                s2[2] = __ffma2_rn(make_float2(wb.x, wb.y), x, s2[2]);
                s2[3] = __ffma2_rn(make_float2(wb.z, wb.w), x, s2[3]);
            }
            unsigned zw[4], aw[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float2 g = gelu2(s2[h]);
                zw[h] = pack_bf16(s2[h].x, s2[h].y);
                aw[h] = pack_bf16(g.x, g.y);
            }
            if (z1) reinterpret_cast<uint4*>(z1 + (size_t)p * C)[cb] = make_uint4(zw[0], zw[1], zw[2], zw[3]);
            reinterpret_cast<uint4*>(a1 + (size_t)p * C)[cb] = make_uint4(aw[0], aw[1], aw[2], aw[3]);
        }
    }
}

// ---------------------------------------------------------------------------------
// tcgen05 (fifth-generation tensor core) helpers. Operands sit in shared memory in the
// no-swizzle K-major layout: "core matrices" of 8 rows x 16 bytes (8 BF16 along K),
// 16 bytes per row; the descriptor gives the byte distance between core matrices
// adjacent along K (leading) and along M or N (stride). Accumulators live in tensor
// memory (TMEM): lane = row of D, column = column of D.

__device__ __forceinline__ uint64_t umma_desc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr unsigned umma_idesc(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(unsigned tmem, uint64_t ad, uint64_t bd, unsigned idesc, unsigned acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(unsigned mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

constexpr long long kSurrWaitCycles = 2000000000LL; // ~1 s of SM clock

// Wait for the phase `parity` of an mbarrier, giving up after `limit` cycles of SM clock
// (~1 s for the kernels). Each try_wait may suspend the warp for up to 0.1 ms (a hint to
// the hardware), so a waiting warp does not spin on the issue slots.
__device__ __forceinline__ bool mbar_wait_limit(unsigned mbar, unsigned parity, long long limit)
{
    const long long t0 = clock64();
    for (;;) {
        unsigned done;
        asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, %3;\nselp.u32 %0, 1, 0, q;\n}\n"
                     : "=r"(done) : "r"(mbar), "r"(parity), "r"(100000u) : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity)
{
    return mbar_wait_limit(mbar, parity, kSurrWaitCycles);
}

#define TMEM_LD_OUT16(r) "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), \
    "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])

// 32 consecutive TMEM columns (x32) or 16 (x16) of this thread's lane.
__device__ __forceinline__ void tmem_ld32(unsigned ta, unsigned* r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                 : TMEM_LD_OUT16(r), TMEM_LD_OUT16((r + 16)) : "r"(ta));
}
__device__ __forceinline__ void tmem_ld16(unsigned ta, unsigned* r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : TMEM_LD_OUT16(r) : "r"(ta));
}
__device__ __forceinline__ void tmem_ld8(unsigned ta, unsigned* r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(ta));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// ---------------------------------------------------------------------------------
// Layers 2-5 on the tensor cores: implicit GEMM, one MMA of M = 128 pixels (one row
// segment of a tile), N output channels, K = 16 input channels per tap and K-half:
//   out[p][n] = sum_tap sum_k w[tap][n][k] in[p + off(tap)][k],  off(tap) = (tap/3 - 1, tap%3 - 1).
// A tile is R rows x 128 columns of one image (R = UR = 4; R = 2 for a forward too small
// to give every SM two tiles, so that a CTA pipelines several). Its (R+2) x 130 x 32
// halo is staged
// by cp.async as four planes of 16-byte channel chunks, so the window of any tap is a
// set of core matrices 16 bytes apart along M (SBO 128 bytes per 8 pixels) and one
// plane apart along K. Weights: [tap][chunk][n][8] (block per tap and chunk).
//
// One persistent CTA per SM (the occupancy of tcgen05 kernels), warp-specialised:
//   warps 0-3   load halos into a two-stage ring (cp.async; each thread waits for its
//               own copies, fences them into the async proxy and arrives on full[s]);
//   warp 4      one thread issues the 4 x 9 x 2 MMAs of a tile into one of two TMEM
//               accumulator sets and commits them to empty[s] (stage free) and
//               tfull[a] (accumulators ready);
//   warps 5-20  read the accumulators (warp w: TMEM lanes 32 (w % 4).., tile row
//               (w - 5) / 4; one pixel per thread, eight channels per tcgen05.ld), apply
//               the epilogue, write 16 bytes per pixel and group and arrive on tempty[a].
// Every mbarrier wait gives up after ~1 s; the CTA then records the failure, drains
// and frees its tensor memory.
//   MODE_FWD (N = 32):  z = acc + b; stores z (if out_z) and GELU(z), BF16.
//   MODE_DGRAD (N = 32): acc is dL/da of the layer below; stores acc GELU'(zaux), BF16.
//   MODE_OUT (N = 16, only n = 0 real): z_5 = acc + b_5 (FP32) and 16 partial sums per
//               tile (one per epilogue warp) in tsum[16 tile + e].
enum { MODE_FWD = 0, MODE_DGRAD = 1, MODE_OUT = 2 };
constexpr int UR = 4, UW = 128, UHW = UW + 2; // default tile height, tile width, halo width
// bytes of one channel-chunk plane of an R-row tile's halo ((R + 2) x 130 pixels x 16
// bytes) and of one halo stage (four planes)
template <int R> __host__ __device__ constexpr int u_plane() { return (R + 2) * UHW * 16; }
template <int R> __host__ __device__ constexpr int u_halo() { return 4 * u_plane<R>(); }
constexpr int U_LOAD_WARPS = 4, U_EPI_WARPS = 16;
constexpr int UMMA_THREADS = (U_LOAD_WARPS + 1 + U_EPI_WARPS) * 32;
constexpr int U_TSUM = U_EPI_WARPS;       // partial sums per tile (MODE_OUT)

struct UGeo {
    int B, H, W;
    int tx, ty;           // tiles per image along x and y
    long long ntiles;
};

inline UGeo make_ugeo(int B, int H, int W, int R = UR)
{
    UGeo g;
    g.B = B; g.H = H; g.W = W;
    g.tx = (W + UW - 1) / UW;
    g.ty = (H + R - 1) / R;
    g.ntiles = (long long)B * g.tx * g.ty;
    return g;
}

template <int N, int R = UR>
constexpr int umma_smem_bytes() { return 9 * 4 * N * 16 + 2 * u_halo<R>(); }

__device__ __forceinline__ void mbar_init(unsigned mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count));
}

// Failure self-test: one thread initialises an mbarrier that nothing ever arrives on
// and waits for it with the tensor-core kernels' own bounded wait, here with a short
// limit; when the wait gives up it raises the network's error flag the way those
// kernels do. No tensor-core operation is issued and no tensor memory is allocated.
__global__ void surr_wait_selftest(long long limit, int* err)
{
    __shared__ __align__(8) unsigned long long bar;
    const unsigned mbar = (unsigned)__cvta_generic_to_shared(&bar);
    mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (!mbar_wait_limit(mbar, 0, limit)) atomicExch(err, 1);
}
__device__ __forceinline__ void mbar_arrive(unsigned mbar)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}

template <int MODE, int N, int R = UR>
__global__ void __launch_bounds__(UMMA_THREADS, 1) surr_conv_umma(const bf16* __restrict__ in, const bf16* __restrict__ wu,
                                                                  const float* __restrict__ bias,
                                                                  const bf16* __restrict__ zaux, bf16* __restrict__ out_z,
                                                                  bf16* __restrict__ out_a, float* __restrict__ z5,
                                                                  double* __restrict__ tsum, const UGeo g,
                                                                  int* __restrict__ err)
{
    constexpr int WBYTES = 9 * 4 * N * 16;
    constexpr int UHR = R + 2;            // halo rows of a tile
    constexpr int UPLANE = u_plane<R>(), UHALO = u_halo<R>();
    constexpr int NSET = R * N;           // TMEM columns of one accumulator set
    constexpr int NCOL = 2 * NSET;        // two sets (a power of two >= 32)
    constexpr unsigned IDESC = umma_idesc(UW, N);
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ws = smem;
    unsigned char* hs = smem + WBYTES;    // stage s at hs + s * UHALO
    __shared__ __align__(8) unsigned long long bars[8]; // full[2], empty[2], tfull[2], tempty[2]
    __shared__ unsigned tslot;
    __shared__ float bv[32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned b_full = smem_u32(&bars[0]), b_empty = smem_u32(&bars[2]);
    const unsigned b_tfull = smem_u32(&bars[4]), b_tempty = smem_u32(&bars[6]);

    pdl_trigger();
    // the prologue (weights, barriers, tensor memory) touches nothing the previous kernel writes
    for (int k = tid; k < WBYTES / 16; k += UMMA_THREADS) cp_async16(ws + k * 16, wu + k * 8);
    cp_commit();
    if (tid < 32) bv[tid] = (MODE == MODE_FWD || (MODE == MODE_OUT && tid == 0)) ? bias[tid] : 0.0f;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(b_full + 8 * s, U_LOAD_WARPS * 32);
            mbar_init(b_empty + 8 * s, 1);
            mbar_init(b_tfull + 8 * s, 1);
            mbar_init(b_tempty + 8 * s, U_EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tslot)), "n"(NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    cp_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); // weights -> tensor core reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tslot;
    const int per = g.tx * g.ty;
    bool failed = false;
    pdl_wait();

    if (warp < U_LOAD_WARPS) {
        // ---- loaders: thread lt copies channel chunk kc = lt % 4 of halo columns
        // hc = lt / 4 + 32 m (m < 5, hc < 130) in all six halo rows
        const int kc = tid & 3, hc0 = tid >> 2;
        long long k = 0;
        for (long long tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++k) {
            const int s = (int)(k & 1);
            if (k >= 2 && !mbar_wait(b_empty + 8 * s, (unsigned)(((k >> 1) - 1) & 1))) { failed = true; break; }
            const int b = (int)tile / per;
            const int rem = (int)tile - b * per;
            const int y0 = (rem / g.tx) * R, x0 = (rem - (rem / g.tx) * g.tx) * UW;
            unsigned char* st = hs + s * UHALO + kc * UPLANE;
            int xo[5];
#pragma unroll
            for (int m = 0; m < 5; ++m) xo[m] = wrap_halo(x0 + hc0 + 32 * m - 1, g.W);
#pragma unroll
            for (int hr = 0; hr < UHR; ++hr) {
                const bf16* row = in + (((size_t)b * g.H + wrap_halo(y0 + hr - 1, g.H)) * g.W) * C + kc * 8;
#pragma unroll
                for (int m = 0; m < 5; ++m) {
                    const int hc = hc0 + 32 * m;
                    if (hc < UHW) cp_async16(st + (hr * UHW + hc) * 16, row + (size_t)xo[m] * C);
                }
            }
            cp_commit();
            cp_wait<0>();
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(b_full + 8 * s);
        }
    } else if (warp == U_LOAD_WARPS) {
        // ---- MMA issuer
        if (lane == 0) {
            const unsigned ws_s = smem_u32(ws), hs_s = smem_u32(hs);
            long long k = 0;
            for (long long tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++k) {
                const int s = (int)(k & 1);
                if (!mbar_wait(b_full + 8 * s, (unsigned)((k >> 1) & 1))) { failed = true; break; }
                if (k >= 2 && !mbar_wait(b_tempty + 8 * s, (unsigned)(((k >> 1) - 1) & 1))) { failed = true; break; }
                tc_fence_after();
                const uint64_t a0 = umma_desc(hs_s + (unsigned)(s * UHALO), UPLANE, 128), b0 = umma_desc(ws_s, N * 16, 128);
                const unsigned acc = tmem + (unsigned)(s * NSET);
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
                        for (int kh = 0; kh < 2; ++kh) {
                            const unsigned aoff = (unsigned)(2 * kh * UPLANE + ((r + tap / 3) * UHW + tap % 3) * 16) >> 4;
                            const unsigned boff = (unsigned)((tap * 4 + 2 * kh) * N * 16) >> 4;
                            umma_bf16(acc + (unsigned)(r * N), a0 + aoff, b0 + boff, IDESC, (tap | kh) != 0);
                        }
                umma_commit(b_empty + 8 * s);
                umma_commit(b_tfull + 8 * s);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue
        // warp e: TMEM lane quarter q4 (fixed by the warp index), tile row r and, when a
        // tile has fewer than four rows, channel group cg of its row (chunks k4 of 8)
        constexpr int KPW = R;                           // of the 4 chunks of 8 channels, per warp
        const int e = warp - U_LOAD_WARPS - 1;          // 0 .. 15
        const int q4 = warp & 3, r = (e >> 2) % R, cg = (e >> 2) / R;
        long long k = 0;
        for (long long tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++k) {
            const int s = (int)(k & 1);
            if (!mbar_wait(b_tfull + 8 * s, (unsigned)((k >> 1) & 1))) { failed = true; break; }
            tc_fence_after();
            const int b = (int)tile / per;
            const int rem = (int)tile - b * per;
            const int y = (rem / g.tx) * R + r, x = (rem - (rem / g.tx) * g.tx) * UW + 32 * q4 + lane;
            const bool valid = y < g.H && x < g.W;
            const size_t p = valid ? ((size_t)b * g.H + y) * g.W + x : 0;
            const unsigned ta = tmem + ((unsigned)(32 * q4) << 16) + (unsigned)(s * NSET + r * N);
            double psum = 0.0;
            if (MODE == MODE_OUT) {
                unsigned v[8];
                if (cg == 0) { // the one real output channel
                    tmem_ld8(ta, v);
                    tmem_wait_ld();
                }
                if (valid && cg == 0) {
                    const float z = __uint_as_float(v[0]) + bv[0];
                    z5[p] = z;
                    psum = z;
                }
            } else {
#pragma unroll 1
                for (int k4 = cg * KPW; k4 < (cg + 1) * KPW; ++k4) {
                    unsigned v[8];
                    tmem_ld8(ta + (unsigned)(k4 * 8), v);
                    tmem_wait_ld();
                    unsigned o[4], zw[4];
                    if (!valid) {
                    } else if (MODE == MODE_FWD) {
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const int c = k4 * 8 + h * 2;
                            const float2 z = __fadd2_rn(make_float2(__uint_as_float(v[2 * h]), __uint_as_float(v[2 * h + 1])),
                                                        make_float2(bv[c], bv[c + 1]));
                            zw[h] = pack_bf16(z.x, z.y);
                            const float2 a = gelu2(z);
                            o[h] = pack_bf16(a.x, a.y);
                        }
                        if (out_z) reinterpret_cast<uint4*>(out_z + p * C)[k4] = make_uint4(zw[0], zw[1], zw[2], zw[3]);
                    } else {
                        const uint4 zv = reinterpret_cast<const uint4*>(zaux + p * C)[k4];
                        const unsigned zz[4] = {zv.x, zv.y, zv.z, zv.w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const float2 d = __fmul2_rn(make_float2(__uint_as_float(v[2 * h]), __uint_as_float(v[2 * h + 1])),
                                                        gelu_grad2(unpack_bf16(zz[h])));
                            o[h] = pack_bf16(d.x, d.y);
                        }
                    }
                    if (valid) reinterpret_cast<uint4*>(out_a + p * C)[k4] = make_uint4(o[0], o[1], o[2], o[3]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b_tempty + 8 * s);
            if (MODE == MODE_OUT) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) psum += __shfl_down_sync(0xffffffffu, psum, o);
                if (lane == 0) tsum[(size_t)tile * U_TSUM + e] = psum;
            }
        }
    }
    if (failed) atomicExch(err, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(NCOL));
}

// ---------------------------------------------------------------------------------
// Weight gradient of a hidden layer on the tensor cores:
//   dW[co][ci][tap] = sum_p gz[p][co] a[p + off(tap)][ci],  db[co] = sum_p gz[p][co].
// Warp w (0..8) owns tap w: a 32 x 32 block (two m16 tiles over co, four n8 tiles over
// ci); the K dimension runs over the 256 pixels of each tile, 16 (one tile row) per
// mma. Pixels outside the image have gz = 0 in shared memory. Per-CTA partials:
// part[cta][co * 288 + ci * 9 + tap] and part[cta][9216 + co].
__global__ void __launch_bounds__(WG_THREADS) surr_wgrad_mma(const bf16* __restrict__ gz, const bf16* __restrict__ a,
                                                             float* __restrict__ part, const Geo g)
{
    extern __shared__ __align__(128) unsigned char smem[];
    bf16* gs = reinterpret_cast<bf16*>(smem);     // [256][PS]
    bf16* hs = gs + TH * TW * PS;                  // [324][PS]
    __shared__ float bsum[8][C];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tid4 = lane & 3;
    const int lq = lane >> 3, lr = lane & 7;
    const int j = warp / 3, i = warp - 3 * (warp / 3);

    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
    float bacc = 0.0f;
    const unsigned gs_base = smem_u32(gs), hs_base = smem_u32(hs);

    for (long long tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
        int b, y0, x0;
        tile_origin(g, tile, b, y0, x0);
        for (int k = tid; k < TH * TW * 4; k += WG_THREADS) {
            const int q = k >> 2, part4 = k & 3;
            const int y = y0 + q / TW, x = x0 + (q % TW);
            bf16* dst = gs + q * PS + part4 * 8;
            if (y < g.H && x < g.W)
                cp_async16(dst, gz + ((((size_t)b * g.H + y) * g.W + x) * C + part4 * 8));
            else
                *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
        }
        load_halo(hs, a, g, tile, tid, WG_THREADS);
        cp_commit();
        cp_wait<0>();
        __syncthreads();

#pragma unroll 2
        for (int kr = 0; kr < TH; ++kr) {
            unsigned af[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int px = kr * TW + (lq >> 1) * 8 + lr;
                ldsm_x4_t(gs_base + (unsigned)(px * PS + mt * 16 + (lq & 1) * 8) * 2u, af[mt][0], af[mt][1], af[mt][2],
                          af[mt][3]);
            }
            unsigned bfr[4][2];
#pragma unroll
            for (int nb = 0; nb < 2; ++nb) {
                const int hp = (kr + j) * HWD + (lq & 1) * 8 + lr + i;
                ldsm_x4_t(hs_base + (unsigned)(hp * PS + nb * 16 + (lq >> 1) * 8) * 2u, bfr[2 * nb][0],
                          bfr[2 * nb][1], bfr[2 * nb + 1][0], bfr[2 * nb + 1][1]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bfr[nt][0], bfr[nt][1]);
        }
        if (warp < 8) {
#pragma unroll
            for (int r = 0; r < 32; ++r) bacc += __bfloat162float(gs[(warp * 32 + r) * PS + lane]);
        }
        __syncthreads();
    }

    float* out = part + (size_t)blockIdx.x * LH_N;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int co = mt * 16 + gid + 8 * (e >> 1);
                const int ci = nt * 8 + 2 * tid4 + (e & 1);
                out[co * 288 + ci * 9 + warp] = acc[mt][nt][e];
            }
    if (warp < 8) bsum[warp][lane] = bacc;
    __syncthreads();
    if (tid < C) {
        float s = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += bsum[w][tid];
        out[9216 + tid] = s;
    }
}

// ---------------------------------------------------------------------------------
// Layer 5 (FP32 units): z_5 = conv3x3(a_4, W_5) + b_5 and per-image block sums of z_5.
// Grid (RED_BLOCKS-or-fewer, B); part[b * gridDim.x + blockIdx.x].
__device__ __forceinline__ double block_sum(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    __syncthreads();
    return s; // valid in thread 0
}

// Deterministic sum of n doubles by one warp (fixed assignment and butterfly order).
__device__ __forceinline__ double warp_sum_ordered(const double* v, int n)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int k = lane; k < n; k += 32) s += v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Deterministic block-wide sum of n doubles: thread i sums v[i], v[i + 256], ... in order,
// then a fixed tree over the 256 thread sums. Valid in thread 0; blockDim.x must be 256.
__device__ __forceinline__ double block_sum_ordered(const double* v, int n, double* red)
{
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) s += v[k];
    red[threadIdx.x] = s;
    __syncthreads();
#pragma unroll
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    return red[0];
}

// phi_out = phi + (z_5 - mean(z_5)) per image; tsum holds partial sums of z_5, those of
// image b being [b * tpi, (b + 1) * tpi). With met (one image), the block also writes
// the surr_metrics partials of phi_out (met[blk], met[nb + blk], met[2 nb + blk], nb =
// gridDim.x), recomputing the neighbours' outputs, which round to the same values.
__global__ void __launch_bounds__(256) surr_residual(const float* __restrict__ phi, const float* __restrict__ z5,
                                                     const double* __restrict__ tsum, int tpi,
                                                     float* __restrict__ out, int H, int W, double* __restrict__ met)
{
    __shared__ double red[256];
    pdl_enter();
    const int b = blockIdx.y;
    const long long HWn = (long long)H * W;
    const double m = block_sum_ordered(tsum + (size_t)b * tpi, tpi, red) / (double)HWn;
    const size_t base = (size_t)b * HWn;
    auto o = [&](long long q) { return (float)((double)phi[base + q] + ((double)z5[base + q] - m)); };
    double sm = 0.0, sp = 0.0, sgr = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < HWn; q += (long long)gridDim.x * blockDim.x) {
        const float fo = o(q);
        out[base + q] = fo;
        if (met) { // the terms of surr_metrics, on the stored values
            const int y = (int)(q / W), x = (int)(q - (long long)y * W);
            const double f = fo;
            sm += f;
            if (f > 0.05 && f < 0.95) {
                const double gx = 0.5 * ((double)o((long long)y * W + wrap1(x + 1, W)) - (double)o((long long)y * W + wrap1(x - 1, W)));
                const double gy = 0.5 * ((double)o((long long)wrap1(y + 1, H) * W + x) - (double)o((long long)wrap1(y - 1, H) * W + x));
                sp += f * (1.0 - f);
                sgr += sqrt(gx * gx + gy * gy);
            }
        }
    }
    if (met) {
        __syncthreads(); // red is reused
        sm = block_sum(sm, red);
        sp = block_sum(sp, red);
        sgr = block_sum(sgr, red);
        if (threadIdx.x == 0) {
            met[blockIdx.x] = sm;
            met[gridDim.x + blockIdx.x] = sp;
            met[2 * gridDim.x + blockIdx.x] = sgr;
        }
    }
}

// Loss partials sum (out - tgt)^2 and sums of g = 2 (out - tgt) / N per image block.
__global__ void __launch_bounds__(256) surr_loss_part(const float* __restrict__ out, const float* __restrict__ tgt,
                                                      double* __restrict__ lpart, double* __restrict__ gpart, int H,
                                                      int W, double two_over_n)
{
    __shared__ double red[8];
    const int b = blockIdx.y;
    const long long HWn = (long long)H * W;
    double sl = 0.0, sg = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < HWn; q += (long long)gridDim.x * blockDim.x) {
        const size_t k = (size_t)b * HWn + q;
        const double d = (double)out[k] - (double)tgt[k];
        sl += d * d;
        sg += (float)(two_over_n * d);
    }
    sl = block_sum(sl, red);
    sg = block_sum(sg, red);
    if (threadIdx.x == 0) {
        lpart[(size_t)b * gridDim.x + blockIdx.x] = sl;
        gpart[(size_t)b * gridDim.x + blockIdx.x] = sg;
    }
}

// dL/dz_5 = g - mean(g) per image (the adjoint of the mean removal).
__global__ void __launch_bounds__(256) surr_gz5(const float* __restrict__ out, const float* __restrict__ tgt,
                                                const double* __restrict__ gpart, float* __restrict__ gz5, int H, int W,
                                                double two_over_n)
{
    __shared__ double mean;
    const int b = blockIdx.y;
    const long long HWn = (long long)H * W;
    if (threadIdx.x < 32) {
        const double sm = warp_sum_ordered(gpart + (size_t)b * gridDim.x, gridDim.x);
        if (threadIdx.x == 0) mean = sm / (double)HWn;
    }
    __syncthreads();
    const float m = (float)mean;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < HWn; q += (long long)gridDim.x * blockDim.x) {
        const size_t k = (size_t)b * HWn + q;
        const float g = (float)(two_over_n * ((double)out[k] - (double)tgt[k]));
        gz5[k] = g - m;
    }
}

// Layer 5 backward per 16 x 16 tile: partials of dW_5 (part[cta][ci * 9 + tap]) and
// db_5 (part[cta][288]); dL/dz_4 = (sum_tap W_5[ci][tap] gz5[p - off(tap)]) GELU'(z_4[p]).
__global__ void __launch_bounds__(256) surr_out_bwd(const bf16* __restrict__ a4, const bf16* __restrict__ z4,
                                                    const float* __restrict__ gz5, const float* __restrict__ params,
                                                    bf16* __restrict__ gz4, float* __restrict__ part, const Geo g)
{
    extern __shared__ __align__(128) unsigned char smem[];
    bf16* hs = reinterpret_cast<bf16*>(smem);          // a_4 halo [324][PS]
    __shared__ float gh[HPX];                           // gz5 halo
    __shared__ float w[L5_N];
    const int tid = threadIdx.x;
    for (int k = tid; k < L5_N; k += blockDim.x)
        w[k] = k < 288 ? __bfloat162float(__float2bfloat16_rn(params[OFF_W5 + k])) : params[OFF_W5 + k];
    // weight gradient: thread (ci, row group rg) owns dW_5[ci][0..8] over tile rows 2 rg, 2 rg + 1,
    // sliding a 3 x 3 window of a_4 channel ci along each row (3 shared loads per pixel)
    const int wci = tid & 31, rg = tid >> 5;
    float acc[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t] = 0.0f;
    float bacc = 0.0f;
    for (long long tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
        int b, y0, x0;
        tile_origin(g, tile, b, y0, x0);
        load_halo(hs, a4, g, tile, tid, 256);
        cp_commit();
        for (int q = tid; q < HPX; q += 256) {
            const int hy = q / HWD, hx = q - hy * HWD;
            const int y = wrap_halo(y0 + hy - 1, g.H), x = wrap_halo(x0 + hx - 1, g.W);
            gh[q] = gz5[((size_t)b * g.H + y) * g.W + x];
        }
        cp_wait<0>();
        __syncthreads();
        const int vr = min(TH, g.H - y0), vc = min(TW, g.W - x0); // valid rows / columns of the tile
#pragma unroll 1
        for (int r = 2 * rg; r < 2 * rg + 2 && r < vr; ++r) {
            float wv[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) wv[j][i] = __bfloat162float(hs[((r + j) * HWD + i) * PS + wci]);
#pragma unroll 1
            for (int c = 0; c < vc; ++c) {
                const float gq = gh[(r + 1) * HWD + c + 1];
                bacc += gq;
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int i = 0; i < 3; ++i) acc[j * 3 + i] = fmaf(gq, wv[j][i], acc[j * 3 + i]);
                if (c + 1 < vc) {
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        wv[j][0] = wv[j][1];
                        wv[j][1] = wv[j][2];
                        wv[j][2] = __bfloat162float(hs[((r + j) * HWD + c + 3) * PS + wci]);
                    }
                }
            }
        }
        // dL/dz_4 at the tile's own pixels
        {
            const int r = tid / TW, c = tid % TW;
            const int y = y0 + r, x = x0 + c;
            if (r < vr && c < vc) {
                float gn[9];
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) gn[tap] = gh[(r + 2 - tap / 3) * HWD + c + 2 - tap % 3];
                const size_t base = (((size_t)b * g.H + y) * g.W + x) * C;
                const uint4* zs = reinterpret_cast<const uint4*>(z4 + base);
                uint4* go = reinterpret_cast<uint4*>(gz4 + base);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint4 zv = zs[k];
                    const unsigned zz[4] = {zv.x, zv.y, zv.z, zv.w};
                    unsigned o[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int ci = k * 8 + h * 2;
                        float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
                        for (int tap = 0; tap < 9; ++tap) {
                            d0 = fmaf(w[ci * 9 + tap], gn[tap], d0);
                            d1 = fmaf(w[(ci + 1) * 9 + tap], gn[tap], d1);
                        }
                        const float2 z = unpack_bf16(zz[h]);
                        o[h] = pack_bf16(d0 * gelu_grad_f(z.x), d1 * gelu_grad_f(z.y));
                    }
                    go[k] = make_uint4(o[0], o[1], o[2], o[3]);
                }
            }
        }
        __syncthreads();
    }
    // the eight row groups' sums, added in order of rg (the halo buffer is free now)
    float* red = reinterpret_cast<float*>(smem);              // [8][L5_N]
#pragma unroll
    for (int t = 0; t < 9; ++t) red[rg * L5_N + wci * 9 + t] = acc[t];
    if (wci == 0) red[rg * L5_N + 288] = bacc;
    __syncthreads();
    float* out = part + (size_t)blockIdx.x * L5_N;
    for (int k = tid; k < L5_N; k += 256) {
        float sum = 0.0f;
        for (int q = 0; q < 8; ++q) sum += red[q * L5_N + k];
        out[k] = sum;
    }
}

// Layer 1 weight gradient per tile: part[cta][co * 27 + ci * 9 + tap] and part[cta][864 + co].
// Thread (co, ci, rg) owns dW_1[co][ci][0..8] over tile rows 4 rg .. 4 rg + 3, sliding a
// 3 x 3 window of input channel ci along each row (one gz load and 3 input loads per
// pixel); the row groups are added in order at the end.
constexpr int IW_THREADS = 384;

__global__ void __launch_bounds__(IW_THREADS) surr_in_wgrad(const bf16* __restrict__ gz1, const float* __restrict__ phi,
                                                            const float* __restrict__ u, const float* __restrict__ v,
                                                            float* __restrict__ part, const Geo g)
{
    __shared__ float gsm[TH * TW][C + 1];   // also the final reduction buffer [4][L1_N]
    __shared__ float xs[3][HPX];
    const int tid = threadIdx.x;
    const int co = tid & 31, ci = (tid >> 5) % 3, rg = tid / 96;
    float acc[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t] = 0.0f;
    float bacc = 0.0f;
    for (long long tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
        int b, y0, x0;
        tile_origin(g, tile, b, y0, x0);
        if (tid < TH * TW) {
            const int r = tid / TW, c = tid % TW;
            const int y = y0 + r, x = x0 + c;
            if (y < g.H && x < g.W) {
                const uint4* src = reinterpret_cast<const uint4*>(gz1 + (((size_t)b * g.H + y) * g.W + x) * C);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint4 vv = src[k];
                    const unsigned ww[4] = {vv.x, vv.y, vv.z, vv.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const float2 f = unpack_bf16(ww[h]);
                        gsm[tid][k * 8 + h * 2] = f.x;
                        gsm[tid][k * 8 + h * 2 + 1] = f.y;
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < C; ++k) gsm[tid][k] = 0.0f; // pixels outside the image add nothing
            }
        }
        for (int q = tid; q < HPX; q += IW_THREADS) {
            const int hy = q / HWD, hx = q - hy * HWD;
            const int y = wrap_halo(y0 + hy - 1, g.H), x = wrap_halo(x0 + hx - 1, g.W);
            const size_t k = ((size_t)b * g.H + y) * g.W + x;
            xs[0][q] = phi[k];
            xs[1][q] = u[k] * U_SCALE;
            xs[2][q] = v[k] * U_SCALE;
        }
        __syncthreads();
#pragma unroll 1
        for (int r = 4 * rg; r < 4 * rg + 4; ++r) {
            float wv[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) wv[j][i] = xs[ci][(r + j) * HWD + i];
#pragma unroll 4
            for (int c = 0; c < TW; ++c) {
                const float gq = gsm[r * TW + c][co];
                bacc += gq;
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int i = 0; i < 3; ++i) acc[j * 3 + i] = fmaf(gq, wv[j][i], acc[j * 3 + i]);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    wv[j][0] = wv[j][1];
                    wv[j][1] = wv[j][2];
                    wv[j][2] = xs[ci][(r + j) * HWD + min(c + 3, HWD - 1)];
                }
            }
        }
        __syncthreads();
    }
    float* red = &gsm[0][0];                 // [4][L1_N]
#pragma unroll
    for (int t = 0; t < 9; ++t) red[rg * L1_N + co * 27 + ci * 9 + t] = acc[t];
    if (ci == 0) red[rg * L1_N + 864 + co] = bacc;
    __syncthreads();
    float* out = part + (size_t)blockIdx.x * L1_N;
    for (int k = tid; k < L1_N; k += IW_THREADS) {
        float sum = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) sum += red[q * L1_N + k];
        out[k] = sum;
    }
}

// grad[k] = sum over c < ncta of part[c][k] in FP64. A block owns 32 consecutive k;
// thread (kx, cy) sums c = cy, cy + 8, ... in order, and the eight sums are added in
// order of cy (deterministic).
__global__ void __launch_bounds__(256) surr_reduce(const float* __restrict__ part, int ncta, int stride, int count,
                                                   float* __restrict__ grad)
{
    __shared__ double sm[8][33];
    const int kx = threadIdx.x & 31, cy = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + kx;
    double acc = 0.0;
    if (k < count)
        for (int c = cy; c < ncta; c += 8) acc += (double)part[(size_t)c * stride + k];
    sm[cy][kx] = acc;
    __syncthreads();
    if (cy == 0 && k < count) {
        double t = 0.0;
#pragma unroll
        for (int y = 0; y < 8; ++y) t += sm[y][kx];
        grad[k] = (float)t;
    }
}

__global__ void surr_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                          const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                          float c2)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.0f - b1) * gk;
        const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

// BF16 tensor-core operands in the [tap][chunk][n][8] layout of surr_conv_umma:
//   wu[l]  (forward, n = co, K = ci):       W_l[co][8 chunk + e][tap]
//   wdu[l] (input gradient, n = ci, K = co): W_l[8 chunk + e][ci][8 - tap]
//   w5u    (layer 5, n < 16, only n = 0):   W_5[0][8 chunk + e][tap]
__global__ void surr_pack(const float* __restrict__ p, bf16* __restrict__ wu, bf16* __restrict__ wdu,
                          bf16* __restrict__ w5u)
{
    const int n_hidden = 3 * 9 * C * C, n5 = 9 * 4 * 16 * 8;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_hidden + n5; k += gridDim.x * blockDim.x) {
        if (k < n_hidden) {
            const int l = k / (9 * C * C), r = k % (9 * C * C);
            const int tap = r / (4 * C * 8), kc = (r / (C * 8)) % 4, n = (r / 8) % C, e = r % 8;
            const float* W = p + OFF_W2 + l * LH_N;                  // [co][ci][tap]
            wu[k] = __float2bfloat16_rn(W[(n * C + kc * 8 + e) * 9 + tap]);
            wdu[k] = __float2bfloat16_rn(W[((kc * 8 + e) * C + n) * 9 + (8 - tap)]);
        } else {
            const int r = k - n_hidden;
            const int tap = r / (4 * 16 * 8), kc = (r / (16 * 8)) % 4, n = (r / 8) % 16, e = r % 8;
            w5u[r] = __float2bfloat16_rn(n == 0 ? p[OFF_W5 + (kc * 8 + e) * 9 + tap] : 0.0f);
        }
    }
}

// Mass and width partials of one field: part[blk] = sum phi, part[nb + blk] = sum over
// the band of phi (1 - phi), part[2 nb + blk] = sum over the band of |grad phi|.
__global__ void __launch_bounds__(256) surr_metrics(const float* __restrict__ phi, int H, int W,
                                                    double* __restrict__ part)
{
    __shared__ double red[8];
    const int HWn = H * W;
    double sm = 0.0, sp = 0.0, sgr = 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < HWn; q += gridDim.x * blockDim.x) {
        const int y = q / W, x = q - y * W;
        const double f = phi[q];
        sm += f;
        if (f > 0.05 && f < 0.95) {
            const double gx = 0.5 * ((double)phi[y * W + wrap1(x + 1, W)] - (double)phi[y * W + wrap1(x - 1, W)]);
            const double gy = 0.5 * ((double)phi[wrap1(y + 1, H) * W + x] - (double)phi[wrap1(y - 1, H) * W + x]);
            sp += f * (1.0 - f);
            sgr += sqrt(gx * gx + gy * gy);
        }
    }
    sm = block_sum(sm, red);
    sp = block_sum(sp, red);
    sgr = block_sum(sgr, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sm;
        part[gridDim.x + blockIdx.x] = sp;
        part[2 * gridDim.x + blockIdx.x] = sgr;
    }
}

} // namespace surr

using namespace surr;

// ---------------------------------------------------------------------------------
// Host side.

constexpr int HYB_DEPTH = 16; // surrogate windows run ahead of one host check

struct lbm_ace_net {
    int dev = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    float* params = nullptr;  // FP32 master [NPARAM]
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* grad = nullptr;
    bf16* wu = nullptr;       // tensor-core operands: [3][9][4][32][8] forward,
    bf16* wdu = nullptr;      //   [3][9][4][32][8] input gradient,
    bf16* w5u = nullptr;      //   [9][4][16][8] layer 5
    int* derr = nullptr;      // set by a kernel whose bounded wait gave up
    long long adam_t = 0;
    bool have_grad = false;
    // activations, sized for cap pixels
    long long cap = 0;
    bf16* z[4] = {nullptr, nullptr, nullptr, nullptr};
    bf16* a[4] = {nullptr, nullptr, nullptr, nullptr};
    bf16* gzb[2] = {nullptr, nullptr};
    float* z5 = nullptr;
    float* gz5 = nullptr;
    float* outb = nullptr;    // phi_out of loss_grad
    double* rpart = nullptr;  int rpart_n = 0;   // per-image reduction partials
    double* rpart2 = nullptr;
    double* tsum = nullptr;   long long tsum_n = 0; // per-tile sums of z_5
    float* wpart = nullptr;   size_t wpart_n = 0; // per-CTA gradient partials
    int conv_grid = 0, out_grid = 0, wg_grid = 0, ob_grid = 0, iw_grid = 0;
    int conv_occ = 0, out_occ = 0;  // resident CTAs per SM reported for the tensor-core kernels
    size_t conv_smem = 0, out_smem = 0, wg_smem = 0, ob_smem = 0;
    size_t conv_smem2 = 0, out_smem2 = 0; // 2-row tiles (small forwards)
    std::vector<double> hpart;
    // hybrid advance: HYB_DEPTH + 1 phase fields (a ring), u, v, and the metric partials of
    // HYB_DEPTH speculative windows
    float* hyb[HYB_DEPTH + 3] = {};
    long long hyb_n = 0;
    double* hyb_part = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_net_err;

int nfail(lbm_ace_net* n, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (n) n->err = buf; else g_net_err = buf;
    return code;
}

#define NCK(net, call)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return nfail((net), e_ == cudaErrorMemoryAllocation ? LBM_ACE_ENOMEM : LBM_ACE_ECUDA,  \
                         "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);     \
    } while (0)

struct NetDevice {
    int prev = -1;
    explicit NetDevice(int d) { cudaGetDevice(&prev); if (prev != d) cudaSetDevice(d); }
    ~NetDevice() { int cur = -1; cudaGetDevice(&cur); if (prev >= 0 && cur != prev) cudaSetDevice(prev); }
};

int grid1(long long n, int sms)
{
    long long g = (n + 255) / 256;
    const long long cap = (long long)sms * 8;
    if (g > cap) g = cap;
    return (int)std::max(1LL, g);
}

int red_blocks(int H, int W)
{
    const long long n = (long long)H * W;
    return (int)std::max(1LL, std::min<long long>(RED_BLOCKS, (n + 255) / 256));
}

int met_blocks(int H, int W)
{
    const long long n = (long long)H * W;
    return (int)std::max(1LL, std::min<long long>(MET_BLOCKS, (n + 255) / 256));
}

void free_acts(lbm_ace_net* n)
{
    for (int l = 0; l < 4; ++l) { cudaFree(n->z[l]); cudaFree(n->a[l]); n->z[l] = n->a[l] = nullptr; }
    for (int k = 0; k < 2; ++k) { cudaFree(n->gzb[k]); n->gzb[k] = nullptr; }
    cudaFree(n->z5); cudaFree(n->gz5); cudaFree(n->outb);
    n->z5 = n->gz5 = n->outb = nullptr;
    n->cap = 0;
}

int ensure_acts(lbm_ace_net* n, long long P, int B, int H = 3, int W = 3)
{
    const long long nt = make_ugeo(B, H, W, 2).ntiles * U_TSUM; // the 2-row tiles are the most
    if (nt > n->tsum_n) {
        cudaFree(n->tsum);
        n->tsum = nullptr;
        n->tsum_n = 0;
        NCK(n, cudaMalloc(&n->tsum, (size_t)nt * sizeof(double)));
        n->tsum_n = nt;
    }
    if (P > n->cap) {
        free_acts(n);
        const size_t act = (size_t)P * C * sizeof(bf16);
        for (int l = 0; l < 4; ++l) {
            NCK(n, cudaMalloc(&n->z[l], act));
            NCK(n, cudaMalloc(&n->a[l], act));
        }
        for (int k = 0; k < 2; ++k) NCK(n, cudaMalloc(&n->gzb[k], act));
        NCK(n, cudaMalloc(&n->z5, (size_t)P * sizeof(float)));
        NCK(n, cudaMalloc(&n->gz5, (size_t)P * sizeof(float)));
        NCK(n, cudaMalloc(&n->outb, (size_t)P * sizeof(float)));
        n->cap = P;
    }
    const int need = std::max(B * RED_BLOCKS, MET_BLOCKS) * 3;
    if (need > n->rpart_n) {
        cudaFree(n->rpart); cudaFree(n->rpart2);
        n->rpart = n->rpart2 = nullptr;
        n->rpart_n = 0;
        NCK(n, cudaMalloc(&n->rpart, (size_t)need * sizeof(double)));
        NCK(n, cudaMalloc(&n->rpart2, (size_t)need * sizeof(double)));
        n->rpart_n = need;
    }
    return LBM_ACE_OK;
}

int check_dims(lbm_ace_net* n, int B, int H, int W)
{
    if (B < 1 || H < 3 || W < 3) return nfail(n, LBM_ACE_EINVAL, "batch %d of %d x %d: need batch >= 1, sides >= 3", B, H, W);
    if ((long long)B * H * W > (1LL << 31) / C)
        return nfail(n, LBM_ACE_EINVAL, "batch %d of %d x %d: too many nodes", B, H, W);
    return LBM_ACE_OK;
}

// Forward pass into n->z / n->a (z stored when keep_z) and out.
template <typename... KArgs, typename... Args>
void launch_chain(void (*kernel)(KArgs...), dim3 grid, int threads, size_t smem, cudaStream_t stream, Args&&... args)
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

// met (B = 1 only): also write the surr_metrics partials of `out` (3 x red_blocks(H, W))
int run_forward(lbm_ace_net* n, const float* phi, const float* u, const float* v, float* out, int B, int H, int W,
                bool keep_z, double* met = nullptr)
{
    // the forward chain is launched with programmatic stream serialisation (each kernel
    // waits for its predecessor with griddepcontrol.wait before reading its output)
    // 2-row tiles when 4-row tiles would not give every conv CTA two (a CTA then
    // pipelines the loads, MMAs and epilogues of several tiles)
    const bool small = make_ugeo(B, H, W).ntiles < 2LL * n->conv_grid;
    const UGeo g = make_ugeo(B, H, W, small ? 2 : UR);
    const long long P = (long long)B * H * W;
    launch_chain(surr_in_fwd, dim3(grid1(P, n->sms)), 256, 0, n->stream, phi, u, v,
                 (const float*)n->params, keep_z ? n->z[0] : nullptr, n->a[0], B, H, W);
    const int grid = (int)std::min<long long>(g.ntiles, n->conv_grid);
    for (int l = 0; l < 3; ++l) {
        launch_chain(small ? surr_conv_umma<MODE_FWD, 32, 2> : surr_conv_umma<MODE_FWD, 32, UR>, dim3(grid),
                     UMMA_THREADS, small ? n->conv_smem2 : n->conv_smem, n->stream,
                     (const bf16*)n->a[l], (const bf16*)(n->wu + (size_t)l * 9 * C * C),
                     (const float*)(n->params + OFF_W2 + l * LH_N + 9216), (const bf16*)nullptr,
                     keep_z ? n->z[l + 1] : (bf16*)nullptr, n->a[l + 1], (float*)nullptr, (double*)nullptr, g,
                     n->derr);
    }
    const int gout = (int)std::min<long long>(g.ntiles, n->out_grid);
    launch_chain(small ? surr_conv_umma<MODE_OUT, 16, 2> : surr_conv_umma<MODE_OUT, 16, UR>, dim3(gout),
                 UMMA_THREADS, small ? n->out_smem2 : n->out_smem, n->stream,
                 (const bf16*)n->a[3], (const bf16*)n->w5u, (const float*)(n->params + OFF_W5 + 288),
                 (const bf16*)nullptr, (bf16*)nullptr, (bf16*)nullptr, n->z5, n->tsum, g, n->derr);
    launch_chain(surr_residual, dim3(red_blocks(H, W), B), 256, 0, n->stream, phi, (const float*)n->z5,
                 (const double*)n->tsum, (int)(g.tx * g.ty * U_TSUM), out, H, W, B == 1 ? met : nullptr);
    NCK(n, cudaGetLastError());
    return LBM_ACE_OK;
}

int check_err(lbm_ace_net* n)
{
    int e = 0;
    NCK(n, cudaMemcpy(&e, n->derr, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        NCK(n, cudaMemset(n->derr, 0, sizeof(int)));
        return nfail(n, LBM_ACE_ETIMEOUT, "a tensor-core wait gave up (tcgen05 commit not observed within ~1 s)");
    }
    return LBM_ACE_OK;
}

int repack(lbm_ace_net* n)
{
    surr_pack<<<grid1(3 * 9 * C * C + 9 * 4 * 16 * 8, n->sms), 256, 0, n->stream>>>(n->params, n->wu, n->wdu, n->w5u);
    NCK(n, cudaGetLastError());
    return LBM_ACE_OK;
}

} // namespace

extern "C" {

int lbm_ace_net_create(int device, void* stream, lbm_ace_net** out)
{
    if (!out) return nfail(nullptr, LBM_ACE_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev)
        return nfail(nullptr, LBM_ACE_ECUDA, "CUDA device %d unavailable (%s)", device,
                     e == cudaSuccess ? "ordinal out of range" : cudaGetErrorString(e));
    lbm_ace_net* n = new (std::nothrow) lbm_ace_net;
    if (!n) return nfail(nullptr, LBM_ACE_ENOMEM, "host allocation failed");
    NetDevice gd(device);
    n->dev = device;
    n->stream = (cudaStream_t)stream;
    auto bail = [&](int rc) { g_net_err = n->err; lbm_ace_net_destroy(n); return rc; };
#define CREATE_CK(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) \
        return bail(nfail(n, e_ == cudaErrorMemoryAllocation ? LBM_ACE_ENOMEM : LBM_ACE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_))); } while (0)
    CREATE_CK(cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, device));
    CREATE_CK(cudaMalloc(&n->params, NPARAM * sizeof(float)));
    CREATE_CK(cudaMalloc(&n->adam_m, NPARAM * sizeof(float)));
    CREATE_CK(cudaMalloc(&n->adam_v, NPARAM * sizeof(float)));
    CREATE_CK(cudaMalloc(&n->grad, NPARAM * sizeof(float)));
    CREATE_CK(cudaMalloc(&n->wu, 3 * 9 * C * C * sizeof(bf16)));
    CREATE_CK(cudaMalloc(&n->wdu, 3 * 9 * C * C * sizeof(bf16)));
    CREATE_CK(cudaMalloc(&n->w5u, 9 * 4 * 16 * 8 * sizeof(bf16)));
    CREATE_CK(cudaMalloc(&n->derr, sizeof(int)));
    CREATE_CK(cudaMemset(n->derr, 0, sizeof(int)));
    CREATE_CK(cudaMemset(n->params, 0, NPARAM * sizeof(float)));
    CREATE_CK(cudaMemset(n->adam_m, 0, NPARAM * sizeof(float)));
    CREATE_CK(cudaMemset(n->adam_v, 0, NPARAM * sizeof(float)));
    CREATE_CK(cudaMemset(n->grad, 0, NPARAM * sizeof(float)));
    CREATE_CK(cudaMemset(n->wu, 0, 3 * 9 * C * C * sizeof(bf16)));
    CREATE_CK(cudaMemset(n->wdu, 0, 3 * 9 * C * C * sizeof(bf16)));
    CREATE_CK(cudaMemset(n->w5u, 0, 9 * 4 * 16 * 8 * sizeof(bf16)));
    // launch shapes: persistent grids of resident CTAs
    n->conv_smem = umma_smem_bytes<32>();
    n->out_smem = umma_smem_bytes<16>();
    n->conv_smem2 = umma_smem_bytes<32, 2>();
    n->out_smem2 = umma_smem_bytes<16, 2>();
    n->wg_smem = (size_t)(TH * TW * PS + HPX * PS) * sizeof(bf16);
    n->ob_smem = (size_t)HPX * PS * sizeof(bf16);
    CREATE_CK(cudaFuncSetAttribute(surr_conv_umma<MODE_FWD, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)n->conv_smem));
    CREATE_CK(cudaFuncSetAttribute(surr_conv_umma<MODE_DGRAD, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)n->conv_smem));
    CREATE_CK(cudaFuncSetAttribute(surr_conv_umma<MODE_OUT, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)n->out_smem));
    CREATE_CK(cudaFuncSetAttribute(surr_conv_umma<MODE_FWD, 32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)n->conv_smem2));
    CREATE_CK(cudaFuncSetAttribute(surr_conv_umma<MODE_OUT, 16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)n->out_smem2));
    CREATE_CK(cudaFuncSetAttribute(surr_conv_umma<MODE_FWD, 32, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    CREATE_CK(cudaFuncSetAttribute(surr_conv_umma<MODE_OUT, 16, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    // the persistent tensor-core kernels want all of the unified L1/shared storage as shared memory
    CREATE_CK(cudaFuncSetAttribute(surr_conv_umma<MODE_FWD, 32>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    CREATE_CK(cudaFuncSetAttribute(surr_conv_umma<MODE_DGRAD, 32>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    CREATE_CK(cudaFuncSetAttribute(surr_conv_umma<MODE_OUT, 16>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    CREATE_CK(cudaFuncSetAttribute(surr_wgrad_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)n->wg_smem));
    int occ = 0;
    // persistent, one CTA per SM (the occupancy the runtime reports for tcgen05 kernels)
    CREATE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, surr_conv_umma<MODE_FWD, 32>, UMMA_THREADS, n->conv_smem));
    n->conv_occ = occ;
    n->conv_grid = n->sms;
    CREATE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, surr_conv_umma<MODE_OUT, 16>, UMMA_THREADS, n->out_smem));
    n->out_occ = occ;
    n->out_grid = n->sms;
    CREATE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, surr_wgrad_mma, WG_THREADS, n->wg_smem));
    n->wg_grid = std::max(1, occ) * n->sms;
    CREATE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, surr_out_bwd, 256, n->ob_smem));
    n->ob_grid = std::max(1, occ) * n->sms;
    CREATE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, surr_in_wgrad, IW_THREADS, 0));
    n->iw_grid = std::max(1, occ) * n->sms;
    n->wpart_n = (size_t)std::max({(size_t)n->wg_grid * LH_N, (size_t)n->ob_grid * L5_N, (size_t)n->iw_grid * L1_N});
    CREATE_CK(cudaMalloc(&n->wpart, n->wpart_n * sizeof(float)));
#undef CREATE_CK
    *out = n;
    return LBM_ACE_OK;
}

int lbm_ace_net_set_params(lbm_ace_net* n, const float* params, size_t count)
{
    if (!n) return nfail(nullptr, LBM_ACE_EINVAL, "net is NULL");
    if (!params || count != (size_t)NPARAM)
        return nfail(n, LBM_ACE_EINVAL, "params must hold %d values (got %zu)", NPARAM, count);
    for (size_t k = 0; k < count; ++k)
        if (!std::isfinite(params[k])) return nfail(n, LBM_ACE_EINVAL, "params[%zu] is not finite", k);
    NetDevice gd(n->dev);
    NCK(n, cudaMemcpyAsync(n->params, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    NCK(n, cudaMemsetAsync(n->adam_m, 0, NPARAM * sizeof(float), n->stream));
    NCK(n, cudaMemsetAsync(n->adam_v, 0, NPARAM * sizeof(float), n->stream));
    n->adam_t = 0;
    n->have_grad = false;
    const int rc = repack(n);
    if (rc) return rc;
    NCK(n, cudaStreamSynchronize(n->stream));
    return LBM_ACE_OK;
}

int lbm_ace_net_get_params(lbm_ace_net* n, float* params, size_t count)
{
    if (!n) return nfail(nullptr, LBM_ACE_EINVAL, "net is NULL");
    if (!params || count != (size_t)NPARAM)
        return nfail(n, LBM_ACE_EINVAL, "params must hold %d values (got %zu)", NPARAM, count);
    NetDevice gd(n->dev);
    NCK(n, cudaMemcpyAsync(params, n->params, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    NCK(n, cudaStreamSynchronize(n->stream));
    return LBM_ACE_OK;
}

int lbm_ace_net_forward(lbm_ace_net* n, const float* phi, const float* u, const float* v, float* phi_out, int batch,
                        int ny, int nx)
{
    if (!n) return nfail(nullptr, LBM_ACE_EINVAL, "net is NULL");
    if (!phi || !u || !v || !phi_out) return nfail(n, LBM_ACE_EINVAL, "an image pointer is NULL");
    if (phi_out == phi || phi_out == u || phi_out == v) return nfail(n, LBM_ACE_EINVAL, "phi_out aliases an input");
    int rc = check_dims(n, batch, ny, nx);
    if (rc) return rc;
    NetDevice gd(n->dev);
    rc = ensure_acts(n, (long long)batch * ny * nx, batch, ny, nx);
    if (rc) return rc;
    return run_forward(n, phi, u, v, phi_out, batch, ny, nx, false);
}

int lbm_ace_net_loss_grad(lbm_ace_net* n, const float* phi, const float* u, const float* v, const float* target,
                          int batch, int ny, int nx, double* loss, float* grad, size_t count)
{
    if (!n) return nfail(nullptr, LBM_ACE_EINVAL, "net is NULL");
    if (!phi || !u || !v || !target) return nfail(n, LBM_ACE_EINVAL, "an image pointer is NULL");
    if (grad && count != (size_t)NPARAM) return nfail(n, LBM_ACE_EINVAL, "grad must hold %d values (got %zu)", NPARAM, count);
    int rc = check_dims(n, batch, ny, nx);
    if (rc) return rc;
    NetDevice gd(n->dev);
    const long long P = (long long)batch * ny * nx;
    rc = ensure_acts(n, P, batch, ny, nx);
    if (rc) return rc;
    rc = run_forward(n, phi, u, v, n->outb, batch, ny, nx, true);
    if (rc) return rc;
    const Geo g = make_geo(batch, ny, nx);
    const int rb = red_blocks(ny, nx);
    const double two_over_n = 2.0 / (double)P;
    surr_loss_part<<<dim3(rb, batch), 256, 0, n->stream>>>(n->outb, target, n->rpart, n->rpart2, ny, nx, two_over_n);
    surr_gz5<<<dim3(rb, batch), 256, 0, n->stream>>>(n->outb, target, n->rpart2, n->gz5, ny, nx, two_over_n);
    // layer 5
    const int gob = (int)std::min<long long>(g.ntiles, n->ob_grid);
    surr_out_bwd<<<gob, 256, n->ob_smem, n->stream>>>(n->a[3], n->z[3], n->gz5, n->params, n->gzb[0], n->wpart, g);
    surr_reduce<<<(L5_N + 31) / 32, 256, 0, n->stream>>>(n->wpart, gob, L5_N, L5_N, n->grad + OFF_W5);
    // layers 4, 3, 2: weight gradient, then dL/dz of the layer below
    const int gwg = (int)std::min<long long>(g.ntiles, n->wg_grid);
    const UGeo ug = make_ugeo(batch, ny, nx);
    const int gcv = (int)std::min<long long>(ug.ntiles, n->conv_grid);
    int cur = 0;
    for (int l = 2; l >= 0; --l) { // hidden layer l + 2 (1-based), input a[l], output gz of z[l]
        surr_wgrad_mma<<<gwg, WG_THREADS, n->wg_smem, n->stream>>>(n->gzb[cur], n->a[l], n->wpart, g);
        surr_reduce<<<(LH_N + 31) / 32, 256, 0, n->stream>>>(n->wpart, gwg, LH_N, LH_N, n->grad + OFF_W2 + l * LH_N);
        surr_conv_umma<MODE_DGRAD, 32><<<gcv, UMMA_THREADS, n->conv_smem, n->stream>>>(
            n->gzb[cur], n->wdu + (size_t)l * 9 * C * C, nullptr, n->z[l], nullptr, n->gzb[cur ^ 1], nullptr, nullptr,
            ug, n->derr);
        cur ^= 1;
    }
    // layer 1
    const int giw = (int)std::min<long long>(g.ntiles, n->iw_grid);
    surr_in_wgrad<<<giw, IW_THREADS, 0, n->stream>>>(n->gzb[cur], phi, u, v, n->wpart, g);
    surr_reduce<<<(L1_N + 31) / 32, 256, 0, n->stream>>>(n->wpart, giw, L1_N, L1_N, n->grad + OFF_W1);
    NCK(n, cudaGetLastError());
    n->have_grad = true;
    if (loss) {
        const size_t np = (size_t)batch * rb;
        n->hpart.resize(np);
        NCK(n, cudaMemcpyAsync(n->hpart.data(), n->rpart, np * sizeof(double), cudaMemcpyDeviceToHost, n->stream));
        NCK(n, cudaStreamSynchronize(n->stream));
        double s = 0.0;
        for (size_t k = 0; k < np; ++k) s += n->hpart[k];
        *loss = s / (double)P;
        rc = check_err(n);
        if (rc) return rc;
        if (!std::isfinite(*loss)) return nfail(n, LBM_ACE_ENUMERIC, "loss is not finite (%g)", *loss);
    }
    if (grad) {
        NCK(n, cudaMemcpyAsync(grad, n->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
        NCK(n, cudaStreamSynchronize(n->stream));
    }
    return LBM_ACE_OK;
}

int lbm_ace_net_adam(lbm_ace_net* n, float lr, float beta1, float beta2, float eps)
{
    if (!n) return nfail(nullptr, LBM_ACE_EINVAL, "net is NULL");
    if (!n->have_grad) return nfail(n, LBM_ACE_EINVAL, "no gradient: call lbm_ace_net_loss_grad first");
    if (!(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return nfail(n, LBM_ACE_EINVAL, "Adam hyper-parameters out of range");
    NetDevice gd(n->dev);
    n->adam_t += 1;
    const double c1 = 1.0 - std::pow((double)beta1, (double)n->adam_t);
    const double c2 = 1.0 - std::pow((double)beta2, (double)n->adam_t);
    surr_adam<<<grid1(NPARAM, n->sms), 256, 0, n->stream>>>(n->params, n->adam_m, n->adam_v, n->grad, NPARAM, lr,
                                                             beta1, beta2, eps, (float)c1, (float)c2);
    NCK(n, cudaGetLastError());
    return repack(n);
}

int lbm_ace_net_gather(lbm_ace_net* n, float* dst, const float* src, const long long* index, int count,
                       long long image_elems)
{
    if (!n) return nfail(nullptr, LBM_ACE_EINVAL, "net is NULL");
    if (!dst || !src || (!index && count > 0) || count < 0 || image_elems < 1)
        return nfail(n, LBM_ACE_EINVAL, "gather: invalid arguments");
    NetDevice gd(n->dev);
    for (int k = 0; k < count; ++k) {
        if (index[k] < 0) return nfail(n, LBM_ACE_EINVAL, "gather: index[%d] = %lld < 0", k, index[k]);
        NCK(n, cudaMemcpyAsync(dst + (size_t)k * image_elems, src + (size_t)index[k] * image_elems,
                               (size_t)image_elems * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
    }
    return LBM_ACE_OK;
}

int lbm_ace_net_metrics(lbm_ace_net* n, const float* phi, int ny, int nx, double* mass, double* width)
{
    if (!n) return nfail(nullptr, LBM_ACE_EINVAL, "net is NULL");
    if (!phi) return nfail(n, LBM_ACE_EINVAL, "phi is NULL");
    int rc = check_dims(n, 1, ny, nx);
    if (rc) return rc;
    NetDevice gd(n->dev);
    rc = ensure_acts(n, 0, 1);
    if (rc) return rc;
    const int rb = met_blocks(ny, nx);
    surr_metrics<<<rb, 256, 0, n->stream>>>(phi, ny, nx, n->rpart);
    NCK(n, cudaGetLastError());
    n->hpart.resize(3 * (size_t)rb);
    NCK(n, cudaMemcpyAsync(n->hpart.data(), n->rpart, 3 * (size_t)rb * sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    NCK(n, cudaStreamSynchronize(n->stream));
    double s[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < 3; ++q)
        for (int k = 0; k < rb; ++k) s[q] += n->hpart[(size_t)q * rb + k];
    if (mass) *mass = s[0];
    if (width) *width = s[2] > 0.0 ? s[1] / s[2] : 0.0;
    if (!std::isfinite(s[0]) || !std::isfinite(s[1]) || !std::isfinite(s[2]))
        return nfail(n, LBM_ACE_ENUMERIC, "phase field is not finite");
    return LBM_ACE_OK;
}

int lbm_ace_net_synchronize(lbm_ace_net* n)
{
    if (!n) return nfail(nullptr, LBM_ACE_EINVAL, "net is NULL");
    NetDevice gd(n->dev);
    NCK(n, cudaStreamSynchronize(n->stream));
    return check_err(n);
}

int lbm_ace_net_wait_selftest(lbm_ace_net* n, long long limit_cycles)
{
    if (!n) return nfail(nullptr, LBM_ACE_EINVAL, "net is NULL");
    if (limit_cycles < 1 || limit_cycles > kSurrWaitCycles)
        return nfail(n, LBM_ACE_EINVAL, "limit_cycles = %lld: must be in [1, %lld]", limit_cycles, kSurrWaitCycles);
    NetDevice gd(n->dev);
    surr_wait_selftest<<<1, 1, 0, n->stream>>>(limit_cycles, n->derr);
    NCK(n, cudaGetLastError());
    NCK(n, cudaStreamSynchronize(n->stream));
    return check_err(n);
}

int lbm_ace_net_launch_shape(const lbm_ace_net* n, int* conv_ctas, int* conv_occupancy, int* out_ctas,
                             int* out_occupancy, int* sms)
{
    if (!n) return nfail(nullptr, LBM_ACE_EINVAL, "net is NULL");
    if (conv_ctas) *conv_ctas = n->conv_grid;
    if (conv_occupancy) *conv_occupancy = n->conv_occ;
    if (out_ctas) *out_ctas = n->out_grid;
    if (out_occupancy) *out_occupancy = n->out_occ;
    if (sms) *sms = n->sms;
    return LBM_ACE_OK;
}

const char* lbm_ace_net_last_error(const lbm_ace_net* n) { return n ? n->err.c_str() : g_net_err.c_str(); }

void lbm_ace_net_destroy(lbm_ace_net* n)
{
    if (!n) return;
    NetDevice gd(n->dev);
    if (n->stream) cudaStreamSynchronize(n->stream); else cudaDeviceSynchronize();
    free_acts(n);
    void* bufs[] = {n->params, n->adam_m, n->adam_v, n->grad, n->wu, n->wdu, n->w5u, n->derr, n->tsum,
                    n->rpart, n->rpart2, n->wpart, n->hyb_part};
    for (void* p : bufs) cudaFree(p);
    for (float* p : n->hyb) cudaFree(p);
    delete n;
}

int lbm_ace_hybrid_advance(lbm_ace_ctx* lat, lbm_ace_net* n, long long windows, double mass_tol, double width_tol,
                           lbm_ace_hybrid_stats* stats)
{
    if (!n) return nfail(nullptr, LBM_ACE_EINVAL, "net is NULL");
    if (!lat) return nfail(n, LBM_ACE_EINVAL, "lattice is NULL");
    if (windows < 0 || !(mass_tol >= 0.0) || !(width_tol >= 0.0))
        return nfail(n, LBM_ACE_EINVAL, "windows must be >= 0 and tolerances >= 0");
    if (lbm_ace_get_stream(lat) != (void*)n->stream)
        return nfail(n, LBM_ACE_EINVAL, "the lattice and the net must work on the same stream");
    lbm_ace_params P;
    int rc = lbm_ace_get_params(lat, &P);
    if (rc) return nfail(n, rc, "lattice: %s", lbm_ace_last_error(lat));
    if (P.velocity_kind == LBM_ACE_VEL_CALLBACK)
        return nfail(n, LBM_ACE_EINVAL, "the hybrid advance needs a vortex, uniform or field velocity");
    if (P.device != n->dev) return nfail(n, LBM_ACE_EINVAL, "the lattice and the net are on different devices");
    const int nx = P.nx, ny = P.ny;
    const long long N = (long long)nx * ny;
    NetDevice gd(n->dev);
    rc = ensure_acts(n, N, 1, ny, nx);
    if (rc) return rc;
    constexpr int NB = HYB_DEPTH + 1;
    if (n->hyb_n < N) {
        for (float*& p : n->hyb) { cudaFree(p); p = nullptr; }
        n->hyb_n = 0;
        for (float*& p : n->hyb) NCK(n, cudaMalloc(&p, (size_t)N * sizeof(float)));
        n->hyb_n = N;
    }
    if (!n->hyb_part) NCK(n, cudaMalloc(&n->hyb_part, (size_t)HYB_DEPTH * 3 * MET_BLOCKS * sizeof(double)));
    float* ring[NB];
    for (int k = 0; k < NB; ++k) ring[k] = n->hyb[k];
    float* u = n->hyb[NB];
    float* v = n->hyb[NB + 1];
    const int rb = red_blocks(ny, nx); // blocks of the residual kernel, which reduces the checks
#define LAT(call) do { const int r_ = (call); if (r_) return nfail(n, r_, "lattice: %s", lbm_ace_last_error(lat)); } while (0)
    lbm_ace_hybrid_stats st;
    std::memset(&st, 0, sizeof st);
    long long t = lbm_ace_steps_done(lat);
    int c = 0; // ring index of the current field
    LAT(lbm_ace_get_phi_device(lat, ring[c]));
    rc = lbm_ace_net_metrics(n, ring[c], ny, nx, &st.mass0, &st.width0);
    if (rc) return rc;
    bool stale = false; // the lattice lags behind ring[c] (surrogate windows since its last step)
    const int K = LBM_ACE_NET_K;
    std::vector<double> hp((size_t)HYB_DEPTH * 3 * rb);
    long long w = 0;
    int run_ahead = HYB_DEPTH; // speculation depth: 1 after a rejection, doubled after each clean group
    while (w < windows) {
        // up to run_ahead surrogate windows back to back, each field in the next ring slot,
        // with its checks reduced on the device; one synchronisation for the group
        const int depth = (int)std::min<long long>(run_ahead, windows - w);
        for (int j = 0; j < depth; ++j) {
            LAT(lbm_ace_velocity_device(lat, (double)(t + (long long)j * K) + 0.5 * K, u, v));
            // the residual kernel also reduces the window's checks (mass and width)
            rc = run_forward(n, ring[(c + j) % NB], u, v, ring[(c + j + 1) % NB], 1, ny, nx, false,
                             n->hyb_part + (size_t)j * 3 * rb);
            if (rc) return rc;
        }
        NCK(n, cudaGetLastError());
        NCK(n, cudaMemcpyAsync(hp.data(), n->hyb_part, (size_t)depth * 3 * rb * sizeof(double), cudaMemcpyDeviceToHost,
                               n->stream));
        NCK(n, cudaStreamSynchronize(n->stream));
        int acc = 0; // windows accepted, in order, before the first that fails a check
        for (; acc < depth; ++acc) {
            double q[3] = {0.0, 0.0, 0.0};
            for (int m = 0; m < 3; ++m)
                for (int k = 0; k < rb; ++k) q[m] += hp[((size_t)acc * 3 + m) * rb + k];
            const double mass = q[0], width = q[2] > 0.0 ? q[1] / q[2] : 0.0;
            if (!std::isfinite(q[0]) || !std::isfinite(q[1]) || !std::isfinite(q[2])) break;
            const double dm = st.mass0 != 0.0 ? std::fabs(mass - st.mass0) / std::fabs(st.mass0) : std::fabs(mass);
            const double dw = st.width0 > 0.0 ? std::fabs(width - st.width0) / st.width0 : (width == 0.0 ? 0.0 : INFINITY);
            if (!(dm <= mass_tol && dw <= width_tol)) break;
            st.max_mass_drift = std::max(st.max_mass_drift, dm);
            st.max_width_dev = std::max(st.max_width_dev, dw);
        }
        if (acc > 0) {
            c = (c + acc) % NB;
            t += (long long)acc * K;
            stale = true;
            st.surrogate_windows += acc;
            st.windows += acc;
            w += acc;
        }
        run_ahead = acc < depth ? 1 : std::min(HYB_DEPTH, 2 * run_ahead);
        if (acc < depth) { // the first rejected window: K lattice Boltzmann steps from ring[c]
            if (stale) LAT(lbm_ace_reset_device(lat, ring[c], t));
            LAT(lbm_ace_step(lat, K));
            LAT(lbm_ace_get_phi_device(lat, ring[c]));
            stale = false;
            t += K;
            st.fallback_windows += 1;
            st.windows += 1;
            w += 1;
        }
    }
    if (stale) LAT(lbm_ace_reset_device(lat, ring[c], t));
    LAT(lbm_ace_synchronize(lat));
#undef LAT
    rc = check_err(n);
    if (rc) return rc;
    if (stats) *stats = st;
    return LBM_ACE_OK;
}

} // extern "C"
