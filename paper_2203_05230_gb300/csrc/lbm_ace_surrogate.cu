// lbm_ace_surrogate.cu -- the learned surrogate declared in include/lbm_ace_surrogate.h:
// a 5-layer periodic 3x3 convolutional network (3 -> 32 -> 32 -> 32 -> 32 -> 1, GELU,
// residual with the image mean of the output removed), its training kernels
// (loss, back-propagation, Adam) and the hybrid advance with the lattice Boltzmann
// fallback.
//
// Kernels (all hand-written):
//   surr_in_fwd      layer 1 on FP32 units: 27 inputs -> 32 outputs per node
//   surr_conv_mma    layers 2-4 forward and their input gradients: implicit GEMM on the
//                    tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulators),
//                    16 x 16 output tiles, 18 x 18 x 32 halo staged by cp.async,
//                    double-buffered, persistent CTAs
//   surr_wgrad_mma   layers 2-4 weight gradients: per-tap GEMM over the pixels on the
//                    tensor cores (ldmatrix.trans operands), per-CTA partials
//   surr_out_fwd / surr_residual   layer 5, mean removal, residual add
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
constexpr int CONV_THREADS = 256;
constexpr int WG_THREADS = 288;       // 9 warps, one per tap
constexpr int RED_BLOCKS = 64;        // blocks per image for per-image reductions
constexpr int W_SMEM = 9 * C * PS;    // packed weights of one layer in shared memory (bf16)

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

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

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
__global__ void __launch_bounds__(256) surr_in_fwd(const float* __restrict__ phi, const float* __restrict__ u,
                                                   const float* __restrict__ v, const float* __restrict__ params,
                                                   bf16* __restrict__ z1, bf16* __restrict__ a1, int B, int H, int W)
{
    __shared__ float w[L1_N];
    for (int k = threadIdx.x; k < L1_N; k += blockDim.x) w[k] = params[OFF_W1 + k];
    __syncthreads();
    const long long P = (long long)B * H * W;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % W);
        const long long r = p / W;
        const int y = (int)(r % H);
        const long long b = r / H;
        float in[27];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int yy = wrap1(y + j - 1, H);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const long long q = (b * H + yy) * W + wrap1(x + i - 1, W);
                in[j * 3 + i] = phi[q];
                in[9 + j * 3 + i] = u[q] * U_SCALE;
                in[18 + j * 3 + i] = v[q] * U_SCALE;
            }
        }
        uint4* zo = reinterpret_cast<uint4*>(z1 + p * C);
        uint4* ao = reinterpret_cast<uint4*>(a1 + p * C);
#pragma unroll 1
        for (int k4 = 0; k4 < 4; ++k4) { // eight output channels per 16-byte store
            unsigned zw[4], aw[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int co = k4 * 8 + h * 2;
                float s0 = w[864 + co], s1 = w[864 + co + 1];
#pragma unroll
                for (int k = 0; k < 27; ++k) {
                    s0 = fmaf(w[co * 27 + k], in[k], s0);
                    s1 = fmaf(w[(co + 1) * 27 + k], in[k], s1);
                }
                zw[h] = pack_bf16(s0, s1);
                aw[h] = pack_bf16(gelu_f(s0), gelu_f(s1));
            }
            if (z1) zo[k4] = make_uint4(zw[0], zw[1], zw[2], zw[3]);
            ao[k4] = make_uint4(aw[0], aw[1], aw[2], aw[3]);
        }
    }
}

// ---------------------------------------------------------------------------------
// Layers 2-4 on the tensor cores. out[p][n] = sum_tap sum_k wpk[tap][n][k] in[p + off(tap)][k]
// with off(tap) = (tap / 3 - 1, tap % 3 - 1).
//   MODE_FWD:   z = out + bias; stores z (if out_z) and GELU(z) (out_a), BF16.
//   MODE_DGRAD: out is dL/da of the layer below; stores dL/dz = out * GELU'(zaux), BF16.
// Each warp owns two tile rows (two m16 tiles of 16 pixels) and all 32 output channels.
enum { MODE_FWD = 0, MODE_DGRAD = 1 };

template <int MODE>
__global__ void __launch_bounds__(CONV_THREADS, 3) surr_conv_mma(const bf16* __restrict__ in, const bf16* __restrict__ wpk,
                                                              const float* __restrict__ bias,
                                                              const bf16* __restrict__ zaux, bf16* __restrict__ out_z,
                                                              bf16* __restrict__ out_a, const Geo g)
{
    extern __shared__ __align__(16) unsigned char smem[];
    bf16* ws = reinterpret_cast<bf16*>(smem);
    bf16* hs = ws + W_SMEM;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tid4 = lane & 3;
    const int lq = lane >> 3, lr = lane & 7;

    for (int k = tid; k < 9 * C * 4; k += CONV_THREADS) {
        const int row = k >> 2, part = k & 3;
        cp_async16(ws + row * PS + part * 8, wpk + row * C + part * 8);
    }
    long long tile = blockIdx.x;
    int buf = 0;
    if (tile < g.ntiles) load_halo(hs, in, g, tile, tid, CONV_THREADS);
    cp_commit();

    float bv[8];
    if (MODE == MODE_FWD) {
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            bv[2 * nt] = bias[nt * 8 + 2 * tid4];
            bv[2 * nt + 1] = bias[nt * 8 + 2 * tid4 + 1];
        }
    }

    const unsigned ws_base = smem_u32(ws);
    for (; tile < g.ntiles; tile += gridDim.x) {
        const long long next = tile + gridDim.x;
        if (next < g.ntiles) load_halo(hs + (buf ^ 1) * (HPX * PS), in, g, next, tid, CONV_THREADS);
        cp_commit();
        cp_wait<1>();
        __syncthreads();

        const unsigned hs_base = smem_u32(hs + buf * (HPX * PS));
        float acc[2][4][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;

        const int r0 = warp * 2;
        // per-lane ldmatrix row addresses at tap (0, 0), k-half 0; every (tap, k-half)
        // adds a compile-time byte offset
        const unsigned a_addr = hs_base + (unsigned)(((r0 * HWD + (lq & 1) * 8 + lr) * PS + (lq >> 1) * 8) * 2);
        const unsigned b_addr = ws_base + (unsigned)((((lq >> 1) * 8 + lr) * PS + (lq & 1) * 8) * 2);
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int j = tap / 3, i = tap % 3;
#pragma unroll
            for (int kh = 0; kh < 2; ++kh) {
                unsigned a[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
                    ldsm_x4(a_addr + (unsigned)((((mt + j) * HWD + i) * PS + kh * 16) * 2), a[mt][0], a[mt][1], a[mt][2],
                            a[mt][3]);
                unsigned bfr[4][2];
#pragma unroll
                for (int nb = 0; nb < 2; ++nb)
                    ldsm_x4(b_addr + (unsigned)(((tap * C + nb * 16) * PS + kh * 16) * 2), bfr[2 * nb][0],
                            bfr[2 * nb][1], bfr[2 * nb + 1][0], bfr[2 * nb + 1][1]);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a[mt], bfr[nt][0], bfr[nt][1]);
            }
        }

        int b, y0, x0;
        tile_origin(g, tile, b, y0, x0);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int y = y0 + r0 + mt;
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                const int x = x0 + gid + hf * 8;
                if (y >= g.H || x >= g.W) continue;
                const size_t base = (((size_t)b * g.H + y) * g.W + x) * C;
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const int co = nt * 8 + 2 * tid4;
                    const float c0 = acc[mt][nt][2 * hf], c1 = acc[mt][nt][2 * hf + 1];
                    if (MODE == MODE_FWD) {
                        const float z0 = c0 + bv[2 * nt], z1 = c1 + bv[2 * nt + 1];
                        if (out_z) *reinterpret_cast<unsigned*>(out_z + base + co) = pack_bf16(z0, z1);
                        *reinterpret_cast<unsigned*>(out_a + base + co) = pack_bf16(gelu_f(z0), gelu_f(z1));
                    } else {
                        const float2 z = unpack_bf16(*reinterpret_cast<const unsigned*>(zaux + base + co));
                        *reinterpret_cast<unsigned*>(out_a + base + co) =
                            pack_bf16(c0 * gelu_grad_f(z.x), c1 * gelu_grad_f(z.y));
                    }
                }
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    cp_wait<0>();
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
    extern __shared__ __align__(16) unsigned char smem[];
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

__global__ void __launch_bounds__(256) surr_out_fwd(const bf16* __restrict__ a4, const float* __restrict__ params,
                                                    float* __restrict__ z5, double* __restrict__ part, int H, int W)
{
    __shared__ float w[L5_N];
    __shared__ double red[8];
    for (int k = threadIdx.x; k < L5_N; k += blockDim.x) w[k] = params[OFF_W5 + k];
    __syncthreads();
    const int b = blockIdx.y;
    const long long HWn = (long long)H * W;
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < HWn; q += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(q / W), x = (int)(q % W);
        float acc = w[288];
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int yy = wrap1(y + tap / 3 - 1, H), xx = wrap1(x + tap % 3 - 1, W);
            const uint4* src = reinterpret_cast<const uint4*>(a4 + (((size_t)b * H + yy) * W + xx) * C);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint4 v = src[k];
                const unsigned vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const float2 f = unpack_bf16(vv[h]);
                    const int ci = k * 8 + h * 2;
                    acc = fmaf(w[ci * 9 + tap], f.x, acc);
                    acc = fmaf(w[(ci + 1) * 9 + tap], f.y, acc);
                }
            }
        }
        z5[(size_t)b * HWn + q] = acc;
        s += acc;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(size_t)b * gridDim.x + blockIdx.x] = s;
}

__device__ __forceinline__ double image_sum(const double* part, int nb)
{
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += part[k];
    return s;
}

// phi_out = phi + (z_5 - mean(z_5)) per image.
__global__ void __launch_bounds__(256) surr_residual(const float* __restrict__ phi, const float* __restrict__ z5,
                                                     const double* __restrict__ part, float* __restrict__ out, int H,
                                                     int W)
{
    __shared__ double mean;
    const int b = blockIdx.y;
    const long long HWn = (long long)H * W;
    if (threadIdx.x == 0) mean = image_sum(part + (size_t)b * gridDim.x, gridDim.x) / (double)HWn;
    __syncthreads();
    const double m = mean;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < HWn; q += (long long)gridDim.x * blockDim.x) {
        const size_t k = (size_t)b * HWn + q;
        out[k] = (float)((double)phi[k] + ((double)z5[k] - m));
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
    if (threadIdx.x == 0) mean = image_sum(gpart + (size_t)b * gridDim.x, gridDim.x) / (double)HWn;
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
    extern __shared__ __align__(16) unsigned char smem[];
    bf16* hs = reinterpret_cast<bf16*>(smem);          // a_4 halo [324][PS]
    __shared__ float gh[HPX];                           // gz5 halo
    __shared__ float w[L5_N];
    const int tid = threadIdx.x;
    for (int k = tid; k < L5_N; k += blockDim.x) w[k] = params[OFF_W5 + k];
    float acc0 = 0.0f, acc1 = 0.0f;
    const int k0 = tid, k1 = tid + 256; // outputs of this thread (k1 valid when < 289)
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
        // weight gradient partials
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int k = s ? k1 : k0;
            if (k >= L5_N) continue;
            float a = 0.0f;
            if (k == 288) {
                for (int r = 0; r < vr; ++r)
                    for (int c = 0; c < vc; ++c) a += gh[(r + 1) * HWD + c + 1];
            } else {
                const int ci = k / 9, tap = k - 9 * (k / 9), j = tap / 3, i = tap % 3;
                for (int r = 0; r < vr; ++r)
                    for (int c = 0; c < vc; ++c)
                        a = fmaf(gh[(r + 1) * HWD + c + 1], __bfloat162float(hs[((r + j) * HWD + c + i) * PS + ci]), a);
            }
            if (s) acc1 += a; else acc0 += a;
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
    float* out = part + (size_t)blockIdx.x * L5_N;
    out[k0] = acc0;
    if (k1 < L5_N) out[k1] = acc1;
}

// Layer 1 weight gradient per tile: part[cta][co * 27 + ci * 9 + tap] and part[cta][864 + co].
__global__ void __launch_bounds__(256) surr_in_wgrad(const bf16* __restrict__ gz1, const float* __restrict__ phi,
                                                     const float* __restrict__ u, const float* __restrict__ v,
                                                     float* __restrict__ part, const Geo g)
{
    __shared__ float gsm[TH * TW][C + 1];
    __shared__ float xs[3][HPX];
    const int tid = threadIdx.x;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (long long tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
        int b, y0, x0;
        tile_origin(g, tile, b, y0, x0);
        {
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
                for (int k = 0; k < C; ++k) gsm[tid][k] = 0.0f;
            }
        }
        for (int q = tid; q < HPX; q += 256) {
            const int hy = q / HWD, hx = q - hy * HWD;
            const int y = wrap_halo(y0 + hy - 1, g.H), x = wrap_halo(x0 + hx - 1, g.W);
            const size_t k = ((size_t)b * g.H + y) * g.W + x;
            xs[0][q] = phi[k];
            xs[1][q] = u[k] * U_SCALE;
            xs[2][q] = v[k] * U_SCALE;
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int k = tid + 256 * s;
            if (k >= L1_N) continue;
            float a = 0.0f;
            if (k >= 864) {
                const int co = k - 864;
                for (int q = 0; q < TH * TW; ++q) a += gsm[q][co];
            } else {
                const int co = k / 27, ci = (k / 9) % 3, tap = k % 9, j = tap / 3, i = tap % 3;
                for (int r = 0; r < TH; ++r)
                    for (int c = 0; c < TW; ++c) a = fmaf(gsm[r * TW + c][co], xs[ci][(r + j) * HWD + c + i], a);
            }
            acc[s] += a;
        }
        __syncthreads();
    }
    float* out = part + (size_t)blockIdx.x * L1_N;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int k = tid + 256 * s;
        if (k < L1_N) out[k] = acc[s];
    }
}

// grad[k] = sum over CTAs of part[cta][k] (FP64, fixed order).
__global__ void surr_reduce(const float* __restrict__ part, int ncta, int stride, int count, float* __restrict__ grad)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < ncta; ++c) s += (double)part[(size_t)c * stride + k];
        grad[k] = (float)s;
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

// BF16 copies of W_2..W_4 for the tensor-core kernels: forward layout wf[l][tap][co][ci]
// and input-gradient layout wd[l][tap'][ci][co] = W[co][ci][8 - tap'].
__global__ void surr_pack(const float* __restrict__ p, bf16* __restrict__ wf, bf16* __restrict__ wd)
{
    const int n = 3 * 9 * C * C;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int l = k / (9 * C * C), r = k % (9 * C * C);
        const int co = r / (C * 9), ci = (r / 9) % C, tap = r % 9;
        const bf16 w = __float2bfloat16_rn(p[OFF_W2 + l * LH_N + r]);
        wf[(size_t)l * 9 * C * C + (tap * C + co) * C + ci] = w;
        wd[(size_t)l * 9 * C * C + ((8 - tap) * C + ci) * C + co] = w;
    }
}

// Mass and width partials of one field: part[blk] = sum phi, part[nb + blk] = sum over
// the band of phi (1 - phi), part[2 nb + blk] = sum over the band of |grad phi|.
__global__ void __launch_bounds__(256) surr_metrics(const float* __restrict__ phi, int H, int W,
                                                    double* __restrict__ part)
{
    __shared__ double red[8];
    const long long HWn = (long long)H * W;
    double sm = 0.0, sp = 0.0, sgr = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < HWn; q += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(q / W), x = (int)(q % W);
        const double f = phi[q];
        sm += f;
        if (f > 0.05 && f < 0.95) {
            const double gx = 0.5 * ((double)phi[(long long)y * W + wrap1(x + 1, W)] - (double)phi[(long long)y * W + wrap1(x - 1, W)]);
            const double gy = 0.5 * ((double)phi[(long long)wrap1(y + 1, H) * W + x] - (double)phi[(long long)wrap1(y - 1, H) * W + x]);
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

struct lbm_ace_net {
    int dev = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    float* params = nullptr;  // FP32 master [NPARAM]
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* grad = nullptr;
    bf16* wf = nullptr;       // [3][9][32][32]
    bf16* wd = nullptr;
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
    float* wpart = nullptr;   size_t wpart_n = 0; // per-CTA gradient partials
    int conv_grid = 0, wg_grid = 0, ob_grid = 0, iw_grid = 0;
    size_t conv_smem = 0, wg_smem = 0, ob_smem = 0;
    std::vector<double> hpart;
    float* hyb[4] = {nullptr, nullptr, nullptr, nullptr}; // hybrid advance: phi, candidate, u, v
    long long hyb_n = 0;
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

void free_acts(lbm_ace_net* n)
{
    for (int l = 0; l < 4; ++l) { cudaFree(n->z[l]); cudaFree(n->a[l]); n->z[l] = n->a[l] = nullptr; }
    for (int k = 0; k < 2; ++k) { cudaFree(n->gzb[k]); n->gzb[k] = nullptr; }
    cudaFree(n->z5); cudaFree(n->gz5); cudaFree(n->outb);
    n->z5 = n->gz5 = n->outb = nullptr;
    n->cap = 0;
}

int ensure_acts(lbm_ace_net* n, long long P, int B)
{
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
    const int need = B * RED_BLOCKS * 3;
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
int run_forward(lbm_ace_net* n, const float* phi, const float* u, const float* v, float* out, int B, int H, int W,
                bool keep_z)
{
    const Geo g = make_geo(B, H, W);
    const long long P = (long long)B * H * W;
    surr_in_fwd<<<grid1(P, n->sms), 256, 0, n->stream>>>(phi, u, v, n->params, keep_z ? n->z[0] : nullptr, n->a[0],
                                                         B, H, W);
    const int grid = (int)std::min<long long>(g.ntiles, n->conv_grid);
    for (int l = 0; l < 3; ++l) {
        surr_conv_mma<MODE_FWD><<<grid, CONV_THREADS, n->conv_smem, n->stream>>>(
            n->a[l], n->wf + (size_t)l * 9 * C * C, n->params + OFF_W2 + l * LH_N + 9216, nullptr,
            keep_z ? n->z[l + 1] : nullptr, n->a[l + 1], g);
    }
    const int rb = red_blocks(H, W);
    surr_out_fwd<<<dim3(rb, B), 256, 0, n->stream>>>(n->a[3], n->params, n->z5, n->rpart, H, W);
    surr_residual<<<dim3(rb, B), 256, 0, n->stream>>>(phi, n->z5, n->rpart, out, H, W);
    NCK(n, cudaGetLastError());
    return LBM_ACE_OK;
}

int repack(lbm_ace_net* n)
{
    surr_pack<<<grid1(3 * 9 * C * C, n->sms), 256, 0, n->stream>>>(n->params, n->wf, n->wd);
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
    CREATE_CK(cudaMalloc(&n->wf, 3 * 9 * C * C * sizeof(bf16)));
    CREATE_CK(cudaMalloc(&n->wd, 3 * 9 * C * C * sizeof(bf16)));
    CREATE_CK(cudaMemset(n->params, 0, NPARAM * sizeof(float)));
    CREATE_CK(cudaMemset(n->adam_m, 0, NPARAM * sizeof(float)));
    CREATE_CK(cudaMemset(n->adam_v, 0, NPARAM * sizeof(float)));
    CREATE_CK(cudaMemset(n->grad, 0, NPARAM * sizeof(float)));
    CREATE_CK(cudaMemset(n->wf, 0, 3 * 9 * C * C * sizeof(bf16)));
    CREATE_CK(cudaMemset(n->wd, 0, 3 * 9 * C * C * sizeof(bf16)));
    // launch shapes: persistent grids of resident CTAs
    n->conv_smem = (size_t)(W_SMEM + 2 * HPX * PS) * sizeof(bf16);
    n->wg_smem = (size_t)(TH * TW * PS + HPX * PS) * sizeof(bf16);
    n->ob_smem = (size_t)HPX * PS * sizeof(bf16);
    CREATE_CK(cudaFuncSetAttribute(surr_conv_mma<MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)n->conv_smem));
    CREATE_CK(cudaFuncSetAttribute(surr_conv_mma<MODE_DGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)n->conv_smem));
    CREATE_CK(cudaFuncSetAttribute(surr_wgrad_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)n->wg_smem));
    int occ = 0;
    CREATE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, surr_conv_mma<MODE_FWD>, CONV_THREADS, n->conv_smem));
    n->conv_grid = std::max(1, occ) * n->sms;
    CREATE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, surr_wgrad_mma, WG_THREADS, n->wg_smem));
    n->wg_grid = std::max(1, occ) * n->sms;
    CREATE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, surr_out_bwd, 256, n->ob_smem));
    n->ob_grid = std::max(1, occ) * n->sms;
    CREATE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, surr_in_wgrad, 256, 0));
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
    rc = ensure_acts(n, (long long)batch * ny * nx, batch);
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
    rc = ensure_acts(n, P, batch);
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
    surr_reduce<<<grid1(L5_N, n->sms), 256, 0, n->stream>>>(n->wpart, gob, L5_N, L5_N, n->grad + OFF_W5);
    // layers 4, 3, 2: weight gradient, then dL/dz of the layer below
    const int gwg = (int)std::min<long long>(g.ntiles, n->wg_grid);
    const int gcv = (int)std::min<long long>(g.ntiles, n->conv_grid);
    int cur = 0;
    for (int l = 2; l >= 0; --l) { // hidden layer l + 2 (1-based), input a[l], output gz of z[l]
        surr_wgrad_mma<<<gwg, WG_THREADS, n->wg_smem, n->stream>>>(n->gzb[cur], n->a[l], n->wpart, g);
        surr_reduce<<<grid1(LH_N, n->sms), 256, 0, n->stream>>>(n->wpart, gwg, LH_N, LH_N, n->grad + OFF_W2 + l * LH_N);
        surr_conv_mma<MODE_DGRAD><<<gcv, CONV_THREADS, n->conv_smem, n->stream>>>(
            n->gzb[cur], n->wd + (size_t)l * 9 * C * C, nullptr, n->z[l], nullptr, n->gzb[cur ^ 1], g);
        cur ^= 1;
    }
    // layer 1
    const int giw = (int)std::min<long long>(g.ntiles, n->iw_grid);
    surr_in_wgrad<<<giw, 256, 0, n->stream>>>(n->gzb[cur], phi, u, v, n->wpart, g);
    surr_reduce<<<grid1(L1_N, n->sms), 256, 0, n->stream>>>(n->wpart, giw, L1_N, L1_N, n->grad + OFF_W1);
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
    const int rb = red_blocks(ny, nx);
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
    return LBM_ACE_OK;
}

const char* lbm_ace_net_last_error(const lbm_ace_net* n) { return n ? n->err.c_str() : g_net_err.c_str(); }

void lbm_ace_net_destroy(lbm_ace_net* n)
{
    if (!n) return;
    NetDevice gd(n->dev);
    if (n->stream) cudaStreamSynchronize(n->stream); else cudaDeviceSynchronize();
    free_acts(n);
    void* bufs[] = {n->params, n->adam_m, n->adam_v, n->grad, n->wf, n->wd, n->rpart, n->rpart2, n->wpart,
                    n->hyb[0], n->hyb[1], n->hyb[2], n->hyb[3]};
    for (void* p : bufs) cudaFree(p);
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
    rc = ensure_acts(n, N, 1);
    if (rc) return rc;
    if (n->hyb_n < N) {
        for (int k = 0; k < 4; ++k) { cudaFree(n->hyb[k]); n->hyb[k] = nullptr; }
        n->hyb_n = 0;
        for (int k = 0; k < 4; ++k) NCK(n, cudaMalloc(&n->hyb[k], (size_t)N * sizeof(float)));
        n->hyb_n = N;
    }
    float* cur = n->hyb[0];
    float* cand = n->hyb[1];
    float* u = n->hyb[2];
    float* v = n->hyb[3];
#define LAT(call) do { const int r_ = (call); if (r_) return nfail(n, r_, "lattice: %s", lbm_ace_last_error(lat)); } while (0)
    lbm_ace_hybrid_stats st;
    std::memset(&st, 0, sizeof st);
    long long t = lbm_ace_steps_done(lat);
    LAT(lbm_ace_get_phi_device(lat, cur));
    rc = lbm_ace_net_metrics(n, cur, ny, nx, &st.mass0, &st.width0);
    if (rc) return rc;
    bool stale = false; // the lattice lags behind cur (surrogate windows since its last step)
    const int K = LBM_ACE_NET_K;
    for (long long w = 0; w < windows; ++w) {
        LAT(lbm_ace_velocity_device(lat, (double)t + 0.5 * K, u, v));
        rc = run_forward(n, cur, u, v, cand, 1, ny, nx, false);
        if (rc) return rc;
        double m = 0.0, wd = 0.0;
        rc = lbm_ace_net_metrics(n, cand, ny, nx, &m, &wd);
        if (rc && rc != LBM_ACE_ENUMERIC) return rc;
        const double dm = st.mass0 != 0.0 ? std::fabs(m - st.mass0) / std::fabs(st.mass0) : std::fabs(m);
        const double dw = st.width0 > 0.0 ? std::fabs(wd - st.width0) / st.width0 : (wd == 0.0 ? 0.0 : INFINITY);
        if (rc == LBM_ACE_OK && dm <= mass_tol && dw <= width_tol) {
            std::swap(cur, cand);
            stale = true;
            st.surrogate_windows += 1;
            st.max_mass_drift = std::max(st.max_mass_drift, dm);
            st.max_width_dev = std::max(st.max_width_dev, dw);
        } else {
            if (stale) LAT(lbm_ace_reset_device(lat, cur, t));
            LAT(lbm_ace_step(lat, K));
            LAT(lbm_ace_get_phi_device(lat, cur));
            stale = false;
            st.fallback_windows += 1;
        }
        t += K;
        st.windows += 1;
    }
    if (stale) LAT(lbm_ace_reset_device(lat, cur, t));
    LAT(lbm_ace_synchronize(lat));
#undef LAT
    n->hyb[0] = cur;
    n->hyb[1] = cand;
    if (stats) *stats = st;
    return LBM_ACE_OK;
}

} // extern "C"
