// ace_step_dev.cuh -- the fused step with populations stored as 16-bit deviations.
//
// Storage: g_i(x) = f*_i(x) - s_i phi(t)(x) in FP16 or BF16 (S), where f*_i is the
// post-collision population of node x and phi(t)(x) its moment in this step; the
// phi plane (FP32) is double-buffered because the next step reads it around each
// node. The split weights s_i (split_of) are dyadic, close to the D2Q9 weights, and
// sum to exactly 1, so f_i = g_i + s_i phi reconstructs the populations without
// adding mass (the nearest FP32 values of 4/9, 1/9, 1/36 sum to 1 + 7.5e-9).
// All arithmetic is FP32; the collision is collide_core, shared with the other kernels.
//
// Pull: f_i(x, t) = g_i(x - c_i) + s_i phi(t - 1)(x - c_i). The kernel is the
// column-pair kernel (ace_step_pair.cuh): two adjacent columns per thread, packed
// 2 x 16-bit loads and stores per plane, x-shifted planes and the phi neighbours
// completed by warp shuffles, loads one row ahead. Traffic per node: 9 x 2 bytes
// read and written plus the phi plane read and written (4 + 4 bytes) = 44 bytes.
//
// Requirement (checked by the host): nx even.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ace_kernels.cuh"
#include "ace_step_pair.cuh"

namespace lbmace {

template <typename S> struct Dev16;
template <>
struct Dev16<__half> {
    __device__ __forceinline__ static float lo(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
    __device__ __forceinline__ static float hi(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
    __device__ __forceinline__ static float one(unsigned short b) { return __half2float(__ushort_as_half(b)); }
    __device__ __forceinline__ static unsigned pack(float a, float b)
    {
        const __half2 h = __floats2half2_rn(a, b); // a in the low half
        return *reinterpret_cast<const unsigned*>(&h);
    }
    __device__ __forceinline__ static unsigned short bits(float a) { return __half_as_ushort(__float2half_rn(a)); }
};
template <>
struct Dev16<__nv_bfloat16> {
    __device__ __forceinline__ static float lo(unsigned w) { return __uint_as_float(w << 16); }
    __device__ __forceinline__ static float hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }
    __device__ __forceinline__ static float one(unsigned short b) { return __uint_as_float((unsigned)b << 16); }
    __device__ __forceinline__ static unsigned pack(float a, float b)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b); // a in the low half
        return *reinterpret_cast<const unsigned*>(&h);
    }
    __device__ __forceinline__ static unsigned short bits(float a) { return __bfloat16_as_ushort(__float2bfloat16_rn(a)); }
};

// Split weights: exact dyadic fractions (1820, 455, 114) / 4096 that sum to 1, within
// 1.1e-4 of the D2Q9 weights. (FP32 weights within 3.4e-9 of w_i that also sum to 1
// were measured worse at 4096^2 over 16384 steps: BF16 phi-L2 1.5e-2 against 6.4e-3.)
__host__ __device__ constexpr float split_of(int i)
{
    return i == 0 ? 1820.0f / 4096.0f : (i < 5 ? 455.0f / 4096.0f : 114.0f / 4096.0f);
}

template <typename S>
struct DevArgs {
    const unsigned short* __restrict__ gin; // g(t-1), 9 planes of 16-bit words
    unsigned short* __restrict__ gout;      // g(t)
    const float* __restrict__ phin;         // phi(t-1)
    float* __restrict__ phout;              // phi(t)
};

// The tile (blockIdx.x, blockIdx.y) of one step. UP: march the rows upwards (march_up).
template <typename S, int MODEL, class Vel, bool UP>
__device__ __forceinline__ void dev_tile(const DevArgs<S>& d, const StepArgs<float>& a, const Vel& vel,
                                         float (*chi_s)[PAIR_COLS + 4], double* red_s)
{
    using C = Dev16<S>;
    const int tx = threadIdx.x;
    const int lane = tx & 31;
    const int x0 = blockIdx.x * PAIR_COLS;
    const int w = min(PAIR_COLS, a.nx - x0); // even
    const bool act = 2 * tx < w;
    const int xa = x0 + (act ? 2 * tx : w - 2);
    const int xb = xa + 1;
    const int xl = xa == 0 ? a.nx - 1 : xa - 1;
    const int xr = xb == a.nx - 1 ? 0 : xb + 1;
    const bool own_left = lane == 0;
    const bool own_right = lane == 31 || 2 * (tx + 1) >= w;
    const int y0 = blockIdx.y * a.rows;
    const int y1 = min(y0 + a.rows, a.ny);
    const int nk = y1 - y0 + 2;
    const unsigned nxu = (unsigned)a.nx, plane = (unsigned)a.plane;
    const unsigned* gw = reinterpret_cast<const unsigned*>(d.gin); // packed pairs (even offsets)

    // halo lanes of warp 0: lanes 0..8 reconstruct population `hi` of the column left
    // of the strip, lanes 16..24 that of the column right of it
    const bool halo = tx < 32 && (lane & 15) < 9;
    const int hi = lane & 15;
    int hcol = 0;
    if (halo) {
        const int c = lane < 16 ? (x0 == 0 ? a.nx - 1 : x0 - 1) : (x0 + w == a.nx ? 0 : x0 + w);
        hcol = wrap_idx(c - cx_of(hi), a.nx);
    }
    const int hcy = halo ? cy_of(hi) : 0;
    const float hs_w = halo ? split_of(hi) : 0.0f;

    const typename Vel::Col ca = vel.col(xa), cb = vel.col(xb);

    struct Raw {            // one source-row set of the deviations
        unsigned v[9];      // packed (xa, xb) pairs
        unsigned short l1, l5, l8, r3, r6, r7; // columns beside the pair, edge lanes only
    };
    struct PhiRaw {         // one row of phi(t-1) around the pair
        float2 v;
        float l, r;
    };
    struct PhiRow { float c[4]; }; // phi(t-1) at columns xl, xa, xb, xr

    Raw nxt;
    PhiRaw pnx;
    float hg = 0.0f, hp = 0.0f; // halo lane: deviation and phi(t-1) at its source node
    typename Vel::Row vr_next{};

    auto load_phi = [&](int row, PhiRaw& q) {
        const unsigned o = (unsigned)row * nxu;
        q.v = *reinterpret_cast<const float2*>(d.phin + (o + (unsigned)xa));
        if (own_left) q.l = d.phin[o + (unsigned)xl];
        if (own_right) q.r = d.phin[o + (unsigned)xr];
    };
    auto unpack_phi = [&](const PhiRaw& q, PhiRow& p) {
        float l = __shfl_up_sync(0xffffffffu, q.v.y, 1);
        float r = __shfl_down_sync(0xffffffffu, q.v.x, 1);
        if (own_left) l = q.l;
        if (own_right) r = q.r;
        p.c[0] = l; p.c[1] = q.v.x; p.c[2] = q.v.y; p.c[3] = r;
    };
    // iteration k pulls row r(k) = y0 - 1 + k (UP: y1 - k) and collides row r(k - 1)
    auto fetch = [&](int k) { // pulled row r(k): deviations, and phi row r(k + 1)
        const int r = wrap_idx(UP ? y1 - k : y0 - 1 + k, a.ny);
        const int rm = r == 0 ? a.ny - 1 : r - 1, rp = r == a.ny - 1 ? 0 : r + 1;
        const unsigned o0 = (unsigned)r * nxu, om = (unsigned)rm * nxu, op = (unsigned)rp * nxu;
        const unsigned ua = (unsigned)xa;
        nxt.v[0] = gw[(o0 + ua) >> 1];
        nxt.v[1] = gw[(plane + o0 + ua) >> 1];
        nxt.v[2] = gw[(2u * plane + om + ua) >> 1];
        nxt.v[3] = gw[(3u * plane + o0 + ua) >> 1];
        nxt.v[4] = gw[(4u * plane + op + ua) >> 1];
        nxt.v[5] = gw[(5u * plane + om + ua) >> 1];
        nxt.v[6] = gw[(6u * plane + om + ua) >> 1];
        nxt.v[7] = gw[(7u * plane + op + ua) >> 1];
        nxt.v[8] = gw[(8u * plane + op + ua) >> 1];
        if (own_left) {
            const unsigned ul = (unsigned)xl;
            nxt.l1 = d.gin[plane + o0 + ul];
            nxt.l5 = d.gin[5u * plane + om + ul];
            nxt.l8 = d.gin[8u * plane + op + ul];
        }
        if (own_right) {
            const unsigned ur = (unsigned)xr;
            nxt.r3 = d.gin[3u * plane + o0 + ur];
            nxt.r6 = d.gin[6u * plane + om + ur];
            nxt.r7 = d.gin[7u * plane + op + ur];
        }
        load_phi(UP ? rm : rp, pnx);
        if (halo) {
            const unsigned hsrc = (unsigned)wrap_idx(r - hcy, a.ny) * nxu + (unsigned)hcol;
            hg = C::one(d.gin[(unsigned)hi * plane + hsrc]);
            hp = d.phin[hsrc];
        }
        const int yc = UP ? y1 - k + 1 : y0 + k - 2;
        if (yc >= y0 && yc < y1) vr_next = vel.rowv(ca, xa, yc);
    };

    // phi(t-1) rows r(k - 1), r(k), r(k + 1) around the pair of the pulled row r(k), in
    // march order: Qb behind, Qc at, Qa ahead (rows r - 1, r, r + 1 when marching down)
    PhiRow Qb, Qc, Qa;
    {
        PhiRaw q;
        load_phi(wrap_idx(UP ? y1 + 1 : y0 - 2, a.ny), q);
        unpack_phi(q, Qc);
        load_phi(wrap_idx(UP ? y1 : y0 - 1, a.ny), q);
        unpack_phi(q, Qa);
    }

    float pa[9], pb[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) pa[i] = pb[i] = 0.0f;
    float pha = 0.0f, phb = 0.0f;
    double msum = 0.0;

    fetch(0);
#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
        Qb = Qc;
        Qc = Qa;
        unpack_phi(pnx, Qa);
        const PhiRow& P0 = UP ? Qa : Qb; // row r - 1
        const PhiRow& P1 = Qc;           // row r
        const PhiRow& P2 = UP ? Qb : Qa; // row r + 1
        // deviations of the pair, shifted planes completed from the neighbour lanes
        unsigned l1 = __shfl_up_sync(0xffffffffu, nxt.v[1], 1) >> 16;
        unsigned l5 = __shfl_up_sync(0xffffffffu, nxt.v[5], 1) >> 16;
        unsigned l8 = __shfl_up_sync(0xffffffffu, nxt.v[8], 1) >> 16;
        unsigned r3 = __shfl_down_sync(0xffffffffu, nxt.v[3], 1) & 0xffffu;
        unsigned r6 = __shfl_down_sync(0xffffffffu, nxt.v[6], 1) & 0xffffu;
        unsigned r7 = __shfl_down_sync(0xffffffffu, nxt.v[7], 1) & 0xffffu;
        if (own_left) { l1 = nxt.l1; l5 = nxt.l5; l8 = nxt.l8; }
        if (own_right) { r3 = nxt.r3; r6 = nxt.r6; r7 = nxt.r7; }
        float fa[9], fb[9];
        // node a reads column xa - c_x, node b column xb - c_x (window columns 1 - c_x,
        // 2 - c_x), row r - c_y (P0, P1, P2 hold rows r - 1, r, r + 1); both nodes at
        // once: f = g + s phi (packed FP32x2)
        auto rec = [&](int i, float ga, float gb, float pa_, float pb_) {
            const float2 r2 = __ffma2_rn(make_float2(split_of(i), split_of(i)), make_float2(pa_, pb_), make_float2(ga, gb));
            fa[i] = r2.x;
            fb[i] = r2.y;
        };
        rec(0, C::lo(nxt.v[0]), C::hi(nxt.v[0]), P1.c[1], P1.c[2]);
        rec(1, C::one((unsigned short)l1), C::lo(nxt.v[1]), P1.c[0], P1.c[1]);
        rec(2, C::lo(nxt.v[2]), C::hi(nxt.v[2]), P0.c[1], P0.c[2]);
        rec(3, C::hi(nxt.v[3]), C::one((unsigned short)r3), P1.c[2], P1.c[3]);
        rec(4, C::lo(nxt.v[4]), C::hi(nxt.v[4]), P2.c[1], P2.c[2]);
        rec(5, C::one((unsigned short)l5), C::lo(nxt.v[5]), P0.c[0], P0.c[1]);
        rec(6, C::hi(nxt.v[6]), C::one((unsigned short)r6), P0.c[2], P0.c[3]);
        rec(7, C::hi(nxt.v[7]), C::one((unsigned short)r7), P2.c[2], P2.c[3]);
        rec(8, C::one((unsigned short)l8), C::lo(nxt.v[8]), P2.c[0], P2.c[1]);
        const float hfk = hg + hs_w * hp;
        // the raw sets are consumed: load the next row now, so it overlaps this whole iteration
        const typename Vel::Row vr = vr_next;
        if (k + 1 < nk) fetch(k + 1);
        float2 s2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < 9; ++i) s2 = __fadd2_rn(s2, make_float2(fa[i], fb[i]));
        const float sa = s2.x, sb = s2.y;
        if (act) {
            float2 c2;
            c2.x = chi_of<float, MODEL>(sa, a);
            c2.y = chi_of<float, MODEL>(sb, a);
            *reinterpret_cast<float2*>(&chi_s[k & 3][2 + 2 * tx]) = c2;
        }
        if (tx < 32) {
            const int base = lane & 16;
            float hs = 0.0f;
#pragma unroll
            for (int j = 0; j < 9; ++j) hs += __shfl_sync(0xffffffffu, hfk, base + j);
            if (lane == 0) chi_s[k & 3][1] = chi_of<float, MODEL>(hs, a);
            if (lane == 16) chi_s[k & 3][w + 2] = chi_of<float, MODEL>(hs, a);
        }
        __syncthreads();
        const float ppa = Qb.c[1], ppb = Qb.c[2]; // phi(t-1) of the colliding row r(k - 1)
        if (k >= 2) {
            const int yc = UP ? y1 - k + 1 : y0 + k - 2;
            const int j = act ? 2 * tx : w - 2;
            // ring slots of rows yc - 1 (S) and yc + 1 (N): the rows pulled at k - 2 and k
            const float* cS = chi_s[(UP ? k : k - 2) & 3] + 1 + j;
            const float* cC = chi_s[(k - 1) & 3] + 1 + j;
            const float* cN = chi_s[(UP ? k - 2 : k) & 3] + 1 + j;
            float2 o2[9];
            collide_pair<float, MODEL>(a, vel, ca, cb, vr, vel.rowv(cb, xb, yc), pa, pb, pha, phb, ppa, ppb, cS, cC, cN,
                                       o2);
            if (act) {
                const unsigned o = (unsigned)yc * nxu + (unsigned)xa;
                unsigned* gout = reinterpret_cast<unsigned*>(d.gout);
                const float2 ph2 = make_float2(-pha, -phb);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const float2 g2 = __ffma2_rn(make_float2(split_of(i), split_of(i)), ph2, o2[i]);
                    gout[(o + (unsigned)i * plane) >> 1] = C::pack(g2.x, g2.y);
                }
                *reinterpret_cast<float2*>(d.phout + o) = make_float2(pha, phb);
                msum += (double)pha + (double)phb;
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) { pa[i] = fa[i]; pb[i] = fb[i]; }
        pha = sa;
        phb = sb;
    }

#pragma unroll
    for (int off = 16; off > 0; off >>= 1) msum += __shfl_down_sync(0xffffffffu, msum, off);
    if (lane == 0) red_s[tx >> 5] = msum;
    __syncthreads();
    if (tx == 0) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < PAIR_THREADS / 32; ++i) s += red_s[i];
        a.mass_part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

template <typename S, int MODEL, class Vel>
__global__ void __launch_bounds__(PAIR_THREADS, 5) ace_step_dev(const DevArgs<S> d, const StepArgs<float> a, const Vel vel)
{
    __shared__ __align__(16) float chi_s[4][PAIR_COLS + 4]; // index j holds column x0 + j - 2
    __shared__ double red_s[PAIR_THREADS / 32];
    // programmatic dependent launch (no-ops for an ordinary launch): see ace_step_pair
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    if (march_up(blockIdx.y, a.tdir))
        dev_tile<S, MODEL, Vel, true>(d, a, vel, chi_s, red_s);
    else
        dev_tile<S, MODEL, Vel, false>(d, a, vel, chi_s, red_s);
}

// ---- state conversions for the deviation storage (init, read-out, checkpoints) ----

// Initial state: g_i(x') = f_i^eq(x' + c_i, 0) - s_i phi0(x') at the source x' = x - c_i
// of each population, phi plane = phi0 (= phi(-1)).
template <typename S, class Vel>
__global__ void ace_init_dev(const double* __restrict__ phi0, unsigned short* __restrict__ g, float* __restrict__ phi,
                             int nx, int ny, Vel vel)
{
    const long long plane = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < plane;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        const float ph = (float)phi0[k];
        float u, v, up, vp, feq[9];
        const typename Vel::Col c = vel.col(x);
        vel.at(c, vel.rowv(c, x, y), u, v, up, vp);
        equilibrium(ph, u, v, feq);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const long long src = (long long)wrap_idx(y - cy_of(i), ny) * nx + wrap_idx(x - cx_of(i), nx);
            g[i * plane + src] = Dev16<S>::bits(feq[i] - split_of(i) * (float)phi0[src]);
        }
        phi[k] = ph;
    }
}

// f_i(x, t) = g_i(x - c_i) + s_i phi(t-1)(x - c_i), as FP64 (f may be null), and
// phi(x, t) = sum_i f_i (FP32 sum in the kernel's order, as FP64; may be null).
template <typename S>
__global__ void ace_pull_state_dev(const unsigned short* __restrict__ g, const float* __restrict__ phi, double* f,
                                   double* phi_t, double* php, int nx, int ny)
{
    const long long plane = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < plane;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const long long src = (long long)wrap_idx(y - cy_of(i), ny) * nx + wrap_idx(x - cx_of(i), nx);
            const float fi = Dev16<S>::one(g[i * plane + src]) + split_of(i) * phi[src];
            s += fi;
            if (f) f[i * plane + k] = (double)fi;
        }
        if (phi_t) phi_t[k] = (double)s;
        if (php) php[k] = (double)phi[k];
    }
}

// Checkpoint write: g_i(x') = f_i(x' + c_i) - s_i phi_prev(x'), phi plane = phi_prev.
template <typename S>
__global__ void ace_push_state_dev(const double* __restrict__ f, const double* __restrict__ php,
                                   unsigned short* __restrict__ g, float* __restrict__ phi, int nx, int ny)
{
    const long long plane = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < plane;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        const float pk = (float)php[k];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const long long dst = (long long)wrap_idx(y + cy_of(i), ny) * nx + wrap_idx(x + cx_of(i), nx);
            g[i * plane + k] = Dev16<S>::bits((float)f[i * plane + dst] - split_of(i) * pk);
        }
        phi[k] = pk;
    }
}

} // namespace lbmace
