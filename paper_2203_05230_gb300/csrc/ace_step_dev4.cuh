// ace_step_dev4.cuh -- the fused step on 16-bit deviation storage with four adjacent
// columns per thread and one independent 128-column strip per warp.
//
// Same storage and arithmetic as ace_step_dev (ace_step_dev.cuh): g_i = f*_i - s_i phi(t)
// in FP16 or BF16, FP32 phi planes ping-ponged, FP32 arithmetic through collide_core. Each
// node gets the same operations on the same values in the same order, so the two kernels
// write bit-identical states; only the FP64 mass partial of a step is summed differently.
//
// What changes is how the work maps onto the SM, for a kernel whose issue slots and
// latencies, not its DRAM bytes, bounded the column-pair form (measured on GB300):
//   * A thread owns the quad of columns xq .. xq + 3 and reads one 64-bit word
//     (4 x 16 bits) per plane and row, so every per-thread cost -- addresses, loop
//     control, the shuffles that complete the x-shifted planes, the lanes at warp edges --
//     is paid once per four nodes instead of once per two.
//   * Each warp marches its own 128-column strip with a private psi ring and its own two
//     halo columns, synchronised by __syncwarp alone: no CTA-wide barrier per row, so a
//     warp never waits for the slowest warp of its CTA.
//   * The pulled populations of the row that collides next are parked in shared memory
//     (9 x 16 bytes per thread, two row buffers) instead of registers.
//   * 3 or 4 CTAs of 128 threads per SM (the template parameter MINB, chosen by the host
//     from the lattice size): at 3, up to 168 registers and no spills; at 4, a
//     128-register cap (a 4-byte spill) and a third more warps to hide latency, which
//     pays on large lattices (4096^2: 105.6k against 101.5k MLUPS) and not on small ones,
//     where the shorter row bands of the one-wave launch cost more (2048^2: 92.1k against
//     95.1k). At 2 CTAs the SM lacks warps.
//   * The row loop is not unrolled: an unrolled body (to rotate the rolling window of
//     phi(t-1) rows without register moves) overflowed the instruction cache, which cost
//     far more than the moves.
//   * The mass partial of phi(t) is accumulated in FP32 parts whose rounded part is an
//     exact integer sum (split_add2i), keeping the FP64 pipe, 1/64 of the FP32 rate on
//     GB300, off the row loop. An FP64 flush every 64 rows under a counter test was
//     predicated into every row iteration by the compiler: 2 FP64-pipe instructions per
//     node, the FP64 pipe 36 % busy; without it, 4096^2 BF16 went from 105.5k to 110.5k
//     MLUPS and 2048^2 from 94.7k to 98.0k.
//
// Requirements (checked by the host): nx a multiple of 4; at most 4095 rows per CTA
// (the integer part of the mass partial is exact for up to 4 x 4095 values below 2).
#pragma once

#include "ace_step_dev.cuh"

namespace lbmace {

constexpr int QUAD_THREADS = 128;
constexpr int QUAD_COLS = 4 * QUAD_THREADS; // columns of a CTA
constexpr int QUAD_STRIP = 128;             // columns of one warp
constexpr int QUAD_WARPS = QUAD_THREADS / 32;
struct QuadSmem {
    float chi[QUAD_WARPS][4][QUAD_STRIP + 8]; // psi ring per warp: index j holds column x0 + j - 4
    float4 park[2][9][QUAD_THREADS];         // pulled f of one row: [buffer][plane][thread] (nodes 0..3)
    double red[QUAD_WARPS];
};

template <typename S, int MODEL, class Vel, bool UP>
__device__ __forceinline__ void dev4_tile(const DevArgs<S>& d, const StepArgs<float>& a, const Vel& vel, QuadSmem& sm)
{
    using C = Dev16<S>;
    const int tx = threadIdx.x;
    const int lane = tx & 31;
    const int wid = tx >> 5;
    const int x0 = (blockIdx.x * QUAD_WARPS + wid) * QUAD_STRIP; // this warp's strip
    const int w = min(QUAD_STRIP, a.nx - x0); // a multiple of 4; <= 0 for a strip past the lattice
    const bool live = w > 0;
    const bool act = 4 * lane < w;
    // threads past a ragged edge redo the last quad; a dead strip's threads point at column 0
    const int xq = live ? x0 + (act ? 4 * lane : w - 4) : 0;
    float (*ring)[QUAD_STRIP + 8] = sm.chi[wid];
    const int xl = xq == 0 ? a.nx - 1 : xq - 1;
    const int xr = xq + 4 == a.nx ? 0 : xq + 4;
    const bool own_left = lane == 0;
    const bool own_right = lane == 31 || 4 * (lane + 1) >= w;
    const int y0 = blockIdx.y * a.rows;
    const int y1 = min(y0 + a.rows, a.ny);
    const int nk = y1 - y0 + 2;
    const unsigned nxu = (unsigned)a.nx, plane = (unsigned)a.plane;
    const uint2* gq = reinterpret_cast<const uint2*>(d.gin); // 4 x 16-bit words (element offset / 4)

    // halo lanes of every warp: lanes 0..8 reconstruct population `hi` of the column left
    // of the strip, lanes 16..24 that of the column right of it
    const bool halo = (lane & 15) < 9;
    const int hi = lane & 15;
    int hcol = 0;
    if (halo && live) {
        const int c = lane < 16 ? (x0 == 0 ? a.nx - 1 : x0 - 1) : (x0 + w == a.nx ? 0 : x0 + w);
        hcol = wrap_idx(c - cx_of(hi), a.nx);
    }
    const int hcy = halo ? cy_of(hi) : 0;
    const float hs_w = halo ? split_of(hi) : 0.0f;

    typename Vel::Col cq[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) cq[j] = vel.col(xq + j);

    struct Raw {                               // one source-row set of the deviations
        uint2 v[9];                            // columns xq .. xq + 3
        unsigned short l1, l5, l8, r3, r6, r7; // xq - 1 (planes 1, 5, 8) and xq + 4 (3, 6, 7): edge lanes
    };
    struct PhiRaw { float4 v; float l, r; };   // phi(t-1) of one row: xq .. xq + 3, edge lanes xq - 1, xq + 4
    struct PhiRow { float c[6]; };             // phi(t-1) at columns xq - 1 .. xq + 4

    Raw nxt;
    PhiRaw pnx;
    float hg = 0.0f, hp = 0.0f;
    typename Vel::Row vr_next{};

    auto load_phi = [&](int row, PhiRaw& q) {
        const unsigned o = (unsigned)row * nxu;
        q.v = *reinterpret_cast<const float4*>(d.phin + (o + (unsigned)xq));
        if (own_left) q.l = d.phin[o + (unsigned)xl];
        if (own_right) q.r = d.phin[o + (unsigned)xr];
    };
    auto unpack_phi = [&](const PhiRaw& q, PhiRow& p) {
        float l = __shfl_up_sync(0xffffffffu, q.v.w, 1);
        float r = __shfl_down_sync(0xffffffffu, q.v.x, 1);
        if (own_left) l = q.l;
        if (own_right) r = q.r;
        p.c[0] = l; p.c[1] = q.v.x; p.c[2] = q.v.y; p.c[3] = q.v.z; p.c[4] = q.v.w; p.c[5] = r;
    };
    // iteration k pulls row r(k) = y0 - 1 + k (UP: y1 - k) and collides row r(k - 1)
    auto fetch = [&](int k) { // raw deviations of row r(k) and the phi(t-1) row r(k + 1)
        const int r = wrap_idx(UP ? y1 - k : y0 - 1 + k, a.ny);
        const int rm = r == 0 ? a.ny - 1 : r - 1, rp = r == a.ny - 1 ? 0 : r + 1;
        const unsigned o0 = (unsigned)r * nxu + (unsigned)xq, om = (unsigned)rm * nxu + (unsigned)xq,
                       op = (unsigned)rp * nxu + (unsigned)xq;
        nxt.v[0] = gq[o0 >> 2];
        nxt.v[1] = gq[(plane + o0) >> 2];
        nxt.v[2] = gq[(2u * plane + om) >> 2];
        nxt.v[3] = gq[(3u * plane + o0) >> 2];
        nxt.v[4] = gq[(4u * plane + op) >> 2];
        nxt.v[5] = gq[(5u * plane + om) >> 2];
        nxt.v[6] = gq[(6u * plane + om) >> 2];
        nxt.v[7] = gq[(7u * plane + op) >> 2];
        nxt.v[8] = gq[(8u * plane + op) >> 2];
        if (own_left) {
            const unsigned dl = (unsigned)xl - (unsigned)xq;
            nxt.l1 = d.gin[plane + o0 + dl];
            nxt.l5 = d.gin[5u * plane + om + dl];
            nxt.l8 = d.gin[8u * plane + op + dl];
        }
        if (own_right) {
            const unsigned dr = (unsigned)xr - (unsigned)xq;
            nxt.r3 = d.gin[3u * plane + o0 + dr];
            nxt.r6 = d.gin[6u * plane + om + dr];
            nxt.r7 = d.gin[7u * plane + op + dr];
        }
        load_phi(UP ? rm : rp, pnx);
        if (halo) {
            const unsigned hsrc = (unsigned)wrap_idx(r - hcy, a.ny) * nxu + (unsigned)hcol;
            hg = C::one(d.gin[(unsigned)hi * plane + hsrc]);
            hp = d.phin[hsrc];
        }
        const int yc = UP ? y1 - k + 1 : y0 + k - 2;
        if (yc >= y0 && yc < y1) vr_next = vel.rowv(cq[0], xq, yc);
    };

    // phi(t-1) window of iteration k: rows r(k - 1) (Wb), r(k) (Wc), r(k + 1) (Wa)
    PhiRow Wb, Wc, Wa;
    {
        PhiRaw q;
        load_phi(wrap_idx(UP ? y1 + 1 : y0 - 2, a.ny), q);
        unpack_phi(q, Wb);
        load_phi(wrap_idx(UP ? y1 : y0 - 1, a.ny), q);
        unpack_phi(q, Wc);
    }
    float4 php = make_float4(0.0f, 0.0f, 0.0f, 0.0f); // phi(t) of the row that collides next
    float2 mlo = make_float2(0.0f, 0.0f);
    unsigned mai = 0u;
    float mmax = 0.0f;

    auto body = [&](int k) {
        unpack_phi(pnx, Wa);
        const PhiRow& P0 = UP ? Wa : Wb; // lattice row r - 1
        const PhiRow& P1 = Wc;           // row r
        const PhiRow& P2 = UP ? Wb : Wa; // row r + 1
        // columns beside the quad of the x-shifted planes, from the neighbouring lanes
        unsigned l1 = __shfl_up_sync(0xffffffffu, nxt.v[1].y, 1) >> 16;
        unsigned l5 = __shfl_up_sync(0xffffffffu, nxt.v[5].y, 1) >> 16;
        unsigned l8 = __shfl_up_sync(0xffffffffu, nxt.v[8].y, 1) >> 16;
        unsigned r3 = __shfl_down_sync(0xffffffffu, nxt.v[3].x, 1) & 0xffffu;
        unsigned r6 = __shfl_down_sync(0xffffffffu, nxt.v[6].x, 1) & 0xffffu;
        unsigned r7 = __shfl_down_sync(0xffffffffu, nxt.v[7].x, 1) & 0xffffu;
        if (own_left) { l1 = nxt.l1; l5 = nxt.l5; l8 = nxt.l8; }
        if (own_right) { r3 = nxt.r3; r6 = nxt.r6; r7 = nxt.r7; }
        // f_i = g_i + s_i phi(t-1) at the source x - c_i of each node (scalar FMAs: the
        // sources of neighbouring nodes do not sit in aligned register pairs); pair 0 =
        // nodes xq, xq + 1, pair 1 = nodes xq + 2, xq + 3
        float2 f[2][9];
        auto rec = [&](int i, const PhiRow& P, int c0, float g0, float g1, float g2, float g3) {
            const float sw = split_of(i);
            f[0][i] = make_float2(__fmaf_rn(sw, P.c[c0], g0), __fmaf_rn(sw, P.c[c0 + 1], g1));
            f[1][i] = make_float2(__fmaf_rn(sw, P.c[c0 + 2], g2), __fmaf_rn(sw, P.c[c0 + 3], g3));
        };
        // column of node j in plane i: xq + j - c_x; its index in a PhiRow: j - c_x + 1
        const uint2* v = nxt.v;
        rec(0, P1, 1, C::lo(v[0].x), C::hi(v[0].x), C::lo(v[0].y), C::hi(v[0].y));
        rec(1, P1, 0, C::one((unsigned short)l1), C::lo(v[1].x), C::hi(v[1].x), C::lo(v[1].y));
        rec(2, P0, 1, C::lo(v[2].x), C::hi(v[2].x), C::lo(v[2].y), C::hi(v[2].y));
        rec(3, P1, 2, C::hi(v[3].x), C::lo(v[3].y), C::hi(v[3].y), C::one((unsigned short)r3));
        rec(4, P2, 1, C::lo(v[4].x), C::hi(v[4].x), C::lo(v[4].y), C::hi(v[4].y));
        rec(5, P0, 0, C::one((unsigned short)l5), C::lo(v[5].x), C::hi(v[5].x), C::lo(v[5].y));
        rec(6, P0, 2, C::hi(v[6].x), C::lo(v[6].y), C::hi(v[6].y), C::one((unsigned short)r6));
        rec(7, P2, 2, C::hi(v[7].x), C::lo(v[7].y), C::hi(v[7].y), C::one((unsigned short)r7));
        rec(8, P2, 0, C::one((unsigned short)l8), C::lo(v[8].x), C::hi(v[8].x), C::lo(v[8].y));
        const float hfk = __fmaf_rn(hs_w, hp, hg);
        // the raw sets are consumed: load the next row now, so it overlaps this whole iteration
        const typename Vel::Row vr = vr_next;
        if (k + 1 < nk) fetch(k + 1);
        float2 s0 = make_float2(0.0f, 0.0f), s1 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            s0 = __fadd2_rn(s0, f[0][i]);
            s1 = __fadd2_rn(s1, f[1][i]);
        }
        float4* park = sm.park[k & 1][0] + tx;
#pragma unroll
        for (int i = 0; i < 9; ++i) park[i * QUAD_THREADS] = make_float4(f[0][i].x, f[0][i].y, f[1][i].x, f[1][i].y);
        if (act) {
            const float4 c4 = make_float4(chi_of<float, MODEL>(s0.x, a), chi_of<float, MODEL>(s0.y, a),
                                          chi_of<float, MODEL>(s1.x, a), chi_of<float, MODEL>(s1.y, a));
            *reinterpret_cast<float4*>(&ring[k & 3][4 + 4 * lane]) = c4;
        }
        {
            const int base = lane & 16;
            float hs = 0.0f;
#pragma unroll
            for (int j = 0; j < 9; ++j) hs += __shfl_sync(0xffffffffu, hfk, base + j);
            if (lane == 0 || lane == 16) ring[k & 3][lane == 0 ? 3 : w + 4] = chi_of<float, MODEL>(hs, a);
        }
        __syncwarp();
        if (k >= 2) {
            const int yc = UP ? y1 - k + 1 : y0 + k - 2;
            const int j = act ? 4 * lane : w - 4; // ring index of column xq - 1 is j + 3
            // ring slots of rows yc - 1 (S) and yc + 1 (N): the rows pulled at k - 2 and k
            const int kS = (UP ? k : k - 2) & 3, kC = (k - 1) & 3, kN = (UP ? k - 2 : k) & 3;
            // chi pairs around the node pairs: [pair][left, centre, right]
            float2 pS[2][3], pC[2][3], pN[2][3];
            auto rd = [&](int slot, float2 (&pp)[2][3]) {
                const float* r = ring[slot] + 3 + j; // column xq - 1
                const float4 c4 = *reinterpret_cast<const float4*>(r + 1);
                const float c[6] = {r[0], c4.x, c4.y, c4.z, c4.w, r[5]};
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int e = 0; e < 3; ++e) pp[h][e] = make_float2(c[2 * h + e], c[2 * h + e + 1]);
            };
            rd(kS, pS);
            rd(kC, pC);
            rd(kN, pN);
            // u(t), u(t-1) of the 4 nodes
            float uu[4], vv[4], up[4], vp[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const typename Vel::Row vq = (Vel::row_uniform || q == 0) ? vr : vel.rowv(cq[q], xq + q, yc);
                vel.at(cq[q], vq, uu[q], vv[q], up[q], vp[q]);
            }
            const float4* pk = sm.park[(k - 1) & 1][0] + tx;
            const float ph[4] = {php.x, php.y, php.z, php.w};
            const float pp[4] = {Wb.c[1], Wb.c[2], Wb.c[3], Wb.c[4]}; // phi(t-1) of row r(k - 1)
            const unsigned o = (unsigned)yc * nxu + (unsigned)xq;
            uint2* gout = reinterpret_cast<uint2*>(d.gout);
            unsigned packed[2][9];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int n0 = 2 * h; // nodes n0, n0 + 1
                float2 fp[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const float4 q4 = pk[i * QUAD_THREADS];
                    fp[i] = h == 0 ? make_float2(q4.x, q4.y) : make_float2(q4.z, q4.w);
                }
                float2 o2[9];
                collide_core<float2, float, MODEL>(
                    a, fp, make_float2(ph[n0], ph[n0 + 1]), make_float2(pp[n0], pp[n0 + 1]),
                    pS[h][0], pS[h][1], pS[h][2], pC[h][0], pC[h][2], pN[h][0], pN[h][1], pN[h][2],
                    make_float2(uu[n0], uu[n0 + 1]), make_float2(vv[n0], vv[n0 + 1]),
                    make_float2(up[n0], up[n0 + 1]), make_float2(vp[n0], vp[n0 + 1]), o2);
                const float2 mph = make_float2(-ph[n0], -ph[n0 + 1]);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const float2 g2 = __ffma2_rn(make_float2(split_of(i), split_of(i)), mph, o2[i]);
                    packed[h][i] = C::pack(g2.x, g2.y);
                }
            }
            if (act) {
#pragma unroll
                for (int i = 0; i < 9; ++i) gout[(o + (unsigned)i * plane) >> 2] = make_uint2(packed[0][i], packed[1][i]);
                st_policy(d.phout + o, php, l2_store_policy_all((a.l2_keep & L2_KEEP_PHI) != 0));
                split_add2i(mai, mlo, make_float2(php.x, php.y));
                split_add2i(mai, mlo, make_float2(php.z, php.w));
                mmax = fmaxf(mmax, fmaxf(fmaxf(fabsf(php.x), fabsf(php.y)), fmaxf(fabsf(php.z), fabsf(php.w))));
            }
        }
        php = make_float4(s0.x, s0.y, s1.x, s1.y);
    };

    if (live) { // a warp strip past the lattice's right edge only joins the final sum
        fetch(0);
#pragma unroll 1
        for (int k = 0; k < nk; ++k) {
            body(k);
            Wb = Wc;
            Wc = Wa;
        }
    }

    double msum;
    if (mmax < 2.0f) {
        msum = split_total_i(mai, mlo, live && act ? 4u * (unsigned)(y1 - y0) : 0u);
    } else { // a value of 2 or more: the FP64 sum of the phi this thread wrote
        msum = 0.0;
        for (int yc = y0; yc < y1; ++yc) {
            const float4 q = *reinterpret_cast<const float4*>(d.phout + ((unsigned)yc * nxu + (unsigned)xq));
            msum += ((double)q.x + (double)q.y) + ((double)q.z + (double)q.w);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) msum += __shfl_down_sync(0xffffffffu, msum, off);
    if (lane == 0) sm.red[wid] = msum;
    __syncthreads();
    if (tx == 0) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < QUAD_WARPS; ++i) s += sm.red[i];
        a.mass_part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

template <typename S, int MODEL, class Vel, int MINB>
__global__ void __launch_bounds__(QUAD_THREADS, MINB)
ace_step_dev4(const DevArgs<S> d, const StepArgs<float> a, const Vel vel)
{
    extern __shared__ __align__(16) unsigned char dev4_smem[];
    QuadSmem& sm = *reinterpret_cast<QuadSmem*>(dev4_smem);
    // programmatic dependent launch (no-ops for an ordinary launch): see ace_step_pair
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    if (march_up(blockIdx.y, a.tdir))
        dev4_tile<S, MODEL, Vel, true>(d, a, vel, sm);
    else
        dev4_tile<S, MODEL, Vel, false>(d, a, vel, sm);
}

} // namespace lbmace
