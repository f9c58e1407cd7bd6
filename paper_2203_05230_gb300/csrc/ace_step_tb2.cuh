// ace_step_tb2.cuh -- two fused steps per launch (temporal blocking), FP32.
//
// The step of ace_step_pair (rows a1-a13 of ace_kernels.cuh) applied twice, n -> n+1 ->
// n+2, with the intermediate populations f*(n+1) kept in shared memory, so a pair of
// steps reads f*(n) and phi(n) from HBM once and writes f*(n+2) and phi(n+2) once: about
// 40 bytes of traffic per node update instead of 80.
//
// A CTA owns output columns [x0, x0 + 256) and rows [y0, y1) and has two warp groups:
//   stage A (warps 0-4): the first step on columns [x0 - 2, x0 + 258), i.e. the output
//     strip plus the two columns on each side that the second step reads, and on rows
//     [y0 - 2, y1 + 2); the code path of ace_step_pair (pair loads, shuffles, psi ring,
//     halo lanes of warp 0), except that the collided populations and phi go to a 4-row
//     ring in shared memory instead of HBM;
//   stage B (warps 5-8): the second step on the output strip; it pulls its populations
//     from the ring, TB_LAG row iterations behind stage A, computes phi and psi (the two
//     halo columns by two lanes of warp 5), collides and writes to HBM.
// Both groups march down the rows in lockstep, two named barriers per row. Every node
// value is computed with the same operations in the same order as by two launches of
// ace_step_pair (the halo columns of a strip are recomputed by the strips beside it), so
// the results are bit-identical (tested).
//
// Requirements (checked by the host): FP32, nx even. phi(n) is read from one plane and
// phi(n+2) written to another (stage A of a neighbouring CTA reads phi(n) around its
// strip), so the host keeps two phi planes and swaps them.
#pragma once

#include "ace_kernels.cuh"

namespace lbmace {

constexpr int TB_COLS = 256;                          // output columns per CTA
constexpr int TB_A_WARPS = 5, TB_B_WARPS = 4;
constexpr int TB_A_THREADS = TB_A_WARPS * 32;         // 130 of 160 pairs active for a full strip
constexpr int TB_THREADS = (TB_A_WARPS + TB_B_WARPS) * 32;
constexpr int TB_RC = TB_COLS + 4;                    // ring column j <-> x0 - 2 + j
constexpr int TB_LAG = 5;                             // stage B runs 5 row iterations behind A

struct TbSmem {
    float f[4][9][TB_RC];        // f*(n+1) of stage A's collided rows (ring by row index & 3)
    float ph[4][TB_RC];          // phi(n+1) of the same rows
    float psa[4][TB_RC + 4];     // stage A psi ring: index j <-> x0 - 4 + j
    float psb[4][TB_RC];         // stage B psi ring: index j <-> x0 - 2 + j
    double red[TB_B_WARPS];
};

// Named barrier 1 over the whole CTA (both warp groups reach it from their own loops).
__device__ __forceinline__ void tb_bar() { asm volatile("bar.sync 1, %0;\n" ::"n"(TB_THREADS) : "memory"); }

// Stage A: step n -> n+1 on columns [x0 - 2, x0 + wb + 2), collided rows y0 - 2 + c for
// c = k - 2 at iteration k (k < nA), into ring slot c & 3.
template <int MODEL, class Vel>
__device__ __forceinline__ void tb2_stage_a(const StepArgs<float>& a, const Vel& vel, TbSmem& S, int x0, int y0, int wb,
                                            int nA, int K)
{
    using V = float2;
    const int tx = threadIdx.x;
    const int lane = tx & 31;
    const int x0a = x0 - 2, w = wb + 4;                // stage A columns [x0a, x0a + w)
    const bool act = 2 * tx < w;
    const int xa = wrap_idx(x0a + (act ? 2 * tx : w - 2), a.nx);
    const int xb = xa + 1;
    const int xl = xa == 0 ? a.nx - 1 : xa - 1;
    const int xr = xb == a.nx - 1 ? 0 : xb + 1;
    const bool own_left = lane == 0;
    const bool own_right = lane == 31 || 2 * (tx + 1) >= w;
    const unsigned nxu = (unsigned)a.nx, plane = (unsigned)a.plane;

    const bool halo = tx < 32 && (lane & 15) < 9;
    const int hi = lane & 15;
    int hcol = 0;
    if (halo) {
        const int c = lane < 16 ? wrap_idx(x0a - 1, a.nx) : wrap_idx(x0a + w, a.nx);
        hcol = wrap_idx(c - cx_of(hi), a.nx);
    }
    const int hcy = halo ? cy_of(hi) : 0;
    const unsigned hbase = (unsigned)(halo ? hi : 0) * plane + (unsigned)hcol;
    const typename Vel::Col ca = vel.col(xa), cb = vel.col(xb);

    struct Raw {
        V v[9];
        float l1, l5, l8, r3, r6, r7;
    };
    Raw nxt;
    float hv = 0.0f;
    float pp_a = 0.0f, pp_b = 0.0f;
    typename Vel::Row vr_next{};

    auto fetch = [&](int k) { // pulled row y0 - 3 + k, and what the row collided at k needs
        const int r = wrap_idx(y0 - 3 + k, a.ny);
        const int rm = r == 0 ? a.ny - 1 : r - 1, rp = r == a.ny - 1 ? 0 : r + 1;
        const unsigned o0 = (unsigned)r * nxu, om = (unsigned)rm * nxu, op = (unsigned)rp * nxu;
        const unsigned ua = (unsigned)xa;
        nxt.v[0] = *reinterpret_cast<const V*>(a.fin + (o0 + ua));
        nxt.v[1] = *reinterpret_cast<const V*>(a.fin + (plane + o0 + ua));
        nxt.v[2] = *reinterpret_cast<const V*>(a.fin + (2u * plane + om + ua));
        nxt.v[3] = *reinterpret_cast<const V*>(a.fin + (3u * plane + o0 + ua));
        nxt.v[4] = *reinterpret_cast<const V*>(a.fin + (4u * plane + op + ua));
        nxt.v[5] = *reinterpret_cast<const V*>(a.fin + (5u * plane + om + ua));
        nxt.v[6] = *reinterpret_cast<const V*>(a.fin + (6u * plane + om + ua));
        nxt.v[7] = *reinterpret_cast<const V*>(a.fin + (7u * plane + op + ua));
        nxt.v[8] = *reinterpret_cast<const V*>(a.fin + (8u * plane + op + ua));
        if (own_left) {
            const unsigned ul = (unsigned)xl;
            nxt.l1 = a.fin[plane + o0 + ul];
            nxt.l5 = a.fin[5u * plane + om + ul];
            nxt.l8 = a.fin[8u * plane + op + ul];
        }
        if (own_right) {
            const unsigned ur = (unsigned)xr;
            nxt.r3 = a.fin[3u * plane + o0 + ur];
            nxt.r6 = a.fin[6u * plane + om + ur];
            nxt.r7 = a.fin[7u * plane + op + ur];
        }
        if (halo) hv = a.fin[hbase + (unsigned)wrap_idx(r - hcy, a.ny) * nxu];
        if (k >= 2) { // the row collided at iteration k: y0 - 2 + (k - 2)
            const int yc = wrap_idx(y0 + k - 4, a.ny);
            if (!a.first) {
                const V p2 = *reinterpret_cast<const V*>(a.phi + ((unsigned)yc * nxu + ua));
                pp_a = p2.x;
                pp_b = p2.y;
            }
            vr_next = vel.rowv(ca, xa, yc);
        }
    };

    float pa[9], pb[9]; // pulled populations of the previous row (collides this iteration)
#pragma unroll
    for (int i = 0; i < 9; ++i) pa[i] = pb[i] = 0.0f;
    float pha = 0.0f, phb = 0.0f;

    fetch(0);
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
        const bool run = k < nA;
        float fa[9], fb[9];
        float sa = 0.0f, sb = 0.0f;
        if (run) {
            float l1 = __shfl_up_sync(0xffffffffu, nxt.v[1].y, 1);
            float l5 = __shfl_up_sync(0xffffffffu, nxt.v[5].y, 1);
            float l8 = __shfl_up_sync(0xffffffffu, nxt.v[8].y, 1);
            float r3 = __shfl_down_sync(0xffffffffu, nxt.v[3].x, 1);
            float r6 = __shfl_down_sync(0xffffffffu, nxt.v[6].x, 1);
            float r7 = __shfl_down_sync(0xffffffffu, nxt.v[7].x, 1);
            if (own_left) { l1 = nxt.l1; l5 = nxt.l5; l8 = nxt.l8; }
            if (own_right) { r3 = nxt.r3; r6 = nxt.r6; r7 = nxt.r7; }
            fa[0] = nxt.v[0].x; fb[0] = nxt.v[0].y;
            fa[1] = l1;         fb[1] = nxt.v[1].x;
            fa[2] = nxt.v[2].x; fb[2] = nxt.v[2].y;
            fa[3] = nxt.v[3].y; fb[3] = r3;
            fa[4] = nxt.v[4].x; fb[4] = nxt.v[4].y;
            fa[5] = l5;         fb[5] = nxt.v[5].x;
            fa[6] = nxt.v[6].y; fb[6] = r6;
            fa[7] = nxt.v[7].y; fb[7] = r7;
            fa[8] = l8;         fb[8] = nxt.v[8].x;
            float2 s2 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int i = 0; i < 9; ++i) s2 = __fadd2_rn(s2, make_float2(fa[i], fb[i]));
            sa = s2.x;
            sb = s2.y;
            if (act) {
                V c2;
                c2.x = chi_of<float, MODEL>(sa, a);
                c2.y = chi_of<float, MODEL>(sb, a);
                *reinterpret_cast<V*>(&S.psa[k & 3][2 + 2 * tx]) = c2;
            }
            const float hvk = hv;
            if (tx < 32) {
                const int base = lane & 16;
                float hs = 0.0f;
#pragma unroll
                for (int j = 0; j < 9; ++j) hs += __shfl_sync(0xffffffffu, hvk, base + j);
                if (lane == 0) S.psa[k & 3][1] = chi_of<float, MODEL>(hs, a);
                if (lane == 16) S.psa[k & 3][w + 2] = chi_of<float, MODEL>(hs, a);
            }
        }
        tb_bar();
        if (run) {
            const float ppa = pp_a, ppb = pp_b;
            const typename Vel::Row vr = vr_next;
            if (k + 1 < nA) fetch(k + 1);
            if (k >= 2) {
                const int c = k - 2;                           // ring row of y0 - 2 + c
                const int yc = wrap_idx(y0 + k - 4, a.ny);
                const int j = act ? 2 * tx : w - 2;            // psa column of xa - 1 is j + 1
                V o2[9];
                collide_pair<float, MODEL>(a, vel, ca, cb, vr, vel.rowv(cb, xb, yc), pa, pb, pha, phb, ppa, ppb,
                                           S.psa[(k - 2) & 3] + 1 + j, S.psa[(k - 1) & 3] + 1 + j,
                                           S.psa[k & 3] + 1 + j, o2);
                if (act) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) *reinterpret_cast<V*>(&S.f[c & 3][i][2 * tx]) = o2[i];
                    *reinterpret_cast<V*>(&S.ph[c & 3][2 * tx]) = make_float2(pha, phb);
                }
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) { pa[i] = fa[i]; pb[i] = fb[i]; }
            pha = sa;
            phb = sb;
        }
        tb_bar();
    }
}

// Stage B: step n+1 -> n+2 on the output strip. Iteration kb (= k - TB_LAG) pulls row
// y0 - 1 + kb from the ring (stage A rows c = kb .. kb + 2) and collides row y0 + kb - 2.
template <int MODEL, class Vel>
__device__ __forceinline__ void tb2_stage_b(const StepArgs<float>& b, const Vel& vel, TbSmem& S, int x0, int y0, int wb,
                                            int nB, int K, double* mass_out)
{
    using V = float2;
    const int tb = threadIdx.x - TB_A_THREADS;
    const int lane = tb & 31;
    const bool act = 2 * tb < wb;
    const int xa = x0 + (act ? 2 * tb : wb - 2);
    const int xb = xa + 1;
    const int j = xa - x0 + 2;                          // ring column of xa
    const unsigned nxu = (unsigned)b.nx, plane = (unsigned)b.plane;
    const typename Vel::Col ca = vel.col(xa), cb = vel.col(xb);
    const bool halo = tb < 32 && (lane == 0 || lane == 16);
    const int jh = lane == 0 ? 1 : wb + 2;              // ring column of x0 - 1 or x0 + wb

    float pa[9], pb[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) pa[i] = pb[i] = 0.0f;
    float pha = 0.0f, phb = 0.0f;
    double msum = 0.0;

#pragma unroll 1
    for (int k = 0; k < K; ++k) {
        const int kb = k - TB_LAG;
        const bool run = kb >= 0 && kb < nB;
        float fa[9], fb[9];
        float sa = 0.0f, sb = 0.0f;
        if (run) {
            // f_i(x, y) = f*_i(x - c_i, y - c_iy): source ring row kb + 1 - c_iy
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float* row = S.f[(kb + 1 - cy_of(i)) & 3][i];
                fa[i] = row[j - cx_of(i)];
                fb[i] = row[j + 1 - cx_of(i)];
            }
            float2 s2 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int i = 0; i < 9; ++i) s2 = __fadd2_rn(s2, make_float2(fa[i], fb[i]));
            sa = s2.x;
            sb = s2.y;
            if (act) {
                V c2;
                c2.x = chi_of<float, MODEL>(sa, b);
                c2.y = chi_of<float, MODEL>(sb, b);
                *reinterpret_cast<V*>(&S.psb[kb & 3][j]) = c2;
            }
            if (halo) {
                float hs = 0.0f;
#pragma unroll
                for (int i = 0; i < 9; ++i) hs += S.f[(kb + 1 - cy_of(i)) & 3][i][jh - cx_of(i)];
                S.psb[kb & 3][jh] = chi_of<float, MODEL>(hs, b);
            }
        }
        tb_bar();
        if (run) {
            if (kb >= 2) {
                const int yc = y0 + kb - 2;
                const float ppa = S.ph[kb & 3][j], ppb = S.ph[kb & 3][j + 1]; // phi(n+1), stage A row kb
                V o2[9];
                collide_pair<float, MODEL>(b, vel, ca, cb, vel.rowv(ca, xa, yc), vel.rowv(cb, xb, yc), pa, pb, pha, phb,
                                           ppa, ppb, S.psb[(kb - 2) & 3] + j - 1, S.psb[(kb - 1) & 3] + j - 1,
                                           S.psb[kb & 3] + j - 1, o2);
                if (act) {
                    const unsigned o = (unsigned)yc * nxu + (unsigned)xa;
#pragma unroll
                    for (int i = 0; i < 9; ++i) *reinterpret_cast<V*>(b.fout + (o + (unsigned)i * plane)) = o2[i];
                    *reinterpret_cast<V*>(b.phi + o) = make_float2(pha, phb);
                    msum += (double)pha + (double)phb;
                }
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) { pa[i] = fa[i]; pb[i] = fb[i]; }
            pha = sa;
            phb = sb;
        }
        tb_bar();
    }

#pragma unroll
    for (int off = 16; off > 0; off >>= 1) msum += __shfl_down_sync(0xffffffffu, msum, off);
    if (lane == 0) S.red[tb >> 5] = msum;
    asm volatile("bar.sync 2, %0;\n" ::"n"(TB_B_WARPS * 32) : "memory");
    if (tb == 0) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < TB_B_WARPS; ++i) s += S.red[i];
        *mass_out = s;
    }
}

// a: step n (fin = f*(n-1) buffer... see host), b: step n+1 (fout, phi plane written,
// mass partials); va / vb: the velocity at the two steps.
template <int MODEL, class Vel>
__global__ void __launch_bounds__(TB_THREADS, 2) ace_step_tb2(const StepArgs<float> a, const StepArgs<float> b,
                                                              const Vel va, const Vel vb)
{
    extern __shared__ __align__(16) unsigned char tb_smem[];
    TbSmem& S = *reinterpret_cast<TbSmem*>(tb_smem);
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    const int x0 = blockIdx.x * TB_COLS, y0 = blockIdx.y * a.rows;
    const int wb = min(TB_COLS, a.nx - x0);               // even
    const int y1 = min(y0 + a.rows, a.ny);
    const int nB = y1 - y0 + 2;
    const int nA = nB + 4;
    const int K = nB + TB_LAG;
    if (threadIdx.x < TB_A_THREADS)
        tb2_stage_a<MODEL>(a, va, S, x0, y0, wb, nA, K);
    else
        tb2_stage_b<MODEL>(b, vb, S, x0, y0, wb, nB, K, &b.mass_part[(long long)blockIdx.y * gridDim.x + blockIdx.x]);
}

} // namespace lbmace
