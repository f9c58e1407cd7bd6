// ace_step_quad.cuh -- the fused FP32 step (rows a1-a13 of ace_kernels.cuh) with four
// adjacent columns per thread and one independent 128-column strip per warp.
//
// The FP32 counterpart of ace_step_dev4 (ace_step_dev4.cuh), same mapping onto the SM:
// a thread owns the quad of columns xq .. xq + 3 and reads one 16-byte word per plane
// and row (the x-shifted planes completed by warp shuffles, edge lanes loading the
// column beside the warp's strip); each warp marches its own strip with a private psi
// ring and two halo columns under __syncwarp; the pulled populations of the row that
// collides next are parked in shared memory; 3 CTAs of 128 threads per SM; the row loop
// is not unrolled; the FP64 mass partial of phi(t) is summed in FP32 parts whose
// rounded part is an exact integer sum (split_add2i, nothing to flush inside the row
// loop: a counter-tested FP64 flush there was predicated into every iteration).
// Every node gets the same arithmetic on the same values as in the other FP32 kernels
// (collide_core, phi summed over planes 0..8 in order), so the states are bit-identical.
//
// Against the column-pair kernel, a warp covers twice the columns, so one wave of
// resident CTAs gives each row band twice the rows: at 1024^2 the pair kernel's bands
// are 6 rows tall and spend a quarter of their work on the two psi rows recomputed at
// each band edge and on filling and draining the row pipeline.
//
// Requirements (checked by the host): nx a multiple of 4; at most 4095 rows per CTA
// (the integer part of the mass partial is exact for up to 4 x 4095 values below 2).
#pragma once

#include "ace_kernels.cuh"
#include "ace_step_pair.cuh"

namespace lbmace {

constexpr int Q32_THREADS = 128;
constexpr int Q32_COLS = 4 * Q32_THREADS; // columns of a CTA
constexpr int Q32_STRIP = 128;            // columns of one warp
constexpr int Q32_WARPS = Q32_THREADS / 32;
constexpr int Q32_MIN_CTAS = 3;

// The f* stores carry an L2 policy (ace_kernels.cuh): with L2_KEEP_F, evict_last on a
// quarter of the lines. Alone it made more of the next step's reads L2 hits from 1536^2
// to 2560^2 (2048^2: 52.1 -> 51.0 us per step), but keeping the phi plane (L2_KEEP_PHI)
// pays more and the two compete for the same lines (2048^2: 47.8 us with phi alone, 49.9
// with both), so the host leaves the bit unset and the f* stores get the normal priority.
struct Quad32Smem {
    float chi[Q32_WARPS][4][Q32_STRIP + 8]; // psi ring per warp: index j holds column x0 + j - 4
    float4 park[2][9][Q32_THREADS];        // pulled f of one row: [buffer][plane][thread] (nodes 0..3)
    double red[Q32_WARPS];
};

// One warp's work: the strip of columns [x0, x0 + 128) (clipped to nx; none when x0 >= nx)
// and rows [y0, y1) of the lattice described by `a`, marching up (UP) or down. ring is
// the warp's psi ring, park the CTA's row buffers (the warp uses the entries of its
// threads, tx = threadIdx.x). Synchronises the warp only. Returns the FP64 sum of the
// phi(t) it wrote (every lane holds it).
template <int MODEL, class Vel, bool UP>
__device__ __forceinline__ double quad32_strip(const StepArgs<float>& a, const Vel& vel, int x0, int y0, int y1,
                                               float (*ring)[Q32_STRIP + 8], float4 (*park_s)[9][Q32_THREADS],
                                               int tx)
{
    const int lane = tx & 31;
    const int w = min(Q32_STRIP, a.nx - x0); // a multiple of 4; <= 0 for a strip past the lattice
    const bool live = w > 0;
    const bool act = 4 * lane < w;
    // threads past a ragged edge redo the last quad; a dead strip's threads point at column 0
    const int xq = live ? x0 + (act ? 4 * lane : w - 4) : 0;
    const int xl = xq == 0 ? a.nx - 1 : xq - 1;
    const int xr = xq + 4 == a.nx ? 0 : xq + 4;
    const bool own_left = lane == 0;
    const bool own_right = lane == 31 || 4 * (lane + 1) >= w;
    const int nk = y1 - y0 + 2;
    const unsigned nxu = (unsigned)a.nx, plane = (unsigned)a.plane;

    // halo lanes of every warp: lanes 0..8 pull population `hi` of the column left of the
    // strip, lanes 16..24 that of the column right of it
    const bool halo = (lane & 15) < 9;
    const int hi = lane & 15;
    int hcol = 0;
    if (halo && live) {
        const int c = lane < 16 ? (x0 == 0 ? a.nx - 1 : x0 - 1) : (x0 + w == a.nx ? 0 : x0 + w);
        hcol = wrap_idx(c - cx_of(hi), a.nx);
    }
    const int hcy = halo ? cy_of(hi) : 0;
    const unsigned hbase = (unsigned)(halo ? hi : 0) * plane + (unsigned)hcol;

    typename Vel::Col cq[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) cq[j] = vel.col(xq + j);

    struct Raw {                 // one source-row set: columns xq .. xq + 3 of the 9 planes
        float4 v[9];
        float l1, l5, l8, r3, r6, r7; // xq - 1 (planes 1, 5, 8) and xq + 4 (3, 6, 7): edge lanes
    };
    Raw nxt;
    const unsigned long long store_policy = l2_store_policy_quarter((a.l2_keep & L2_KEEP_F) != 0);
    float hv = 0.0f;
    float4 pp_next = make_float4(0.0f, 0.0f, 0.0f, 0.0f); // phi(t-1) of the row that collides next
    typename Vel::Row vr_next{};

    // iteration k pulls row r(k) = y0 - 1 + k (UP: y1 - k) and collides row r(k - 1)
    auto fetch = [&](int k) {
        const int r = wrap_idx(UP ? y1 - k : y0 - 1 + k, a.ny);
        const int rm = r == 0 ? a.ny - 1 : r - 1, rp = r == a.ny - 1 ? 0 : r + 1;
        const unsigned o0 = (unsigned)r * nxu + (unsigned)xq, om = (unsigned)rm * nxu + (unsigned)xq,
                       op = (unsigned)rp * nxu + (unsigned)xq;
        const float* fin = a.fin;
        nxt.v[0] = *reinterpret_cast<const float4*>(fin + o0);
        nxt.v[1] = *reinterpret_cast<const float4*>(fin + (plane + o0));
        nxt.v[2] = *reinterpret_cast<const float4*>(fin + (2u * plane + om));
        nxt.v[3] = *reinterpret_cast<const float4*>(fin + (3u * plane + o0));
        nxt.v[4] = *reinterpret_cast<const float4*>(fin + (4u * plane + op));
        nxt.v[5] = *reinterpret_cast<const float4*>(fin + (5u * plane + om));
        nxt.v[6] = *reinterpret_cast<const float4*>(fin + (6u * plane + om));
        nxt.v[7] = *reinterpret_cast<const float4*>(fin + (7u * plane + op));
        nxt.v[8] = *reinterpret_cast<const float4*>(fin + (8u * plane + op));
        if (own_left) {
            const unsigned dl = (unsigned)xl - (unsigned)xq;
            nxt.l1 = fin[plane + o0 + dl];
            nxt.l5 = fin[5u * plane + om + dl];
            nxt.l8 = fin[8u * plane + op + dl];
        }
        if (own_right) {
            const unsigned dr = (unsigned)xr - (unsigned)xq;
            nxt.r3 = fin[3u * plane + o0 + dr];
            nxt.r6 = fin[6u * plane + om + dr];
            nxt.r7 = fin[7u * plane + op + dr];
        }
        if (halo) hv = fin[hbase + (unsigned)wrap_idx(r - hcy, a.ny) * nxu];
        const int yc = UP ? y1 - k + 1 : y0 + k - 2;
        if (yc >= y0 && yc < y1) {
            if (!a.first) pp_next = *reinterpret_cast<const float4*>(a.phi + ((unsigned)yc * nxu + (unsigned)xq));
            vr_next = vel.rowv(cq[0], xq, yc);
        }
    };

    float4 php = make_float4(0.0f, 0.0f, 0.0f, 0.0f); // phi(t) of the row that collides next
    float2 mlo = make_float2(0.0f, 0.0f);
    unsigned mai = 0u;
    float mmax = 0.0f;

    auto body = [&](int k) {
        // columns beside the quad of the x-shifted planes, from the neighbouring lanes
        float l1 = __shfl_up_sync(0xffffffffu, nxt.v[1].w, 1);
        float l5 = __shfl_up_sync(0xffffffffu, nxt.v[5].w, 1);
        float l8 = __shfl_up_sync(0xffffffffu, nxt.v[8].w, 1);
        float r3 = __shfl_down_sync(0xffffffffu, nxt.v[3].x, 1);
        float r6 = __shfl_down_sync(0xffffffffu, nxt.v[6].x, 1);
        float r7 = __shfl_down_sync(0xffffffffu, nxt.v[7].x, 1);
        if (own_left) { l1 = nxt.l1; l5 = nxt.l5; l8 = nxt.l8; }
        if (own_right) { r3 = nxt.r3; r6 = nxt.r6; r7 = nxt.r7; }
        // pulled f_i of the 4 nodes: planes with c_x = +1 read column x - 1, c_x = -1
        // column x + 1; pair 0 = nodes xq, xq + 1, pair 1 = nodes xq + 2, xq + 3
        const float4* v = nxt.v;
        float2 f[2][9];
        f[0][0] = make_float2(v[0].x, v[0].y); f[1][0] = make_float2(v[0].z, v[0].w);
        f[0][1] = make_float2(l1, v[1].x);     f[1][1] = make_float2(v[1].y, v[1].z);
        f[0][2] = make_float2(v[2].x, v[2].y); f[1][2] = make_float2(v[2].z, v[2].w);
        f[0][3] = make_float2(v[3].y, v[3].z); f[1][3] = make_float2(v[3].w, r3);
        f[0][4] = make_float2(v[4].x, v[4].y); f[1][4] = make_float2(v[4].z, v[4].w);
        f[0][5] = make_float2(l5, v[5].x);     f[1][5] = make_float2(v[5].y, v[5].z);
        f[0][6] = make_float2(v[6].y, v[6].z); f[1][6] = make_float2(v[6].w, r6);
        f[0][7] = make_float2(v[7].y, v[7].z); f[1][7] = make_float2(v[7].w, r7);
        f[0][8] = make_float2(l8, v[8].x);     f[1][8] = make_float2(v[8].y, v[8].z);
        const float hvk = hv;
        const float4 ppc = pp_next;
        // the raw sets are consumed: load the next row now, so it overlaps this whole iteration
        const typename Vel::Row vr = vr_next;
        if (k + 1 < nk) fetch(k + 1);
        float2 s0 = make_float2(0.0f, 0.0f), s1 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            s0 = __fadd2_rn(s0, f[0][i]);
            s1 = __fadd2_rn(s1, f[1][i]);
        }
        float4* park = park_s[k & 1][0] + tx;
#pragma unroll
        for (int i = 0; i < 9; ++i) park[i * Q32_THREADS] = make_float4(f[0][i].x, f[0][i].y, f[1][i].x, f[1][i].y);
        if (act) {
            const float4 c4 = make_float4(chi_of<float, MODEL>(s0.x, a), chi_of<float, MODEL>(s0.y, a),
                                          chi_of<float, MODEL>(s1.x, a), chi_of<float, MODEL>(s1.y, a));
            *reinterpret_cast<float4*>(&ring[k & 3][4 + 4 * lane]) = c4;
        }
        {
            const int base = lane & 16;
            float hs = 0.0f;
#pragma unroll
            for (int j = 0; j < 9; ++j) hs += __shfl_sync(0xffffffffu, hvk, base + j);
            if (lane == 0 || lane == 16) ring[k & 3][lane == 0 ? 3 : w + 4] = chi_of<float, MODEL>(hs, a);
        }
        __syncwarp();
        if (k >= 2) {
            const int yc = UP ? y1 - k + 1 : y0 + k - 2;
            const int j = act ? 4 * lane : w - 4; // ring index of column xq - 1 is j + 3
            // ring slots of rows yc - 1 (S) and yc + 1 (N): the rows pulled at k - 2 and k
            const int kS = (UP ? k : k - 2) & 3, kC = (k - 1) & 3, kN = (UP ? k - 2 : k) & 3;
            float2 pS[2][3], pC[2][3], pN[2][3]; // chi pairs around the node pairs: [pair][left, centre, right]
            auto rd = [&](int slot, float2 (&pq)[2][3]) {
                const float* r = ring[slot] + 3 + j; // column xq - 1
                const float4 c4 = *reinterpret_cast<const float4*>(r + 1);
                const float c[6] = {r[0], c4.x, c4.y, c4.z, c4.w, r[5]};
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int e = 0; e < 3; ++e) pq[h][e] = make_float2(c[2 * h + e], c[2 * h + e + 1]);
            };
            rd(kS, pS);
            rd(kC, pC);
            rd(kN, pN);
            float uu[4], vv[4], up[4], vp[4]; // u(t), u(t-1) of the 4 nodes
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const typename Vel::Row vq = (Vel::row_uniform || q == 0) ? vr : vel.rowv(cq[q], xq + q, yc);
                vel.at(cq[q], vq, uu[q], vv[q], up[q], vp[q]);
            }
            const float4* pk = park_s[(k - 1) & 1][0] + tx;
            const float ph[4] = {php.x, php.y, php.z, php.w};
            const float pp[4] = {ppc.x, ppc.y, ppc.z, ppc.w};
            const unsigned o = (unsigned)yc * nxu + (unsigned)xq;
            float2 o2[2][9];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int n0 = 2 * h; // nodes n0, n0 + 1
                float2 fp[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const float4 q4 = pk[i * Q32_THREADS];
                    fp[i] = h == 0 ? make_float2(q4.x, q4.y) : make_float2(q4.z, q4.w);
                }
                collide_core<float2, float, MODEL>(
                    a, fp, make_float2(ph[n0], ph[n0 + 1]), make_float2(pp[n0], pp[n0 + 1]),
                    pS[h][0], pS[h][1], pS[h][2], pC[h][0], pC[h][2], pN[h][0], pN[h][1], pN[h][2],
                    make_float2(uu[n0], uu[n0 + 1]), make_float2(vv[n0], vv[n0 + 1]),
                    make_float2(up[n0], up[n0 + 1]), make_float2(vp[n0], vp[n0 + 1]), o2[h]);
            }
            if (act) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    st_policy(a.fout + (o + (unsigned)i * plane), make_float4(o2[0][i].x, o2[0][i].y, o2[1][i].x, o2[1][i].y),
                              store_policy);
                st_policy(a.phi + o, php, l2_store_policy_all((a.l2_keep & L2_KEEP_PHI) != 0));
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
        for (int k = 0; k < nk; ++k) body(k);
    }

    double msum;
    if (mmax < 2.0f) {
        msum = split_total_i(mai, mlo, live && act ? 4u * (unsigned)(y1 - y0) : 0u);
    } else { // a value of 2 or more: the FP64 sum of the phi this thread wrote
        msum = 0.0;
        for (int yc = y0; yc < y1; ++yc) {
            const float4 q = *reinterpret_cast<const float4*>(a.phi + ((unsigned)yc * nxu + (unsigned)xq));
            msum += ((double)q.x + (double)q.y) + ((double)q.z + (double)q.w);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) msum += __shfl_xor_sync(0xffffffffu, msum, off);
    return msum;
}

// One CTA of the single-lattice kernel: warp wid takes strip blockIdx.x * 4 + wid of the
// row band blockIdx.y (a.rows tall); the warps' mass sums go, in warp order, to the CTA's
// partial.
template <int MODEL, class Vel, bool UP>
__device__ __forceinline__ void quad32_tile(const StepArgs<float>& a, const Vel& vel, Quad32Smem& sm)
{
    const int tx = threadIdx.x;
    const int wid = tx >> 5;
    const int x0 = (blockIdx.x * Q32_WARPS + wid) * Q32_STRIP; // this warp's strip
    const int y0 = blockIdx.y * a.rows;
    const int y1 = min(y0 + a.rows, a.ny);
    const double msum = quad32_strip<MODEL, Vel, UP>(a, vel, x0, y0, y1, sm.chi[wid], sm.park, tx);
    if ((tx & 31) == 0) sm.red[wid] = msum;
    __syncthreads();
    if (tx == 0) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < Q32_WARPS; ++i) s += sm.red[i];
        a.mass_part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

template <int MODEL, class Vel>
__global__ void __launch_bounds__(Q32_THREADS, Q32_MIN_CTAS) ace_step_quad(const StepArgs<float> a, const Vel vel)
{
    extern __shared__ __align__(16) unsigned char quad32_smem[];
    Quad32Smem& sm = *reinterpret_cast<Quad32Smem*>(quad32_smem);
    // programmatic dependent launch (no-ops for an ordinary launch): see ace_step_pair
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    if (march_up(blockIdx.y, a.tdir))
        quad32_tile<MODEL, Vel, true>(a, vel, sm);
    else
        quad32_tile<MODEL, Vel, false>(a, vel, sm);
}

} // namespace lbmace
