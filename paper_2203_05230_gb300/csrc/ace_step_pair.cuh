// ace_step_pair.cuh -- the fused step (rows a1-a13 of ace_kernels.cuh) with two
// adjacent columns per thread, to cut the instructions spent per node.
//
// A CTA of 128 threads owns 256 consecutive columns; thread t owns the pair
// (xa, xa + 1) = (x0 + 2t, x0 + 2t + 1) and marches down `rows` rows. Each of the 9
// population planes of a source row is read with one 8- (FP32) or 16-byte (FP64)
// load per pair. For the planes shifted in x the column beside the pair comes from
// the neighbouring lane's load by a warp shuffle; only the lanes at a warp or strip
// edge load it themselves. The loads of row r + 1 are issued while row r - 1
// collides and are unpacked (shuffles) only when row r + 1 is processed, so no
// shuffle waits on memory. psi goes into a 4-slot shared-memory ring as pairs; the
// two halo columns of the strip are recomputed by lanes of warp 0 as in ace_step.
// The per-node arithmetic is collide_node_row, shared with the other variants, and
// phi is summed in the same order, so all variants agree bit for bit. Stores are
// pairs too. Row bands alternate their march direction from band to band and from step
// to step (march_up), so a band's halo rows and the previous step's last rows are read
// from L2 rather than DRAM.
//
// Requirement (checked by the host): nx even, so every pair is aligned.
#pragma once

#include "ace_kernels.cuh"

namespace lbmace {

constexpr int PAIR_THREADS = 128;
constexpr int PAIR_COLS = 2 * PAIR_THREADS;

// March direction of row band `by` in a step with parity tdir (t & 1): alternate bands
// march in opposite directions and every band turns round at the next step. Two
// neighbouring bands then reach their common edge together, so the rows both of them
// read there (each band's halo) come from DRAM once and are found in L2 by the other;
// and each step starts on the rows the previous step wrote last, still in L2.
__device__ __forceinline__ bool march_up(unsigned by, int tdir) { return ((by + (unsigned)tdir) & 1u) != 0; }

// One tile: columns [x0, x0 + 256) (clipped to nx) and rows [y0, y0 + a.rows) of the
// lattice described by `a`. chi_s (4 x (PAIR_COLS + 4), 16-byte aligned: ring index j
// holds column x0 + j - 2) and red_s (PAIR_THREADS / 32 doubles) are the CTA's shared
// memory; thread 0 writes the tile's FP64 mass of phi(t) to *mass_out. Ends with a
// barrier, so the CTA can take another tile right after.
// UP: march the rows from y1 - 1 up to y0 instead of down from y0; every node gets the
// same arithmetic on the same values, only the order of the FP64 mass partial changes.
template <typename T, int MODEL, class Vel, bool UP = false>
__device__ __forceinline__ void pair_tile(const StepArgs<T>& a, const Vel& vel, int x0, int y0,
                                          T (*chi_s)[PAIR_COLS + 4], double* red_s, double* mass_out)
{
    using V = typename Pair2<T>::type;
    const int tx = threadIdx.x;
    const int lane = tx & 31;
    const int w = min(PAIR_COLS, a.nx - x0); // even
    const bool act = 2 * tx < w;
    const int xa = x0 + (act ? 2 * tx : w - 2); // threads past a ragged edge redo the last pair
    const int xb = xa + 1;
    const int xl = xa == 0 ? a.nx - 1 : xa - 1;     // column left of the pair
    const int xr = xb == a.nx - 1 ? 0 : xb + 1;     // column right of the pair
    const bool own_left = lane == 0;                // no lane to the left in this warp
    const bool own_right = lane == 31 || 2 * (tx + 1) >= w; // no active lane to the right
    const int y1 = min(y0 + a.rows, a.ny);
    const int nk = y1 - y0 + 2;
    const unsigned nxu = (unsigned)a.nx, plane = (unsigned)a.plane;

    // halo lanes of warp 0 (as in ace_step)
    const bool halo = tx < 32 && (lane & 15) < 9;
    const int hi = lane & 15;
    int hcol = 0;
    if (halo) {
        const int c = lane < 16 ? (x0 == 0 ? a.nx - 1 : x0 - 1) : (x0 + w == a.nx ? 0 : x0 + w);
        hcol = wrap_idx(c - cx_of(hi), a.nx);
    }
    const int hcy = halo ? cy_of(hi) : 0;
    const unsigned hbase = (unsigned)(halo ? hi : 0) * plane + (unsigned)hcol;

    const typename Vel::Col ca = vel.col(xa), cb = vel.col(xb);

    // raw loads of one source row set: the 9 pairs and, for edge lanes, the 6 columns
    // beside the pair of the shifted planes (1, 5, 8 on the left; 3, 6, 7 on the right)
    struct Raw {
        V v[9];
        T l1, l5, l8, r3, r6, r7;
    };
    Raw nxt;
    T hv = T(0);
    T pp_a = T(0), pp_b = T(0); // phi(t-1) of the row that collides next
    typename Vel::Row vr_next{};

    // iteration k pulls row r(k) = y0 - 1 + k (UP: y1 - k) and collides row r(k - 1)
    auto fetch = [&](int k) { // pulled row r(k), plus what row r(k - 1) needs to collide
        const int r = wrap_idx(UP ? y1 - k : y0 - 1 + k, a.ny);
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
        const int yc = UP ? y1 - k + 1 : y0 + k - 2;
        if (yc >= y0 && yc < y1) {
            if (!a.first) {
                const V p2 = *reinterpret_cast<const V*>(a.phi + ((unsigned)yc * nxu + ua));
                pp_a = p2.x;
                pp_b = p2.y;
            }
            vr_next = vel.rowv(ca, xa, yc);
        }
    };

    // pulled populations f_i of the pair from a raw row set (shuffles for the shifted planes)
    auto unpack = [&](const Raw& q, T (&fa)[9], T (&fb)[9]) {
        T l1 = __shfl_up_sync(0xffffffffu, q.v[1].y, 1);
        T l5 = __shfl_up_sync(0xffffffffu, q.v[5].y, 1);
        T l8 = __shfl_up_sync(0xffffffffu, q.v[8].y, 1);
        T r3 = __shfl_down_sync(0xffffffffu, q.v[3].x, 1);
        T r6 = __shfl_down_sync(0xffffffffu, q.v[6].x, 1);
        T r7 = __shfl_down_sync(0xffffffffu, q.v[7].x, 1);
        if (own_left) { l1 = q.l1; l5 = q.l5; l8 = q.l8; }
        if (own_right) { r3 = q.r3; r6 = q.r6; r7 = q.r7; }
        // planes with c_x = +1 read x - 1, planes with c_x = -1 read x + 1
        fa[0] = q.v[0].x; fb[0] = q.v[0].y;
        fa[1] = l1;       fb[1] = q.v[1].x;
        fa[2] = q.v[2].x; fb[2] = q.v[2].y;
        fa[3] = q.v[3].y; fb[3] = r3;
        fa[4] = q.v[4].x; fb[4] = q.v[4].y;
        fa[5] = l5;       fb[5] = q.v[5].x;
        fa[6] = q.v[6].y; fb[6] = r6;
        fa[7] = q.v[7].y; fb[7] = r7;
        fa[8] = l8;       fb[8] = q.v[8].x;
    };

    T pa[9], pb[9]; // pulled populations of the previous row (collides this iteration)
#pragma unroll
    for (int i = 0; i < 9; ++i) pa[i] = pb[i] = T(0);
    T pha = T(0), phb = T(0);
    double msum = 0.0;

    fetch(0);
#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
        T fa[9], fb[9];
        unpack(nxt, fa, fb);
        const T hvk = hv;
        // what the row colliding below needs from the raw set, before it is refilled
        const T ppa = pp_a, ppb = pp_b;
        const typename Vel::Row vr = vr_next;
        if (k + 1 < nk) fetch(k + 1); // the loads of row k + 1 overlap this whole iteration
        T sa, sb; // phi of both nodes, summed in order 0..8 like every other variant
        if constexpr (sizeof(T) == 4) {
            float2 s2 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int i = 0; i < 9; ++i) s2 = __fadd2_rn(s2, make_float2(fa[i], fb[i]));
            sa = s2.x;
            sb = s2.y;
        } else {
            sa = T(0);
            sb = T(0);
#pragma unroll
            for (int i = 0; i < 9; ++i) { sa += fa[i]; sb += fb[i]; }
        }
        if (act) {
            V c2;
            c2.x = chi_of<T, MODEL>(sa, a);
            c2.y = chi_of<T, MODEL>(sb, a);
            *reinterpret_cast<V*>(&chi_s[k & 3][2 + 2 * tx]) = c2;
        }
        if (tx < 32) {
            const int base = lane & 16;
            T hs = T(0);
#pragma unroll
            for (int j = 0; j < 9; ++j) hs += __shfl_sync(0xffffffffu, hvk, base + j);
            if (lane == 0) chi_s[k & 3][1] = chi_of<T, MODEL>(hs, a);
            if (lane == 16) chi_s[k & 3][w + 2] = chi_of<T, MODEL>(hs, a);
        }
        __syncthreads();
        if (k >= 2) {
            const int yc = UP ? y1 - k + 1 : y0 + k - 2;
            const int j = act ? 2 * tx : w - 2; // ring column of xa - 1 is j + 1
            // ring slots of rows yc - 1 (S) and yc + 1 (N): the rows pulled at k - 2 and k
            const int ks = UP ? k : k - 2, kn = UP ? k - 2 : k;
            V o2[9];
            collide_pair<T, MODEL>(a, vel, ca, cb, vr, vel.rowv(cb, xb, yc), pa, pb, pha, phb, ppa, ppb,
                                   chi_s[ks & 3] + 1 + j, chi_s[(k - 1) & 3] + 1 + j, chi_s[kn & 3] + 1 + j, o2);
            if (act) {
                const unsigned o = (unsigned)yc * nxu + (unsigned)xa;
#pragma unroll
                for (int i = 0; i < 9; ++i) *reinterpret_cast<V*>(a.fout + (o + (unsigned)i * plane)) = o2[i];
                V p2;
                p2.x = pha;
                p2.y = phb;
                if constexpr (sizeof(T) == 4) // the phi plane's L2 policy (ace_kernels.cuh)
                    st_policy(a.phi + o, p2, l2_store_policy_all((a.l2_keep & L2_KEEP_PHI) != 0));
                else
                    *reinterpret_cast<V*>(a.phi + o) = p2;
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
        *mass_out = s;
    }
    __syncthreads();
}

template <typename T, int MODEL, class Vel>
__global__ void __launch_bounds__(PAIR_THREADS, sizeof(T) == 4 ? 5 : 1) ace_step_pair(const StepArgs<T> a, const Vel vel)
{
    __shared__ __align__(16) T chi_s[4][PAIR_COLS + 4];
    __shared__ double red_s[PAIR_THREADS / 32];
    // Programmatic dependent launch: let the next step's CTAs be scheduled as slots free
    // up, and wait for the previous step (all of its memory) before touching the state.
    // Both are no-ops for an ordinary launch.
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    double* mp = &a.mass_part[(long long)blockIdx.y * gridDim.x + blockIdx.x];
    if (march_up(blockIdx.y, a.tdir))
        pair_tile<T, MODEL, Vel, true>(a, vel, blockIdx.x * PAIR_COLS, blockIdx.y * a.rows, chi_s, red_s, mp);
    else
        pair_tile<T, MODEL, Vel, false>(a, vel, blockIdx.x * PAIR_COLS, blockIdx.y * a.rows, chi_s, red_s, mp);
}

} // namespace lbmace
