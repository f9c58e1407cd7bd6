// ace_step_warp.cuh -- the fused step (rows a1-a13 of ace_kernels.cuh) with each warp
// working on its own 32-column strip, so no CTA-wide barrier sits in the row loop.
//
// A CTA covers TILE_X columns as four independent warps. Warp j owns columns
// [x0 + 32 j, x0 + 32 j + 32) and marches down `rows` rows with a warp-private 4-slot
// ring of psi rows in shared memory, ordered by __syncwarp alone. psi at the two
// columns beside the warp's strip is recomputed from the populations by lanes 0..8
// (left) and 16..24 (right), summed in the interior's order. Everything the
// collision of row r - 1 needs from memory -- the populations of row r + 1, phi(t-1)
// of row r and the velocity factors of row r -- is requested one row ahead, so the
// loop only waits on loads issued a full row earlier. The collision and stores are
// collide_node, shared with the other variants, so all variants agree bit for bit.
#pragma once

#include "ace_kernels.cuh"

namespace lbmace {

constexpr int WARP_COLS = 32;

template <typename T, int MODEL, class Vel>
__global__ void __launch_bounds__(TILE_X) ace_step_warp(const StepArgs<T> a, const Vel vel)
{
    __shared__ T chi_s[TILE_X / WARP_COLS][4][WARP_COLS + 2];
    __shared__ double red_s[TILE_X / 32];

    const int tx = threadIdx.x;
    const int lane = tx & 31;
    const int wid = tx >> 5;
    const int xs = blockIdx.x * TILE_X + wid * WARP_COLS; // first column of this warp's strip
    const int ww = max(0, min(WARP_COLS, a.nx - xs));     // strip width (0: nothing to do)
    const bool act = lane < ww;
    const int x = act ? xs + lane : (ww > 0 ? xs : 0);
    const int xm = x == 0 ? a.nx - 1 : x - 1;
    const int xp = x == a.nx - 1 ? 0 : x + 1;
    const int y0 = blockIdx.y * a.rows;
    const int y1 = min(y0 + a.rows, a.ny);
    const int nk = y1 - y0 + 2; // rows y0-1 .. y1 get phi and chi
    T (*chi)[WARP_COLS + 2] = chi_s[wid];

    // halo lanes: 0..8 pull population `hi` of the column left of the strip, 16..24
    // that of the column right of it
    const bool halo = ww > 0 && (lane & 15) < 9;
    const int hi = lane & 15;
    int hcol = 0;
    if (halo) {
        const int c = lane < 16 ? (xs == 0 ? a.nx - 1 : xs - 1) : (xs + ww == a.nx ? 0 : xs + ww);
        hcol = wrap_idx(c - cx_of(hi), a.nx);
    }
    const int hcy = halo ? cy_of(hi) : 0;
    const T* hplane = a.fin + (long long)(halo ? hi : 0) * a.plane;
    const typename Vel::Col vcol = vel.col(x);

    T ra[9], rb[9], rc[9]; // pulled row r, row r - 1, row r + 1 (prefetched)
    T hv = T(0);           // this lane's halo population of the row being pulled
    T pp_next = T(0);      // phi(t-1) of the row that collides next
    typename Vel::Row vr_next{}; // velocity factors of that row
    T phb = T(0);
    double msum = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) ra[i] = rb[i] = rc[i] = T(0);

    // Requests for pull index k: the populations of row r = y0 - 1 + k, and phi(t-1)
    // and the velocity factors of row y0 + k - 2, which collides in the row() call
    // that pulls row r.
    auto fetch = [&](int k, T (&dst)[9]) {
        const int r = wrap_idx(y0 - 1 + k, a.ny);
        if (act) pull_row(a.fin, a.plane, a.nx, r, wrap_idx(r - 1, a.ny), wrap_idx(r + 1, a.ny), x, xm, xp, dst);
        if (halo) hv = hplane[(long long)wrap_idx(r - hcy, a.ny) * a.nx + hcol];
        const int yc = y0 + k - 2;
        if (yc >= y0 && yc < y1) {
            if (act && !a.first) pp_next = a.phi[(long long)yc * a.nx + x];
            vr_next = vel.rowv(vcol, x, yc);
        }
    };
    if (ww > 0) fetch(0, ra);

    // pulled row r = y0 - 1 + k in `cur`; row r - 1 (in `prev`) collides; `next`
    // receives row r + 1
    auto row = [&](int k, const T (&cur)[9], const T (&prev)[9], T (&next)[9]) {
        T ph = T(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) ph += cur[i];
        if (act) chi[k & 3][1 + lane] = chi_of<T, MODEL>(ph, a);
        {
            const int base = lane & 16;
            T hs = T(0);
#pragma unroll
            for (int j = 0; j < 9; ++j) hs += __shfl_sync(0xffffffffu, hv, base + j);
            if (lane == 0) chi[k & 3][0] = chi_of<T, MODEL>(hs, a);
            if (lane == 16) chi[k & 3][ww + 1] = chi_of<T, MODEL>(hs, a);
        }
        __syncwarp();
        const T pp = pp_next;                 // for row r - 1 = y0 + k - 2 (fetched with row r)
        const typename Vel::Row vr = vr_next;
        if (k + 1 < nk) fetch(k + 1, next);
        if (k >= 2 && act) {
            const int yc = y0 + k - 2;
            collide_node_row<T, MODEL>(a, vel, vcol, vr, x, yc, prev, phb, pp, chi[(k - 2) & 3] + lane,
                                       chi[(k - 1) & 3] + lane, chi[k & 3] + lane);
            a.phi[(long long)yc * a.nx + x] = phb;
            msum += (double)phb;
        }
        phb = ph;
    };
    if (ww > 0) {
#pragma unroll 1
        for (int k = 0; k < nk; ++k) {
            row(k, ra, rb, rc);
#pragma unroll
            for (int i = 0; i < 9; ++i) { rb[i] = ra[i]; ra[i] = rc[i]; }
        }
    }

#pragma unroll
    for (int off = 16; off > 0; off >>= 1) msum += __shfl_down_sync(0xffffffffu, msum, off);
    if (lane == 0) red_s[wid] = msum;
    __syncthreads();
    if (tx == 0) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < TILE_X / 32; ++i) s += red_s[i];
        a.mass_part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

} // namespace lbmace
