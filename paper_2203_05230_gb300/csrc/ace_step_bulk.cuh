// ace_step_bulk.cuh -- the fused step (rows a1-a13 of ace_kernels.cuh) with its
// population reads staged through shared memory by the bulk-copy engine.
//
// A CTA owns TX consecutive columns (one thread each) and marches down `rows` rows.
// One producer thread streams, for each source row it needs, the 9 population planes
// over columns [x0 - H, x0 + w + H) (H = 16 bytes of halo on each side) and the phi
// row of its own columns into a ring of STAGES shared-memory stages, with
// cp.async.bulk completing on one mbarrier per stage. The copies run several rows
// ahead of the arithmetic, so many bytes are in flight per SM without holding them in
// registers. The periodic wrap in x is handled by splitting a row's column range at
// the lattice edge into at most three 16-byte aligned segments. All threads then pull
// f_i(x, t) = f*_i(x - c_i, t - 1) from shared memory, and the collision and stores
// are those of ace_step (collide_node), so both kernels give identical results.
//
// Requirements (checked by the host): nx * sizeof(T) a multiple of 16 and nx >= H.
// Every wait on an mbarrier is bounded; on timeout the CTA sets *err, waits (bounded)
// for the copies it issued, and returns.
#pragma once

#include "ace_kernels.cuh"

namespace lbmace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~`limit` clock cycles and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

constexpr long long kWaitLimitCycles = 4000000000LL; // ~2 s at 2 GHz

template <typename T, int TX, int STAGES>
struct BulkSmem {
    static constexpr int H = 16 / (int)sizeof(T); // halo columns per side (16 bytes)
    static constexpr int W = TX + 2 * H;           // staged columns per plane row
    uint64_t bar[STAGES];
    alignas(16) T f[STAGES][9][W];
    alignas(16) T phi[STAGES][TX];
    T chi[4][TX + 2];
    double red[TX / 32];
};

template <typename T, int MODEL, class Vel, int TX, int STAGES>
__global__ void __launch_bounds__(TX) ace_step_bulk(const StepArgs<T> a, const Vel vel, int* err)
{
    using Sm = BulkSmem<T, TX, STAGES>;
    constexpr int H = Sm::H;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Sm& sm = *reinterpret_cast<Sm*>(smem_raw);

    const int tx = threadIdx.x;
    const int lane = tx & 31;
    const int x0 = blockIdx.x * TX;
    const int w = min(TX, a.nx - x0);
    const bool act = tx < w;
    const int x = x0 + (act ? tx : 0);
    const int y0 = blockIdx.y * a.rows;
    const int y1 = min(y0 + a.rows, a.ny);
    const int nk = y1 - y0 + 2;   // pulled rows y0-1 .. y1
    const int nsrc = nk + 2;      // source rows y0-2 .. y1+1 (source index q <-> row y0-2+q)

    // Producer: stage source index q (9 planes with halo, plus the phi row when the
    // row is one this CTA collides).
    auto issue = [&](int q) {
        const int st = q % STAGES;
        const int row = wrap_idx(y0 - 2 + q, a.ny);
        const bool with_phi = (q >= 2) && (q < nsrc - 2);
        const uint32_t bytes = (uint32_t)((9 * (w + 2 * H) + (with_phi ? w : 0)) * sizeof(T));
        mbar_expect_tx(&sm.bar[st], bytes);
        const int lo = x0 - H, hi = x0 + w + H;
        const long long rowoff = (long long)row * a.nx;
        for (int i = 0; i < 9; ++i) {
            const T* plane = a.fin + (long long)i * a.plane + rowoff;
            T* dst = sm.f[st][i];
            if (lo < 0) bulk_g2s(dst, plane + (a.nx + lo), (uint32_t)(-lo * sizeof(T)), &sm.bar[st]);
            const int m0 = lo < 0 ? 0 : lo, m1 = hi > a.nx ? a.nx : hi;
            bulk_g2s(dst + (m0 - lo), plane + m0, (uint32_t)((m1 - m0) * sizeof(T)), &sm.bar[st]);
            if (hi > a.nx) bulk_g2s(dst + (a.nx - lo), plane, (uint32_t)((hi - a.nx) * sizeof(T)), &sm.bar[st]);
        }
        if (with_phi) bulk_g2s(sm.phi[st], a.phi + rowoff + x0, (uint32_t)(w * sizeof(T)), &sm.bar[st]);
    };

    if (tx == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&sm.bar[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    int issued = 0; // producer's count of issued source indices
    if (tx == 0) {
        for (; issued < STAGES && issued < nsrc; ++issued) issue(issued);
    }

    const typename Vel::Col vcol = vel.col(x);
    T ra[9], rb[9]; // pulled row r, row r - 1
#pragma unroll
    for (int i = 0; i < 9; ++i) ra[i] = rb[i] = T(0);
    T phb = T(0);
    double msum = 0.0;    // FP64 column sum of phi over this thread's rows
    bool ok = true;       // this thread's waits all completed
    bool aborted = false; // some thread's wait gave up (uniform across the CTA)
    int waited = 0;       // source indices this thread has seen complete

    // Pulled row r = y0 - 1 + k into `cur`; row r - 1 (in `prev`) collides once psi of
    // rows r - 2 .. r is in the ring. Returns false when the CTA gives up.
    auto row = [&](int k, T (&cur)[9], const T (&prev)[9]) -> bool {
        // sources k, k+1, k+2 (rows r-1, r, r+1) must be in
        for (; waited <= k + 2; ++waited)
            if (ok && !mbar_wait_bounded(&sm.bar[waited % STAGES], (uint32_t)((waited / STAGES) & 1), kWaitLimitCycles))
                ok = false;
        T ph = T(0);
        if (act) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int q = k + 1 - cy_of(i);
                cur[i] = sm.f[q % STAGES][i][tx + H - cx_of(i)];
                ph += cur[i];
            }
            sm.chi[k & 3][1 + tx] = chi_of<T, MODEL>(ph, a);
        }
        // psi at the columns left (x0 - 1) and right (x0 + w) of the strip
        if (tx == 0 || tx == w - 1) {
            for (int side = 0; side < 2; ++side) {
                if ((side == 0 && tx != 0) || (side == 1 && tx != w - 1)) continue;
                const int col = side == 0 ? H - 1 : w + H; // staged column of the halo node
                T hs = T(0);
#pragma unroll
                for (int i = 0; i < 9; ++i) hs += sm.f[(k + 1 - cy_of(i)) % STAGES][i][col - cx_of(i)];
                sm.chi[k & 3][side == 0 ? 0 : w + 1] = chi_of<T, MODEL>(hs, a);
            }
        }
        if (__syncthreads_or(!ok)) return false; // a barrier whose result every thread shares

        // refill the stage freed by source index k - 1 (consumed by all threads)
        if (tx == 0 && k >= 1 && issued < nsrc) {
            fence_proxy_async_smem();
            issue(issued);
            ++issued;
        }
        if (k >= 2 && act) {
            const int yc = y0 + k - 2; // source index k
            const T pp = sm.phi[k % STAGES][tx];
            collide_node<T, MODEL>(a, vel, vcol, x, yc, prev, phb, pp, sm.chi[(k - 2) & 3] + tx,
                                   sm.chi[(k - 1) & 3] + tx, sm.chi[k & 3] + tx);
            a.phi[(long long)yc * a.nx + x] = phb;
            msum += (double)phb;
        }
        phb = ph;
        return true;
    };
#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
        if (!row(k, ra, rb)) { aborted = true; break; }
#pragma unroll
        for (int i = 0; i < 9; ++i) rb[i] = ra[i];
    }

    if (aborted) {
        // give up: record it, let this CTA's copies in flight (at most the last STAGES
        // issued, one per stage) land with a bounded wait, and return
        if (tx == 0) {
            atomicExch(err, 1);
            for (int q = issued > STAGES ? issued - STAGES : 0; q < issued; ++q)
                mbar_wait_bounded(&sm.bar[q % STAGES], (uint32_t)((q / STAGES) & 1), kWaitLimitCycles);
        }
        return;
    }

#pragma unroll
    for (int off = 16; off > 0; off >>= 1) msum += __shfl_down_sync(0xffffffffu, msum, off);
    if (lane == 0) sm.red[tx >> 5] = msum;
    __syncthreads();
    if (tx == 0) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < TX / 32; ++i) s += sm.red[i];
        a.mass_part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

} // namespace lbmace
