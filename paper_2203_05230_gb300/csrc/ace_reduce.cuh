// ace_reduce.cuh -- global mass reductions over a stored lattice state (FP64, FP32 and
// 16-bit deviation storage), each finished by its last CTA into a result block.
//
// The global mass sum_x sum_i f_i(x, t) of the state is the conserved quantity of the
// scheme (Eq. 12 summed over the lattice; mass conservation, Section 2.2). The step
// kernels reduce phi(t) per CTA themselves (row a13); these kernels read the whole
// stored state on request.
#pragma once

#include "ace_kernels.cuh"
#include "ace_step_dev.cuh"

namespace lbmace {

// Neumaier-compensated accumulation.
__device__ __forceinline__ void neumaier(double& s, double& c, double v)
{
    const double t = s + v;
    c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
}

constexpr int RED_THREADS = 256;

// Partial sums of n values of T: each thread sums a fixed strided subset with
// compensation, the CTA combines in a fixed tree order. Deterministic.
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) ace_sum_partials(const T* __restrict__ v, long long n,
                                                                double* __restrict__ part)
{
    __shared__ double sh[RED_THREADS];
    double s = 0.0, c = 0.0;
    for (long long k = blockIdx.x * (long long)RED_THREADS + threadIdx.x; k < n;
         k += (long long)gridDim.x * RED_THREADS)
        neumaier(s, c, (double)v[k]);
    sh[threadIdx.x] = s + c;
    __syncthreads();
    for (int h = RED_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Mass accumulator of one thread over groups of four FP32 values (split_add2i), with the
// largest magnitude seen. The integer sum is exact while every value is below 2 in
// magnitude (every population and phi of a lattice in practice) and the thread adds at
// most 8192 values (the host sizes the grid for that); a thread that saw a larger value
// (or an infinity) sums its values again in FP64 instead. A NaN reaches lo and the total.
struct MassAccI {
    unsigned ai = 0u, nv = 0u;
    float2 lo = make_float2(0.0f, 0.0f);
    float vmax = 0.0f;
    __device__ __forceinline__ void add(float4 q)
    {
        vmax = fmaxf(vmax, fmaxf(fmaxf(fabsf(q.x), fabsf(q.y)), fmaxf(fabsf(q.z), fabsf(q.w))));
        split_add2i(ai, lo, make_float2(q.x, q.y));
        split_add2i(ai, lo, make_float2(q.z, q.w));
        nv += 4u;
    }
    __device__ __forceinline__ bool exact() const { return vmax < 2.0f; }
    __device__ __forceinline__ double total() const { return split_total_i(ai, lo, nv); }
};
constexpr long long MASS_VALUES_PER_THREAD = 8192; // bound of MassAccI's exact integer sum

// Grid of a global-mass reduction over `values` values with a kernel that keeps `occ`
// CTAs of RED_THREADS threads resident per SM: one wave of resident CTAs, or more CTAs
// when a thread would otherwise add more than MASS_VALUES_PER_THREAD values (the bound
// of MassAccI; 16 values of slack for the grid-stride rounding of the two value kinds).
inline int mass_reduction_grid(int sms, int occ, long long values)
{
    const long long per_cta = (MASS_VALUES_PER_THREAD - 16) * RED_THREADS;
    long long g = (long long)sms * (occ < 1 ? 1 : occ);
    const long long need = (values + per_cta - 1) / per_cta;
    if (need > g) g = need;
    return (int)g;
}

// Fixed-order CTA sum of one double per thread into part[blockIdx.x]: a shuffle tree in
// each warp, then the warps' sums in warp order by thread 0.
__device__ __forceinline__ void block_sum_to(double v, double* sh, double* part)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < RED_THREADS / 32; ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

// Fixed-order compensated sum of part[0 .. n) by the CTA's RED_THREADS threads: each a
// Neumaier sum over a strided subset, then a pairwise tree whose nodes add two
// (sum, compensation) pairs with an error-free two-sum of the sums. Returns the total
// in thread 0.
__device__ __forceinline__ double block_final_sum(const double* part, int n, double* ss, double* sc)
{
    double s = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < n; k += RED_THREADS) neumaier(s, c, part[k]);
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int h = RED_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            const double a = ss[threadIdx.x], b = ss[threadIdx.x + h];
            const double t = a + b;
            const double bp = t - a;
            const double err = (a - (t - bp)) + (b - bp); // two-sum: a + b = t + err exactly
            ss[threadIdx.x] = t;
            sc[threadIdx.x] += sc[threadIdx.x + h] + err;
        }
        __syncthreads();
    }
    return ss[0] + sc[0];
}

// The result of a finished sum: out[0] = the sum; out[1] = the device wait-failure flag
// *err (0 when err is null), so a host that reads out after synchronising needs no copy.
// out may point into mapped host memory.
__device__ __forceinline__ void write_result(double* out, double total, const int* err)
{
    out[0] = total;
    out[1] = err ? (double)*err : 0.0;
}

// After every CTA has written its partial: the CTA that finishes last (a ticket counter
// in global memory, zero between calls) sums all partials in their fixed order, writes
// the result (write_result) and resets the counter. Saves the separate finishing launch;
// the result does not depend on which CTA finishes last.
__device__ __forceinline__ void finish_in_last_block(const double* part, unsigned* done, double* out, const int* err,
                                                     double* ss, double* sc)
{
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence(); // this CTA's partial is visible before its ticket
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double total = block_final_sum(part, gridDim.x, ss, sc);
    if (threadIdx.x == 0) {
        write_result(out, total, err);
        *done = 0u;
    }
}

// Partial sums of n FP32 values (16-byte aligned) for the global mass: groups of four
// independent 16-byte loads per thread, MassAccI over a fixed strided subset of the
// groups of four (the grid gives each thread at most MASS_VALUES_PER_THREAD values), the
// n % 4 last values in FP64 by the first threads of CTA 0, then a fixed tree per CTA and
// the final sum in the last CTA. Deterministic, and bound by HBM bandwidth rather than by
// the FP64 pipe: per value one FP32 add pair, one integer add and one max.
static __global__ void __launch_bounds__(RED_THREADS) ace_sum_partials_f32(const float* __restrict__ v, long long n,
                                                                           double* __restrict__ part,
                                                                           unsigned* done, double* out,
                                                                           const int* err)
{
    __shared__ double sh[RED_THREADS], sc[RED_THREADS];
    const float4* v4 = reinterpret_cast<const float4*>(v);
    const long long n4 = n >> 2;
    const long long stride = (long long)gridDim.x * RED_THREADS;
    const long long first = blockIdx.x * (long long)RED_THREADS + threadIdx.x;
    MassAccI acc;
    long long k = first;
    // groups of four independent 16-byte loads, software-pipelined: the next group's loads
    // are issued before this group is added (35.0 -> 32.9 us at 2048^2)
    float4 q0{}, q1{}, q2{}, q3{};
    bool have = k + 3 * stride < n4;
    if (have) {
        q0 = v4[k]; q1 = v4[k + stride]; q2 = v4[k + 2 * stride]; q3 = v4[k + 3 * stride];
    }
    while (have) {
        const long long kn = k + 4 * stride;
        const bool next = kn + 3 * stride < n4;
        float4 r0{}, r1{}, r2{}, r3{};
        if (next) {
            r0 = v4[kn]; r1 = v4[kn + stride]; r2 = v4[kn + 2 * stride]; r3 = v4[kn + 3 * stride];
        }
        acc.add(q0);
        acc.add(q1);
        acc.add(q2);
        acc.add(q3);
        q0 = r0; q1 = r1; q2 = r2; q3 = r3;
        k = kn;
        have = next;
    }
    for (; k < n4; k += stride) acc.add(v4[k]);
    double s;
    if (acc.exact()) {
        s = acc.total();
    } else { // a value of 2 or more in magnitude: this thread's values again, in FP64
        s = 0.0;
        for (k = first; k < n4; k += stride) {
            const float4 q = v4[k];
            s += ((double)q.x + (double)q.y) + ((double)q.z + (double)q.w);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < (n & 3)) s += (double)v[4 * n4 + threadIdx.x];
    block_sum_to(s, sh, part);
    finish_in_last_block(part, done, out, err, sh, sc);
}

// Final sum of n partials by one CTA (block_final_sum), for partials written by kernels
// that do not finish their own sums; writes the result as write_result does.
static __global__ void __launch_bounds__(RED_THREADS) ace_finalize(const double* __restrict__ part, int n,
                                                                   double* __restrict__ out, const int* err)
{
    __shared__ double ss[RED_THREADS], sc[RED_THREADS];
    const double total = block_final_sum(part, n, ss, sc);
    if (threadIdx.x == 0) write_result(out, total, err);
}

// Partial sums of the stored state's mass: the 9 deviation planes (n16 16-bit values,
// 16-byte aligned) plus the phi plane (n values, FP32, 16-byte aligned); the split
// weights sum to 1, so sum_i f_i = sum_i g_i + phi at every node. Groups of four
// independent 16-byte loads (32 values) per thread, widened exactly to FP32 and summed
// by MassAccI (a thread that saw a value of 2 or more sums its values again in FP64);
// the ragged ends in FP64 by the first threads of CTA 0; a fixed tree per CTA and the
// final sum in the last CTA. The grid gives each thread at most MASS_VALUES_PER_THREAD
// values. Deterministic.
template <typename S>
__global__ void __launch_bounds__(RED_THREADS) ace_sum_partials_dev(const unsigned short* __restrict__ g,
                                                                    const float* __restrict__ phi, long long n,
                                                                    double* __restrict__ part, unsigned* done,
                                                                    double* out, const int* err)
{
    using C = Dev16<S>;
    __shared__ double sh[RED_THREADS], sc[RED_THREADS];
    const long long n16 = 9 * n, ng = n16 >> 3, np = n >> 2;
    const uint4* g8 = reinterpret_cast<const uint4*>(g);
    const float4* p4 = reinterpret_cast<const float4*>(phi);
    const long long stride = (long long)gridDim.x * RED_THREADS;
    const long long first = blockIdx.x * (long long)RED_THREADS + threadIdx.x;
    MassAccI acc;
    auto add8 = [&](const uint4 q) {
        acc.add(make_float4(C::lo(q.x), C::hi(q.x), C::lo(q.y), C::hi(q.y)));
        acc.add(make_float4(C::lo(q.z), C::hi(q.z), C::lo(q.w), C::hi(q.w)));
    };
    long long k = first;
    // groups of four independent 16-byte loads, software-pipelined as in ace_sum_partials_f32
    uint4 q0{}, q1{}, q2{}, q3{};
    bool have = k + 3 * stride < ng;
    if (have) {
        q0 = g8[k]; q1 = g8[k + stride]; q2 = g8[k + 2 * stride]; q3 = g8[k + 3 * stride];
    }
    while (have) {
        const long long kn = k + 4 * stride;
        const bool next = kn + 3 * stride < ng;
        uint4 r0{}, r1{}, r2{}, r3{};
        if (next) {
            r0 = g8[kn]; r1 = g8[kn + stride]; r2 = g8[kn + 2 * stride]; r3 = g8[kn + 3 * stride];
        }
        add8(q0);
        add8(q1);
        add8(q2);
        add8(q3);
        q0 = r0; q1 = r1; q2 = r2; q3 = r3;
        k = kn;
        have = next;
    }
    for (; k < ng; k += stride) add8(g8[k]);
    for (k = first; k < np; k += stride) acc.add(p4[k]);
    double s;
    if (acc.exact()) {
        s = acc.total();
    } else { // a value of 2 or more in magnitude: this thread's values again, in FP64
        s = 0.0;
        for (k = first; k < ng; k += stride) {
            const uint4 q = g8[k];
            const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) s += (double)C::lo(w[j]) + (double)C::hi(w[j]);
        }
        for (k = first; k < np; k += stride) {
            const float4 q = p4[k];
            s += ((double)q.x + (double)q.y) + ((double)q.z + (double)q.w);
        }
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x < (n16 & 7)) s += (double)C::one(g[8 * ng + threadIdx.x]);
        if (threadIdx.x < (n & 3)) s += (double)phi[4 * np + threadIdx.x];
    }
    block_sum_to(s, sh, part);
    finish_in_last_block(part, done, out, err, sh, sc);
}

} // namespace lbmace
