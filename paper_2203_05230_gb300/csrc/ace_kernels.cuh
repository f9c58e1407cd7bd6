// ace_kernels.cuh -- device code of the GB300 (sm_103a) lattice Boltzmann step for
// the modified conservative Allen-Cahn equation (Liang, arXiv 2203.05230).
//
// One fused kernel per time step (ace_step) does, for every node of its tile:
//   a1 pull-stream        f_i(x, t) = f*_i(x - c_i, t - 1)             (Eq. 9, periodic)
//   a2 moment             phi = sum_i f_i                               (Eq. 12)
//   a3 signed distance    psi = eps ln((phi_c + d)/(1 - phi_c + d))     (Eq. 13, clip)
//   a4 isotropic gradient grad psi = sum_i w_i c_i psi(x + c_i) / c_s^2
//   a5 normal             n = grad psi / (|grad psi| + d)               (Eq. 13)
//   a6 sharpening         S = (1/(4 eps)) (1 - tanh^2(psi/(2 eps)))     (Eqs. 6, 11)
//                           evaluated as (1 - ((2 phi_c - 1)/(1 + 2 d))^2)/(4 eps),
//                           an exact rewrite since tanh(psi/(2 eps)) = (2 phi_c - 1)/(1 + 2 d)
//   a7 velocity           Eq. 14 from separable 1-D tables (no memory traffic per node)
//   a8 time derivative    d_t(phi u) = phi(t) u(t) - phi(t-1) u(t-1)   (explicit Euler)
//   a9 forcing            F_i = w_i c_i . (d_t(phi u) + c_s^2 S n) / c_s^2   (Eq. 11)
//   a10 equilibrium       f_i^eq = w_i phi (1 + c_i . u / c_s^2)       (Eq. 10)
//   a11 collision         f*_i = f_i - (f_i - f_i^eq)/tau + (1 - 1/(2 tau)) F_i  (Eq. 9),
//                           evaluated as (1 - 1/tau) f_i + w_i (A + c_i . B) with f*_0 the
//                           remainder phi - sum_{i>=1} f*_i (exact mass in any precision)
//   a12 store             f*_i (SoA planes) and phi(t) (becomes phi(t-1) of the next step)
//   a13 mass partial      one FP64 sum of phi per CTA
//
// Data layout in HBM: populations are 9 SoA planes [9][ny][nx] (x fastest) in two
// ping-pong buffers holding post-collision values f*(t-1); the phi plane [ny][nx]
// holds phi(t-1) and is overwritten in place with phi(t) by the thread that reads it.
//
// Tiling: a CTA owns TILE_X consecutive columns (one per thread) and marches down
// `rows` rows. For each row r it pulls the 9 populations, forms phi and psi, and
// keeps psi in a 4-slot shared-memory ring of rows; the collision of row r - 1 runs
// once psi of rows r - 2 .. r is there. psi at the two columns left and right of
// the strip (the stencil's halo) is recomputed from the populations by lanes of
// warp 0, and the strip recomputes psi on one row above and below its range.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmace {

constexpr int TILE_X = 128;

// L2 eviction priority of a kernel's stores, set by the host per lattice (StepArgs::
// l2_keep): a policy from createpolicy rides on each st.global.L2::cache_hint. A step
// reads first the rows the step before wrote last (alternating march), and what it reads
// is dead once read, so letting written lines outlast read ones turns more of the next
// step's reads into L2 hits where the kept data fits the L2 (measured on GB300).
constexpr int L2_KEEP_F = 1, L2_KEEP_PHI = 2;

// evict_last on `frac` of the lines when keep, else the normal priority (both policies
// are made and one is selected: no branch)
__device__ __forceinline__ unsigned long long l2_store_policy_quarter(bool keep)
{
    unsigned long long last, normal;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 0.25;" : "=l"(last));
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(normal));
    return keep ? last : normal;
}
__device__ __forceinline__ unsigned long long l2_store_policy_all(bool keep)
{
    unsigned long long last, normal;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(last));
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(normal));
    return keep ? last : normal;
}
__device__ __forceinline__ void st_policy(float* p, float4 v, unsigned long long policy)
{
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
                 :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(policy) : "memory");
}
__device__ __forceinline__ void st_policy(float* p, float2 v, unsigned long long policy)
{
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;"
                 :: "l"(p), "f"(v.x), "f"(v.y), "l"(policy) : "memory");
}

// D2Q9 velocity set and weights (Section 2.2, after Eq. 10):
// 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)
__host__ __device__ constexpr int cx_of(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
template <typename T>
__host__ __device__ constexpr T w_of(int i)
{
    return i == 0 ? T(4) / T(9) : (i < 5 ? T(1) / T(9) : T(1) / T(36));
}

__device__ __forceinline__ float dlog(float v) { return logf(v); }
__device__ __forceinline__ double dlog(double v) { return log(v); }
__device__ __forceinline__ float dsqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double dsqrt(double v) { return sqrt(v); }

__device__ __forceinline__ int wrap_idx(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

enum { MODEL_MODIFIED = 0, MODEL_CONSERVATIVE = 1 };

// Scalar parameters of one step.
template <typename T>
struct StepArgs {
    const T* __restrict__ fin; // f*(t-1), 9 planes
    T* __restrict__ fout;      // f*(t), 9 planes
    T* phi;                    // in: phi(t-1); out: phi(t)
    double* mass_part;         // one FP64 partial per CTA
    int nx, ny;
    long long plane;           // nx * ny
    int rows;                  // rows per CTA
    int first;                 // t == 0: no time-derivative term
    int tdir;                  // t & 1: march direction of the row bands (column-pair kernels)
    int l2_keep = 0;           // L2 priority of the stores (bits; 0 = normal): L2_KEEP_F = f* of
                               // the FP32 quad kernel evict_last on a quarter of the lines (unset),
                               // L2_KEEP_PHI = the phi plane evict_last (FP32 and 16-bit kernels)
    T omega;                   // 1 / tau
    T fpref;                   // 1 - 1 / (2 tau)
    T eps, inv_eps, inv4eps;   // eps, 1/eps, 1/(4 eps)
    T delta, inv1p2d;          // regulariser d, 1/(1 + 2 d)
};

// Prescribed velocities. `col(x)` holds what depends on x only, `rowv(col, x, y)` what
// else a thread needs for node (x, y) (so it can be requested ahead of use), and
// `at(col, row, ...)` gives u(t) and u(t-1) from the two.
template <typename T>
struct VelVortex { // Eq. 14: u = A sx2[x] s2y[y] c(t), v = -A sy2[y] s2x[x] c(t)
    const T* sx2; const T* s2x; const T* sy2; const T* s2y;
    T amp, ct, ctm1;
    static constexpr bool row_uniform = true; // rowv does not depend on the column
    struct Col { T sx2, s2x; };
    struct Row { T sy2, s2y; };
    __device__ __forceinline__ Col col(int x) const { return {sx2[x], s2x[x]}; }
    __device__ __forceinline__ Row rowv(const Col&, int, int y) const { return {sy2[y], s2y[y]}; }
    __device__ __forceinline__ void at(const Col& c, const Row& r, T& u, T& v, T& up, T& vp) const
    {
        const T us = amp * c.sx2 * r.s2y;
        const T vs = -amp * r.sy2 * c.s2x;
        u = us * ct; v = vs * ct; up = us * ctm1; vp = vs * ctm1;
    }
};

template <typename T>
struct VelUniform {
    T ux, uy;
    static constexpr bool row_uniform = true;
    struct Col {};
    struct Row {};
    __device__ __forceinline__ Col col(int) const { return {}; }
    __device__ __forceinline__ Row rowv(const Col&, int, int) const { return {}; }
    __device__ __forceinline__ void at(const Col&, const Row&, T& u, T& v, T& up, T& vp) const
    {
        u = ux; v = uy; up = ux; vp = uy;
    }
};

template <typename T>
struct VelPlanes { // device FP64 planes of u(t), v(t), u(t-1), v(t-1)
    const double* u; const double* v; const double* up; const double* vp;
    int nx;
    static constexpr bool row_uniform = false;
    struct Col {};
    struct Row { T u, v, up, vp; };
    __device__ __forceinline__ Col col(int) const { return {}; }
    __device__ __forceinline__ Row rowv(const Col&, int x, int y) const
    {
        const long long k = (long long)y * nx + x;
        return {T(u[k]), T(v[k]), T(up[k]), T(vp[k])};
    }
    __device__ __forceinline__ void at(const Col&, const Row& r, T& uu, T& vv, T& upp, T& vpp) const
    {
        uu = r.u; vv = r.v; upp = r.up; vpp = r.vp;
    }
};

// Eq. 10, f_i^eq = w_i phi (1 + c_i . u / c_s^2), with f_0^eq taken as the remainder
// phi - sum_{i>=1} f_i^eq. Since c_0 = 0 this equals w_0 phi in real arithmetic; in
// floating point it makes the equilibrium carry exactly the mass phi whatever the
// rounding of the weights (in FP32 the nine weights sum to 1 + 7.5e-9, which would add
// omega * phi * 7.5e-9 of mass at every node and step).
template <typename T>
__device__ __forceinline__ void equilibrium(T ph, T u, T v, T* feq)
{
    T rest = T(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const T cu = T(cx_of(i)) * u + T(cy_of(i)) * v;
        feq[i] = w_of<T>(i) * ph * (T(1) + T(3) * cu);
        rest += feq[i];
    }
    feq[0] = ph - rest;
}

// chi is the field whose isotropic gradient gives the normal: psi (Eq. 13) for the
// paper's model, phi for the conservative-ACE ablation (Eq. 1).
// psi of Eq. 13 from the clipped phi. FP64: one log of the ratio. FP32: the hardware
// base-2 logarithm of numerator and denominator (no division); its ~1e-7 absolute
// error in psi only perturbs the direction of n, far below FP32 storage rounding.
__device__ __forceinline__ double psi_clipped(double pc, double eps, double delta)
{
    return eps * log((pc + delta) / (1.0 - pc + delta));
}
__device__ __forceinline__ float psi_clipped(float pc, float eps, float delta)
{
    return (eps * 0.69314718055994531f) * (__log2f(pc + delta) - __log2f(1.0f - pc + delta));
}

// 1 / (|g| + delta) for the normal of Eq. 13. FP32 uses the hardware reciprocal square
// root and reciprocal (the normal's direction, not its last bits, enters Eq. 11).
__device__ __forceinline__ double inv_norm(double g2, double delta) { return 1.0 / (sqrt(g2) + delta); }
__device__ __forceinline__ float inv_norm(float g2, float delta)
{
    // |g| = g2 / sqrt(g2); below 1e-30 (far under delta) the floor only keeps 0 * inf away
    const float g = g2 * rsqrtf(fmaxf(g2, 1e-30f));
    return __fdividef(1.0f, g + delta);
}

__device__ __forceinline__ float clip01(float v) { return fminf(fmaxf(v, 0.0f), 1.0f); }
__device__ __forceinline__ double clip01(double v) { return fmin(fmax(v, 0.0), 1.0); }

template <typename T, int MODEL>
__device__ __forceinline__ T chi_of(T ph, const StepArgs<T>& a)
{
    if (MODEL == MODEL_MODIFIED) {
        return psi_clipped(clip01(ph), a.eps, a.delta);
    } else {
        return ph;
    }
}

template <typename T> struct Pair2;
template <> struct Pair2<float> { using type = float2; };
template <> struct Pair2<double> { using type = double2; };

// Arithmetic with explicit rounding and no contraction left to the compiler, on one
// node (float, double) or on two nodes at once (float2, the packed FP32x2 instructions
// of sm_100 and later). Each float2 lane rounds exactly like the float operation, so
// every kernel variant computes bit-identical populations.
template <typename V> struct Ar;
template <>
struct Ar<float> {
    using S = float;
    __device__ __forceinline__ static float c(float s) { return s; }
    __device__ __forceinline__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ __forceinline__ static float sub(float a, float b) { return __fsub_rn(a, b); }
    __device__ __forceinline__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ __forceinline__ static float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    __device__ __forceinline__ static float neg(float a) { return -a; }
    template <class F> __device__ __forceinline__ static float map(float a, F f) { return f(a); }
};
template <>
struct Ar<double> {
    using S = double;
    __device__ __forceinline__ static double c(double s) { return s; }
    __device__ __forceinline__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ __forceinline__ static double sub(double a, double b) { return __dsub_rn(a, b); }
    __device__ __forceinline__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ __forceinline__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    __device__ __forceinline__ static double neg(double a) { return -a; }
    template <class F> __device__ __forceinline__ static double map(double a, F f) { return f(a); }
};
template <>
struct Ar<float2> {
    using S = float;
    __device__ __forceinline__ static float2 c(float s) { return make_float2(s, s); }
    __device__ __forceinline__ static float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    __device__ __forceinline__ static float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
    __device__ __forceinline__ static float2 sub(float2 a, float2 b) { return __fadd2_rn(a, neg(b)); }
    __device__ __forceinline__ static float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    __device__ __forceinline__ static float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
    template <class F> __device__ __forceinline__ static float2 map(float2 a, F f) { return make_float2(f(a.x), f(a.y)); }
};

// Steps a4-a11 on V (one node, or two nodes as float2): gradient of chi from the
// stencil (cS*, cC*, cN*: rows yc - 1, yc, yc + 1; l/c/r: columns x - 1, x, x + 1),
// normal, sharpening, time derivative, forcing, equilibrium and BGK. f: pulled
// populations f_i(x, t); ph = phi(x, t); pp = phi(x, t - 1); u, v at t and up, vp at
// t - 1. Writes the post-collision populations to fs.
template <typename V, typename T, int MODEL>
__device__ __forceinline__ void collide_core(const StepArgs<T>& a, const V* f, V ph, V pp, V cSl, V cSc, V cSr, V cCl,
                                             V cCr, V cNl, V cNc, V cNr, V u, V v, V up, V vp, V* fs)
{
    using R = Ar<V>;
    const V third = R::c(T(1) / T(3)), twelfth = R::c(T(1) / T(12));
    // 3 sum_i w_i c_i chi(x + c_i): axis neighbours weigh 3/9, diagonals 3/36
    const V gx = R::fma(R::sub(cCr, cCl), third, R::mul(R::add(R::sub(cNr, cNl), R::sub(cSr, cSl)), twelfth));
    const V gy = R::fma(R::sub(cNc, cSc), third, R::mul(R::sub(R::add(cNr, cNl), R::add(cSr, cSl)), twelfth));
    const V inv = R::map(R::fma(gx, gx, R::mul(gy, gy)), [&](T g2) { return inv_norm(g2, a.delta); });
    const V nxv = R::mul(gx, inv), nyv = R::mul(gy, inv);
    V S;
    if (MODEL == MODEL_MODIFIED) {
        const V pc = R::map(ph, [](T q) { return clip01(q); });
        const V th = R::mul(R::fma(R::c(T(2)), pc, R::c(T(-1))), R::c(a.inv1p2d));
        S = R::mul(R::fma(R::neg(th), th, R::c(T(1))), R::c(a.inv4eps));
    } else {
        S = R::mul(R::mul(ph, R::sub(R::c(T(1)), ph)), R::c(a.inv_eps));
    }
    V dx = R::c(T(0)), dy = R::c(T(0));
    if (!a.first) {
        dx = R::fma(ph, u, R::neg(R::mul(pp, up)));
        dy = R::fma(ph, v, R::neg(R::mul(pp, vp)));
    }
    const V S3 = R::mul(S, third);
    const V Gx = R::fma(S3, nxv, dx); // bracket of Eq. 11: d_t(phi u) + c_s^2 S n
    const V Gy = R::fma(S3, nyv, dy);
    // Eqs. 9-11 folded: f*_i = (1 - omega) f_i + w_i (A + c_i . B) with A = omega phi
    // and B = 3 (omega phi u + (1 - 1/(2 tau)) G); f*_0 is the remainder phi - sum_{i>=1}
    // f*_i (sum_i f*_i = phi holds exactly in real arithmetic), so the collision
    // conserves mass in any precision whatever the rounding of the weights.
    const V om1 = R::c(T(1) - a.omega);
    const V A = R::mul(R::c(a.omega), ph);
    const V fp = R::c(a.fpref), three = R::c(T(3));
    const V Bx = R::mul(three, R::fma(A, u, R::mul(fp, Gx)));
    const V By = R::mul(three, R::fma(A, v, R::mul(fp, Gy)));
    const V w1 = R::c(w_of<T>(1)), w5 = R::c(w_of<T>(5));
    fs[1] = R::fma(f[1], om1, R::mul(w1, R::add(A, Bx)));
    fs[2] = R::fma(f[2], om1, R::mul(w1, R::add(A, By)));
    fs[3] = R::fma(f[3], om1, R::mul(w1, R::sub(A, Bx)));
    fs[4] = R::fma(f[4], om1, R::mul(w1, R::sub(A, By)));
    const V Bp = R::add(Bx, By), Bm = R::sub(Bx, By);
    fs[5] = R::fma(f[5], om1, R::mul(w5, R::add(A, Bp)));
    fs[6] = R::fma(f[6], om1, R::mul(w5, R::sub(A, Bm)));
    fs[7] = R::fma(f[7], om1, R::mul(w5, R::sub(A, Bp)));
    fs[8] = R::fma(f[8], om1, R::mul(w5, R::add(A, Bm)));
    V rest = fs[1];
#pragma unroll
    for (int i = 2; i < 9; ++i) rest = R::add(rest, fs[i]);
    fs[0] = R::sub(ph, rest);
}

// Steps a4-a12 for one node (x, yc) with T arithmetic: collide_core, then the 9
// stores of f* (or, when `out` is given, the values written there for the caller).
// cS/cC/cN point at column x - 1 of rows yc - 1, yc, yc + 1 of the chi ring.
template <typename T, int MODEL, class Vel>
__device__ __forceinline__ void collide_node_row(const StepArgs<T>& a, const Vel& vel, const typename Vel::Col& vcol,
                                                 const typename Vel::Row& vrow, int x, int yc, const T* f, T ph,
                                                 T pp, const T* cS, const T* cC, const T* cN, bool store = true,
                                                 T* out = nullptr)
{
    T u, v, up, vp;
    vel.at(vcol, vrow, u, v, up, vp);
    T fs[9];
    collide_core<T, T, MODEL>(a, f, ph, pp, cS[0], cS[1], cS[2], cC[0], cC[2], cN[0], cN[1], cN[2], u, v, up, vp, fs);
    if (out) {
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i] = fs[i];
    } else if (store) {
        // 32-bit element offsets (9 nx ny < 2^31 is checked on the host); the plane
        // offsets i * plane are the same for the whole warp
        const unsigned o = (unsigned)yc * (unsigned)a.nx + (unsigned)x;
#pragma unroll
        for (int i = 0; i < 9; ++i) a.fout[o + (unsigned)i * (unsigned)a.plane] = fs[i];
    }
}

// Two adjacent nodes (xa, xa + 1) of row yc: collide_core on float2 (packed FP32x2)
// for FP32, twice on double for FP64. rS/rC/rN point at column xa - 1 of rows yc - 1,
// yc, yc + 1 (four consecutive ring entries). Writes f* of both nodes as pairs.
template <typename T, int MODEL, class Vel>
__device__ __forceinline__ void collide_pair(const StepArgs<T>& a, const Vel& vel, const typename Vel::Col& ca,
                                             const typename Vel::Col& cb, const typename Vel::Row& vra,
                                             const typename Vel::Row& vrb, const T* fa, const T* fb, T pha, T phb,
                                             T ppa, T ppb, const T* rS, const T* rC, const T* rN,
                                             typename Pair2<T>::type* out)
{
    T ua, va, upa, vpa, ub, vb, upb, vpb;
    vel.at(ca, vra, ua, va, upa, vpa);
    vel.at(cb, vrb, ub, vb, upb, vpb);
    if constexpr (sizeof(T) == 4) {
        float2 f2[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f2[i] = make_float2(fa[i], fb[i]);
        collide_core<float2, float, MODEL>(
            a, f2, make_float2(pha, phb), make_float2(ppa, ppb), make_float2(rS[0], rS[1]), make_float2(rS[1], rS[2]),
            make_float2(rS[2], rS[3]), make_float2(rC[0], rC[1]), make_float2(rC[2], rC[3]), make_float2(rN[0], rN[1]),
            make_float2(rN[1], rN[2]), make_float2(rN[2], rN[3]), make_float2(ua, ub), make_float2(va, vb),
            make_float2(upa, upb), make_float2(vpa, vpb), out);
    } else {
        T oa[9], ob[9];
        collide_core<T, T, MODEL>(a, fa, pha, ppa, rS[0], rS[1], rS[2], rC[0], rC[2], rN[0], rN[1], rN[2], ua, va, upa,
                                  vpa, oa);
        collide_core<T, T, MODEL>(a, fb, phb, ppb, rS[1], rS[2], rS[3], rC[1], rC[3], rN[1], rN[2], rN[3], ub, vb, upb,
                                  vpb, ob);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            out[i].x = oa[i];
            out[i].y = ob[i];
        }
    }
}

template <typename T, int MODEL, class Vel>
__device__ __forceinline__ void collide_node(const StepArgs<T>& a, const Vel& vel, const typename Vel::Col& vcol,
                                             int x, int yc, const T* f, T ph, T pp,
                                             const T* cS, const T* cC, const T* cN, bool store = true)
{
    collide_node_row<T, MODEL>(a, vel, vcol, vel.rowv(vcol, x, yc), x, yc, f, ph, pp, cS, cC, cN, store);
}

// Population i of node (x, y) at time t, pulled from f*(t-1) at (x - c_i, y - c_i).
// ro_m/ro_0/ro_p are the element offsets of rows r-1, r, r+1 (wrapped, times nx) and
// xm/x/xp the wrapped columns; 32-bit offsets with warp-uniform plane strides.
template <typename T>
__device__ __forceinline__ void pull_row(const T* __restrict__ fin, unsigned plane, unsigned ro_m, unsigned ro_0,
                                         unsigned ro_p, unsigned xm, unsigned x, unsigned xp, T* f)
{
    f[0] = fin[ro_0 + x];
    f[1] = fin[plane + ro_0 + xm];
    f[2] = fin[2u * plane + ro_m + x];
    f[3] = fin[3u * plane + ro_0 + xp];
    f[4] = fin[4u * plane + ro_p + x];
    f[5] = fin[5u * plane + ro_m + xm];
    f[6] = fin[6u * plane + ro_m + xp];
    f[7] = fin[7u * plane + ro_p + xp];
    f[8] = fin[8u * plane + ro_p + xm];
}

// The same with row indices (used by the variants that index rows directly).
template <typename T>
__device__ __forceinline__ void pull_row(const T* __restrict__ fin, long long plane, int nx,
                                         int r, int rm, int rp, int x, int xm, int xp, T* f)
{
    const unsigned n = (unsigned)nx;
    pull_row(fin, (unsigned)plane, (unsigned)rm * n, (unsigned)r * n, (unsigned)rp * n, (unsigned)xm, (unsigned)x,
             (unsigned)xp, f);
}

template <typename T, int MODEL, class Vel>
__global__ void __launch_bounds__(TILE_X, sizeof(T) == 4 ? 8 : 1) ace_step(const StepArgs<T> a, const Vel vel)
{
    __shared__ T chi_s[4][TILE_X + 2];
    __shared__ double red_s[TILE_X / 32];

    const int tx = threadIdx.x;
    const int lane = tx & 31;
    const int x0 = blockIdx.x * TILE_X;
    const int w = min(TILE_X, a.nx - x0);
    const bool act = tx < w;
    // threads beyond a ragged strip's width work on its last column and store nothing
    const int x = x0 + (act ? tx : w - 1);
    const int xm = x == 0 ? a.nx - 1 : x - 1;
    const int xp = x == a.nx - 1 ? 0 : x + 1;
    const int y0 = blockIdx.y * a.rows;
    const int y1 = min(y0 + a.rows, a.ny);
    const int nk = y1 - y0 + 2; // rows y0-1 .. y1 get phi and chi
    const unsigned nxu = (unsigned)a.nx, plane = (unsigned)a.plane;

    // Halo lanes of warp 0: lanes 0..8 pull population `hi` of the column left of
    // the strip, lanes 16..24 that of the column right of it.
    const bool halo = tx < 32 && (lane & 15) < 9;
    const int hi = lane & 15;
    int hcol = 0;
    if (halo) {
        const int c = lane < 16 ? (x0 == 0 ? a.nx - 1 : x0 - 1) : (x0 + w == a.nx ? 0 : x0 + w);
        hcol = wrap_idx(c - cx_of(hi), a.nx);
    }
    const int hcy = halo ? cy_of(hi) : 0;
    const unsigned hbase = (unsigned)(halo ? hi : 0) * plane + (unsigned)hcol;

    const typename Vel::Col vcol = vel.col(x);

    T ra[9], rb[9], rc[9]; // pulled row r, row r - 1, row r + 1 (prefetched)
    T hv = T(0);
    T phb = T(0);
    double msum = 0.0; // FP64 column sum of phi over this thread's rows

    // rows r - 1, r, r + 1 of the row being pulled, as element offsets
    int r = wrap_idx(y0 - 1, a.ny);
    auto load = [&](int rr, T (&dst)[9]) {
        const int rm = rr == 0 ? a.ny - 1 : rr - 1, rp = rr == a.ny - 1 ? 0 : rr + 1;
        pull_row(a.fin, plane, (unsigned)rm * nxu, (unsigned)rr * nxu, (unsigned)rp * nxu, (unsigned)xm,
                 (unsigned)x, (unsigned)xp, dst);
        if (halo) hv = a.fin[hbase + (unsigned)wrap_idx(rr - hcy, a.ny) * nxu];
    };
    load(r, ra);
#pragma unroll
    for (int i = 0; i < 9; ++i) rb[i] = rc[i] = T(0);

#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
        // row r = y0 - 1 + k: phi (Eq. 12) and chi into the ring slot k & 3
        T ph = T(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) ph += ra[i];
        if (act) chi_s[k & 3][1 + tx] = chi_of<T, MODEL>(ph, a);
        if (tx < 32) {
            const int base = lane & 16;
            T hs = T(0);
#pragma unroll
            for (int j = 0; j < 9; ++j) hs += __shfl_sync(0xffffffffu, hv, base + j);
            if (lane == 0) chi_s[k & 3][0] = chi_of<T, MODEL>(hs, a);
            if (lane == 16) chi_s[k & 3][w + 1] = chi_of<T, MODEL>(hs, a);
        }
        __syncthreads();
        r = r == a.ny - 1 ? 0 : r + 1;
        if (k + 1 < nk) load(r, rc); // row r + 1 while row r - 1 collides
        if (k >= 2) {
            // collide row yc = y0 + k - 2 with its pulled populations rb and phi phb
            const int yc = y0 + k - 2;
            const unsigned po = (unsigned)yc * nxu + (unsigned)x;
            const T pp = a.first ? T(0) : a.phi[po];
            const int j = act ? tx : w - 1; // stencil column in the ring
            collide_node<T, MODEL>(a, vel, vcol, x, yc, rb, phb, pp, chi_s[(k - 2) & 3] + j,
                                   chi_s[(k - 1) & 3] + j, chi_s[k & 3] + j, act);
            if (act) {
                a.phi[po] = phb;
                msum += (double)phb;
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) { rb[i] = ra[i]; ra[i] = rc[i]; }
        phb = ph;
    }

    // a13: block-reduced mass of phi(t) over the CTA's nodes, fixed order.
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) msum += __shfl_down_sync(0xffffffffu, msum, off);
    if (lane == 0) red_s[tx >> 5] = msum;
    __syncthreads();
    if (tx == 0) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < TILE_X / 32; ++i) s += red_s[i];
        a.mass_part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// Initial state: f_i(x, 0) = f_i^eq(phi0(x), u(x, 0)). Stored as the post-collision
// buffer f*(-1) from which the first step pulls, f*_i(x - c_i) = f_i(x, 0): each node
// pushes its 9 equilibria to x - c_i.
template <typename T, class Vel>
__global__ void ace_init(const double* __restrict__ phi0, T* __restrict__ fst, T* __restrict__ phi,
                         int nx, int ny, Vel vel)
{
    const long long plane = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < plane;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        const T ph = T(phi0[k]);
        T u, v, up, vp, feq[9];
        const typename Vel::Col c = vel.col(x);
        vel.at(c, vel.rowv(c, x, y), u, v, up, vp);
        equilibrium(ph, u, v, feq);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            fst[i * plane + (long long)wrap_idx(y - cy_of(i), ny) * nx + wrap_idx(x - cx_of(i), nx)] = feq[i];
        phi[k] = ph;
    }
}

// phi(x, t) = sum_i f*_i(x - c_i, t - 1) (Eq. 12 after streaming), as FP64.
template <typename T>
__global__ void ace_moment(const T* __restrict__ fst, double* __restrict__ out, int nx, int ny)
{
    const long long plane = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < plane;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        T s = T(0);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            s += fst[i * plane + (long long)wrap_idx(y - cy_of(i), ny) * nx + wrap_idx(x - cx_of(i), nx)];
        out[k] = (double)s;
    }
}

// Checkpoint read: f_i(x, t) = f*_i(x - c_i, t - 1) as FP64, and phi(t-1).
template <typename T>
__global__ void ace_pull_state(const T* __restrict__ fst, const T* __restrict__ phi,
                               double* __restrict__ f, double* __restrict__ php, int nx, int ny)
{
    const long long plane = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < plane;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[i * plane + k] =
                (double)fst[i * plane + (long long)wrap_idx(y - cy_of(i), ny) * nx + wrap_idx(x - cx_of(i), nx)];
        php[k] = (double)phi[k];
    }
}

// Checkpoint write: f*_i(x) = f_i(x + c_i) rounded to T, phi plane = phi(t-1).
template <typename T>
__global__ void ace_push_state(const double* __restrict__ f, const double* __restrict__ php,
                               T* __restrict__ fst, T* __restrict__ phi, int nx, int ny)
{
    const long long plane = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < plane;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            fst[i * plane + k] =
                T(f[i * plane + (long long)wrap_idx(y + cy_of(i), ny) * nx + wrap_idx(x + cx_of(i), nx)]);
        phi[k] = T(php[k]);
    }
}

// Running sum of FP32 values split into a part rounded to a multiple of 2^-16, summed
// exactly as an integer, and a remainder summed in FP32, two values at a time. It keeps
// per-value sums on the FP32 and integer pipes (GB300 runs FP64 at 1/64 of the FP32
// rate) and needs no flush inside a loop. For |v| < 64, t = v + 192 lies in [128, 256),
// where consecutive FP32 values are 2^-16 apart; hence bits(t) - bits(192) =
// (t - 192) * 2^16 exactly, t - 192 is v rounded to a multiple of 2^-16, and the
// remainder v - (t - 192), below 2^-17, is exact as well. ai adds the raw bit patterns of
// t modulo 2^32; with nv values added, ai - nv * bits(192) is the exact sum of the
// rounded parts in units of 2^-16 while that sum stays below 2^15 in magnitude (8192
// values below 2 each, say). The FP32 sum of the remainders carries the only rounding,
// about 1e-14 of a lattice's total.
__device__ __forceinline__ void split_add2i(unsigned& ai, float2& lo, float2 v)
{
    const float2 t = __fadd2_rn(v, make_float2(192.0f, 192.0f));
    const float2 h = __fadd2_rn(t, make_float2(-192.0f, -192.0f));
    ai += __float_as_uint(t.x) + __float_as_uint(t.y);
    lo = __fadd2_rn(lo, __fadd2_rn(v, make_float2(-h.x, -h.y)));
}

__device__ __forceinline__ double split_total_i(unsigned ai, float2 lo, unsigned nv)
{
    const int m = (int)(ai - nv * 0x43400000u); // 0x43400000 = bits(192.0f)
    return (double)m * 0x1p-16 + ((double)lo.x + (double)lo.y);
}

} // namespace lbmace
