// Persistent trajectory kernel for relic overdensity profiles (sm_103a).
//
// One thread integrates TPT trajectories (one per (radius, |P0|, mu) triple,
// Sec. II.C) backward from z0 = 0 to z_end with classical RK4 in u = ln a
// (Eq. eoms), the force being the closed-form gradient of the compensated,
// growing NFW halo (App. A).  The state (x, y, vx, vy) stays in registers for
// the whole integration; the per-step coefficients (background, growth,
// coupling at the three RK stage times, built in FP64 on the host) are read as
// warp-uniform vector loads, either staged once per request into shared memory
// or (GTAB) in place through the L1 cache.  At the end the Liouville map
// f0 = f_init(P_i) (Sec. II.C) and the weight of the trajectory in
// Eq. localdensity are applied, once per relic mass read from the trajectory
// (Sec. III), and each tile's sum is formed by a warp-shuffle + shared-memory tree.  Tile sums land in a per-request
// array; the CTA that completes the last tile of a radius adds them in tile
// order (so every result is bitwise independent of scheduling and of what
// else shares the launch) and writes n/nbar.
//
// Work distribution: CTAs of a persistent grid pull tile indices from one
// atomic counter; a tile is `tile` consecutive trajectories of one radius of
// one request, so uneven batches of requests share one launch.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <type_traits>

#include "nuprof_internal.h"

namespace nuprof {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Force evaluation: m = Mhat(r, z) / r^3, so that gradPhi / F = m * (x, y).
//   Mhat = I(r/(r_s (1+z))) / I(c) - (r/R)^3   for r < r200 (1+z)
//        = 1 - (r/R)^3                         for r < R
//        = 0                                   otherwise          (App. A)
// which gives m = sel / r^3 - 1/R^3 with sel = I/I(c) inside the NFW edge and
// 1 in the shell, and m = 0 beyond R.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float rsqrt_approx(float v)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ float lg2_approx(float v)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ float rcp_approx(float v)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// I(y) = ln(1+y) - y/(1+y) (Eq. nfw) in FP32.  For small y the two terms
// cancel, so inside the NFW part I = y^2 g(y) with g = I/y^2 approximated by a
// rational function N(y)/D(y) (nfw_rational_fit.py).  Two fits exist, and a
// request uses one of them for all of its evaluations:
//   wide:   degrees 4 and 5 on 0 <= y <= 16 (6e-8 relative, 3e-7 after float32
//           rounding; every coefficient positive), for halos with c > 8;
//   narrow: degrees 4 and 4 on 0 <= y <= 8 (6e-8, 3e-7), one fused
//           multiply-add cheaper, for halos with c <= 8, whose NFW part never
//           reaches y = 8.
// Above y = 16 (halos with c > 16) the two terms differ by more than a factor
// 1.5 and are subtracted directly, with the hardware base-2 logarithm and
// reciprocal (rcp(-u) = -1/u exactly).
__device__ __forceinline__ float nfw_N16(float y)
{
    float p = 3.952767202e-06f;
    p = fmaf(p, y, 2.387282439e-03f);
    p = fmaf(p, y, 6.631398201e-02f);
    p = fmaf(p, y, 3.795046508e-01f);
    p = fmaf(p, y, 5.000000596e-01f);
    return p;
}

__device__ __forceinline__ float nfw_D16(float y)
{
    float p = 5.989100318e-04f;
    p = fmaf(p, y, 3.099172190e-02f);
    p = fmaf(p, y, 3.629413843e-01f);
    p = fmaf(p, y, 1.422382593e+00f);
    p = fmaf(p, y, 2.092346668e+00f);
    p = fmaf(p, y, 1.0f);
    return p;
}

__device__ __forceinline__ float nfw_N8(float y)
{
    float p = -4.539978363e-06f;
    p = fmaf(p, y, 4.568357544e-04f);
    p = fmaf(p, y, 4.554858804e-02f);
    p = fmaf(p, y, 3.421576917e-01f);
    p = fmaf(p, y, 5.000000000e-01f);
    return p;
}

__device__ __forceinline__ float nfw_D8(float y)
{
    float p = 1.647129469e-02f;
    p = fmaf(p, y, 2.829689085e-01f);
    p = fmaf(p, y, 1.281258702e+00f);
    p = fmaf(p, y, 2.017652512e+00f);
    p = fmaf(p, y, 1.0f);
    return p;
}

// Largest concentration served by the narrow fit.
constexpr float kNarrowMaxC = 8.0f;

// y = r^2 rs is passed together with u = 1 + y formed as one fused
// multiply-add from r^2 and rs (every FP32 product that feeds a sum is written
// as an explicit fused multiply-add, here and in the packed path, so that no
// compiler contraction decides the rounding).
__device__ __forceinline__ float nfw_I_log(float y, float u)
{
    return fmaf(lg2_approx(u), 0.693147180559945309f, y * rcp_approx(-u));
}

// Same in FP64, accurate to a few ulp for every y.  With t = y/(1+y),
// I = -ln(1-t) - t = t^2 sum_{k>=0} t^k/(k+2), a series of positive terms; for
// t < 1/2 (y < 1) it is summed by Horner through k = 50 (truncation below
// 1e-16 relative), above that the two terms no longer cancel badly.
__device__ __forceinline__ double nfw_I(double y)
{
    const double t = y / (1.0 + y);
    if (t < 0.5) {
        double p = 1.0 / 52.0;
#pragma unroll   // fully: the coefficients 1/(k+2) become compile-time constants
        for (int k = 49; k >= 0; --k) p = fma(p, t, 1.0 / (double)(k + 2));
        return (t * t) * p;
    }
    return log1p(y) - t;
}

// Steps between two tests of the early exit (a power of two).
constexpr int kExitEvery = 4;

// Added to r^2 in FP32 so that a trajectory through r = 0 exactly gets a
// finite reciprocal square root.
constexpr float kR2Guard = 1e-20f;

// A trajectory is finished when its velocity can no longer change: it lies
// beyond R, where the gradient is exactly zero (mass compensation, App. A),
// and the straight line it follows from there along the integration direction
// (-v: the backward step moves it along -v) does not come back within R
// before z_end.  That holds when it recedes (x . v <= 0); when the line's
// closest approach to the centre, b^2 = r^2 - (x . v)^2 / v^2, stays beyond R
// (App. B's first criterion, for rays that miss the halo); or when the
// trajectory is too slow to cover the distance r - R before z_end (App. B's
// second criterion, v I_io < r - R), with irem the remaining force-free
// distance per unit speed of the discrete map.  All three are exact here
// because nothing acts outside R.  The factor kMiss keeps the tests safe
// against the rounding of the stepped positions (relative deviations below
// 1e-4 from the straight line).
template <typename T>
__device__ __forceinline__ bool escapes(T r2, T dot, T v2, T R2, T R, T irem)
{
    const T kMiss = T(1.001);
    if (!(r2 >= R2)) return false;
    if (dot <= T(0) || (r2 - kMiss * R2) * v2 >= dot * dot) return true;
    const T reach = R + sqrt(v2) * irem;          // farthest start that still reaches R
    return r2 >= kMiss * (reach * reach);
}

// c: the NFW edge r = r200 (1+z) in y = r S; narrow: c <= 8, the request uses
// the narrow rational fit.
struct HaloF32 { float invIc, invR3, R2, R, c; bool narrow; };
struct HaloF64 { double invIc, invR3, R2, R; };

// Branch tallies of force evaluations, kept only by the counting variant of the
// kernel (used once, untimed, to turn the data-dependent work into an exact
// algorithmic flop count): beyond R, shell, NFW part on the first branch of
// I(y) (FP32: the rational function; FP64: the series), NFW part on the
// logarithm branch, and the trajectory-steps of
// unfinished trajectories.  Steps that a finished trajectory runs only because
// its warp is still busy are not counted (they are not needed work); the sixth
// count is every lane-step the warps ran, needed or not (padding lanes too).
struct NoTally {
    __device__ __forceinline__ void add(int) {}
    __device__ __forceinline__ void set_live(bool) {}
    __device__ __forceinline__ void ran(unsigned) {}
};
struct Tally {
    unsigned n[6] = {0u, 0u, 0u, 0u, 0u, 0u};   // 4 branches, live steps, lane-steps run
    bool live = true;                           // only unfinished trajectories count
    __device__ __forceinline__ void add(int k) { n[k] += live ? 1u : 0u; }
    __device__ __forceinline__ void set_live(bool v)
    {
        live = v;
        n[4] += v ? 1u : 0u;
    }
    __device__ __forceinline__ void ran(unsigned k) { n[5] += k; }
};

// The compensated halo's gradient vanishes beyond R, and the NFW term only
// enters inside r200 (1+z): both tests are branches, so a warp whose lanes
// are all beyond R (or all in the shell) skips that work.  The result is the
// same value the full expression gives (0, resp. sel = 1).
//
// FP32 arithmetic of one evaluation, fixed per branch so that every code path
// (scalar, packed, any warp composition) gives a lane the same bits.  With
// rs = S/r and the table's T = S/I(c) (so y = r S = r^2 rs):
//   beyond R:              m = 0
//   NFW, y < Yq:           m = (N(y) (rs T)) rcp(D(y)) - 1/R^3
//                          (I rinv^3 / I(c) = y^2 g rinv^3 / I(c) = g S^2 rinv / I(c))
//   NFW, Yq <= y < c:      m = (I(y)/I(c)) rinv^3 - 1/R^3
//   shell:                 m = rinv^2 rinv - 1/R^3 (one rounding)
// Yq, the stage's bound of the rational branch (the FP32 table's C_Q slots),
// is min(c, 16, (1 - 1e-3) R S): y < Yq implies r < R with a margin far above
// the rounding of y, so that one compare classifies a lane.  The NFW part is
// y < c (the edge r = r200 (1+z) is y = c exactly), tested on y itself; the
// FP64 path tests r^2 against the table's squared edge.  The two tests differ
// only in the rounding at the edge, where the mass is continuous.
// The r -> 0 guard is folded into r^2 itself: r^2 = x^2 + (y^2 + 1e-20) with
// two fused multiply-adds, which changes the bits of r^2 only below ~2e-13 kpc^2.
__device__ __forceinline__ float guarded_r2(float x, float y)
{
    return fmaf(x, x, fmaf(y, y, kR2Guard));
}

template <class Ctr = NoTally>
__device__ __forceinline__ float accel_m(float x, float y, float S, float Yq, float T,
                                         const HaloF32& hc, Ctr& ctr)
{
    const float r2 = guarded_r2(x, y);
    float m = 0.0f;
    if (r2 < hc.R2) {
        const float rinv = rsqrt_approx(r2);
        const float rs = rinv * S;
        const float ys = r2 * rs;
        if (ys < Yq) {
            ctr.add(2);
            const float n = hc.narrow ? nfw_N8(ys) : nfw_N16(ys);
            const float d = hc.narrow ? nfw_D8(ys) : nfw_D16(ys);
            m = fmaf(n * (rs * T), rcp_approx(d), -hc.invR3);
        } else {
            const float rinv2 = rinv * rinv;
            if (ys < hc.c) {
                ctr.add(3);
                const float sel = nfw_I_log(ys, fmaf(r2, rs, 1.0f)) * hc.invIc;
                m = fmaf(sel, rinv2 * rinv, -hc.invR3);
            } else {
                ctr.add(1);
                m = fmaf(rinv2, rinv, -hc.invR3);
            }
        }
    } else {
        ctr.add(0);
    }
    return m;
}

template <class Ctr = NoTally>
__device__ __forceinline__ double accel_m(double x, double y, double S, double Q, double,
                                          const HaloF64& hc, Ctr& ctr)
{
    const double r2 = fma(x, x, y * y);
    double m = 0.0;
    if (r2 < hc.R2) {
        const double rinv = rsqrt(fmax(r2, 1e-200));
        const double rinv3 = rinv * rinv * rinv;
        double sel = 1.0;
        if (r2 < Q) {
            const double ys = (r2 * rinv) * S;
            ctr.add(ys < 1.0 ? 2 : 3);
            sel = nfw_I(ys) * hc.invIc;
        } else {
            ctr.add(1);
        }
        m = fma(sel, rinv3, -hc.invR3);
    } else {
        ctr.add(0);
    }
    return m;
}

template <typename T> struct PrecTraits;
template <> struct PrecTraits<float> {
    using Halo = HaloF32;
    static __device__ __forceinline__ Halo halo(const DevProblem& P)
    {
        const float c = (float)P.c_nfw;
        return {(float)P.invIc, (float)P.invR3, (float)P.R2, (float)sqrt(P.R2), c, c <= kNarrowMaxC};
    }
};
template <> struct PrecTraits<double> {
    using Halo = HaloF64;
    static __device__ __forceinline__ Halo halo(const DevProblem& P)
    {
        return {P.invIc, P.invR3, P.R2, sqrt(P.R2)};
    }
};

// Initial distribution f(q) (Sec. II.C, Sec. IV.B), evaluated in FP64 in both
// precision modes (it runs once per trajectory and mass, in the epilogue).
// The tabulated kind is linear in ln q between log-spaced nodes (stored in
// FP64), the first value below the first node and 0 above the last.
__device__ __forceinline__ double relic_f_table(const DevProblem& P, double q)
{
    const double* t = reinterpret_cast<const double*>(P.ftab);
    const int n = P.n_ftab;
    if (!(q > P.ftab_q0)) return t[0];
    if (q > P.ftab_q1) return 0.0;
    const double u = log(q / P.ftab_q0) * P.ftab_scale;
    if (u >= (double)(n - 1)) return t[n - 1];
    const int k = (int)u;
    const double w = u - (double)k;
    return t[k] + w * (t[k + 1] - t[k]);
}

__device__ __forceinline__ double relic_f_dev(const DevProblem& P, double q)
{
    if (P.f_kind == NU_F_TABLE) return relic_f_table(P, q);
    if (P.f_kind == NU_F_FREEZEIN) {
        const double qq = fmax(q, 1e-300);
        return exp(-qq) / sqrt(qq);
    }
    return 1.0 / (1.0 + exp(q - P.f_p0));
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// One classical RK4 step of size -h for one trajectory (Eq. eoms in ln a).
// c points at the step's C_COUNT coefficients (see CoefSlot).  Every product-sum
// is an explicit fused multiply-add, so the packed two-trajectory variant
// below performs exactly the same roundings.
template <typename T, class Ctr>
__device__ __forceinline__ void rk4_step(T& x, T& y, T& vx, T& vy, const T* c,
                                         const typename PrecTraits<T>::Halo& hc, Ctr& ctr)
{
    const T m1 = accel_m(x, y, c[C_S0], c[C_Q0], c[C_T0], hc, ctr);
    const T p1 = c[C_B1] * m1;
    const T X2 = fmaT(c[C_MA1], vx, x), Y2 = fmaT(c[C_MA1], vy, y);
    const T VX2 = fmaT(p1, x, vx), VY2 = fmaT(p1, y, vy);

    const T m2 = accel_m(X2, Y2, c[C_S1], c[C_Q1], c[C_T1], hc, ctr);
    const T p2 = c[C_B2] * m2;
    const T X3 = fmaT(c[C_MA2], VX2, x), Y3 = fmaT(c[C_MA2], VY2, y);
    const T VX3 = fmaT(p2, X2, vx), VY3 = fmaT(p2, Y2, vy);

    const T m3 = accel_m(X3, Y3, c[C_S1], c[C_Q1], c[C_T1], hc, ctr);
    const T p3 = c[C_B3] * m3;
    const T X4 = fmaT(c[C_MA3], VX3, x), Y4 = fmaT(c[C_MA3], VY3, y);
    const T VX4 = fmaT(p3, X3, vx), VY4 = fmaT(p3, Y3, vy);

    const T m4 = accel_m(X4, Y4, c[C_S2], c[C_Q2], c[C_T2], hc, ctr);
    const T p4 = c[C_B4] * m4;

    // x' = x - (h/6) (A_a v + 2 A_m V2 + 2 A_m V3 + A_b V4)
    const T nx = fmaT(c[C_W2], VX4, fmaT(c[C_W1], VX2 + VX3, fmaT(c[C_W0], vx, x)));
    const T ny = fmaT(c[C_W2], VY4, fmaT(c[C_W1], VY2 + VY3, fmaT(c[C_W0], vy, y)));
    // v' = v + (h/6) (BF_a m1 x + 2 BF_m m2 X2 + 2 BF_m m3 X3 + BF_b m4 X4)
    const T p2x2 = p2 * T(2);   // exact doubling
    const T third = T(1) / T(3);
    const T tx = fmaT(p3, X3, fmaT(p2x2, X2, p1 * x));
    const T ty = fmaT(p3, Y3, fmaT(p2x2, Y2, p1 * y));
    const T nvx = fmaT(p4, X4, fmaT(tx, third, vx));
    const T nvy = fmaT(p4, Y4, fmaT(ty, third, vy));
    x = nx;
    y = ny;
    vx = nvx;
    vy = nvy;
}

// ---------------------------------------------------------------------------
// Packed FP32x2 path: two trajectories per thread held as register pairs, every
// arithmetic operation issued as one f32x2 instruction (fma/mul/add.rn.f32x2).
// Each component sees exactly the operations of the scalar path above, in the
// same order, so the results are bitwise those of the two-trajectory scalar
// kernel; only selects, comparisons and the special functions stay scalar.
// The coefficients come from a table with every value stored twice ({c, c}),
// so a 16-byte shared load yields two ready operand pairs.
// ---------------------------------------------------------------------------
struct f2 {
    unsigned long long v;
};

__device__ __forceinline__ f2 pk(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float f2lo(f2 a)
{
    float l, h;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(a.v));
    return l;
}
__device__ __forceinline__ float f2hi(f2 a)
{
    float l, h;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(a.v));
    return h;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 dup(float a) { return pk(a, a); }

struct HaloX2 {
    f2 invIc, neg_invR3;
    float R2, c;
};

// N(y) and D(y) of the rational g for both lanes (see nfw_N16, nfw_D16 and
// nfw_N8, nfw_D8); NARROW selects the fit.
template <bool NARROW>
__device__ __forceinline__ f2 nfw_N_x2(f2 y)
{
    f2 p;
    if constexpr (NARROW) {
        p = dup(-4.539978363e-06f);
        p = fma2(p, y, dup(4.568357544e-04f));
        p = fma2(p, y, dup(4.554858804e-02f));
        p = fma2(p, y, dup(3.421576917e-01f));
        p = fma2(p, y, dup(5.000000000e-01f));
    } else {
        p = dup(3.952767202e-06f);
        p = fma2(p, y, dup(2.387282439e-03f));
        p = fma2(p, y, dup(6.631398201e-02f));
        p = fma2(p, y, dup(3.795046508e-01f));
        p = fma2(p, y, dup(5.000000596e-01f));
    }
    return p;
}
template <bool NARROW>
__device__ __forceinline__ f2 nfw_D_x2(f2 y)
{
    f2 p;
    if constexpr (NARROW) {
        p = dup(1.647129469e-02f);
        p = fma2(p, y, dup(2.829689085e-01f));
        p = fma2(p, y, dup(1.281258702e+00f));
        p = fma2(p, y, dup(2.017652512e+00f));
        p = fma2(p, y, dup(1.0f));
    } else {
        p = dup(5.989100318e-04f);
        p = fma2(p, y, dup(3.099172190e-02f));
        p = fma2(p, y, dup(3.629413843e-01f));
        p = fma2(p, y, dup(1.422382593e+00f));
        p = fma2(p, y, dup(2.092346668e+00f));
        p = fma2(p, y, dup(1.0f));
    }
    return p;
}

// I(y) on the logarithm branch for both lanes (see nfw_I_log).
__device__ __forceinline__ f2 nfw_I_log_x2(f2 y, f2 u)
{
    const float ua = f2lo(u), ub = f2hi(u);
    const f2 lg = pk(lg2_approx(ua), lg2_approx(ub));
    const f2 rn = pk(rcp_approx(-ua), rcp_approx(-ub));
    return fma2(lg, dup(0.693147180559945309f), mul2(y, rn));
}

// Geometry of one force evaluation for both lanes of a register pair:
// guarded r^2, 1/r, rs = S/r and y = r^2 rs, and per lane whether it is on
// the rational branch of the NFW part (y < Yq, which implies r < R).
struct Geo2 {
    f2 r2, rinv, rs, ys;
    bool q0, q1;
};

__device__ __forceinline__ Geo2 geometry_x2(f2 x, f2 y, f2 S, f2 Yq)
{
    Geo2 g;
    g.r2 = fma2(x, x, fma2(y, y, dup(kR2Guard)));
    g.rinv = pk(rsqrt_approx(f2lo(g.r2)), rsqrt_approx(f2hi(g.r2)));
    g.rs = mul2(g.rinv, S);
    g.ys = mul2(g.r2, g.rs);
    g.q0 = f2lo(g.ys) < f2lo(Yq);
    g.q1 = f2hi(g.ys) < f2hi(Yq);
    return g;
}

// Per-branch formulas of accel_m for both lanes (FP32, the same operations).
template <bool NARROW>
__device__ __forceinline__ f2 m_rational_x2(const Geo2& g, f2 T, const HaloX2& hc)
{
    const f2 nr = mul2(nfw_N_x2<NARROW>(g.ys), mul2(g.rs, T));
    const f2 d = nfw_D_x2<NARROW>(g.ys);
    return fma2(nr, pk(rcp_approx(f2lo(d)), rcp_approx(f2hi(d))), hc.neg_invR3);
}
__device__ __forceinline__ f2 m_log_x2(const Geo2& g, f2 rinv2, const HaloX2& hc)
{
    const f2 sel = mul2(nfw_I_log_x2(g.ys, fma2(g.r2, g.rs, dup(1.0f))), hc.invIc);
    return fma2(sel, mul2(rinv2, g.rinv), hc.neg_invR3);
}
__device__ __forceinline__ f2 m_shell_x2(const Geo2& g, f2 rinv2, const HaloX2& hc)
{
    return fma2(rinv2, g.rinv, hc.neg_invR3);
}
// shell or beyond R (0), for lanes outside the NFW edge
__device__ __forceinline__ f2 m_out_x2(const Geo2& g, const HaloX2& hc)
{
    const f2 ms = m_shell_x2(g, mul2(g.rinv, g.rinv), hc);
    return pk(f2lo(g.r2) < hc.R2 ? f2lo(ms) : 0.0f, f2hi(g.r2) < hc.R2 ? f2hi(ms) : 0.0f);
}
// any mix of branches: each formula that some lane of the warp needs,
// evaluated for both lanes and selected per lane
template <bool NARROW>
__device__ __forceinline__ f2 m_mixed_x2(const Geo2& g, f2 T, const HaloX2& hc, bool need_log)
{
    const f2 rinv2 = mul2(g.rinv, g.rinv);
    const f2 mq = m_rational_x2<NARROW>(g, T, hc);
    const f2 ml = need_log ? m_log_x2(g, rinv2, hc) : dup(0.0f);
    const f2 ms = m_shell_x2(g, rinv2, hc);
    const bool n0 = f2lo(g.ys) < hc.c, n1 = f2hi(g.ys) < hc.c;
    const bool in0 = f2lo(g.r2) < hc.R2, in1 = f2hi(g.r2) < hc.R2;
    return pk(!in0 ? 0.0f : g.q0 ? f2lo(mq) : n0 ? f2lo(ml) : f2lo(ms),
              !in1 ? 0.0f : g.q1 ? f2hi(mq) : n1 ? f2hi(ml) : f2hi(ms));
}

// m = Mhat/r^3 at two independent points (a, b) of both lanes: lane by lane
// the values of accel_m (FP32).  Within one RK4 step the first two stages'
// positions depend only on the step's start state, and so do the last two
// given the first two, so their force evaluations are independent and run
// interleaved.  One warp vote covers all four lane-evaluations (the two
// points of a pair almost always share their branch): every one on the
// rational branch of the NFW part (the common case: it covers the whole NFW
// part of halos with c <= 16), every one outside the NFW edge (shell or
// beyond R), or any mix (each formula that a lane needs evaluated for all and
// selected per lane).  All lanes of the warp execute this function together
// (the integration loop is warp-uniform).
template <bool NARROW>
__device__ __forceinline__ void accel_m_pair_x2(f2 xa, f2 ya, f2 Sa, f2 Ya, f2 Ta,
                                                f2 xb, f2 yb, f2 Sb, f2 Yb, f2 Tb,
                                                const HaloX2& hc, f2& ma, f2& mb)
{
    const Geo2 ga = geometry_x2(xa, ya, Sa, Ya);
    const Geo2 gb = geometry_x2(xb, yb, Sb, Yb);
    const unsigned full = 0xffffffffu;
    if (__all_sync(full, ga.q0 && ga.q1 && gb.q0 && gb.q1)) {
        ma = m_rational_x2<NARROW>(ga, Ta, hc);
        mb = m_rational_x2<NARROW>(gb, Tb, hc);
        return;
    }
    // lanes inside R and inside the NFW edge
    const bool na0 = f2lo(ga.r2) < hc.R2 && f2lo(ga.ys) < hc.c;
    const bool na1 = f2hi(ga.r2) < hc.R2 && f2hi(ga.ys) < hc.c;
    const bool nb0 = f2lo(gb.r2) < hc.R2 && f2lo(gb.ys) < hc.c;
    const bool nb1 = f2hi(gb.r2) < hc.R2 && f2hi(gb.ys) < hc.c;
    if (__all_sync(full, !(na0 || na1 || nb0 || nb1))) {
        ma = m_out_x2(ga, hc);
        mb = m_out_x2(gb, hc);
        return;
    }
    // a lane of the NFW part above the rational branch (only halos with c > 16)
    const bool la = (na0 && !ga.q0) || (na1 && !ga.q1);
    const bool lb = (nb0 && !gb.q0) || (nb1 && !gb.q1);
    const bool need_log = __any_sync(full, la || lb);
    ma = m_mixed_x2<NARROW>(ga, Ta, hc, need_log);
    mb = m_mixed_x2<NARROW>(gb, Tb, hc, need_log);
}

// One 16-byte entry of the duplicated table (two slots, each a {c, c} pair).
template <bool GTAB>
__device__ __forceinline__ ulonglong2 coef_pair(const uint4* src4, int q)
{
    const uint4 w = GTAB ? __ldg(&src4[q]) : src4[q];
    return make_ulonglong2(((unsigned long long)w.y << 32) | w.x,
                           ((unsigned long long)w.w << 32) | w.z);
}

// rk4_step for two trajectories at once.  src4 points at the step's 10 x 16
// bytes of the duplicated table (slot j -> floats 2j, 2j+1); each entry is
// loaded where it is first needed, which keeps the table out of registers.
// The four force evaluations run as two independent pairs (stages 1 and 2,
// then 3 and 4); every value is formed by the same operations as in rk4_step.
template <bool GTAB, bool NARROW>
__device__ __forceinline__ void rk4_step_x2(f2& x, f2& y, f2& vx, f2& vy, const uint4* src4,
                                            const HaloX2& hc)
{
    const ulonglong2 q0 = coef_pair<GTAB>(src4, 0);
    const f2 MA1{q0.x}, MA2{q0.y};
    const f2 X2 = fma2(MA1, vx, x), Y2 = fma2(MA1, vy, y);
    const ulonglong2 q5 = coef_pair<GTAB>(src4, 5), q6 = coef_pair<GTAB>(src4, 6);
    const ulonglong2 q7 = coef_pair<GTAB>(src4, 7), q8 = coef_pair<GTAB>(src4, 8);
    const f2 S0{q5.x}, S1{q5.y}, Yq0{q6.y}, Yq1{q7.x}, T0{q8.x}, T1{q8.y};
    f2 m1, m2;
    accel_m_pair_x2<NARROW>(x, y, S0, Yq0, T0, X2, Y2, S1, Yq1, T1, hc, m1, m2);
    const ulonglong2 q1 = coef_pair<GTAB>(src4, 1), q2 = coef_pair<GTAB>(src4, 2);
    const f2 MA3{q1.x}, B1{q1.y}, B2{q2.x};
    const f2 p1 = mul2(B1, m1);
    const f2 VX2 = fma2(p1, x, vx), VY2 = fma2(p1, y, vy);
    const f2 p2 = mul2(B2, m2);
    const f2 VX3 = fma2(p2, X2, vx), VY3 = fma2(p2, Y2, vy);
    const f2 X3 = fma2(MA2, VX2, x), Y3 = fma2(MA2, VY2, y);
    const f2 X4 = fma2(MA3, VX3, x), Y4 = fma2(MA3, VY3, y);

    const ulonglong2 q9 = coef_pair<GTAB>(src4, 9);
    const f2 S2{q6.x}, Yq2{q7.y}, T2{q9.x};
    f2 m3, m4;
    accel_m_pair_x2<NARROW>(X3, Y3, S1, Yq1, T1, X4, Y4, S2, Yq2, T2, hc, m3, m4);
    const ulonglong2 q3 = coef_pair<GTAB>(src4, 3), q4 = coef_pair<GTAB>(src4, 4);
    const f2 B3{q2.y}, B4{q3.x}, W0{q3.y}, W1{q4.x}, W2{q4.y};
    const f2 p3 = mul2(B3, m3);
    const f2 VX4 = fma2(p3, X3, vx), VY4 = fma2(p3, Y3, vy);
    const f2 p4 = mul2(B4, m4);

    const f2 nx = fma2(W2, VX4, fma2(W1, add2(VX2, VX3), fma2(W0, vx, x)));
    const f2 ny = fma2(W2, VY4, fma2(W1, add2(VY2, VY3), fma2(W0, vy, y)));
    const f2 p2x2 = mul2(p2, dup(2.0f));   // exact doubling
    const f2 third = dup(1.0f / 3.0f);
    const f2 tx = fma2(p3, X3, fma2(p2x2, X2, mul2(p1, x)));
    const f2 ty = fma2(p3, Y3, fma2(p2x2, Y2, mul2(p1, y)));
    vx = fma2(p4, X4, fma2(tx, third, vx));
    vy = fma2(p4, Y4, fma2(ty, third, vy));
    x = nx;
    y = ny;
}

// The packed step loop of one tile for steps [s_begin, s_end): early-exit test
// every kExitEvery steps, then an RK4 step of both lanes.  NARROW is fixed per
// request (the rational fit its force uses), so the tile chooses the loop once.
template <bool GTAB, bool NARROW>
__device__ __forceinline__ void packed_steps(f2& X, f2& Y, f2& VX, f2& VY, const float* tab,
                                             int s_begin, int s_end, bool act0, bool act1,
                                             bool done, const HaloX2& h2, float R)
{
    for (int n = s_begin; n < s_end; ++n) {
        if (((n - s_begin) & (kExitEvery - 1)) == 0) {
            const f2 r2 = fma2(X, X, mul2(Y, Y));
            const f2 dot = fma2(X, VX, mul2(Y, VY));
            const f2 v2 = fma2(VX, VX, mul2(VY, VY));
            const float irem = tab[(size_t)n * 2 * C_COUNT + 2 * C_IREM];
            const bool fin0 = !act0 || escapes(f2lo(r2), f2lo(dot), f2lo(v2), h2.R2, R, irem);
            const bool fin1 = !act1 || escapes(f2hi(r2), f2hi(dot), f2hi(v2), h2.R2, R, irem);
            done |= fin0 && fin1;
            if (__all_sync(0xffffffffu, done)) break;
        }
        rk4_step_x2<GTAB, NARROW>(X, Y, VX, VY,
                                  reinterpret_cast<const uint4*>(tab + (size_t)n * 2 * C_COUNT), h2);
    }
}

// ---------------------------------------------------------------------------
// Work queue of a resident launch (see QueueCtl).  Thread 0 of a CTA has
// claimed tile g; it returns g once the host has published it, or -1 when the
// launch ends: the queue was closed (or has expired) with g beyond its last
// published tile, or this CTA's wait ran past the limit and it expired the
// queue itself (by compare-and-swap on the same word the host publishes
// through, so the tile it gave up on can never be published afterwards).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long load_acquire_sys(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.sys.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned load_acquire_sys(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.sys.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ int queue_wait(QueueCtl* q, unsigned g, int* n_probs)
{
    const unsigned long long t0 = globaltimer_ns();
    bool asked = false;
    for (;;) {
        const unsigned long long w = load_acquire_sys(&q->word);
        const unsigned published = (unsigned)w;
        if (g < published) {
            *n_probs = (int)load_acquire_sys(&q->n_probs);
            return (int)g;
        }
        if ((unsigned)(w >> 32) != kQueueOpen) return -1;
        if (!asked) {
            atomicExch_system(&q->want_work, 1u);
            asked = true;
        }
        if (globaltimer_ns() - t0 > q->wait_limit_ns) {
            const unsigned long long expired = ((unsigned long long)kQueueExpired << 32) | published;
            if (atomicCAS_system(&q->word, w, expired) == w) return -1;
            continue;                          // the host changed the word: look again
        }
        __nanosleep(2000);
    }
}

// The packed path asks for two 512-thread CTAs per SM (at most 64 registers):
// it issues few instructions per trajectory, so it needs many warps to hide
// the latency of its dependent chains.
template <typename T, int TPT, bool COUNT, bool PACKED = false, bool GTAB = false>
__global__ void __launch_bounds__(512, PACKED ? 2 : 1)
traj_kernel(const DevProblem* __restrict__ probs, const int* __restrict__ tile_prefix,
            int n_probs, int n_tiles, unsigned* __restrict__ tile_counter,
            unsigned long long* __restrict__ tallies, QueueCtl* queue)
{
    using Ctr = typename std::conditional<COUNT, Tally, NoTally>::type;
    Ctr ctr;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s_coef = reinterpret_cast<T*>(smem_raw);
    __shared__ int s_tile;
    __shared__ int s_req;
    __shared__ int s_last;
    // the descriptor of the tile's request, read through L2 (requests published
    // into a resident launch are never served from a stale L1 line)
    __shared__ __align__(16) DevProblem s_prob;
    __shared__ double s_red[32][2];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    int cur = -1;

    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned claimed = atomicAdd(tile_counter, 1u);
            int np = n_probs;
            int t = queue ? queue_wait(queue, claimed, &np)
                          : (claimed < (unsigned)n_tiles ? (int)claimed : -1);
            // request that owns global tile t: last p with tile_prefix[p] <= t
            if (t >= 0) {
                int lo = 0, hi = np - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (__ldcg(&tile_prefix[mid]) <= t) lo = mid; else hi = mid - 1;
                }
                s_req = lo;
            }
            s_tile = t;
        }
        __syncthreads();
        const int g = s_tile;
        if (g < 0) break;
        const int lo = s_req;
        {
            constexpr int kWords = (int)(sizeof(DevProblem) / sizeof(unsigned));
            static_assert(sizeof(DevProblem) % sizeof(unsigned) == 0, "descriptor words");
            const unsigned* src = reinterpret_cast<const unsigned*>(probs + lo);
            unsigned* dst = reinterpret_cast<unsigned*>(&s_prob);
            for (int i = threadIdx.x; i < kWords; i += blockDim.x) dst[i] = __ldcg(&src[i]);
        }
        __syncthreads();
        const DevProblem& P = s_prob;
        const int n_steps = P.n_steps;

        // coefficient table: staged once per request into shared memory, or
        // (GTAB) read in place through the L1 cache with warp-uniform loads
        const T* tab = GTAB ? reinterpret_cast<const T*>(PACKED ? P.coef2 : P.coef) : s_coef;
        if (!GTAB && lo != cur) {   // stage this request's table (uniform branch)
            const float4* src = reinterpret_cast<const float4*>(PACKED ? P.coef2 : P.coef);
            float4* dst = reinterpret_cast<float4*>(s_coef);
            const int n16 = (int)((size_t)n_steps * C_COUNT * sizeof(T) * (PACKED ? 2 : 1) / 16);
            for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldg(&src[i]);
            __syncthreads();
            cur = lo;
        }

        const int tps = P.tiles_per_seg;
        const int lt = g - __ldcg(&tile_prefix[lo]);
        const int seg = lt / tps;
        const int tis = lt - seg * tps;
        const int n_mu = P.n_mu;
        const int n_seg = P.n_q * n_mu;
        const typename PrecTraits<T>::Halo hc = PrecTraits<T>::halo(P);
        const T x0 = reinterpret_cast<const T*>(P.x0)[seg];

        // steps of this launch: all of them, or one chunk of a served request
        const int s_begin = P.step_begin;
        const int s_end = P.step_end > 0 ? P.step_end : n_steps;
        T* state = reinterpret_cast<T*>(P.state);

        T x[TPT], y[TPT], vx[TPT], vy[TPT];
        bool act[TPT];
        bool done = true;            // every trajectory of this lane is finished
#pragma unroll
        for (int i = 0; i < TPT; ++i) {
            const int t = tis * P.tile + i * blockDim.x + threadIdx.x;
            act[i] = t < n_seg;
            done &= !act[i];
            const int tt = act[i] ? t : 0;
            if (state && s_begin > 0) {          // resume a served request
                const T* st = state + ((size_t)seg * n_seg + tt) * 4;
                x[i] = st[0];
                y[i] = st[1];
                vx[i] = st[2];
                vy[i] = st[3];
            } else {                             // Sec. II.C initial conditions
                const int j = tt / n_mu, k = tt - (tt / n_mu) * n_mu;
                const T v0 = reinterpret_cast<const T*>(P.v0)[j];
                x[i] = x0;
                y[i] = T(0);
                vx[i] = v0 * reinterpret_cast<const T*>(P.mu)[k];
                vy[i] = v0 * reinterpret_cast<const T*>(P.smu)[k];
            }
        }

        // A finished trajectory (escapes(): beyond R on a line that never
        // re-enters) keeps its velocity for every later step, and q_i depends
        // on v alone.  A warp stops integrating once all of its lanes are in that state
        // (padding lanes of a ragged tile start finished); the test runs every
        // kExitEvery steps, and a finished lane that keeps stepping with its
        // warp stays beyond R with its velocity unchanged.  All lanes of the
        // warp reach the vote, so the full mask is valid.
        if constexpr (PACKED) {
            static_assert(TPT == 2, "packed path holds two trajectories");
            f2 X = pk(x[0], x[1]), Y = pk(y[0], y[1]);
            f2 VX = pk(vx[0], vx[1]), VY = pk(vy[0], vy[1]);
            const HaloX2 h2{dup(hc.invIc), dup(-hc.invR3), hc.R2, hc.c};
            const float* ftab = reinterpret_cast<const float*>(tab);
            if (hc.narrow)
                packed_steps<GTAB, true>(X, Y, VX, VY, ftab, s_begin, s_end, act[0], act[1], done,
                                         h2, hc.R);
            else
                packed_steps<GTAB, false>(X, Y, VX, VY, ftab, s_begin, s_end, act[0], act[1], done,
                                          h2, hc.R);
            x[0] = f2lo(X); x[1] = f2hi(X);
            y[0] = f2lo(Y); y[1] = f2hi(Y);
            vx[0] = f2lo(VX); vx[1] = f2hi(VX);
            vy[0] = f2lo(VY); vy[1] = f2hi(VY);
        } else {
            bool fin_i[TPT];
#pragma unroll
            for (int i = 0; i < TPT; ++i) fin_i[i] = !act[i];
            for (int n = s_begin; n < s_end; ++n) {
                if (((n - s_begin) & (kExitEvery - 1)) == 0) {
                    bool fin = true;
#pragma unroll
                    for (int i = 0; i < TPT; ++i) {
                        fin_i[i] = !act[i] || escapes(fma(x[i], x[i], y[i] * y[i]),
                                                      fma(x[i], vx[i], y[i] * vy[i]),
                                                      fma(vx[i], vx[i], vy[i] * vy[i]), hc.R2,
                                                      hc.R, tab[(size_t)n * C_COUNT + C_IREM]);
                        fin &= fin_i[i];
                    }
                    done |= fin;
                    if (__all_sync(0xffffffffu, done)) break;
                }
                ctr.ran(TPT);
                T c[C_COUNT];
                const float4* c4 = reinterpret_cast<const float4*>(tab + (size_t)n * C_COUNT);
#pragma unroll
                for (int q = 0; q < (int)(C_COUNT * sizeof(T) / 16); ++q)
                    reinterpret_cast<float4*>(c)[q] = GTAB ? __ldg(&c4[q]) : c4[q];
#pragma unroll
                for (int i = 0; i < TPT; ++i) {
                    ctr.set_live(!fin_i[i] && !done);
                    rk4_step<T, Ctr>(x[i], y[i], vx[i], vy[i], c, hc, ctr);
                }
            }
        }

        if (state && s_end < n_steps) {          // more chunks follow: keep the state
#pragma unroll
            for (int i = 0; i < TPT; ++i) {
                if (!act[i]) continue;
                const int t = tis * P.tile + i * blockDim.x + threadIdx.x;
                T* st = state + ((size_t)seg * n_seg + t) * 4;
                st[0] = x[i];
                st[1] = y[i];
                st[2] = vx[i];
                st[3] = vy[i];
            }
            __syncthreads();   // every thread has read s_tile before it is reused
            continue;
        }

        // Liouville map and the weight of each trajectory in Eq. localdensity,
        // in FP64 from the final state (in the mixed mode its FP32 components
        // widened exactly).  The final momentum is that of the fiducial mass;
        // mass a of a mass-reuse request reads it scaled by s_a (Sec. III).
        double qf[TPT];
#pragma unroll
        for (int i = 0; i < TPT; ++i) {
            const double ux = (double)vx[i], uy = (double)vy[i];
            qf[i] = sqrt(fma(ux, ux, uy * uy)) * P.q_scale;
            if (P.qi && act[i]) {
                const int t = tis * P.tile + i * blockDim.x + threadIdx.x;
                reinterpret_cast<T*>(P.qi)[(size_t)seg * n_seg + t] = (T)qf[i];
            }
        }
        // momentum and direction nodes of each trajectory (recomputed here
        // rather than kept live through the step loop)
        int tj[TPT], tk[TPT];
#pragma unroll
        for (int i = 0; i < TPT; ++i) {
            const int t = act[i] ? tis * P.tile + i * blockDim.x + threadIdx.x : 0;
            tj[i] = t / n_mu;
            tk[i] = t - tj[i] * n_mu;
        }
        const int nm = P.n_mass;
        double* part = P.partials + ((size_t)seg * tps + tis) * 2 * nm;
        for (int a = 0; a < nm; ++a) {
            const double sa = P.mass_s[a];
            double acc = 0.0, accc = 0.0;
#pragma unroll
            for (int i = 0; i < TPT; ++i) {
                if (!act[i]) continue;
                const double f = relic_f_dev(P, qf[i] * sa);
                const double wm = P.wmu[tk[i]];
                acc += P.wq[tj[i]] * wm * f;
                accc += P.wqc[tj[i]] * wm * f;
            }
            // tile sum: warp shuffle, then the warps in order
            acc = warp_sum(acc);
            accc = warp_sum(accc);
            if (lane == 0) {
                s_red[warp][0] = acc;
                s_red[warp][1] = accc;
            }
            __syncthreads();
            if (warp == 0) {
                double t0 = lane < nwarps ? s_red[lane][0] : 0.0;
                double t1 = lane < nwarps ? s_red[lane][1] : 0.0;
                t0 = warp_sum(t0);
                t1 = warp_sum(t1);
                if (lane == 0) {
                    part[2 * a] = t0;
                    part[2 * a + 1] = t1;
                }
            }
            __syncthreads();   // s_red is reused by the next mass
        }
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(&P.seg_count[seg], 1u);
            s_last = (prev == (unsigned)(tps - 1));
        }
        __syncthreads();

        if (s_last && warp == 0) {   // this CTA finished the radius: add tiles in order
            __threadfence();
            const double* sp = P.partials + (size_t)seg * tps * 2 * nm;
            for (int a = 0; a < nm; ++a) {
                double t0 = 0.0, t1 = 0.0;
                for (int i = lane; i < tps; i += 32) {
                    t0 += __ldcg(&sp[(size_t)i * 2 * nm + 2 * a]);
                    t1 += __ldcg(&sp[(size_t)i * 2 * nm + 2 * a + 1]);
                }
                t0 = warp_sum(t0);
                t1 = warp_sum(t1);
                if (lane == 0) {
                    const double ratio = t0 * P.norms[2 * a];
                    const double ratio_c = t1 * P.norms[2 * a + 1];
                    P.out[(size_t)a * P.n_radii + seg] = ratio;
                    P.err[(size_t)a * P.n_radii + seg] = fabs(ratio - ratio_c) / (3.0 * fabs(ratio));
                    if (!isfinite(ratio)) atomicOr(P.status, 1);
                }
            }
            if (lane == 0) {
                P.seg_count[seg] = 0u;              // ready for the next run
                if (P.done_flag) {                  // serving: signal the request's last radius
                    __threadfence_system();
                    if (atomicAdd(P.done_count, 1u) == (unsigned)P.n_radii - 1u) {
                        __threadfence_system();
                        *P.done_flag = 1u;
                    }
                }
            }
        }
        // the next iteration's first __syncthreads orders s_tile/s_last reuse
    }
    if constexpr (COUNT) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            unsigned long long v = ctr.n[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) atomicAdd(&tallies[k], v);
        }
    }
}

// Force probe: m = Mhat/r^3 from the same device function the integrator
// uses, at radius r[i] on the x axis and RK stage (half-step index) `stage`.
template <typename T>
__global__ void force_probe_kernel(const DevProblem* __restrict__ prob, int stage,
                                   const double* __restrict__ r, int n, double* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const DevProblem& P = *prob;
    const T* c = reinterpret_cast<const T*>(P.coef);
    // stage 2k -> S0/Q0 of step k; 2k+1 -> S1/Q1 of step k; 2N -> S2/Q2 of step N-1
    const int k = stage >= 2 * P.n_steps ? P.n_steps - 1 : stage / 2;
    const int slot = stage >= 2 * P.n_steps ? 2 : (stage & 1);
    const T S = c[(size_t)k * C_COUNT + C_S0 + slot];
    const T Q = c[(size_t)k * C_COUNT + C_Q0 + slot];
    const T Tq = c[(size_t)k * C_COUNT + C_T0 + slot];
    const typename PrecTraits<T>::Halo hc = PrecTraits<T>::halo(P);
    NoTally none;
    out[i] = (double)accel_m((T)r[i], T(0), S, Q, Tq, hc, none);
}

int launch_force_probe(int precision, const DevProblem* d_prob, int stage, const double* d_r, int n,
                       double* d_out, void* stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = (n + 127) / 128;
    if (precision == NU_FP64)
        force_probe_kernel<double><<<grid, 128, 0, s>>>(d_prob, stage, d_r, n, d_out);
    else
        force_probe_kernel<float><<<grid, 128, 0, s>>>(d_prob, stage, d_r, n, d_out);
    if (cudaGetLastError() != cudaSuccess) return NU_ECUDA;
    count_launch();
    return NU_OK;
}

size_t coef_smem_bytes(int precision, int n_steps, int tpt)
{
    // the packed path stages the duplicated table (two floats per coefficient)
    const size_t per = precision == NU_FP64 ? sizeof(double) : sizeof(float) * (tpt == 3 ? 2 : 1);
    return (size_t)n_steps * C_COUNT * per;
}

template <typename T, int TPT, bool COUNT, bool PACKED = false, bool GTAB = false>
static int launch_t(int block, int grid, size_t smem, const DevProblem* d_probs, const int* d_prefix,
                    int n_probs, int n_tiles, unsigned* d_counter, unsigned long long* d_tallies,
                    cudaStream_t s, QueueCtl* d_queue = nullptr)
{
    auto k = traj_kernel<T, TPT, COUNT, PACKED, GTAB>;
    if (GTAB) smem = 0;
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return NU_ECUDA;
    }
    k<<<grid, block, smem, s>>>(d_probs, d_prefix, n_probs, n_tiles, d_counter, d_tallies, d_queue);
    if (cudaGetLastError() != cudaSuccess) return NU_ECUDA;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
        count_launch();   // captured launches are counted when the graph is replayed
    return NU_OK;
}

template <bool GTAB>
static int launch_shape(int precision, int tpt, int block, int grid, size_t smem,
                        const DevProblem* d_probs, const int* d_prefix, int n_probs, int n_tiles,
                        unsigned* d_counter, cudaStream_t s, QueueCtl* q)
{
    if (precision == NU_FP64) {
        if (tpt == 2) return launch_t<double, 2, false, false, GTAB>(block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, nullptr, s, q);
        return launch_t<double, 1, false, false, GTAB>(block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, nullptr, s, q);
    }
    if (tpt == 3) return launch_t<float, 2, false, true, GTAB>(block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, nullptr, s, q);
    if (tpt == 2) return launch_t<float, 2, false, false, GTAB>(block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, nullptr, s, q);
    return launch_t<float, 1, false, false, GTAB>(block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, nullptr, s, q);
}

int launch_traj(int precision, int tpt, int block, int grid, size_t smem, const DevProblem* d_probs,
                const int* d_prefix, int n_probs, int n_tiles, unsigned* d_counter, void* stream,
                bool gtab, QueueCtl* d_queue)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (gtab || smem > kMaxStagedSmem)   // a table too large to stage is read through L1
        return launch_shape<true>(precision, tpt, block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, s, d_queue);
    return launch_shape<false>(precision, tpt, block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, s, d_queue);
}

template <bool GTAB>
static int launch_tally_shape(int precision, int tpt, int block, int grid, size_t smem,
                              const DevProblem* d_probs, const int* d_prefix, int n_probs,
                              int n_tiles, unsigned* d_counter, unsigned long long* d_tallies,
                              cudaStream_t s)
{
    if (precision == NU_FP64) {
        if (tpt == 2) return launch_t<double, 2, true, false, GTAB>(block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, d_tallies, s);
        return launch_t<double, 1, true, false, GTAB>(block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, d_tallies, s);
    }
    if (tpt >= 2) return launch_t<float, 2, true, false, GTAB>(block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, d_tallies, s);
    return launch_t<float, 1, true, false, GTAB>(block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, d_tallies, s);
}

int launch_traj_tally(int precision, int tpt, int block, int grid, size_t smem,
                      const DevProblem* d_probs, const int* d_prefix, int n_probs, int n_tiles,
                      unsigned* d_counter, unsigned long long* d_tallies, void* stream)
{
    // the tallies are trajectory facts: every shape integrates the same values
    // (for a packed batch the scalar two-trajectory kernel counts, bitwise the
    // same computation; it stages the plain table, which needs less than smem)
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (smem > kMaxStagedSmem)
        return launch_tally_shape<true>(precision, tpt, block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, d_tallies, s);
    return launch_tally_shape<false>(precision, tpt, block, grid, smem, d_probs, d_prefix, n_probs, n_tiles, d_counter, d_tallies, s);
}

template <typename T, int TPT, bool PACKED = false, bool GTAB = false>
static int occ_t(int block, size_t smem, int* out)
{
    auto k = traj_kernel<T, TPT, false, PACKED, GTAB>;
    if (GTAB) smem = 0;
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return NU_ECUDA;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, block, smem) != cudaSuccess)
        return NU_ECUDA;
    return NU_OK;
}

template <bool GTAB>
static int occ_shape(int precision, int tpt, int block, size_t smem, int* out)
{
    if (precision == NU_FP64)
        return tpt == 2 ? occ_t<double, 2, false, GTAB>(block, smem, out) : occ_t<double, 1, false, GTAB>(block, smem, out);
    if (tpt == 3) return occ_t<float, 2, true, GTAB>(block, smem, out);
    return tpt == 2 ? occ_t<float, 2, false, GTAB>(block, smem, out) : occ_t<float, 1, false, GTAB>(block, smem, out);
}

int max_ctas_per_sm(int precision, int tpt, int block, size_t smem, int* out, bool gtab)
{
    return (gtab || smem > kMaxStagedSmem) ? occ_shape<true>(precision, tpt, block, smem, out)
                : occ_shape<false>(precision, tpt, block, smem, out);
}

}  // namespace nuprof
