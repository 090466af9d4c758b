// gp_sweep.cuh -- CN line-solve kernels for one axis of the split-step step.
//
// Every line along the swept axis solves the CN system (paper, "Summary of
// revisions": calclux / calcluy / calcluz)
//     -c phi[t-1] + (1+2c) phi[t] - c phi[t+1] = c psi[t-1] + (1-2c) psi[t] + c psi[t+1]
// on its n = N-2 interior nodes with zero end nodes, by the Thomas algorithm
// on precomputed recursion coefficients (inverse pivots ip[t] and
// multipliers cp[t], built once per dt on the host in FP64):
//     forward   dp[t] = (r[t] + c dp[t-1]) ip[t]
//     backward  phi[t] = dp[t] - cp[t] phi[t+1],  phi[n-1] = dp[n-1].
// The tables hold ip[t] - 1 (small, about -2c) rather than ip[t], and the
// forward step forms u + u (ip - 1) with fused multiply-adds: |ip| is close
// to one, so a rounded ip would act as a gain error on every dp, the same in
// every step, and in real time that is a steady norm drift (about 3e-8 per
// FP32 sweep); stored as a deviation its rounding error is ~|2c| smaller.
//
// Every value is read once from one buffer and written once to the other
// (sweeps are out of place, ping-ponging between two arrays).  A line is cut
// into segments of seg_len interior nodes, one thread per (line, segment),
// which gives the GPU enough independent sequential recurrences to cover
// memory latency.  Both recurrences contract: an error in dp[t-1] reaches
// dp[t] multiplied by c ip[t] = -cp[t], and an error in phi[t+1] reaches
// phi[t] multiplied by -cp[t], with |cp| < 1.  So
//  - a segment starting at t_b runs the forward sweep from t_b - (W+1) with
//    dp = 0 there (the line start needs no warm-up): the error at t_b is at
//    most |cp|_max^(W+2) * max|dp|;
//  - the backward sweep is windowed: dp values sit in a register ring of
//    B + W entries, and once dp[t0 .. t0+B+W-1] are known the chunk
//    phi[t0 .. t0+B-1] is recovered by starting the backward recurrence at
//    t0+B+W-1 with phi ~ dp (dropping cp * phi[t0+B+W]); the dropped term
//    reaches phi[t0+B-1] through W+1 factors, i.e. |cp|_max^(W+1) max|phi|.
// The host picks W so that |cp|_max^(W+1) is within half the unit roundoff
// (below the rounding of one operation), or uses the exact two-pass form (window 0, one segment), which
// stages dp in the output and reads it back.  The last chunk of a line is
// solved exactly from phi[n-1] = dp[n-1].
//
// The x sweep carries the fused potential-plus-nonlinear kick (calcnu),
// applied to each value as it is loaded, together with the pending
// renormalisation factor of the previous imaginary-time step; the z sweep
// carries the fused norm reduction (two-stage, deterministic, FP64 across
// threads) whose last block writes the next renormalisation factor.
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "gp_internal.h"

namespace gpcn {

template <typename R> struct cx;
template <> struct __align__(8) cx<float> { float re, im; };
template <> struct __align__(16) cx<double> { double re, im; };

// Read-only loads of coefficient-table entries (uniform across a warp).
__device__ __forceinline__ float ldc(const float *p) { return __ldg(p); }
__device__ __forceinline__ double ldc(const double *p) { return __ldg(p); }
__device__ __forceinline__ cx<float> ldc(const cx<float> *p) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return cx<float>{v.x, v.y};
}
__device__ __forceinline__ cx<double> ldc(const cx<double> *p) {
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    return cx<double>{v.x, v.y};
}

__device__ __forceinline__ float g_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double g_expm1(double x) { return expm1(x); }
__device__ __forceinline__ void g_sincos(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void g_sincos(double x, double *s, double *c) { sincos(x, s, c); }

// Short Taylor polynomials for the kick's small arguments (textbook series,
// Horner form).  Each is used only where its truncation error is below a
// quarter of the unit roundoff of the factor it forms; larger arguments fall
// back to expm1 / sincos.
//   FP32: sin through x^5, cos through x^6 for |x| <= 0.2 (next terms
//         x^7/7!, x^8/8! below 2^-26 relative); exp(-y) - 1 through y^4 for
//         |y| <= 0.05 (next term below 2^-27 of exp(-y)).
//   FP64: sin through x^9, cos through x^10 for |x| <= 0.1 (next terms below
//         2^-58 relative); exp(-y) - 1 through y^7 for |y| <= 0.02 (next
//         term below 2^-60 of exp(-y)).
// Imaginary-time factors are formed as deviations from one (exp(-y) - 1,
// and the trap tables hold exp(-dt V_a) - 1): a factor rounded once near one
// and applied at every step acts as a potential error of u / dt (u the unit
// roundoff), the same at every step, which shifts the FP32 fixed point (by
// about 7e-6 of mu on the 480x400x320 grid at dt = 0.1 d^2); a deviation
// rounded once is off by u |dt V|, a potential error of u |V|.
template <typename R> struct Series;
template <> struct Series<float> {
    static constexpr float kTrig = 0.2f, kExp = 0.05f;
    __device__ __forceinline__ static void sincos(float x, float *sn, float *cs) {
        const float x2 = x * x;
        *sn = x * fmaf(x2, fmaf(x2, 1.f / 120.f, -1.f / 6.f), 1.f);
        *cs = fmaf(x2, fmaf(x2, fmaf(x2, -1.f / 720.f, 1.f / 24.f), -0.5f), 1.f);
    }
    __device__ __forceinline__ static float expm1m(float y) {  // exp(-y) - 1
        return y * fmaf(y, fmaf(y, fmaf(y, 1.f / 24.f, -1.f / 6.f), 0.5f), -1.f);
    }
};
template <> struct Series<double> {
    static constexpr double kTrig = 0.1, kExp = 0.02;
    __device__ __forceinline__ static void sincos(double x, double *sn, double *cs) {
        const double x2 = x * x;
        *sn = x * fma(x2, fma(x2, fma(x2, fma(x2, 1.0 / 362880.0, -1.0 / 5040.0), 1.0 / 120.0),
                              -1.0 / 6.0), 1.0);
        *cs = fma(x2, fma(x2, fma(x2, fma(x2, fma(x2, -1.0 / 3628800.0, 1.0 / 40320.0), -1.0 / 720.0),
                                  1.0 / 24.0), -0.5), 1.0);
    }
    __device__ __forceinline__ static double expm1m(double y) {  // exp(-y) - 1
        return y * fma(y, fma(y, fma(y, fma(y, fma(y, fma(y, -1.0 / 5040.0, 1.0 / 720.0), -1.0 / 120.0),
                                              1.0 / 24.0), -1.0 / 6.0), 0.5), -1.0);
    }
};
// The library functions are called out of line: every load site of the x
// sweep inlines the kick, and inlined full-range sincos / exp code at each of
// them would crowd the instruction cache for a path that is rarely taken.
template <typename R> __device__ __noinline__ cx<R> sincos_full(R x) {
    cx<R> r;
    g_sincos(x, &r.im, &r.re);
    return r;
}
template <typename R> __device__ __noinline__ R expm1m_full(R y) { return g_expm1(-y); }
template <typename R> __device__ __forceinline__ void kick_sincos(R x, R *sn, R *cs) {
    if (fabs(x) <= Series<R>::kTrig) {
        Series<R>::sincos(x, sn, cs);
    } else {
        const cx<R> r = sincos_full(x);
        *sn = r.im;
        *cs = r.re;
    }
}
// exp(-y) - 1
template <typename R> __device__ __forceinline__ R kick_expm1m(R y) {
    return fabs(y) <= Series<R>::kExp ? Series<R>::expm1m(y) : expm1m_full(y);
}
// Deviation from one of the imaginary-time kick factor
// (1 + ex)(1 + eyz)(1 + m): the trap part of the node and line, then the
// nonlinear part m = exp(-dt g |q|^2) - 1.
template <typename R> __device__ __forceinline__ R kick_dev(R ex, R eyz, R m) {
    const R t = fma(ex, eyz, ex + eyz);
    return fma(t, m, t + m);
}

// Per-site kick state of one x line.  Imaginary time: exp(-dt V) is the
// product of per-axis factors exp(-dt V_x(i)) (a table of deviations from
// one) and exp(-dt (V_y(j) + V_z(k))) (fixed along the line, held as its
// deviation from one), times exp(-dt g |psi|^2); the kicked value is
// q + q D with D the product's deviation from one (kick_dev).
// Real time: theta = dt V_x(i) (a table) + dt (V_y(j) + V_z(k)) (fixed along
// the line) + dt g |psi|^2, and exp(-i theta).
template <typename R> struct KickState {
    R s;              // pending renormalisation factor
    R dtg;            // dt * g
    R eyz;            // exp(-dt (V_y + V_z)) - 1 of the line (imaginary time)
    const R *ex;      // exp(-dt V_x(i)) - 1 per node (imaginary time)
    R pyz;            // dt (V_y + V_z) of the line (real time)
    const R *px;      // dt V_x(i) per node (real time)
    R xo, xd, xc;     // x(i) = xo + i xd and dt V_x(i) = xc x(i)^2 (real time, computed in place)
};

// Per-thread sum: plain FP64, or FP32 with an error-free two-sum
// compensation term (Knuth) so that long FP32 sums keep FP64-like accuracy.
template <typename R> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float t = s + x;
        float bp = t - s;
        c += (s - (t - bp)) + (x - bp);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// ------------------------------------------------------------------ forms
// A form gives the arithmetic of one step of the recurrences on values of
// type V, and how V maps to the element layout in memory (MemV): identity
// for one line; the packed pair forms keep the two lines' values in
// component-wise float2 registers.
template <typename V_> struct LineForm {
    static constexpr int kLines = 1;
    static constexpr bool kChunkKick = false;  // kick_chunk: a chunk of nodes kicked at once
    using MemV = V_;
    __device__ __forceinline__ static V_ load(MemV m) { return m; }
    __device__ __forceinline__ static MemV store(V_ v) { return v; }
};

// Chunk kicks work in groups of at most kKickGroup nodes (bounds the
// registers the group's phases and scaled values hold).
constexpr int kKickGroup = 8;

// Imaginary time, real field: c = kappa, coefficients real.
template <typename R> struct FImagReal : LineForm<R> {
    using Real = R;
    using V = R;
    using C = R;
    __device__ __forceinline__ static V zero() { return R(0); }
    __device__ __forceinline__ static V rhs(V pm, V p0, V p1, R k) {
        return fma(k, (pm + p1) - R(2) * p0, p0);
    }
    __device__ __forceinline__ static V fwd(V r, V dprev, R k, C ipm1) {
        const V u = fma(k, dprev, r);
        return fma(u, ipm1, u);
    }
    __device__ __forceinline__ static V back(V dp, C cp, V phi) { return fma(-cp, phi, dp); }
    __device__ __forceinline__ static R abs2(V v) { return v * v; }
    __device__ __forceinline__ static V kick(V p, const KickState<R> &k, int node) {
        const V q = p * k.s;
        return fma(q, kick_dev(__ldg(k.ex + node), k.eyz, kick_expm1m(k.dtg * (q * q))), q);
    }
    // kick of NB consecutive nodes from node0: table loads issued together,
    // one series-range test per group, values equal kick's
    static constexpr bool kChunkKick = true;
    template <int NB> __device__ __forceinline__ static void kick_chunk(V (&v)[NB], const KickState<R> &k, int node0) {
#pragma unroll
        for (int g0 = 0; g0 < NB; g0 += kKickGroup) {
            constexpr int G = NB < kKickGroup ? NB : kKickGroup;
            R ex[G], q[G], y[G];
            bool small = true;
#pragma unroll
            for (int i = 0; i < G; ++i) ex[i] = __ldg(k.ex + node0 + g0 + i);
#pragma unroll
            for (int i = 0; i < G; ++i) {
                q[i] = v[g0 + i] * k.s;
                y[i] = k.dtg * (q[i] * q[i]);
                small = small && fabs(y[i]) <= Series<R>::kExp;
            }
            if (small) {
#pragma unroll
                for (int i = 0; i < G; ++i) v[g0 + i] = fma(q[i], kick_dev(ex[i], k.eyz, Series<R>::expm1m(y[i])), q[i]);
            } else {
#pragma unroll
                for (int i = 0; i < G; ++i) v[g0 + i] = kick(v[g0 + i], k, node0 + g0 + i);
            }
        }
    }
};

// Imaginary time, complex field: c = kappa real, applied to both parts.
template <typename R> struct FImagCplx : LineForm<cx<R>> {
    using Real = R;
    using V = cx<R>;
    using C = R;
    __device__ __forceinline__ static V zero() { return V{R(0), R(0)}; }
    __device__ __forceinline__ static V rhs(V pm, V p0, V p1, R k) {
        return V{fma(k, (pm.re + p1.re) - R(2) * p0.re, p0.re),
                 fma(k, (pm.im + p1.im) - R(2) * p0.im, p0.im)};
    }
    __device__ __forceinline__ static V fwd(V r, V dprev, R k, C ipm1) {
        const R ure = fma(k, dprev.re, r.re), uim = fma(k, dprev.im, r.im);
        return V{fma(ure, ipm1, ure), fma(uim, ipm1, uim)};
    }
    __device__ __forceinline__ static V back(V dp, C cp, V phi) {
        return V{fma(-cp, phi.re, dp.re), fma(-cp, phi.im, dp.im)};
    }
    __device__ __forceinline__ static R abs2(V v) { return fma(v.re, v.re, v.im * v.im); }
    __device__ __forceinline__ static V kick(V p, const KickState<R> &k, int node) {
        const V q{p.re * k.s, p.im * k.s};
        const R f = kick_dev(__ldg(k.ex + node), k.eyz, kick_expm1m(k.dtg * abs2(q)));
        return V{fma(q.re, f, q.re), fma(q.im, f, q.im)};
    }
    static constexpr bool kChunkKick = true;
    template <int NB> __device__ __forceinline__ static void kick_chunk(V (&v)[NB], const KickState<R> &k, int node0) {
#pragma unroll
        for (int g0 = 0; g0 < NB; g0 += kKickGroup) {
            constexpr int G = NB < kKickGroup ? NB : kKickGroup;
            R ex[G], y[G];
            V q[G];
            bool small = true;
#pragma unroll
            for (int i = 0; i < G; ++i) ex[i] = __ldg(k.ex + node0 + g0 + i);
#pragma unroll
            for (int i = 0; i < G; ++i) {
                q[i] = V{v[g0 + i].re * k.s, v[g0 + i].im * k.s};
                y[i] = k.dtg * abs2(q[i]);
                small = small && fabs(y[i]) <= Series<R>::kExp;
            }
            if (small) {
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    const R f = kick_dev(ex[i], k.eyz, Series<R>::expm1m(y[i]));
                    v[g0 + i] = V{fma(q[i].re, f, q[i].re), fma(q[i].im, f, q[i].im)};
                }
            } else {
#pragma unroll
                for (int i = 0; i < G; ++i) v[g0 + i] = kick(v[g0 + i], k, node0 + g0 + i);
            }
        }
    }
};

// Real time, complex field: c = i kappa, coefficients complex.
template <typename R> struct FRealTime : LineForm<cx<R>> {
    using Real = R;
    using V = cx<R>;
    using C = cx<R>;
    __device__ __forceinline__ static V zero() { return V{R(0), R(0)}; }
    __device__ __forceinline__ static V rhs(V pm, V p0, V p1, R k) {
        // r = p0 + i k (pm + p1 - 2 p0)
        R dre = (pm.re + p1.re) - R(2) * p0.re;
        R dim = (pm.im + p1.im) - R(2) * p0.im;
        return V{fma(-k, dim, p0.re), fma(k, dre, p0.im)};
    }
    __device__ __forceinline__ static V fwd(V r, V dprev, R k, C ipm1) {
        // u = r + i k dprev;  u ip = u + u (ip - 1)
        const R ure = fma(-k, dprev.im, r.re);
        const R uim = fma(k, dprev.re, r.im);
        return V{fma(ure, ipm1.re, fma(-uim, ipm1.im, ure)), fma(ure, ipm1.im, fma(uim, ipm1.re, uim))};
    }
    __device__ __forceinline__ static V back(V dp, C cp, V phi) {
        // dp - cp * phi
        R pre = fma(cp.re, phi.re, -cp.im * phi.im);
        R pim = fma(cp.re, phi.im, cp.im * phi.re);
        return V{dp.re - pre, dp.im - pim};
    }
    __device__ __forceinline__ static R abs2(V v) { return fma(v.re, v.re, v.im * v.im); }
    __device__ __forceinline__ static V kick(V p, const KickState<R> &k, int node) {
        const V q{p.re * k.s, p.im * k.s};
        const R theta = fma(k.dtg, abs2(q), __ldg(k.px + node) + k.pyz);
        R sn, cs;
        kick_sincos(theta, &sn, &cs);
        // exp(-i theta) q
        return V{fma(cs, q.re, sn * q.im), fma(cs, q.im, -sn * q.re)};
    }
    static constexpr bool kChunkKick = true;
    template <int NB> __device__ __forceinline__ static void kick_chunk(V (&v)[NB], const KickState<R> &k, int node0) {
#pragma unroll
        for (int g0 = 0; g0 < NB; g0 += kKickGroup) {
            constexpr int G = NB < kKickGroup ? NB : kKickGroup;
            R px[G], th[G];
            V q[G];
            bool small = true;
#pragma unroll
            for (int i = 0; i < G; ++i) px[i] = __ldg(k.px + node0 + g0 + i);
#pragma unroll
            for (int i = 0; i < G; ++i) {
                q[i] = V{v[g0 + i].re * k.s, v[g0 + i].im * k.s};
                th[i] = fma(k.dtg, abs2(q[i]), px[i] + k.pyz);
                small = small && fabs(th[i]) <= Series<R>::kTrig;
            }
            if (small) {
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    R sn, cs;
                    Series<R>::sincos(th[i], &sn, &cs);
                    v[g0 + i] = V{fma(cs, q[i].re, sn * q[i].im), fma(cs, q[i].im, -sn * q[i].re)};
                }
            } else {
#pragma unroll
                for (int i = 0; i < G; ++i) v[g0 + i] = kick(v[g0 + i], k, node0 + g0 + i);
            }
        }
    }
};

// Two adjacent lines advanced together by one thread: every operation is
// applied to both, the recursion coefficients are shared, and a pair of
// elements moves as one 8- or 16-byte access.
template <class F> struct FPair {
    using Real = typename F::Real;
    using E = typename F::V;
    struct __align__(2 * sizeof(E)) V { E a, b; };
    using C = typename F::C;
    static constexpr int kLines = 2;
    using MemV = V;
    __device__ __forceinline__ static V load(MemV m) { return m; }
    __device__ __forceinline__ static MemV store(V v) { return v; }
    __device__ __forceinline__ static V zero() { return V{F::zero(), F::zero()}; }
    __device__ __forceinline__ static V rhs(V pm, V p0, V p1, Real k) {
        return V{F::rhs(pm.a, p0.a, p1.a, k), F::rhs(pm.b, p0.b, p1.b, k)};
    }
    __device__ __forceinline__ static V fwd(V r, V dprev, Real k, C ipm1) {
        return V{F::fwd(r.a, dprev.a, k, ipm1), F::fwd(r.b, dprev.b, k, ipm1)};
    }
    __device__ __forceinline__ static V back(V dp, C cp, V phi) {
        return V{F::back(dp.a, cp, phi.a), F::back(dp.b, cp, phi.b)};
    }
    __device__ __forceinline__ static Real abs2(V v) { return F::abs2(v.a) + F::abs2(v.b); }
    __device__ __forceinline__ static V kick2(V v, const KickState<Real> &ka, const KickState<Real> &kb, int node) {
        return V{F::kick(v.a, ka, node), F::kick(v.b, kb, node)};
    }
    static constexpr bool kChunkKick = F::kChunkKick;
    template <int NB>
    __device__ __forceinline__ static void kick_chunk(V (&v)[NB], const KickState<Real> &ka,
                                                      const KickState<Real> &kb, int node0) {
        E a[NB], b[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            a[q] = v[q].a;
            b[q] = v[q].b;
        }
        F::template kick_chunk<NB>(a, ka, node0);
        F::template kick_chunk<NB>(b, kb, node0);
#pragma unroll
        for (int q = 0; q < NB; ++q) v[q] = V{a[q], b[q]};
    }
};

// Packed FP32 pairs: the two lines' values of each component share one
// float2, and each FP32 operation of the scalar form becomes one paired
// operation (fma / mul / add .f32x2, round to nearest) on both lines, in the
// same order, so the results equal the scalar form's.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

struct PRealTimeF {
    using Real = float;
    using F = FRealTime<float>;
    using C = cx<float>;
    struct __align__(16) V { float2 re, im; };  // (line a, line b) per component
    using MemV = typename FPair<F>::V;
    static constexpr int kLines = 2;
    __device__ __forceinline__ static V load(MemV m) {
        return V{make_float2(m.a.re, m.b.re), make_float2(m.a.im, m.b.im)};
    }
    __device__ __forceinline__ static MemV store(V v) {
        MemV m;
        m.a = cx<float>{v.re.x, v.im.x};
        m.b = cx<float>{v.re.y, v.im.y};
        return m;
    }
    __device__ __forceinline__ static V zero() { return V{dup2(0.f), dup2(0.f)}; }
    __device__ __forceinline__ static V rhs(V pm, V p0, V p1, float k) {
        const float2 dre = fma2(dup2(-2.f), p0.re, add2(pm.re, p1.re));
        const float2 dim = fma2(dup2(-2.f), p0.im, add2(pm.im, p1.im));
        return V{fma2(dup2(-k), dim, p0.re), fma2(dup2(k), dre, p0.im)};
    }
    __device__ __forceinline__ static V fwd(V r, V dprev, float k, C ipm1) {
        const float2 ure = fma2(dup2(-k), dprev.im, r.re);
        const float2 uim = fma2(dup2(k), dprev.re, r.im);
        return V{fma2(ure, dup2(ipm1.re), fma2(uim, dup2(-ipm1.im), ure)),
                 fma2(ure, dup2(ipm1.im), fma2(uim, dup2(ipm1.re), uim))};
    }
    __device__ __forceinline__ static V back(V dp, C cp, V phi) {
        const float2 pre = fma2(dup2(cp.re), phi.re, mul2(dup2(-cp.im), phi.im));
        const float2 pim = fma2(dup2(cp.re), phi.im, mul2(dup2(cp.im), phi.re));
        return V{sub2(dp.re, pre), sub2(dp.im, pim)};
    }
    __device__ __forceinline__ static float abs2(V v) {
        const float2 s = fma2(v.re, v.re, mul2(v.im, v.im));
        return s.x + s.y;
    }
    // Kick of both lines: shared scale, dt g and dt V_x (given as px);
    // per-line dt (V_y + V_z).  The scaled values q and the phase
    // theta = dt V_x + dt (V_y + V_z) + dt g |q|^2.
    __device__ __forceinline__ static float2 kick_phase(V p, const KickState<float> &ka, const KickState<float> &kb,
                                                        float px, float2 &qre, float2 &qim) {
        const float2 s = dup2(ka.s);
        qre = mul2(p.re, s);
        qim = mul2(p.im, s);
        const float2 a2 = fma2(qre, qre, mul2(qim, qim));
        const float2 base = add2(dup2(px), make_float2(ka.pyz, kb.pyz));
        return fma2(dup2(ka.dtg), a2, base);
    }
    __device__ __forceinline__ static bool kick_small(float2 th) {
        return fabsf(th.x) <= Series<float>::kTrig && fabsf(th.y) <= Series<float>::kTrig;
    }
    // exp(-i theta) q, theta within the series range.
    __device__ __forceinline__ static V kick_series(float2 th, float2 qre, float2 qim) {
        const float2 x2 = mul2(th, th);
        const float2 sn = mul2(th, fma2(x2, fma2(x2, dup2(1.f / 120.f), dup2(-1.f / 6.f)), dup2(1.f)));
        const float2 cs = fma2(x2, fma2(x2, fma2(x2, dup2(-1.f / 720.f), dup2(1.f / 24.f)), dup2(-0.5f)), dup2(1.f));
        return V{fma2(cs, qre, mul2(sn, qim)), fma2(cs, qim, mul2(make_float2(-sn.x, -sn.y), qre))};
    }
    // dt V_x at x node `node`, computed in registers: the same formula as the
    // x phase table, in FP32 (about 1e-11 from the table's FP64-rounded value
    // at the benchmark's dt), instead of a dependent table load per node.
    __device__ __forceinline__ static float px_of(const KickState<float> &k, int node) {
        const float x = fmaf((float)node, k.xd, k.xo);
        return k.xc * (x * x);
    }
    __device__ __forceinline__ static V kick2(V p, const KickState<float> &ka, const KickState<float> &kb,
                                              int node) {
        float2 qre, qim;
        const float2 th = kick_phase(p, ka, kb, px_of(ka, node), qre, qim);
        if (kick_small(th)) return kick_series(th, qre, qim);
        float2 sn, cs;
        kick_sincos(th.x, &sn.x, &cs.x);
        kick_sincos(th.y, &sn.y, &cs.y);
        return V{fma2(cs, qre, mul2(sn, qim)), fma2(cs, qim, mul2(make_float2(-sn.x, -sn.y), qre))};
    }
    // Kick of NB consecutive nodes (node0 ...): one test per chunk selects
    // the series for all of them; a chunk with any phase outside the series
    // range takes kick2 node by node.  Either way every value equals kick2's.
    static constexpr bool kChunkKick = true;
    template <int NB>
    __device__ __forceinline__ static void kick_chunk(V (&v)[NB], const KickState<float> &ka,
                                                      const KickState<float> &kb, int node0) {
        float px[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) px[q] = px_of(ka, node0 + q);
        float2 th[NB], qre[NB], qim[NB];
        bool small = true;
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            th[q] = kick_phase(v[q], ka, kb, px[q], qre[q], qim[q]);
            small = small && kick_small(th[q]);
        }
        if (small) {
#pragma unroll
            for (int q = 0; q < NB; ++q) v[q] = kick_series(th[q], qre[q], qim[q]);
        } else {
#pragma unroll
            for (int q = 0; q < NB; ++q) v[q] = kick2(v[q], ka, kb, node0 + q);
        }
    }
};

// exp(-y) - 1 by the FP32 series of Series<float>::expm1m, on two lines at once.
__device__ __forceinline__ float2 expm1m_series2(float2 y) {
    return mul2(y, fma2(y, fma2(y, fma2(y, dup2(1.f / 24.f), dup2(-1.f / 6.f)), dup2(0.5f)), dup2(-1.f)));
}
// kick_dev on two lines: the node's x deviation ex, the lines' deviations eyz.
__device__ __forceinline__ float2 kick_dev2(float ex, float2 eyz, float2 m) {
    const float2 t = fma2(dup2(ex), eyz, add2(dup2(ex), eyz));
    return fma2(t, m, add2(t, m));
}

// Packed FP32 pairs of the imaginary-time forms, in the same operation order
// as FImagReal<float> / FImagCplx<float> (results equal the scalar forms').
struct PImagRealF {
    using Real = float;
    using F = FImagReal<float>;
    using C = float;
    using V = float2;                     // (line a, line b)
    using MemV = typename FPair<F>::V;
    static constexpr int kLines = 2;
    __device__ __forceinline__ static V load(MemV m) { return make_float2(m.a, m.b); }
    __device__ __forceinline__ static MemV store(V v) { return MemV{v.x, v.y}; }
    __device__ __forceinline__ static V zero() { return dup2(0.f); }
    __device__ __forceinline__ static V rhs(V pm, V p0, V p1, float k) {
        return fma2(dup2(k), fma2(dup2(-2.f), p0, add2(pm, p1)), p0);
    }
    __device__ __forceinline__ static V fwd(V r, V dprev, float k, C ipm1) {
        const float2 u = fma2(dup2(k), dprev, r);
        return fma2(u, dup2(ipm1), u);
    }
    __device__ __forceinline__ static V back(V dp, C cp, V phi) { return fma2(dup2(-cp), phi, dp); }
    __device__ __forceinline__ static float abs2(V v) {
        const float2 s = mul2(v, v);
        return s.x + s.y;
    }
    // q, y = dt g q^2 of both lines
    __device__ __forceinline__ static float2 kick_arg(V p, const KickState<float> &ka, float2 &q) {
        q = mul2(p, dup2(ka.s));
        return mul2(dup2(ka.dtg), mul2(q, q));
    }
    __device__ __forceinline__ static bool kick_small(float2 y) {
        return fabs(y.x) <= Series<float>::kExp && fabs(y.y) <= Series<float>::kExp;
    }
    // q + q D, D the kick factor's deviation from one (m = exp(-y) - 1).
    __device__ __forceinline__ static V kick_apply(float2 q, float ex, const KickState<float> &ka,
                                                   const KickState<float> &kb, float2 m) {
        return fma2(q, kick_dev2(ex, make_float2(ka.eyz, kb.eyz), m), q);
    }
    __device__ __forceinline__ static V kick2(V p, const KickState<float> &ka, const KickState<float> &kb,
                                              int node) {
        float2 q;
        const float2 y = kick_arg(p, ka, q);
        const float ex = __ldg(ka.ex + node);
        if (kick_small(y)) return kick_apply(q, ex, ka, kb, expm1m_series2(y));
        return kick_apply(q, ex, ka, kb, make_float2(kick_expm1m(y.x), kick_expm1m(y.y)));
    }
    static constexpr bool kChunkKick = true;
    template <int NB>
    __device__ __forceinline__ static void kick_chunk(V (&v)[NB], const KickState<float> &ka,
                                                      const KickState<float> &kb, int node0) {
#pragma unroll
        for (int g0 = 0; g0 < NB; g0 += kKickGroup) {
            constexpr int G = NB < kKickGroup ? NB : kKickGroup;
            float ex[G];
            float2 q[G], y[G];
            bool small = true;
#pragma unroll
            for (int i = 0; i < G; ++i) ex[i] = __ldg(ka.ex + node0 + g0 + i);
#pragma unroll
            for (int i = 0; i < G; ++i) {
                y[i] = kick_arg(v[g0 + i], ka, q[i]);
                small = small && kick_small(y[i]);
            }
            if (small) {
#pragma unroll
                for (int i = 0; i < G; ++i) v[g0 + i] = kick_apply(q[i], ex[i], ka, kb, expm1m_series2(y[i]));
            } else {
#pragma unroll
                for (int i = 0; i < G; ++i) v[g0 + i] = kick2(v[g0 + i], ka, kb, node0 + g0 + i);
            }
        }
    }
};

struct PImagCplxF {
    using Real = float;
    using F = FImagCplx<float>;
    using C = float;
    struct __align__(16) V { float2 re, im; };  // (line a, line b) per component
    using MemV = typename FPair<F>::V;
    static constexpr int kLines = 2;
    __device__ __forceinline__ static V load(MemV m) {
        return V{make_float2(m.a.re, m.b.re), make_float2(m.a.im, m.b.im)};
    }
    __device__ __forceinline__ static MemV store(V v) {
        MemV m;
        m.a = cx<float>{v.re.x, v.im.x};
        m.b = cx<float>{v.re.y, v.im.y};
        return m;
    }
    __device__ __forceinline__ static V zero() { return V{dup2(0.f), dup2(0.f)}; }
    __device__ __forceinline__ static V rhs(V pm, V p0, V p1, float k) {
        return V{PImagRealF::rhs(pm.re, p0.re, p1.re, k), PImagRealF::rhs(pm.im, p0.im, p1.im, k)};
    }
    __device__ __forceinline__ static V fwd(V r, V dprev, float k, C ipm1) {
        return V{PImagRealF::fwd(r.re, dprev.re, k, ipm1), PImagRealF::fwd(r.im, dprev.im, k, ipm1)};
    }
    __device__ __forceinline__ static V back(V dp, C cp, V phi) {
        return V{PImagRealF::back(dp.re, cp, phi.re), PImagRealF::back(dp.im, cp, phi.im)};
    }
    __device__ __forceinline__ static float abs2(V v) {
        const float2 s = fma2(v.re, v.re, mul2(v.im, v.im));
        return s.x + s.y;
    }
    __device__ __forceinline__ static float2 kick_arg(V p, const KickState<float> &ka, V &q) {
        const float2 s = dup2(ka.s);
        q = V{mul2(p.re, s), mul2(p.im, s)};
        return mul2(dup2(ka.dtg), fma2(q.re, q.re, mul2(q.im, q.im)));
    }
    __device__ __forceinline__ static V kick_apply(V q, float ex, const KickState<float> &ka,
                                                   const KickState<float> &kb, float2 m) {
        const float2 f = kick_dev2(ex, make_float2(ka.eyz, kb.eyz), m);
        return V{fma2(q.re, f, q.re), fma2(q.im, f, q.im)};
    }
    __device__ __forceinline__ static V kick2(V p, const KickState<float> &ka, const KickState<float> &kb,
                                              int node) {
        V q;
        const float2 y = kick_arg(p, ka, q);
        const float ex = __ldg(ka.ex + node);
        if (PImagRealF::kick_small(y)) return kick_apply(q, ex, ka, kb, expm1m_series2(y));
        return kick_apply(q, ex, ka, kb, make_float2(kick_expm1m(y.x), kick_expm1m(y.y)));
    }
    static constexpr bool kChunkKick = true;
    template <int NB>
    __device__ __forceinline__ static void kick_chunk(V (&v)[NB], const KickState<float> &ka,
                                                      const KickState<float> &kb, int node0) {
#pragma unroll
        for (int g0 = 0; g0 < NB; g0 += kKickGroup) {
            constexpr int G = NB < kKickGroup ? NB : kKickGroup;
            float ex[G];
            V q[G];
            float2 y[G];
            bool small = true;
#pragma unroll
            for (int i = 0; i < G; ++i) ex[i] = __ldg(ka.ex + node0 + g0 + i);
#pragma unroll
            for (int i = 0; i < G; ++i) {
                y[i] = kick_arg(v[g0 + i], ka, q[i]);
                small = small && PImagRealF::kick_small(y[i]);
            }
            if (small) {
#pragma unroll
                for (int i = 0; i < G; ++i) v[g0 + i] = kick_apply(q[i], ex[i], ka, kb, expm1m_series2(y[i]));
            } else {
#pragma unroll
                for (int i = 0; i < G; ++i) v[g0 + i] = kick2(v[g0 + i], ka, kb, node0 + g0 + i);
            }
        }
    }
};

// Four adjacent lines of a real field in imaginary time: lines (0, 1) in
// the first float2 and (2, 3) in the second, every operation PImagRealF's
// on both halves (results equal the scalar form's).  A node of the four
// lines is one 16-byte access, so each row a warp reads or writes on a
// strided axis is 512 contiguous bytes instead of the pair form's 256.
struct PImagRealQ {
    using Real = float;
    using F = FImagReal<float>;
    using C = float;
    using P = PImagRealF;
    struct __align__(16) V { float2 a, b; };
    struct __align__(16) MemV { float x, y, z, w; };
    static constexpr int kLines = 4;
    static constexpr bool kChunkKick = true;
    __device__ __forceinline__ static V load(MemV m) { return V{make_float2(m.x, m.y), make_float2(m.z, m.w)}; }
    __device__ __forceinline__ static MemV store(V v) { return MemV{v.a.x, v.a.y, v.b.x, v.b.y}; }
    __device__ __forceinline__ static V zero() { return V{dup2(0.f), dup2(0.f)}; }
    __device__ __forceinline__ static V rhs(V pm, V p0, V p1, float k) {
        return V{P::rhs(pm.a, p0.a, p1.a, k), P::rhs(pm.b, p0.b, p1.b, k)};
    }
    __device__ __forceinline__ static V fwd(V r, V dprev, float k, C ipm1) {
        return V{P::fwd(r.a, dprev.a, k, ipm1), P::fwd(r.b, dprev.b, k, ipm1)};
    }
    __device__ __forceinline__ static V back(V dp, C cp, V phi) {
        return V{P::back(dp.a, cp, phi.a), P::back(dp.b, cp, phi.b)};
    }
    __device__ __forceinline__ static float abs2(V v) { return P::abs2(v.a) + P::abs2(v.b); }
    // Kick of the four lines (scale, dt g and the x factor shared; the line
    // factors exp(-dt (V_y + V_z)) from each line's state).
    __device__ __forceinline__ static V kick4(V p, const KickState<float> (&k)[4], int node) {
        float2 qa, qb;
        const float2 ya = P::kick_arg(p.a, k[0], qa), yb = P::kick_arg(p.b, k[0], qb);
        const float ex = __ldg(k[0].ex + node);
        const float2 ea = P::kick_small(ya) ? expm1m_series2(ya) : make_float2(kick_expm1m(ya.x), kick_expm1m(ya.y));
        const float2 eb = P::kick_small(yb) ? expm1m_series2(yb) : make_float2(kick_expm1m(yb.x), kick_expm1m(yb.y));
        return V{P::kick_apply(qa, ex, k[0], k[1], ea), P::kick_apply(qb, ex, k[2], k[3], eb)};
    }
    template <int NB>
    __device__ __forceinline__ static void kick_chunk(V (&v)[NB], const KickState<float> (&k)[4], int node0) {
#pragma unroll
        for (int g0 = 0; g0 < NB; g0 += kKickGroup) {
            constexpr int G = NB < kKickGroup ? NB : kKickGroup;
            float ex[G];
            float2 qa[G], qb[G], ya[G], yb[G];
            bool small = true;
#pragma unroll
            for (int i = 0; i < G; ++i) ex[i] = __ldg(k[0].ex + node0 + g0 + i);
#pragma unroll
            for (int i = 0; i < G; ++i) {
                ya[i] = P::kick_arg(v[g0 + i].a, k[0], qa[i]);
                yb[i] = P::kick_arg(v[g0 + i].b, k[0], qb[i]);
                small = small && P::kick_small(ya[i]) && P::kick_small(yb[i]);
            }
            if (small) {
#pragma unroll
                for (int i = 0; i < G; ++i)
                    v[g0 + i] = V{P::kick_apply(qa[i], ex[i], k[0], k[1], expm1m_series2(ya[i])),
                                  P::kick_apply(qb[i], ex[i], k[2], k[3], expm1m_series2(yb[i]))};
            } else {
#pragma unroll
                for (int i = 0; i < G; ++i) v[g0 + i] = kick4(v[g0 + i], k, node0 + g0 + i);
            }
        }
    }
};

// FP16 storage of a real field in imaginary time (FP32 arithmetic): the
// forms above with 2-byte elements in memory, widened on load and rounded
// to nearest on store.  FImagRealH is the single-line form (its values are
// FP32 in registers; StoreOf gives its memory element), PImagRealH the pair
// and QImagRealH the four-line form.  There is no single-line strided form:
// cp.async moves 4, 8 or 16 bytes, so the strided axes take pairs or quads.
struct FImagRealH : FImagReal<float> {
    using MemV = __half;
    __device__ __forceinline__ static float load(MemV m) { return __half2float(m); }
    __device__ __forceinline__ static MemV store(float v) { return __float2half_rn(v); }
};
struct __align__(4) Half2 { __half a, b; };
struct __align__(8) Half4 { __half x, y, z, w; };
struct PImagRealH : PImagRealF {
    using F = FImagRealH;
    using MemV = Half2;
    // one packed conversion each way
    __device__ __forceinline__ static V load(MemV m) { return __half22float2(__halves2half2(m.a, m.b)); }
    __device__ __forceinline__ static MemV store(V v) {
        const __half2 h = __float22half2_rn(v);
        return MemV{__low2half(h), __high2half(h)};
    }
};
struct QImagRealH : PImagRealQ {
    using F = FImagRealH;
    using MemV = Half4;
    __device__ __forceinline__ static V load(MemV m) {
        return V{__half22float2(__halves2half2(m.x, m.y)), __half22float2(__halves2half2(m.z, m.w))};
    }
    __device__ __forceinline__ static MemV store(V v) {
        const __half2 a = __float22half2_rn(v.a), b = __float22half2_rn(v.b);
        return MemV{__low2half(a), __high2half(a), __low2half(b), __high2half(b)};
    }
};
// The memory element of a single-line form's field.
template <class F> struct StoreOf { using type = typename F::V; };
template <> struct StoreOf<FImagRealH> { using type = __half; };
template <class F> using store_t = typename StoreOf<F>::type;

// The paired form of a single-line form.
template <class F> struct PairForm { using type = FPair<F>; };
template <> struct PairForm<FRealTime<float>> { using type = PRealTimeF; };
template <> struct PairForm<FImagReal<float>> { using type = PImagRealF; };
template <> struct PairForm<FImagCplx<float>> { using type = PImagCplxF; };
template <> struct PairForm<FImagRealH> { using type = PImagRealH; };
// The four-line form of a single-line form, where there is one.
template <class F> struct QuadForm { using type = void; };
template <> struct QuadForm<FImagReal<float>> { using type = PImagRealQ; };
template <> struct QuadForm<FImagRealH> { using type = QImagRealH; };
template <class F> constexpr bool has_quad() { return !std::is_void<typename QuadForm<F>::type>::value; }

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum `v` over the block in a fixed order; valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = (lane < (int)((blockDim.x + 31) >> 5)) ? red[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// Block partial of sum |phi|^2, then the last block to finish sums the
// partials in block order and writes the norm (and the renormalisation
// factor) -- deterministic whatever the block completion order.  `block` and
// `nblocks` number the blocks of one condensate (all of the grid for a single
// condensate; one instance's share of a batched launch).
__device__ __forceinline__ void norm_finalize(double v, const SweepArgs &a, unsigned block, unsigned nblocks) {
    __shared__ double red[32];
    __shared__ int is_last;
    double bsum = block_sum(v, red);
    if (threadIdx.x == 0) {
        a.partials[block] = bsum;
        __threadfence();
        unsigned prev = atomicAdd(a.counter, 1u);
        is_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) s += __ldcg(a.partials + b);
    double total = block_sum(s, red);
    if (threadIdx.x == 0) {
        double nrm = a.dV * total;
        *a.norm_out = nrm;
        if (a.want_scale) *a.scale_out = 1.0 / sqrt(nrm);
        *a.counter = 0u;
    }
}

// ------------------------------------------------------------------ async copies
// Global -> shared copies that bypass registers (cp.async); a copy whose
// source is out of range writes zeros (source size 0).
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int src = valid ? BYTES : 0;
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem), "n"(BYTES),
                     "r"(src)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Wait until at most `pending` of this thread's newest copy groups are in flight.
__device__ __forceinline__ void cp_async_wait(int pending) {
    switch (pending) {
    case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    }
}

// ------------------------------------------------------------------ one segment
// Outputs per chunk of the windowed solve: 16, or 8 for 16-byte elements
// (complex FP64) to bound the register ring.
template <typename V> __host__ __device__ constexpr int chunk_len() { return sizeof(V) >= 16 ? 8 : 16; }
// Chunks in a line's input ring: two readable, two in flight.
constexpr int kRingChunks = 4;

// Windowed Thomas solve of the interior nodes [tb, te) of a line of n
// interior unknowns; the coefficient tables hold their last values from
// tconst on.
// interior unknowns.  Inputs are read by interior position p (node p+1;
// positions outside [0, n) read 0) after io.need(p_end) has made the
// positions [p_end - B, p_end) readable; outputs go through io.put(t0, q, v)
// (position t0 + q) and io.flush(t0, count).
// One full chunk: dp[t0+W .. t0+W+B-1] forward, then phi[t0 .. t0+B-1] by
// the windowed backward sweep.  SETTLED: every coefficient the chunk uses
// equals the table's last entry (cp and ip reach their fixed point a few
// nodes into the line and stay there to FP rounding), so they are read once
// per thread instead of once per node.
template <class F, typename R, int B, int W, bool SETTLED, class IO>
__device__ __forceinline__ void window_chunk(int t0, typename F::V (&D)[B + W], typename F::V &pm, typename F::V &p0,
                                             typename F::V &p1, typename F::V &dprev, R kap,
                                             const typename F::C *__restrict__ cp,
                                             const typename F::C *__restrict__ ipm1, typename F::C cps,
                                             typename F::C ips, IO &io) {
    using V = typename F::V;
    io.need(t0 + W + 2 + B);
    V in[B];  // the chunk's inputs, positions t0+W+2 .. t0+W+B+1 (kicked as one chunk on the x sweep)
    io.vals(t0 + W + 2, in);
#pragma unroll
    for (int q = 0; q < B; ++q) {
        dprev = F::fwd(F::rhs(pm, p0, p1, kap), dprev, kap, SETTLED ? ips : ldc(ipm1 + t0 + W + q));
        D[W + q] = dprev;
        pm = p0;
        p0 = p1;
        p1 = in[q];
    }
    V phi = D[B + W - 1];
#pragma unroll
    for (int q = B + W - 2; q >= B; --q) phi = F::back(D[q], SETTLED ? cps : ldc(cp + t0 + q), phi);
#pragma unroll
    for (int q = B - 1; q >= 0; --q) {
        phi = F::back(D[q], SETTLED ? cps : ldc(cp + t0 + q), phi);
        io.put(t0, q, phi);
    }
    io.flush(t0, B);
#pragma unroll
    for (int q = 0; q < W; ++q) D[q] = D[B + q];
}

template <class F, typename R, int B, int W, class IO>
__device__ __forceinline__ void solve_segment(int n, int tb, int te, int tconst, R kap,
                                              const typename F::C *__restrict__ cp,
                                              const typename F::C *__restrict__ ipm1, IO &io) {
    using V = typename F::V;
    using C = typename F::C;
    // forward warm-up from dp = 0 at tw (exact when tw == 0: node 0 is 0)
    const int tw = tb > W + 1 ? tb - (W + 1) : 0;
    // the segment behaves as a line ending at e: W look-ahead values beyond
    // te start the windowed backward sweep of its last chunk
    const int e = min(te + W, n);
    io.start(tw - 1, e + 2);
    io.need(tw + 2);
    V pm = io.val(tw - 1);
    V p0 = io.val(tw);
    V p1 = io.val(tw + 1);
    V dprev = F::zero();
    for (int t = tw; t < tb; ++t) {
        dprev = F::fwd(F::rhs(pm, p0, p1, kap), dprev, kap, ldc(ipm1 + t));
        pm = p0;
        p0 = p1;
        io.need(t + 3);
        p1 = io.val(t + 2);
    }
    const int m = e - tb;
    V D[B + W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
        if (q < m) {
            dprev = F::fwd(F::rhs(pm, p0, p1, kap), dprev, kap, ldc(ipm1 + tb + q));
            D[q] = dprev;
            pm = p0;
            p0 = p1;
            io.need(tb + q + 3);
            p1 = io.val(tb + q + 2);
        }
    }
    int t0 = tb;
    // chunks before the coefficients settle read the tables; the rest keep
    // the settled values in registers
    const C cps = ldc(cp + n - 1), ips = ldc(ipm1 + n - 1);
    for (; t0 + B + W <= e && t0 < tconst; t0 += B)
        window_chunk<F, R, B, W, false>(t0, D, pm, p0, p1, dprev, kap, cp, ipm1, cps, ips, io);
    for (; t0 + B + W <= e; t0 += B)
        window_chunk<F, R, B, W, true>(t0, D, pm, p0, p1, dprev, kap, cp, ipm1, cps, ips, io);
    const int rem = e - t0;  // 0 <= rem < B + W: finish from dp[e-1]
    io.need(e + 2);
#pragma unroll
    for (int q = W; q < B + W; ++q) {
        if (q < rem) {
            dprev = F::fwd(F::rhs(pm, p0, p1, kap), dprev, kap, ldc(ipm1 + t0 + q));
            D[q] = dprev;
            pm = p0;
            p0 = p1;
            p1 = io.val(t0 + q + 2);
        }
    }
    V phi = F::zero();
#pragma unroll
    for (int q = B + W - 1; q >= 0; --q) {
        if (q < rem) {
            phi = F::back(D[q], ldc(cp + t0 + q), (q == rem - 1) ? F::zero() : phi);
            if (t0 + q < te) io.put(t0, q, phi);
        }
    }
    io.flush(t0, min(rem, te - t0));
}

// Exact two-pass Thomas over a whole line (window 0): dp is staged in the
// output and read back by the backward sweep.  Direct loads and stores.
template <class F, typename R, class IO>
__device__ __forceinline__ void solve_line_exact(int n, R kap, const typename F::C *__restrict__ cp,
                                                 const typename F::C *__restrict__ ipm1, IO &io) {
    using V = typename F::V;
    V pm = F::zero();
    V p0 = io.load1(0);
    V p1 = io.load1(1);
    V dprev = F::zero();
    for (int t = 0; t < n; ++t) {
        dprev = F::fwd(F::rhs(pm, p0, p1, kap), dprev, kap, ldc(ipm1 + t));
        pm = p0;
        p0 = p1;
        p1 = io.load1(t + 2);
        if (t < n - 1) io.stage(t, dprev);
    }
    V phi = dprev;
    io.put1(n - 1, phi);
    for (int t = n - 2; t >= 0; --t) {
        phi = F::back(io.unstage(t), ldc(cp + t), phi);
        io.put1(t, phi);
    }
}

// ------------------------------------------------------------------ kick / norm hooks
// The x sweep applies the kick to every value it reads; the z sweep adds
// |phi|^2 of every value it writes to the thread's norm sum.
template <typename R, int KIND> __device__ __forceinline__ void kick_init(KickState<R> &k, const SweepArgs &a,
                                                                          long long L) {
    const int j = (int)(L / a.nz), kk = (int)(L % a.nz);
    k.s = (R)__ldg(a.scale);
    k.dtg = (R)(a.dt * a.g);
    k.ex = static_cast<const R *>(a.kick_ex);
    if (a.kick_ex) {
        const R ey = __ldg(static_cast<const R *>(a.kick_ey) + j), ez = __ldg(static_cast<const R *>(a.kick_ez) + kk);
        k.eyz = fma(ey, ez, ey + ez);  // (1 + ey)(1 + ez) - 1
    } else {
        k.eyz = R(0);
    }
    k.px = static_cast<const R *>(a.phase_ex);
    k.pyz = a.phase_ex ? __ldg(static_cast<const R *>(a.phase_ey) + j) + __ldg(static_cast<const R *>(a.phase_ez) + kk)
                       : R(0);
    k.xo = (R)a.origin[0];
    k.xd = (R)a.d[0];
    k.xc = (R)(a.dt * a.half_w2[0]);
}

// F is the single-line form; M is F (one line per thread) or its pair or
// quad form.
template <class F, class M, typename R, int KIND> struct Hooks {
    using V = typename M::V;
    static constexpr int NL = M::kLines;
    KickState<R> k[NL];
    Acc<R> *acc;
    __device__ __forceinline__ void init(const SweepArgs &a, long long L) {
        if (KIND == K_X) {
#pragma unroll
            for (int q = 0; q < NL; ++q) kick_init<R, KIND>(k[q], a, L + q);
        }
    }
    __device__ __forceinline__ V on_load(int p, V v) const {
        if constexpr (KIND == K_X) {
            if constexpr (NL == 4) v = M::kick4(v, k, p + 1);
            else if constexpr (NL == 2) v = M::kick2(v, k[0], k[1], p + 1);
            else v = F::kick(v, k[0], p + 1);
        }
        return v;
    }
    // on_load of NB consecutive positions p .. p+NB-1.
    template <int NB> __device__ __forceinline__ void on_load_chunk(int p, V (&v)[NB]) const {
        if constexpr (KIND == K_X) {
            if constexpr (NL == 4) {
                M::template kick_chunk<NB>(v, k, p + 1);
            } else if constexpr (M::kChunkKick && NL == 2) {
                M::template kick_chunk<NB>(v, k[0], k[1], p + 1);
            } else if constexpr (M::kChunkKick) {
                M::template kick_chunk<NB>(v, k[0], p + 1);
            } else {
#pragma unroll
                for (int q = 0; q < NB; ++q) v[q] = on_load(p + q, v[q]);
            }
        }
    }
    __device__ __forceinline__ void on_store(V v) const {
        if (KIND == K_Z) acc->add(M::abs2(v));
    }
};

// Direct per-thread access, for the exact two-pass form.
template <class F, class M, typename R, int KIND> struct DirectIO {
    using V = typename M::V;
    using MV = typename M::MemV;
    const MV *in;
    MV *out;
    long long st;
    int n;
    Hooks<F, M, R, KIND> hk;
    __device__ __forceinline__ V load1(int t) const {
        if (t < 0 || t >= n) return M::zero();
        return hk.on_load(t, M::load(in[(long long)(t + 1) * st]));
    }
    __device__ __forceinline__ void put1(int t, V v) const {
        out[(long long)(t + 1) * st] = M::store(v);
        hk.on_store(v);
    }
    __device__ __forceinline__ void stage(int t, V v) const { out[(long long)(t + 1) * st] = M::store(v); }
    __device__ __forceinline__ V unstage(int t) const { return M::load(out[(long long)(t + 1) * st]); }
};

// ------------------------------------------------------------------ strided axes
// One thread owns one segment of one line (element stride st); consecutive
// threads own lines adjacent in memory, so each cp.async instruction of a
// warp reads one contiguous row.  Each thread streams its line through a
// private column of a shared ring, ring[position % R][thread], R = 4 chunks:
// while one chunk is consumed the next two are in flight.
template <class F, class M, typename R, int B, int KIND> struct ColumnIO {
    using V = typename M::V;
    using MV = typename M::MemV;
    static constexpr int RL = kRingChunks * B;  // ring length (power of two)
    const MV *in;
    MV *out;
    MV *ring;     // this thread's column: element p at ring[(p - s0) % RL * T]
    long long st;
    int n, T, s0, limit, issued, ready;
    Hooks<F, M, R, KIND> hk;
    __device__ __forceinline__ void issue() {
        const int pb = s0 + issued * B;
        // the chunk's B ring rows are consecutive: (pb + e - s0) mod RL =
        // ((issued B) mod RL) + e, since RL is a multiple of B
        MV *slot = ring + ((issued * B) & (RL - 1)) * T;
        if (pb >= 0 && pb + B <= n) {
            // the whole chunk inside the line (every chunk but a line's
            // first and last): no per-element range test or select
            const MV *g = in + (long long)(pb + 1) * st;
#pragma unroll
            for (int e = 0; e < B; ++e) cp_async<sizeof(MV)>(slot + e * T, g + e * st, true);
        } else {
#pragma unroll
            for (int e = 0; e < B; ++e) {
                const int p = pb + e;
                const bool ok = p >= 0 && p < n;
                cp_async<sizeof(MV)>(slot + e * T, ok ? in + (long long)(p + 1) * st : in, ok);
            }
        }
        cp_async_commit();
        ++issued;
    }
    __device__ __forceinline__ void start(int first, int lim) {
        s0 = first;
        limit = lim;
        issued = ready = 0;
        while (issued < kRingChunks - 1 && s0 + issued * B < limit) issue();
    }
    __device__ __forceinline__ void need(int p_end) {
        const int c = (p_end - 1 - s0) / B;
        if (c < ready) return;
        cp_async_wait(issued - 1 - c);
        ready = c + 1;
        while (issued <= c + kRingChunks - 2 && s0 + issued * B < limit) issue();
    }
    __device__ __forceinline__ V val(int p) const {
        return hk.on_load(p, M::load(ring[((p - s0) & (RL - 1)) * T]));
    }
    template <int NB> __device__ __forceinline__ void vals(int p, V (&v)[NB]) const {
#pragma unroll
        for (int q = 0; q < NB; ++q) v[q] = M::load(ring[((p + q - s0) & (RL - 1)) * T]);
        hk.on_load_chunk(p, v);
    }
    __device__ __forceinline__ void put(int t0, int q, V v) const {
        out[(long long)(t0 + q + 1) * st] = M::store(v);
        hk.on_store(v);
    }
    __device__ __forceinline__ void flush(int, int) const {}
};

template <class F, int LPT> struct LinesPerThread { using M = F; };
template <class F> struct LinesPerThread<F, 2> { using M = typename PairForm<F>::type; };
template <class F> struct LinesPerThread<F, 4> { using M = typename QuadForm<F>::type; };

// One thread per (line, segment), or per (group of LPT = 2 or 4 adjacent
// lines, segment); blockIdx.y is the segment.  Window 0 selects the exact
// two-pass form over whole lines with direct access.
template <class F, typename R, int W, int KIND, int LPT>
__device__ __forceinline__ double lines_body(const SweepArgs &a, unsigned bx, unsigned seg,
                                             unsigned char *smem_raw) {
    using M = typename LinesPerThread<F, LPT>::M;
    using V = typename M::V;
    using MV = typename M::MemV;
    using C = typename F::C;
    constexpr int B = chunk_len<MV>();
    const long long L = ((long long)bx * blockDim.x + threadIdx.x) * LPT;
    Acc<R> acc;
    if (L < a.n_lines) {
        const long long off = (L / a.inner) * a.outer_stride + (L % a.inner);
        const MV *in = reinterpret_cast<const MV *>(static_cast<const store_t<F> *>(a.psi) + off);
        MV *out = reinterpret_cast<MV *>(static_cast<store_t<F> *>(a.psi_out) + off);
        const long long st = a.stride / LPT;  // stride in units of MV
        const int n = a.N - 2;
        const C *cp = static_cast<const C *>(a.cp);
        const C *ipm1 = static_cast<const C *>(a.ip);
        if (seg == 0) out[0] = M::store(M::zero());
        if ((int)seg == a.n_seg - 1) out[(long long)(a.N - 1) * st] = M::store(M::zero());
        if constexpr (W > 0) {
            ColumnIO<F, M, R, B, KIND> io;
            io.in = in;
            io.out = out;
            io.st = st;
            io.n = n;
            io.T = blockDim.x;
            io.ring = reinterpret_cast<MV *>(smem_raw) + threadIdx.x;
            io.hk.acc = &acc;
            io.hk.init(a, L);
            const int tb = seg * a.seg_len;
            const int te = (int)seg == a.n_seg - 1 ? n : tb + a.seg_len;
            solve_segment<M, R, B, W>(n, tb, te, a.t_const, (R)a.kappa, cp, ipm1, io);
        } else {
            DirectIO<F, M, R, KIND> io;
            io.in = in;
            io.out = out;
            io.st = st;
            io.n = n;
            io.hk.acc = &acc;
            io.hk.init(a, L);
            solve_line_exact<M, R>(n, (R)a.kappa, cp, ipm1, io);
        }
    }
    return acc.value();
}

// One thread per (line, segment), or per (pair of adjacent lines, segment)
// when LPT = 2; blockIdx.y is the segment.  Window 0 selects the exact
// two-pass form over whole lines with direct access.
template <class F, typename R, int W, int KIND, int LPT>
__global__ void __launch_bounds__(256, 1) sweep_lines_kernel(SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const double v = lines_body<F, R, W, KIND, LPT>(a, blockIdx.x, blockIdx.y, smem_raw);
    if (KIND == K_Z) norm_finalize(v, a, blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y);
}

template <typename V> __host__ __device__ constexpr size_t column_ring_bytes(int threads) {
    return (size_t)kRingChunks * chunk_len<V>() * threads * sizeof(V);
}

// ------------------------------------------------------------------ contiguous axis
// A warp owns one segment of 32 consecutive stride-1 lines (one contiguous
// block of 32 * N elements).  Input chunks of B values per line are copied
// cooperatively (each cp.async instruction covers 32/B lines x B consecutive
// elements) into a per-warp ring, ring[line][position % R] (rows padded by
// one element against bank conflicts), two chunks ahead of the consumer;
// lane l reads row l.  Outputs are collected in a padded tile, row l per
// lane, and written back cooperatively.
template <class F, typename R, int B, int W> struct TileIO {
    using V = typename F::V;
    static constexpr int RL = kRingChunks * B;   // ring length per line (power of two)
    static constexpr int RS = RL + 1;            // padded ring row
    static constexpr int OS = B + W + 1;         // padded output row
    static constexpr int LPI = 32 / B;           // lines per cooperative instruction
    const V *in0;                                // node 0 of the warp's first line
    V *out0;
    V *ring, *otile;
    int N, n, lane, nvalid, s0, limit, issued, ready;
    Acc<R> *acc;
    R csum;  // |phi|^2 of the chunk being written (added to acc per chunk)
    // Per-lane constants of the cooperative copies: lane copies element e of
    // lines qb, qb + LPI, qb + 2 LPI, ... (its first `nit` of them are valid).
    int e, qb, nit;
    const V *src_lane;  // in0 + qb * N + 1 + e
    V *dst_lane;        // ring + qb * RS
    __device__ __forceinline__ void setup() {
        e = lane % B;
        qb = lane / B;
        nit = qb < nvalid ? (nvalid - qb + LPI - 1) / LPI : 0;
        src_lane = in0 + (long long)qb * N + 1 + e;
        dst_lane = ring + qb * RS;
    }
    __device__ __forceinline__ void issue() {
        const int pb = s0 + issued * B;
        const int p = pb + e;
        const bool pos_ok = p >= 0 && p < n;
        const int ro = (issued * B + e) & (RL - 1);
        const V *src = src_lane + pb;
        V *dst = dst_lane + ro;
#pragma unroll 4
        for (int it = 0; it < B; ++it) {
            const bool ok = pos_ok && it < nit;
            cp_async<sizeof(V)>(dst, ok ? src : in0, ok);
            src += (long long)LPI * N;
            dst += LPI * RS;
        }
        cp_async_commit();
        ++issued;
    }
    __device__ __forceinline__ void start(int first, int lim) {
        s0 = first;
        limit = lim;
        issued = ready = 0;
        while (issued < kRingChunks - 1 && s0 + issued * B < limit) issue();
    }
    __device__ __forceinline__ void need(int p_end) {
        const int c = (p_end - 1 - s0) / B;
        if (c < ready) return;
        __syncwarp();  // every lane is done with the chunk slot about to be refilled
        cp_async_wait(issued - 1 - c);
        __syncwarp();  // the chunk written by all lanes' copies is visible to all lanes
        ready = c + 1;
        while (issued <= c + kRingChunks - 2 && s0 + issued * B < limit) issue();
    }
    __device__ __forceinline__ V val(int p) const { return ring[lane * RS + ((p - s0) & (RL - 1))]; }
    template <int NB> __device__ __forceinline__ void vals(int p, V (&v)[NB]) const {
#pragma unroll
        for (int q = 0; q < NB; ++q) v[q] = val(p + q);
    }
    __device__ __forceinline__ void put(int, int q, V v) {
        otile[lane * OS + q] = v;
        csum += F::abs2(v);
    }
    // Write positions t0 .. t0+count-1 of the 32 lines back to global memory.
    __device__ __forceinline__ void flush(int t0, int count) {
        if (lane < nvalid) acc->add(csum);
        csum = R(0);
        __syncwarp();
        if (count == B) {
            V *dst = out0 + (long long)qb * N + t0 + 1 + e;
            const V *src = otile + qb * OS + e;
#pragma unroll 4
            for (int it = 0; it < B; ++it) {
                if (it < nit) *dst = *src;
                dst += (long long)LPI * N;
                src += LPI * OS;
            }
        } else {
            for (int q = 0; q < nvalid; ++q)
                for (int ee = lane; ee < count; ee += 32) out0[(long long)q * N + t0 + 1 + ee] = otile[q * OS + ee];
        }
        __syncwarp();
    }
};

template <typename V, int W> __host__ __device__ constexpr size_t tile_warp_bytes() {
    return (size_t)32 * ((kRingChunks * chunk_len<V>() + 1) + (chunk_len<V>() + W + 1)) * sizeof(V);
}
constexpr int kTileWarps = 2;

template <class F, typename R, int W>
__device__ __forceinline__ double contig_body(const SweepArgs &a, unsigned bx, unsigned seg,
                                              unsigned char *smem_raw) {
    using V = typename F::V;
    using C = typename F::C;
    constexpr int B = chunk_len<V>();
    using IO = TileIO<F, R, B, W>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long L0 = ((long long)bx * (blockDim.x >> 5) + warp) * 32;
    Acc<R> acc;
    if (L0 < a.n_lines) {
        IO io;
        V *wbase = reinterpret_cast<V *>(smem_raw + warp * tile_warp_bytes<V, W>());
        io.ring = wbase;
        io.otile = wbase + 32 * IO::RS;
        io.in0 = static_cast<const V *>(a.psi) + L0 * a.N;
        io.out0 = static_cast<V *>(a.psi_out) + L0 * a.N;
        io.N = a.N;
        io.n = a.N - 2;
        io.lane = lane;
        io.nvalid = (int)min(32LL, a.n_lines - L0);
        io.acc = &acc;
        io.csum = R(0);
        io.setup();
        if (lane < io.nvalid) {
            if (seg == 0) io.out0[(long long)lane * a.N] = F::zero();
            if ((int)seg == a.n_seg - 1) io.out0[(long long)lane * a.N + a.N - 1] = F::zero();
        }
        const int tb = seg * a.seg_len;
        const int te = (int)seg == a.n_seg - 1 ? io.n : tb + a.seg_len;
        solve_segment<F, R, B, W>(io.n, tb, te, a.t_const, (R)a.kappa, static_cast<const C *>(a.cp),
                                  static_cast<const C *>(a.ip), io);
    }
    return acc.value();
}

template <class F, typename R, int W>
__global__ void __launch_bounds__(kTileWarps * 32, 1) sweep_contig_kernel(SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const double v = contig_body<F, R, W>(a, blockIdx.x, blockIdx.y, smem_raw);
    norm_finalize(v, a, blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y);
}

// ------------------------------------------------------------------ batched launches
// Many condensates in one launch: instance i owns the blocks
// [first[i], first[i+1]) of a 1D grid, laid out as its single-condensate grid
// (bx fastest, then the segment).  Each instance has its own argument block
// (buffers, sizes, coefficients, norm partials and counter).
struct BatchDesc {
    const SweepArgs *args;    // per instance
    const unsigned *first;    // n + 1 prefix sums of blocks
    const unsigned *gridx;    // per instance: blocks along x of its own grid
    int n;
};

__device__ __forceinline__ int find_instance(const BatchDesc &d, unsigned b) {
    int lo = 0, hi = d.n - 1;
    while (lo < hi) {  // last i with first[i] <= b
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(d.first + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class F, typename R, int W, int KIND, int LPT>
__global__ void __launch_bounds__(256, 1) batch_lines_kernel(BatchDesc d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int i = find_instance(d, blockIdx.x);
    const SweepArgs a = d.args[i];
    const unsigned local = blockIdx.x - __ldg(d.first + i);
    const unsigned gx = __ldg(d.gridx + i);
    const unsigned nblocks = __ldg(d.first + i + 1) - __ldg(d.first + i);
    const double v = lines_body<F, R, W, KIND, LPT>(a, local % gx, local / gx, smem_raw);
    if (KIND == K_Z) norm_finalize(v, a, local, nblocks);
}

template <class F, typename R, int W>
__global__ void __launch_bounds__(kTileWarps * 32, 1) batch_contig_kernel(BatchDesc d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int i = find_instance(d, blockIdx.x);
    const SweepArgs a = d.args[i];
    const unsigned local = blockIdx.x - __ldg(d.first + i);
    const unsigned gx = __ldg(d.gridx + i);
    const unsigned nblocks = __ldg(d.first + i + 1) - __ldg(d.first + i);
    const double v = contig_body<F, R, W>(a, local % gx, local / gx, smem_raw);
    norm_finalize(v, a, local, nblocks);
}

}  // namespace gpcn
