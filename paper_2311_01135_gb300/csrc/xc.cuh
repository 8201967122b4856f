// Closed-shell B3LYP (VWN5) energy density and its first derivatives on the
// device.  The paper supports only B3LYP (Section 3.2, "Libxc") and obtains
// the potential by automatic differentiation; here the derivatives are
// written out analytically.
//
//   e(rho, sigma) = 0.80 e_Slater + 0.72 de_B88 + 0.19 e_VWN5 + 0.81 e_LYP
//   (the remaining 0.20 exact exchange enters the Fock matrix through K),
//   v_rho = de/drho,  v_sigma = de/dsigma,  sigma = |grad rho|^2.
//
// Pieces (closed shell, rho total density):
//  Slater: -(3/4)(3/pi)^(1/3) rho^(4/3)                            (Dirac 1930)
//  B88:    -2^(1/3) beta sigma rho^(-4/3) / g(x),  g = 1 + 6 beta x asinh x,
//          x = 2^(1/3) sqrt(sigma) / rho^(4/3), beta = 0.0042       (Becke 1988)
//  VWN5:   rho eps_c(r_s), paramagnetic fit with A = 0.0310907, x0 = -0.10498,
//          b = 3.72744, c = 12.9352, x = sqrt(r_s)                 (VWN 1980)
//  LYP:    -a rho/(1 + d r) - a b E/(1 + d r) [C_F rho - rho^(-5/3) sigma (1/24 + 7 delta/72)],
//          r = rho^(-1/3), E = exp(-c r), delta = c r + d r/(1 + d r)
//          (Lee-Yang-Parr 1988 in the Miehlich et al. 1989 form)
// Points with rho < 1e-10 contribute nothing; sigma is floored at 1e-20.
#pragma once
#include <cuda_runtime.h>

namespace xc {

template <typename T> __host__ __device__ __forceinline__ T cbrt_(T x);
template <> __host__ __device__ __forceinline__ double cbrt_(double x) { return cbrt(x); }
template <> __host__ __device__ __forceinline__ float cbrt_(float x) { return cbrtf(x); }
template <typename T> __host__ __device__ __forceinline__ T log_(T x);
template <> __host__ __device__ __forceinline__ double log_(double x) { return log(x); }
template <> __host__ __device__ __forceinline__ float log_(float x) { return logf(x); }
template <typename T> __host__ __device__ __forceinline__ T atan_(T x);
template <> __host__ __device__ __forceinline__ double atan_(double x) { return atan(x); }
template <> __host__ __device__ __forceinline__ float atan_(float x) { return atanf(x); }
template <typename T> __host__ __device__ __forceinline__ T asinh_(T x);
template <> __host__ __device__ __forceinline__ double asinh_(double x) { return asinh(x); }
template <> __host__ __device__ __forceinline__ float asinh_(float x) { return asinhf(x); }
template <typename T> __host__ __device__ __forceinline__ T exp_(T x);
template <> __host__ __device__ __forceinline__ double exp_(double x) { return exp(x); }
template <> __host__ __device__ __forceinline__ float exp_(float x) { return expf(x); }
template <typename T> __host__ __device__ __forceinline__ T sqrt_(T x);
template <> __host__ __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
template <> __host__ __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }

constexpr double RHO_CUT = 1e-10;
constexpr double SIGMA_FLOOR = 1e-20;

template <typename T>
__host__ __device__ __forceinline__ void b3lyp(T rho, T sigma, T &e, T &vr, T &vs) {
    if (!(rho >= (T)RHO_CUT)) {
        e = vr = vs = (T)0;
        return;
    }
    if (sigma < (T)SIGMA_FLOOR) sigma = (T)SIGMA_FLOOR;
    const T r13 = cbrt_(rho);          // rho^(1/3)
    const T rm13 = (T)1 / r13;         // rho^(-1/3)
    const T r43 = rho * r13;           // rho^(4/3)
    const T rm43 = rm13 / rho;         // rho^(-4/3)

    // ---- Slater (weight 1 - a0 = 0.80):  C_x = (3/4)(3/pi)^(1/3)
    const T Cx = (T)0.73855876638202240588;
    T e_s = -Cx * r43;
    T v_s = -(T)(4.0 / 3.0) * Cx * r13;

    // ---- B88 gradient correction (weight 0.72)
    const T beta = (T)0.0042;
    const T K = (T)1.2599210498948731648 * beta;  // 2^(1/3) beta
    const T sq = sqrt_(sigma);
    const T x = (T)1.2599210498948731648 * sq * rm43;
    const T ash = asinh_(x);
    const T g = (T)1 + (T)6 * beta * x * ash;
    const T gp = (T)6 * beta * (ash + x / sqrt_((T)1 + x * x));
    const T ig = (T)1 / g;
    T e_b = -K * sigma * rm43 * ig;
    T vr_b = (T)(4.0 / 3.0) * K * sigma * rm43 / rho * (ig - x * gp * ig * ig);
    T vs_b = -K * rm43 * (ig - (T)0.5 * x * gp * ig * ig);

    // ---- VWN5 (weight 0.19), r_s = (3/(4 pi rho))^(1/3) = 0.62035049089940001667 rho^(-1/3)
    const T A = (T)0.0310907, x0 = (T)-0.10498, bv = (T)3.72744, cv = (T)12.9352;
    const T Qv = (T)6.15199081975908;        // sqrt(4c - b^2)
    const T X0 = x0 * x0 + bv * x0 + cv;
    const T rs = (T)0.62035049089940001667 * rm13;
    const T xs = sqrt_(rs);
    const T Xx = xs * xs + bv * xs + cv;
    const T at = atan_(Qv / ((T)2 * xs + bv));
    const T l1 = log_(xs * xs / Xx);
    const T l2 = log_((xs - x0) * (xs - x0) / Xx);
    const T eps_c = A * (l1 + (T)2 * bv / Qv * at - bv * x0 / X0 * (l2 + (T)2 * (bv + (T)2 * x0) / Qv * at));
    const T dXx = (T)2 * xs + bv;
    const T deps_dx = A * ((T)2 / xs - dXx / Xx - bv / Xx
                           - bv * x0 / X0 * ((T)2 / (xs - x0) - dXx / Xx - (bv + (T)2 * x0) / Xx));
    // d eps/d rho = deps/dx * dx/drs * drs/drho = deps_dx * (1/(2x)) * (-rs/(3 rho))
    T e_v = rho * eps_c;
    T v_v = eps_c - deps_dx * xs / (T)6;  // eps - (rs/3) deps/drs, deps/drs = deps_dx / (2x)

    // ---- LYP (weight 0.81)
    const T la = (T)0.04918, lb = (T)0.132, lc = (T)0.2533, ld = (T)0.349;
    const T CF = (T)2.8712340001881918;      // (3/10)(3 pi^2)^(2/3)
    const T den = (T)1 / ((T)1 + ld * rm13);
    const T Ec = exp_(-lc * rm13);
    const T delta = lc * rm13 + ld * rm13 * den;
    const T h = (T)(1.0 / 24.0) + (T)(7.0 / 72.0) * delta;
    const T rm53 = rm43 * rm13;                       // rho^(-5/3)
    const T rm83 = rm53 / rho;                        // rho^(-8/3)
    T e_l = -la * rho * den - la * lb * Ec * den * (CF * rho - rm53 * sigma * h);
    T vs_l = la * lb * Ec * den * rm53 * h;
    T vr_l = -la * den - la * ld * rm13 * den * den / (T)3
             - la * lb * CF * Ec * den * ((T)1 + lc * rm13 / (T)3 + ld * rm13 * den / (T)3)
             + la * lb * sigma * Ec * den * rm83 *
                   (h * (lc * rm13 / (T)3 + ld * rm13 * den / (T)3 - (T)(5.0 / 3.0))
                    - (T)(7.0 / 216.0) * rm13 * (lc + ld * den - ld * ld * rm13 * den * den));

    e = (T)0.80 * e_s + (T)0.72 * e_b + (T)0.19 * e_v + (T)0.81 * e_l;
    vr = (T)0.80 * v_s + (T)0.72 * vr_b + (T)0.19 * v_v + (T)0.81 * vr_l;
    vs = (T)0.72 * vs_b + (T)0.81 * vs_l;
}

// The same functional in three independent weighted parts (0: 0.80 Slater +
// 0.72 B88, 1: 0.19 VWN5, 2: 0.81 LYP) whose sum is b3lyp(); lets three warp
// groups evaluate one block of points in parallel.  Same formulas, same
// cutoffs; only the order of the final sum differs.
template <typename T>
__host__ __device__ __forceinline__ void b3lyp_part(int part, T rho, T sigma, T &e, T &vr, T &vs) {
    e = vr = vs = (T)0;
    if (!(rho >= (T)RHO_CUT)) return;
    if (sigma < (T)SIGMA_FLOOR) sigma = (T)SIGMA_FLOOR;
    const T r13 = cbrt_(rho);
    const T rm13 = (T)1 / r13;
    const T rm43 = rm13 / rho;
    if (part == 0) {
        const T r43 = rho * r13;
        const T Cx = (T)0.73855876638202240588;
        const T beta = (T)0.0042;
        const T K = (T)1.2599210498948731648 * beta;
        const T sq = sqrt_(sigma);
        const T x = (T)1.2599210498948731648 * sq * rm43;
        const T ash = asinh_(x);
        const T g = (T)1 + (T)6 * beta * x * ash;
        const T gp = (T)6 * beta * (ash + x / sqrt_((T)1 + x * x));
        const T ig = (T)1 / g;
        e = (T)0.80 * (-Cx * r43) + (T)0.72 * (-K * sigma * rm43 * ig);
        vr = (T)0.80 * (-(T)(4.0 / 3.0) * Cx * r13) +
             (T)0.72 * ((T)(4.0 / 3.0) * K * sigma * rm43 / rho * (ig - x * gp * ig * ig));
        vs = (T)0.72 * (-K * rm43 * (ig - (T)0.5 * x * gp * ig * ig));
    } else if (part == 1) {
        const T A = (T)0.0310907, x0 = (T)-0.10498, bv = (T)3.72744, cv = (T)12.9352;
        const T Qv = (T)6.15199081975908;
        const T X0 = x0 * x0 + bv * x0 + cv;
        const T rs = (T)0.62035049089940001667 * rm13;
        const T xs = sqrt_(rs);
        const T Xx = xs * xs + bv * xs + cv;
        const T at = atan_(Qv / ((T)2 * xs + bv));
        const T l1 = log_(xs * xs / Xx);
        const T l2 = log_((xs - x0) * (xs - x0) / Xx);
        const T eps_c = A * (l1 + (T)2 * bv / Qv * at - bv * x0 / X0 * (l2 + (T)2 * (bv + (T)2 * x0) / Qv * at));
        const T dXx = (T)2 * xs + bv;
        const T deps_dx = A * ((T)2 / xs - dXx / Xx - bv / Xx
                               - bv * x0 / X0 * ((T)2 / (xs - x0) - dXx / Xx - (bv + (T)2 * x0) / Xx));
        e = (T)0.19 * (rho * eps_c);
        vr = (T)0.19 * (eps_c - deps_dx * xs / (T)6);
    } else {
        const T la = (T)0.04918, lb = (T)0.132, lc = (T)0.2533, ld = (T)0.349;
        const T CF = (T)2.8712340001881918;
        const T den = (T)1 / ((T)1 + ld * rm13);
        const T Ec = exp_(-lc * rm13);
        const T delta = lc * rm13 + ld * rm13 * den;
        const T h = (T)(1.0 / 24.0) + (T)(7.0 / 72.0) * delta;
        const T rm53 = rm43 * rm13;
        const T rm83 = rm53 / rho;
        e = (T)0.81 * (-la * rho * den - la * lb * Ec * den * (CF * rho - rm53 * sigma * h));
        vs = (T)0.81 * (la * lb * Ec * den * rm53 * h);
        vr = (T)0.81 * (-la * den - la * ld * rm13 * den * den / (T)3
                        - la * lb * CF * Ec * den * ((T)1 + lc * rm13 / (T)3 + ld * rm13 * den / (T)3)
                        + la * lb * sigma * Ec * den * rm83 *
                              (h * (lc * rm13 / (T)3 + ld * rm13 * den / (T)3 - (T)(5.0 / 3.0))
                               - (T)(7.0 / 216.0) * rm13 * (lc + ld * den - ld * ld * rm13 * den * den)));
    }
}

}  // namespace xc
