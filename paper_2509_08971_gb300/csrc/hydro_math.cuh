// Device arithmetic of the hydro stage: ideal-gas closure, minmod limiter,
// piecewise-linear face states and the HLLC flux.
//
// Physics: Eq. "conservative form" (S = 0) and Eq. "fluxes" of the HARD paper
// with p = (gamma-1) e; numerics of Sec. 2.2.2 with minmod-limited PLM face
// states and the HLLC solver (Toro, ch. 10) with Davis wave-speed bounds.
//
// The FP64 functions evaluate every formula in one fixed operation order and
// are compiled without FMA contraction, so each + - * / sqrt is one IEEE
// operation.  The FP32 functions trade that for fewer instructions
// (reciprocals, the one-sided branch-free HLLC form).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "vec2.cuh"

namespace hh {

constexpr int NF = 5;

// Rotated-frame component order per physical axis: (normal, tangent 1,
// tangent 2) as indices into the momentum / velocity slots 1..3.
template <int AX> struct Rot;
template <> struct Rot<0> { static constexpr int n = 1, t1 = 2, t2 = 3; };
template <> struct Rot<1> { static constexpr int n = 2, t1 = 1, t2 = 3; };
template <> struct Rot<2> { static constexpr int n = 3, t1 = 1, t2 = 2; };

// ---------------------------------------------------------------- minmod --
// Zero unless both slopes have the same strict sign; otherwise the smaller
// magnitude (a on a tie).  A sign test, so tiny slopes never underflow.
__device__ __forceinline__ double minmod(double a, double b) {
    if (a > 0.0 && b > 0.0) return (a <= b) ? a : b;
    if (a < 0.0 && b < 0.0) return (-a <= -b) ? a : b;
    return 0.0;
}
__device__ __forceinline__ float minmod(float a, float b) { return vminmod(a, b); }

// ------------------------------------------------- fused multiply-adds --
// Both element types are compiled without automatic FMA contraction, so the
// rounding of every expression is fixed by the source and identical in every
// kernel that uses these functions.  FP64 keeps a*b + c as two roundings (the
// oracle's order); FP32 fuses it explicitly.
__device__ __forceinline__ double madd(double a, double b, double c) { return a * b + c; }
__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }

// acc - diff / dx: FP64 divides (oracle order), FP32 multiplies by the
// precomputed 1/dx it is handed instead.
__device__ __forceinline__ double sub_over_dx(double acc, double diff, double dx) {
    return acc - diff / dx;
}
__device__ __forceinline__ float sub_over_dx(float acc, float diff, float inv_dx) {
    return fmaf(-diff, inv_dx, acc);
}

// ------------------------------------------------------- closure helpers --
// Conserved -> primitive W = (rho, u, v, w, p), p = (gamma-1)(E - rho|v|^2/2).
__device__ __forceinline__ void cons_to_prim(const double U[NF], double gm1, double W[NF]) {
    double rho = U[0];
    double u = U[1] / rho;
    double v = U[2] / rho;
    double w = U[3] / rho;
    double kin = 0.5 * rho * (u * u + v * v + w * w);
    W[0] = rho; W[1] = u; W[2] = v; W[3] = w;
    W[4] = gm1 * (U[4] - kin);
}
__device__ __forceinline__ void cons_to_prim(const float U[NF], float gm1, float W[NF]) {
    float rho = U[0];
    float ir = vrcp(rho);
    float u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
    float kin = 0.5f * fmaf(U[1], u, fmaf(U[2], v, U[3] * w));
    W[0] = rho; W[1] = u; W[2] = v; W[3] = w;
    W[4] = gm1 * (U[4] - kin);
}

// Non-physical test on a primitive state (also catches NaN).
template <typename T>
__device__ __forceinline__ bool nonphys(const T W[NF]) {
    return !(W[0] > T(0)) || !(W[4] > T(0));
}

// ------------------------------------------------------------------ HLLC --
// FP64: the four-branch textbook form, one fixed evaluation order.
// Wn = (rho, un, t1, t2, p) in the frame whose normal is component 1.
__device__ __forceinline__ void hllc_normal(const double WL[NF], const double WR[NF],
                                            double gamma, double gm1, double /*igm1*/,
                                            double F[NF]) {
    double UL[NF], FL[NF], UR[NF], FR[NF];
    {
        double rho = WL[0], un = WL[1], t1 = WL[2], t2 = WL[3], p = WL[4];
        double E = p / gm1 + 0.5 * rho * (un * un + t1 * t1 + t2 * t2);
        UL[0] = rho; UL[1] = rho * un; UL[2] = rho * t1; UL[3] = rho * t2; UL[4] = E;
        FL[0] = rho * un; FL[1] = rho * un * un + p; FL[2] = rho * un * t1;
        FL[3] = rho * un * t2; FL[4] = (E + p) * un;
    }
    {
        double rho = WR[0], un = WR[1], t1 = WR[2], t2 = WR[3], p = WR[4];
        double E = p / gm1 + 0.5 * rho * (un * un + t1 * t1 + t2 * t2);
        UR[0] = rho; UR[1] = rho * un; UR[2] = rho * t1; UR[3] = rho * t2; UR[4] = E;
        FR[0] = rho * un; FR[1] = rho * un * un + p; FR[2] = rho * un * t1;
        FR[3] = rho * un * t2; FR[4] = (E + p) * un;
    }
    double rL = WL[0], uL = WL[1], pL = WL[4];
    double rR = WR[0], uR = WR[1], pR = WR[4];
    double cL = sqrt(gamma * pL / rL);
    double cR = sqrt(gamma * pR / rR);
    double SL = fmin(uL - cL, uR - cR);
    double SR = fmax(uL + cL, uR + cR);
    double Sstar = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR))
                 / (rL * (SL - uL) - rR * (SR - uR));
    if (0.0 <= SL) {
#pragma unroll
        for (int f = 0; f < NF; ++f) F[f] = FL[f];
        return;
    }
    if (SR <= 0.0) {
#pragma unroll
        for (int f = 0; f < NF; ++f) F[f] = FR[f];
        return;
    }
    bool left = Sstar >= 0.0;
    double r = left ? rL : rR, u = left ? uL : uR, p = left ? pL : pR;
    double t1 = left ? WL[2] : WR[2], t2 = left ? WL[3] : WR[3];
    double SK = left ? SL : SR;
    double fac = r * (SK - u) / (SK - Sstar);
    double Us[NF];
    Us[0] = fac;
    Us[1] = fac * Sstar;
    Us[2] = fac * t1;
    Us[3] = fac * t2;
    double EK = left ? UL[4] : UR[4];
    Us[4] = fac * (EK / r + (Sstar - u) * (Sstar + p / (r * (SK - u))));
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        double UKf = left ? UL[f] : UR[f];
        double FKf = left ? FL[f] : FR[f];
        F[f] = FKf + SK * (Us[f] - UKf);
    }
}

// FP32: the one-sided form of vec2.cuh (hllc_core), F = F_K + s (U*_K - U_K),
// with s = 0 reproducing the supersonic branches without a branch.
__device__ __forceinline__ void hllc_normal(const float WL[NF], const float WR[NF], float gamma,
                                            float /*gm1*/, float igm1, float F[NF]) {
    hllc_core<float>(WL, WR, gamma, igm1, F);
}

// Face flux through a face whose normal is physical axis AX, from the
// primitives of the four cells i-1, i, i+1, i+2 around the face i+1/2:
//   dq_m = minmod(q_m - q_{m-1}, q_{m+1} - q_m)
//   q_L = q_i + dq_i/2,   q_R = q_{i+1} - dq_{i+1}/2,   F = HLLC(q_L, q_R).
template <int AX, typename T>
__device__ __forceinline__ void hllc_axis(const T qL[NF], const T qR[NF], T gamma, T gm1, T igm1,
                                          T F[NF]) {
    using R = Rot<AX>;
    T WL[NF] = {qL[0], qL[R::n], qL[R::t1], qL[R::t2], qL[4]};
    T WR[NF] = {qR[0], qR[R::n], qR[R::t1], qR[R::t2], qR[4]};
    T Fn[NF];
    hllc_normal(WL, WR, gamma, gm1, igm1, Fn);
    F[0] = Fn[0];
    F[R::n] = Fn[1];
    F[R::t1] = Fn[2];
    F[R::t2] = Fn[3];
    F[4] = Fn[4];
}

template <int AX>
__device__ __forceinline__ void face_flux4(const double q0[NF], const double q1[NF],
                                           const double q2[NF], const double q3[NF], double gamma,
                                           double gm1, double igm1, double F[NF]) {
    double qL[NF], qR[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        double dqi = minmod(q1[f] - q0[f], q2[f] - q1[f]);
        double dqi1 = minmod(q2[f] - q1[f], q3[f] - q2[f]);
        qL[f] = madd(0.5, dqi, q1[f]);
        qR[f] = madd(-0.5, dqi1, q2[f]);
    }
    hllc_axis<AX>(qL, qR, gamma, gm1, igm1, F);
}
template <int AX>
__device__ __forceinline__ void face_flux4(const float q0[NF], const float q1[NF],
                                           const float q2[NF], const float q3[NF], float gamma,
                                           float gm1, float igm1, float F[NF]) {
    float qL[NF], qR[NF];
    plm_faces<float>(q0, q1, q2, q3, qL, qR);
    hllc_axis<AX>(qL, qR, gamma, gm1, igm1, F);
}

// Signal rate of one cell: sum over the active axes of (|v_d| + c)/dx_d.
// `act` and `dx` are indexed by physical axis; summed in physical order.
__device__ __forceinline__ double cell_rate(const double W[NF], double gamma, const bool act[3],
                                            const double dx[3]) {
    double cs = sqrt(gamma * W[4] / W[0]);
    double r = 0.0;
    if (act[0]) r += (fabs(W[1]) + cs) / dx[0];
    if (act[1]) r += (fabs(W[2]) + cs) / dx[1];
    if (act[2]) r += (fabs(W[3]) + cs) / dx[2];
    return r;
}
__device__ __forceinline__ float cell_rate(const float W[NF], float gamma, const bool act[3],
                                           const float inv_dx[3]) {
    float cs = vsqrt(gamma * W[4] * vrcp(W[0]));
    float r = 0.0f;
    if (act[0]) r = fmaf(fabsf(W[1]) + cs, inv_dx[0], r);
    if (act[1]) r = fmaf(fabsf(W[2]) + cs, inv_dx[1], r);
    if (act[2]) r = fmaf(fabsf(W[3]) + cs, inv_dx[2], r);
    return r;
}

// Order-preserving bits of a non-negative rate (NaN sorts above +inf).
__device__ __forceinline__ unsigned long long rate_bits(double r) {
    return (unsigned long long)__double_as_longlong(r);
}
__device__ __forceinline__ unsigned long long rate_bits(float r) {
    // widen exactly to double so both element types share one slot format
    return (unsigned long long)__double_as_longlong((double)r);
}

}  // namespace hh
