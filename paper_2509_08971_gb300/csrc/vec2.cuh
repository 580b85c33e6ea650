// FP32 arithmetic of the face flux, written once over a value type V with
// small operation helpers (vadd, vfma, vminmod, ...).  Every operation is a
// single IEEE operation with the rounding written in the source (explicit
// fmaf, single-instruction approximate reciprocal and square root), so each
// kernel that evaluates a face rounds it identically.  (Packed f32x2
// arithmetic rounds lane for lane like these scalar operations as long as the
// assembler is kept from contracting a packed product into a packed sum; it
// was measured in the stage kernel, bit-identical, and did not speed it up,
// so it is not used.)
//
// Formulas: minmod-limited PLM face states and the one-sided HLLC flux with
// Davis wave-speed bounds (see hydro_math.cuh for the statement).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hh {

// ---- arithmetic, scalar ----
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float vrcp(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float vrsqrt(float a) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float vsqrt(float a) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
// minmod: min(|a|,|b|) carrying the XOR of the signs is >= 0 exactly when the
// slopes agree; clamp at 0 and give it a's sign (three ALU operations)
__device__ __forceinline__ float vminmod(float a, float b) {
    float r;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return copysignf(fmaxf(r, 0.0f), a);
}
__device__ __forceinline__ bool vge0(float a) { return a >= 0.0f; }
__device__ __forceinline__ float vsel(bool c, float a, float b) { return c ? a : b; }

template <class V> __device__ __forceinline__ V splat(float a);
template <> __device__ __forceinline__ float splat<float>(float a) { return a; }

// ---- face states: q_L = q_i + dq_i/2, q_R = q_{i+1} - dq_{i+1}/2 ----
template <class V>
__device__ __forceinline__ void plm_faces(const V q0[5], const V q1[5], const V q2[5],
                                          const V q3[5], V qL[5], V qR[5]) {
    const V half = splat<V>(0.5f), mhalf = splat<V>(-0.5f);
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        const V d0 = vsub(q1[f], q0[f]);
        const V d1 = vsub(q2[f], q1[f]);
        const V d2 = vsub(q3[f], q2[f]);
        qL[f] = vfma(half, vminmod(d0, d1), q1[f]);
        qR[f] = vfma(mhalf, vminmod(d1, d2), q2[f]);
    }
}

// ---- one-sided HLLC on rotated states W = (rho, un, t1, t2, p) ----
//   F = F_K + s (U*_K - U_K), K = L if S* >= 0 else R,
//   s = min(S_L, 0) for K = L, max(S_R, 0) for K = R.
// Written with four reciprocal / reciprocal-square-root operations per face:
//   c_K = (gamma p_K) / sqrt(gamma p_K rho_K)               (= sqrt(gamma p_K / rho_K)),
//   S*  = [p_R - p_L + m_L u_L - m_R u_R] / (m_L - m_R),    m_K = rho_K (S_K - u_K),
//   f   = m_K / (S_K - S*)                                  (rho* of the star state),
//   f e* = [(S_K - u_K) E_K + (S* - u_K)(m_K S* + p_K)] / (S_K - S*),
//   F_t = F_rho t_K for both tangential components (the tangential velocity
//         is t_K on the whole K side of the contact, star state included),
// the energy term being the star energy rho_K (S_K-u_K)/(S_K-S*) [E_K/rho_K +
// (S*-u_K)(S* + p_K/(rho_K (S_K-u_K)))] with m_K / rho_K = S_K - u_K taken out.
// The root's argument is kept at or above the smallest normal number, so a
// zero pressure gives c = 0 rather than 0 * inf.
template <class V>
__device__ __forceinline__ void hllc_core(const V WL[5], const V WR[5], V gamma, V igm1,
                                          V F[5]) {
    const V zero = splat<V>(0.0f), half = splat<V>(0.5f), tiny = splat<V>(1.17549435e-38f);
    const V rL = WL[0], uL = WL[1], pL = WL[4];
    const V rR = WR[0], uR = WR[1], pR = WR[4];
    const V gpL = vmul(gamma, pL), gpR = vmul(gamma, pR);
    const V cL = vmul(gpL, vrsqrt(vmax(vmul(gpL, rL), tiny)));
    const V cR = vmul(gpR, vrsqrt(vmax(vmul(gpR, rR), tiny)));
    const V SL = vmin(vsub(uL, cL), vsub(uR, cR));
    const V SR = vmax(vadd(uL, cL), vadd(uR, cR));
    const V aL = vsub(SL, uL), aR = vsub(SR, uR);       // < 0, > 0
    const V mL = vmul(rL, aL), mR = vmul(rR, aR);
    const V num = vfma(vneg(mR), uR, vfma(mL, uL, vsub(pR, pL)));
    const V Sstar = vmul(num, vrcp(vsub(mL, mR)));
    const auto left = vge0(Sstar);
    const V r = vsel(left, rL, rR), u = vsel(left, uL, uR), p = vsel(left, pL, pR);
    const V t1 = vsel(left, WL[2], WR[2]), t2 = vsel(left, WL[3], WR[3]);
    const V m = vsel(left, mL, mR), a = vsel(left, aL, aR);
    const V SK = vsel(left, SL, SR);
    const V s = vsel(left, vmin(SL, zero), vmax(SR, zero));
    const V ke = vfma(u, u, vfma(t1, t1, vmul(t2, t2)));
    const V E = vfma(p, igm1, vmul(vmul(half, r), ke));
    const V r2 = vrcp(vsub(SK, Sstar));
    const V fac = vmul(m, r2);                          // rho_K (S_K - u_K) / (S_K - S*)
    const V mu = vmul(r, u);
    const V fes = vmul(r2, vfma(vsub(Sstar, u), vfma(m, Sstar, p), vmul(a, E)));
    const V dr = vsub(fac, r);
    F[0] = vfma(s, dr, mu);
    F[1] = vfma(s, vsub(vmul(fac, Sstar), mu), vfma(mu, u, p));
    F[2] = vmul(F[0], t1);                              // tangential momentum moves with the mass
    F[3] = vmul(F[0], t2);
    F[4] = vfma(s, vsub(fes, E), vmul(vadd(E, p), u));
}

}  // namespace hh
