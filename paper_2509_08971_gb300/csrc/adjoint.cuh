// Adjoint (vector-Jacobian product) of one Runge-Kutta stage.
//
// A stage is  U_out = a U0 + b (U_c + dt L(U_c))  with L the flux difference
// of Sec. 2.2.2 (stage 1: a = 0, b = 1; stage 2: a = b = 1/2).  Given the
// cotangent G of U_out, the stage's VJP is
//     dU_c  = b G + J_L(U_c)^T lambda,     lambda = b dt G
//     dU0   = a G
//     dgamma = (dL/dgamma)^T lambda
// J_L^T lambda is assembled face by face.  L_i = -sum_d (F_{i+1/2} - F_{i-1/2})/dx_d,
// so the cotangent of the face flux F_{m-1/2} between cells m-1 and m is
//     Fbar = (lambda_m - lambda_{m-1}) / dx          (lambda of a ghost cell = 0).
// Each face then runs its flux backwards: HLLC (the region the forward pass
// took; Davis min/max and minmod pass the cotangent to the argument they
// selected), the piecewise-linear face states, and lands on the primitive
// states of its four stencil cells, mapped back through the boundary map (a
// reflecting wall negates the normal velocity).  A per-cell pass then applies
// the transpose of the conserved-to-primitive map and the RK combine.
//
// gamma enters through p = (gamma-1)(E - rho|v|^2/2) of every cell, the
// sound speeds c = sqrt(gamma p / rho) and the face energies
// E = p/(gamma-1) + rho|v|^2/2.
#pragma once
#include "hydro_math.cuh"
#include "pdl.h"
#include "stage_kernel.cuh"

namespace hh {

// The face and cell passes are launched as programmatic dependents (pdl.h):
// each waits for the pass before it on the device and triggers the next one
// when its loop is done.
// The primitive cotangent accumulator holds one 8-slot record per cell (5
// used), so that FP32 contributions land with one 16-byte vector reduction
// plus one scalar reduction.
constexpr int GW_STRIDE = 8;

__device__ __forceinline__ void accumulate_cell(float* rec, const float v[NF]) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(rec), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3])
                 : "memory");
    atomicAdd(rec + 4, v[4]);
}
__device__ __forceinline__ void accumulate_cell(double* rec, const double v[NF]) {
#pragma unroll
    for (int f = 0; f < NF; ++f) atomicAdd(rec + f, v[f]);
}

// Division and square root of the adjoint: FP64 exact IEEE operations (the
// order of the formulas below is the oracle transcription's); FP32 through the
// approximate reciprocal and square root that the FP32 forward stage uses.
__device__ __forceinline__ double adiv(double a, double b) { return a / b; }
__device__ __forceinline__ float adiv(float a, float b) { return a * vrcp(b); }
__device__ __forceinline__ double asqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float asqrt(float a) { return vsqrt(a); }

template <typename T>
struct AdjArgs {
    const T* Uc;          // state the flux difference is taken of
    const T* gout;        // cotangent of the stage output
    T lam;                // lambda = lam * gout  (b * dt)
    T* gW;                // primitive cotangent accumulator, one record of GW_STRIDE per cell
    double* g_gamma;      // accumulated d/dgamma
    long long N;
    int n[3];             // kernel-axis extents
    int bc_lo[3], bc_hi[3];
    T gamma, gm1;
    T dxk[3];             // per kernel axis: dx (FP64) or 1/dx (FP32)
    // z faces of kind BC_HALO (a slab of a decomposed mesh): the ghost planes
    // of Uc below / above the slab ([5][2][ny][nx], z fastest-but-one) and the
    // accumulators of the primitive cotangent the faces scatter onto them
    // ([2][ny][nx] records of GW_STRIDE)
    const T* zg[2];
    T* gwg[2];
};

// Which argument minmod selected: 0 none, 1 a, 2 b (the forward rule).
template <typename T>
__device__ __forceinline__ int minmod_sel(T a, T b) {
    if (a > T(0) && b > T(0)) return (a <= b) ? 1 : 2;
    if (a < T(0) && b < T(0)) return (-a <= -b) ? 1 : 2;
    return 0;
}

// Reverse of the physical normal flux F(W) = (r u, r u^2 + p, r u v, r u w, (E+p) u),
// E = p/(gamma-1) + r|v|^2/2, accumulated into Wb and gb.
template <typename T>
__device__ __forceinline__ void flux_vjp(const T W[NF], T gamma, const T Fb[NF], T Wb[NF],
                                         T& Eb) {
    const T r = W[0], u = W[1], v = W[2], w = W[3], p = W[4];
    const T g1 = gamma - T(1);
    const T E = adiv(p, g1) + T(0.5) * r * (u * u + v * v + w * w);
    Wb[0] += Fb[0] * u + Fb[1] * u * u + Fb[2] * u * v + Fb[3] * u * w;
    Wb[1] += Fb[0] * r + Fb[1] * T(2) * r * u + Fb[2] * r * v + Fb[3] * r * w + Fb[4] * (E + p);
    Wb[2] += Fb[2] * r * u;
    Wb[3] += Fb[3] * r * u;
    Wb[4] += Fb[1] + Fb[4] * u;
    Eb += Fb[4] * u;
}

// Reverse of E = p/(gamma-1) + r|v|^2/2.
template <typename T>
__device__ __forceinline__ void energy_vjp(const T W[NF], T gamma, T Eb, T Wb[NF], T& gb) {
    const T r = W[0], u = W[1], v = W[2], w = W[3], p = W[4];
    const T g1 = gamma - T(1);
    Wb[0] += Eb * T(0.5) * (u * u + v * v + w * w);
    Wb[1] += Eb * r * u;
    Wb[2] += Eb * r * v;
    Wb[3] += Eb * r * w;
    Wb[4] += adiv(Eb, g1);
    gb -= adiv(Eb * p, g1 * g1);
}

// Reverse of c = sqrt(gamma p / r).
template <typename T>
__device__ __forceinline__ void sound_vjp(const T W[NF], T gamma, T c, T cb, T Wb[NF], T& gb) {
    const T r = W[0], p = W[4];
    const T zb = adiv(cb, T(2) * c);         // z = gamma p / r
    gb += adiv(zb * p, r);
    Wb[4] += adiv(zb * gamma, r);
    Wb[0] -= adiv(zb * gamma * p, r * r);
}

// HLLC on rotated states (normal along slot 1): recompute the forward pass,
// then push Fb back onto WLb, WRb (overwritten) and gb (added).
template <typename T>
__device__ void hllc_vjp(const T WL[NF], const T WR[NF], T gamma, const T Fb[NF], T WLb[NF],
                         T WRb[NF], T& gb) {
#pragma unroll
    for (int f = 0; f < NF; ++f) WLb[f] = WRb[f] = T(0);
    const T g1 = gamma - T(1);
    const T rL = WL[0], uL = WL[1], pL = WL[4];
    const T rR = WR[0], uR = WR[1], pR = WR[4];
    const T cL = asqrt(adiv(gamma * pL, rL)), cR = asqrt(adiv(gamma * pR, rR));
    const T aL = uL - cL, aR = uR - cR, bL = uL + cL, bR = uR + cR;
    const bool minL = aL <= aR, maxL = bL >= bR;     // which side set S_L / S_R
    const T SL = minL ? aL : aR;
    const T SR = maxL ? bL : bR;
    T ELb = T(0), ERb = T(0);
    if (T(0) <= SL) {                                // supersonic to the right: F = F_L
        flux_vjp(WL, gamma, Fb, WLb, ELb);
        energy_vjp(WL, gamma, ELb, WLb, gb);
        return;
    }
    if (SR <= T(0)) {                                // supersonic to the left: F = F_R
        flux_vjp(WR, gamma, Fb, WRb, ERb);
        energy_vjp(WR, gamma, ERb, WRb, gb);
        return;
    }
    const T mL = rL * (SL - uL), mR = rR * (SR - uR);
    const T num = pR - pL + mL * uL - mR * uR;
    const T den = mL - mR;
    const T Ss = adiv(num, den);
    const bool left = Ss >= T(0);
    const T* WK = left ? WL : WR;
    T* WKb = left ? WLb : WRb;
    const T rK = WK[0], uK = WK[1], vK = WK[2], wK = WK[3], pK = WK[4];
    const T EK = adiv(pK, g1) + T(0.5) * rK * (uK * uK + vK * vK + wK * wK);
    const T SK = left ? SL : SR;
    const T mK = left ? mL : mR;
    const T D = SK - Ss;
    const T fac = adiv(mK, D);
    const T A = Ss - uK;
    const T q = adiv(pK, mK);
    const T Bq = Ss + q;
    const T es = adiv(EK, rK) + A * Bq;
    const T Us[NF] = {fac, fac * Ss, fac * vK, fac * wK, fac * es};
    const T UK[NF] = {rK, rK * uK, rK * vK, rK * wK, EK};
    // F = F_K + S_K (U* - U_K)
    T EKb = T(0), SKb = T(0), Ssb = T(0), mKb = T(0);
    flux_vjp(WK, gamma, Fb, WKb, EKb);
#pragma unroll
    for (int f = 0; f < NF; ++f) SKb += Fb[f] * (Us[f] - UK[f]);
    // U_K = (r, r u, r v, r w, E)
    WKb[0] += -SK * (Fb[0] + Fb[1] * uK + Fb[2] * vK + Fb[3] * wK);
    WKb[1] += -SK * Fb[1] * rK;
    WKb[2] += -SK * Fb[2] * rK;
    WKb[3] += -SK * Fb[3] * rK;
    EKb += -SK * Fb[4];
    // U* = fac (1, S*, v, w, es)
    const T facb = SK * (Fb[0] + Fb[1] * Ss + Fb[2] * vK + Fb[3] * wK + Fb[4] * es);
    Ssb += SK * Fb[1] * fac;
    WKb[2] += SK * Fb[2] * fac;
    WKb[3] += SK * Fb[3] * fac;
    const T esb = SK * Fb[4] * fac;
    // es = E/r + A Bq
    EKb += adiv(esb, rK);
    WKb[0] -= adiv(esb * EK, rK * rK);
    const T Ab = esb * Bq, Bqb = esb * A;
    Ssb += Bqb;                                      // Bq = S* + q
    WKb[4] += adiv(Bqb, mK);                         // q = p / m
    mKb -= adiv(Bqb * pK, mK * mK);
    Ssb += Ab;                                       // A = S* - u
    WKb[1] -= Ab;
    mKb += adiv(facb, D);                            // fac = m / D
    const T Db = adiv(-facb * mK, D * D);
    SKb += Db;                                       // D = S_K - S*
    Ssb -= Db;
    energy_vjp(WK, gamma, EKb, WKb, gb);
    // S* = num / den
    const T numb = adiv(Ssb, den);
    const T denb = adiv(-Ssb * Ss, den);
    T mLb = denb + numb * uL + (left ? mKb : T(0));
    T mRb = -denb - numb * uR + (left ? T(0) : mKb);
    WRb[4] += numb;
    WLb[4] -= numb;
    WLb[1] += numb * mL;
    WRb[1] -= numb * mR;
    T SLb = left ? SKb : T(0), SRb = left ? T(0) : SKb;
    // m_L = r_L (S_L - u_L), m_R = r_R (S_R - u_R)
    WLb[0] += mLb * (SL - uL);
    SLb += mLb * rL;
    WLb[1] -= mLb * rL;
    WRb[0] += mRb * (SR - uR);
    SRb += mRb * rR;
    WRb[1] -= mRb * rR;
    // Davis bounds
    T cLb = T(0), cRb = T(0);
    if (minL) { WLb[1] += SLb; cLb -= SLb; } else { WRb[1] += SLb; cRb -= SLb; }
    if (maxL) { WLb[1] += SRb; cLb += SRb; } else { WRb[1] += SRb; cRb += SRb; }
    sound_vjp(WL, gamma, cL, cLb, WLb, gb);
    sound_vjp(WR, gamma, cR, cRb, WRb, gb);
}

// The reverse of one face's flux along physical axis PA: from the primitives
// q of its four stencil cells (boundary map and reflections applied), the
// lambdas of the two cells it separates (zero for a cell outside the mesh)
// and the kernel-axis width parameter, the cotangents qb of the four stencil
// primitives (reflections not yet undone) and the face's explicit d/dgamma.
template <typename T, int PA>
__device__ __forceinline__ void face_vjp_core(const T q[4][NF], const T ll[NF], const T lr[NF],
                                              T dxk, T gamma, T qb[4][NF], T& gb) {
    using R = Rot<PA>;
    // face flux cotangent (lambda_m - lambda_{m-1}) / dx
    T Fb[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) Fb[f] = sub_over_dx(T(0), ll[f] - lr[f], dxk);
    // forward face states, remembering the minmod selections
    T qL[NF], qR[NF];
    int s1[NF], s2[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const T d0 = q[1][f] - q[0][f], d1 = q[2][f] - q[1][f], d2 = q[3][f] - q[2][f];
        s1[f] = minmod_sel(d0, d1);
        s2[f] = minmod_sel(d1, d2);
        const T m1 = s1[f] == 1 ? d0 : (s1[f] == 2 ? d1 : T(0));
        const T m2 = s2[f] == 1 ? d1 : (s2[f] == 2 ? d2 : T(0));
        qL[f] = madd(T(0.5), m1, q[1][f]);
        qR[f] = madd(T(-0.5), m2, q[2][f]);
    }
    const T WL[NF] = {qL[0], qL[R::n], qL[R::t1], qL[R::t2], qL[4]};
    const T WR[NF] = {qR[0], qR[R::n], qR[R::t1], qR[R::t2], qR[4]};
    const T Fn_b[NF] = {Fb[0], Fb[R::n], Fb[R::t1], Fb[R::t2], Fb[4]};
    T WLb[NF], WRb[NF];
    gb = T(0);
    hllc_vjp(WL, WR, gamma, Fn_b, WLb, WRb, gb);
    T qLb[NF], qRb[NF];
    qLb[0] = WLb[0]; qLb[R::n] = WLb[1]; qLb[R::t1] = WLb[2]; qLb[R::t2] = WLb[3]; qLb[4] = WLb[4];
    qRb[0] = WRb[0]; qRb[R::n] = WRb[1]; qRb[R::t1] = WRb[2]; qRb[R::t2] = WRb[3]; qRb[4] = WRb[4];
    // face states backwards onto the four stencil primitives
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        qb[0][f] = T(0); qb[1][f] = qLb[f]; qb[2][f] = qRb[f]; qb[3][f] = T(0);
        const T s1b = T(0.5) * qLb[f], s2b = T(-0.5) * qRb[f];
        if (s1[f] == 1) { qb[1][f] += s1b; qb[0][f] -= s1b; }
        if (s1[f] == 2) { qb[2][f] += s1b; qb[1][f] -= s1b; }
        if (s2[f] == 1) { qb[2][f] += s2b; qb[1][f] -= s2b; }
        if (s2[f] == 2) { qb[3][f] += s2b; qb[2][f] -= s2b; }
    }
}

// The reverse of one face's contribution to L: the face between cells m-1
// and m along kernel axis KA (physical axis PA), at transverse coordinates
// c3 (c3[KA] = m), scattered onto its four stencil cells.
template <typename T, int KA, int PA>
__device__ __forceinline__ void face_vjp_one(const AdjArgs<T>& A, const int c3[3], double& gacc) {
    using R = Rot<PA>;
    const int na = A.n[KA];
    const int m = c3[KA];
    long long src[4];
    bool flip[4];
    int side[4];                                       // -1: a cell of this mesh; 0 / 1: ghost plane
    T q[4][NF];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        int c[3] = {c3[0], c3[1], c3[2]};
        const int cm = m - 2 + s;
        side[s] = -1;
        if (KA == 2 && ((cm < 0 && A.bc_lo[2] == BC_HALO) || (cm >= na && A.bc_hi[2] == BC_HALO))) {
            // a neighbouring slab's cell: planes -2, -1 / na, na+1 of the ghost buffers
            side[s] = cm < 0 ? 0 : 1;
            const int k = cm < 0 ? cm + 2 : cm - na;
            flip[s] = false;
            src[s] = ((long long)k * A.n[1] + c[1]) * A.n[0] + c[0];
            const long long gs = 2ll * A.n[1] * A.n[0];
            T U[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) U[f] = A.zg[side[s]][f * gs + src[s]];
            cons_to_prim(U, A.gm1, q[s]);
            continue;
        }
        c[KA] = bc_map(cm, na, A.bc_lo[KA], A.bc_hi[KA], flip[s]);
        src[s] = ((long long)c[2] * A.n[1] + c[1]) * A.n[0] + c[0];
        T U[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) U[f] = A.Uc[f * A.N + src[s]];
        if (flip[s]) U[R::n] = -U[R::n];
        cons_to_prim(U, A.gm1, q[s]);
    }
    T ll[NF], lr[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        lr[f] = m < na ? A.lam * A.gout[f * A.N + src[2]] : T(0);
        ll[f] = m > 0 ? A.lam * A.gout[f * A.N + src[1]] : T(0);
    }
    T qb[4][NF], gb;
    face_vjp_core<T, PA>(q, ll, lr, A.dxk[KA], A.gamma, qb, gb);
    gacc += (double)gb;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (flip[s]) qb[s][R::n] = -qb[s][R::n];
        const bool any = qb[s][0] != T(0) || qb[s][1] != T(0) || qb[s][2] != T(0) ||
                         qb[s][3] != T(0) || qb[s][4] != T(0);
        T* acc = side[s] < 0 ? A.gW : A.gwg[side[s]];
        if (any) accumulate_cell(acc + src[s] * GW_STRIDE, qb[s]);
    }
}

// All faces of a stage in one launch, one thread per face.  The index space
// is DIM copies (one per axis, axis slowest, so that a warp evaluates faces
// of one axis) of the cell grid extended by one along every active axis, x
// fastest (coalesced): the point (i0, i1, i2) of copy d owns the face of axis
// d on the low side of cell (i0, i1, i2) when the other two indices are in
// range.
// 128-thread blocks, seven per SM (72 registers in FP32): every face of a
// 256^2 mesh is resident at once, so the launch takes one pass of the VJP's
// long dependency chain instead of two.
constexpr int FACES_VJP_THREADS = 128;
template <typename T, int DIM, int PX, int PY>
__global__ void __launch_bounds__(FACES_VJP_THREADS, 7) faces_vjp_kernel(const AdjArgs<T> A) {
    griddep_wait();
    // 32-bit index arithmetic (the launcher keeps DIM * total below 2^31)
    const unsigned e0 = A.n[0] + 1, e1 = DIM >= 2 ? A.n[1] + 1 : 1, e2 = DIM >= 3 ? A.n[2] + 1 : 1;
    const unsigned total = e0 * e1 * e2;
    double gacc = 0.0;
    for (unsigned g = blockIdx.x * blockDim.x + threadIdx.x; g < DIM * total;
         g += gridDim.x * blockDim.x) {
        const unsigned axis = g / total;
        const unsigned e = g - axis * total;
        const unsigned row = e / e0;
        const int c3[3] = {(int)(e - row * e0), (int)(row % e1), (int)(row / e1)};
        const bool in0 = c3[0] < A.n[0], in1 = DIM < 2 || c3[1] < A.n[1];
        const bool in2 = DIM < 3 || c3[2] < A.n[2];
        if (axis == 0) {
            if (in1 && in2) face_vjp_one<T, 0, PX>(A, c3, gacc);
        } else if (axis == 1) {
            if (DIM >= 2 && in0 && in2) face_vjp_one<T, 1, PY>(A, c3, gacc);
        } else {
            if (DIM >= 3 && in0 && in1) face_vjp_one<T, 2, 2>(A, c3, gacc);
        }
    }
    griddep_launch_dependents();
    // block sum of the explicit d/dgamma, one atomic per block
    __shared__ double red[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gacc += __shfl_xor_sync(0xffffffffu, gacc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = gacc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        if (s != 0.0) atomicAdd(A.g_gamma, s);
    }
}

// Per cell: the transpose of the conserved-to-primitive map applied to the
// accumulated primitive cotangent (which it may clear after reading), plus the
// RK combine:
//     out_c  (=|+=)  b G + J_prim^T gW,      out0 = a G  (when out0 != null)
// and d/dgamma of p = (gamma-1)(E - kin): gW_p * p / (gamma - 1).
template <typename T>
__global__ void __launch_bounds__(256) cell_vjp_kernel(const T* Uc, T* gW, const T* G, T b, T a,
                                                       T* out_c, bool accumulate, T* out0,
                                                       long long N, T gamma, double* g_gamma,
                                                       bool clear_gW) {
    griddep_wait();
    double gacc = 0.0;
    const T g1 = gamma - T(1);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        // every load first (the stores below could alias them as far as the
        // compiler knows), so that the cell takes one round trip to memory
        T U[NF], W[NF], Wb[NF], Gc[NF], Oc[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            U[f] = Uc[f * N + c];
            Wb[f] = gW[c * GW_STRIDE + f];
            Gc[f] = G[f * N + c];
            Oc[f] = accumulate ? out_c[f * N + c] : T(0);
        }
        if (clear_gW) {
#pragma unroll
            for (int f = 0; f < NF; ++f) gW[c * GW_STRIDE + f] = T(0);   // ready for the next use
        }
        cons_to_prim(U, g1, W);
        const T r = W[0], u = W[1], v = W[2], w = W[3];
        T Ub[NF];
        Ub[1] = adiv(Wb[1], r) - Wb[4] * g1 * u;
        Ub[2] = adiv(Wb[2], r) - Wb[4] * g1 * v;
        Ub[3] = adiv(Wb[3], r) - Wb[4] * g1 * w;
        Ub[4] = Wb[4] * g1;
        Ub[0] = Wb[0] - adiv(Wb[1] * u + Wb[2] * v + Wb[3] * w, r) +
                Wb[4] * g1 * T(0.5) * (u * u + v * v + w * w);
        gacc += (double)adiv(Wb[4] * W[4], g1);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const T val = b * Gc[f] + Ub[f];
            out_c[f * N + c] = accumulate ? Oc[f] + val : val;
            if (out0) out0[f * N + c] = a * Gc[f];
        }
    }
    griddep_launch_dependents();
    __shared__ double red[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gacc += __shfl_xor_sync(0xffffffffu, gacc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = gacc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        if (s != 0.0) atomicAdd(g_gamma, s);
    }
}

// A neighbouring slab's ghost-plane accumulator added into this slab's
// accumulator: `from` ([2][ny][nx] records) lands on planes k0, k0+1.
template <typename T>
__global__ void __launch_bounds__(256) add_ghost_cotangent_kernel(T* gW, const T* from,
                                                                  long long plane_records, int k0) {
    const long long n = 2 * plane_records * GW_STRIDE;
    T* dst = gW + (long long)k0 * plane_records * GW_STRIDE;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] += from[i];
}

}  // namespace hh
