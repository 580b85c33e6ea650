// Second scheme of the stage update: WENO5-Z face states of the primitives
// and the HLL flux (Sec. 2.2.2: the paper's own reconstruction and Riemann
// solver), three ghost layers per active axis.  Same mesh, boundary kinds,
// RK stage combine and epilogues as the PLM-minmod + HLLC kernels.
//
//   WENO5-Z (Borges, Carmona, Costa, Don 2008), value at the right face of
//   the middle cell of v0..v4 (cell averages):
//     candidates  p0 = (2 v0 - 7 v1 + 11 v2)/6, p1 = (-v1 + 5 v2 + 2 v3)/6,
//                 p2 = (2 v2 + 5 v3 - v4)/6
//     indicators  b0 = 13/12 (v0 - 2v1 + v2)^2 + 1/4 (v0 - 4v1 + 3v2)^2
//                 b1 = 13/12 (v1 - 2v2 + v3)^2 + 1/4 (v1 - v3)^2
//                 b2 = 13/12 (v2 - 2v3 + v4)^2 + 1/4 (3v2 - 4v3 + v4)^2
//     weights     a_k = d_k (1 + |b0 - b2| / (b_k + eps)), d = (1, 6, 3)/10,
//                 eps = 1e-30; value = sum a_k p_k / sum a_k
//   The right state of a face is the same function of the mirrored stencil.
//
//   HLL (Harten, Lax, van Leer 1983) with the Davis bounds
//     S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R):
//     F = F_L (0 <= S_L), F_R (S_R <= 0),
//         (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L) otherwise.
//
// FP64 evaluates every formula in the written order with IEEE division and
// square root (one rounding per operation, no contraction); FP32 multiplies
// by approximate reciprocals and square roots.
//
// Tiling: as stage_kernel (a TX x TY column marching its z-chunk), with a
// (TX+6) x (TY+6) primitive plane in shared memory and, along z, each thread
// holding its column's last six primitives in registers: plane j yields the
// z face between cells j-3 and j-2, and cell j-3 completes.
#pragma once
#include "stage_kernel.cuh"

namespace hh {

constexpr int WENO_G = 3;                 // ghost layers

// ---------------------------------------------------------------- WENO5-Z --
__device__ __forceinline__ double weno5z(double v0, double v1, double v2, double v3, double v4) {
    const double p0 = (2.0 * v0 - 7.0 * v1 + 11.0 * v2) / 6.0;
    const double p1 = (-v1 + 5.0 * v2 + 2.0 * v3) / 6.0;
    const double p2 = (2.0 * v2 + 5.0 * v3 - v4) / 6.0;
    const double s0 = v0 - 2.0 * v1 + v2, t0 = v0 - 4.0 * v1 + 3.0 * v2;
    const double s1 = v1 - 2.0 * v2 + v3, t1 = v1 - v3;
    const double s2 = v2 - 2.0 * v3 + v4, t2 = 3.0 * v2 - 4.0 * v3 + v4;
    const double b0 = 13.0 / 12.0 * s0 * s0 + 0.25 * t0 * t0;
    const double b1 = 13.0 / 12.0 * s1 * s1 + 0.25 * t1 * t1;
    const double b2 = 13.0 / 12.0 * s2 * s2 + 0.25 * t2 * t2;
    const double tau = fabs(b0 - b2);
    const double a0 = 0.1 * (1.0 + tau / (b0 + 1e-30));
    const double a1 = 0.6 * (1.0 + tau / (b1 + 1e-30));
    const double a2 = 0.3 * (1.0 + tau / (b2 + 1e-30));
    return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2);
}
__device__ __forceinline__ float weno5z(float v0, float v1, float v2, float v3, float v4) {
    const float sixth = 1.0f / 6.0f;
    const float p0 = (2.0f * v0 - 7.0f * v1 + 11.0f * v2) * sixth;
    const float p1 = (-v1 + 5.0f * v2 + 2.0f * v3) * sixth;
    const float p2 = (2.0f * v2 + 5.0f * v3 - v4) * sixth;
    const float s0 = v0 - 2.0f * v1 + v2, t0 = v0 - 4.0f * v1 + 3.0f * v2;
    const float s1 = v1 - 2.0f * v2 + v3, t1 = v1 - v3;
    const float s2 = v2 - 2.0f * v3 + v4, t2 = 3.0f * v2 - 4.0f * v3 + v4;
    const float c = 13.0f / 12.0f;
    const float b0 = fmaf(c * s0, s0, 0.25f * t0 * t0);
    const float b1 = fmaf(c * s1, s1, 0.25f * t1 * t1);
    const float b2 = fmaf(c * s2, s2, 0.25f * t2 * t2);
    const float tau = fabsf(b0 - b2);
    const float a0 = 0.1f * fmaf(tau, vrcp(b0 + 1e-30f), 1.0f);
    const float a1 = 0.6f * fmaf(tau, vrcp(b1 + 1e-30f), 1.0f);
    const float a2 = 0.3f * fmaf(tau, vrcp(b2 + 1e-30f), 1.0f);
    return fmaf(a0, p0, fmaf(a1, p1, a2 * p2)) * vrcp(a0 + a1 + a2);
}

// -------------------------------------------------------------------- HLL --
// Rotated primitive states W = (rho, un, t1, t2, p), normal along slot 1.
__device__ __forceinline__ void hll_normal(const double WL[NF], const double WR[NF],
                                           double gamma, double gm1, double F[NF]) {
    double UL[NF], FL[NF], UR[NF], FR[NF];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const double* W = s == 0 ? WL : WR;
        double* U = s == 0 ? UL : UR;
        double* G = s == 0 ? FL : FR;
        const double rho = W[0], un = W[1], t1 = W[2], t2 = W[3], p = W[4];
        const double E = p / gm1 + 0.5 * rho * (un * un + t1 * t1 + t2 * t2);
        U[0] = rho; U[1] = rho * un; U[2] = rho * t1; U[3] = rho * t2; U[4] = E;
        G[0] = rho * un; G[1] = rho * un * un + p; G[2] = rho * un * t1;
        G[3] = rho * un * t2; G[4] = (E + p) * un;
    }
    const double cL = sqrt(gamma * WL[4] / WL[0]);
    const double cR = sqrt(gamma * WR[4] / WR[0]);
    const double SL = fmin(WL[1] - cL, WR[1] - cR);
    const double SR = fmax(WL[1] + cL, WR[1] + cR);
    if (0.0 <= SL) {
#pragma unroll
        for (int f = 0; f < NF; ++f) F[f] = FL[f];
    } else if (SR <= 0.0) {
#pragma unroll
        for (int f = 0; f < NF; ++f) F[f] = FR[f];
    } else {
#pragma unroll
        for (int f = 0; f < NF; ++f)
            F[f] = (SR * FL[f] - SL * FR[f] + SL * SR * (UR[f] - UL[f])) / (SR - SL);
    }
}
__device__ __forceinline__ void hll_normal(const float WL[NF], const float WR[NF], float gamma,
                                           float igm1, float F[NF]) {
    float UL[NF], FL[NF], UR[NF], FR[NF];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const float* W = s == 0 ? WL : WR;
        float* U = s == 0 ? UL : UR;
        float* G = s == 0 ? FL : FR;
        const float rho = W[0], un = W[1], t1 = W[2], t2 = W[3], p = W[4];
        const float mu = rho * un;
        const float E = fmaf(p, igm1, 0.5f * rho * fmaf(un, un, fmaf(t1, t1, t2 * t2)));
        U[0] = rho; U[1] = mu; U[2] = rho * t1; U[3] = rho * t2; U[4] = E;
        G[0] = mu; G[1] = fmaf(mu, un, p); G[2] = mu * t1; G[3] = mu * t2; G[4] = (E + p) * un;
    }
    const float cL = vsqrt(gamma * WL[4] * vrcp(WL[0]));
    const float cR = vsqrt(gamma * WR[4] * vrcp(WR[0]));
    const float SL = fminf(WL[1] - cL, WR[1] - cR);
    const float SR = fmaxf(WL[1] + cL, WR[1] + cR);
    // one branch-free form: the upwind cases are the clamped speeds 0 <= SL
    // (F_L) and SR <= 0 (F_R) of the same expression
    const float sl = fminf(SL, 0.0f), sr = fmaxf(SR, 0.0f);
    const float inv = vrcp(sr - sl);
#pragma unroll
    for (int f = 0; f < NF; ++f)
        F[f] = (sr * FL[f] - sl * FR[f] + sl * sr * (UR[f] - UL[f])) * inv;
}

// Face flux along physical axis AX from the six cells q0..q5 around the face
// (the face sits between q2 and q3).
template <int AX, typename T>
__device__ __forceinline__ void weno_face(const T q[6][NF], T gamma, T gx, T F[NF]) {
    using R = Rot<AX>;
    T qL[NF], qR[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        qL[f] = weno5z(q[0][f], q[1][f], q[2][f], q[3][f], q[4][f]);
        qR[f] = weno5z(q[5][f], q[4][f], q[3][f], q[2][f], q[1][f]);
    }
    const T WL[NF] = {qL[0], qL[R::n], qL[R::t1], qL[R::t2], qL[4]};
    const T WR[NF] = {qR[0], qR[R::n], qR[R::t1], qR[R::t2], qR[4]};
    T Fn[NF];
    hll_normal(WL, WR, gamma, gx, Fn);
    F[0] = Fn[0];
    F[R::n] = Fn[1];
    F[R::t1] = Fn[2];
    F[R::t2] = Fn[3];
    F[4] = Fn[4];
}

// Both face values of the middle cell of v0..v4: `right` at its right face
// (weno5z(v0, .., v4)) and `left` at its left face (weno5z of the mirrored
// stencil v4, .., v0).  The mirrored stencil has the indicators (b2, b1, b0)
// and the same tau5, so in FP32 one pass shares the three ratios
// tau5 / (b_k + eps) (candidate k of the left value takes the linear weight
// d_k with the ratio of b_{2-k}) and the candidates' differences.
// FP64 (the parity path) evaluates the two values exactly as weno5z of the
// stencil and of its mirror, so that they round like the oracle's.
__device__ __forceinline__ void weno5z_pair(double v0, double v1, double v2, double v3, double v4,
                                            double& right, double& left) {
    right = weno5z(v0, v1, v2, v3, v4);
    left = weno5z(v4, v3, v2, v1, v0);
}
__device__ __forceinline__ void weno5z_pair(float v0, float v1, float v2, float v3, float v4,
                                            float& right, float& left) {
    // The candidates as offsets from v2, in terms of the indicators' own
    // differences: with u_k = s_k / 12 and w_k = t_k / 4, the right value's
    // candidates are v2 + (u0 + w0), v2 + (u1 - w1), v2 + (u2 - w2).  The
    // mirrored stencil has s' = (s2, s1, s0) and t' = (t2, -t1, t0), so the
    // left value's are v2 + (u2 + w2), v2 + (u1 + w1), v2 + (u0 - w0).  Each
    // value is then v2 + sum a_k (p_k - v2) / sum a_k.
    // The indicators' differences from the four first differences d_k of
    // the stencil: s0 = d01 - d12, t0 = d01 - 3 d12, s1 = d12 - d23,
    // t1 = d12 + d23, s2 = d23 - d34, t2 = 3 d23 - d34 (d_ab = v_a - v_b).
    const float c = 13.0f / 12.0f, twelfth = 1.0f / 12.0f;
    const float d01 = v0 - v1, d12 = v1 - v2, d23 = v2 - v3, d34 = v3 - v4;
    const float s0 = d01 - d12, t0 = fmaf(-3.0f, d12, d01);
    const float s1 = d12 - d23, t1 = d12 + d23;
    const float s2 = d23 - d34, t2 = fmaf(3.0f, d23, -d34);
    const float w0 = 0.25f * t0, w1 = 0.25f * t1, w2 = 0.25f * t2;    // exact
    const float b0 = fmaf(c * s0, s0, w0 * t0);
    const float b1 = fmaf(c * s1, s1, w1 * t1);
    const float b2 = fmaf(c * s2, s2, w2 * t2);
    const float tau = fabsf(b0 - b2);
    const float r0 = tau * vrcp(b0 + 1e-30f), r1 = tau * vrcp(b1 + 1e-30f),
                r2 = tau * vrcp(b2 + 1e-30f);
    const float a0 = fmaf(0.1f, r0, 0.1f), a1 = fmaf(0.6f, r1, 0.6f), a2 = fmaf(0.3f, r2, 0.3f);
    const float l0 = fmaf(0.1f, r2, 0.1f), l2 = fmaf(0.3f, r0, 0.3f);
    // candidate offsets u_k +- w_k with u_k = s_k / 12
    const float e0p = fmaf(s0, twelfth, w0), e0m = fmaf(s0, twelfth, -w0);
    const float e1p = fmaf(s1, twelfth, w1), e1m = fmaf(s1, twelfth, -w1);
    const float e2p = fmaf(s2, twelfth, w2), e2m = fmaf(s2, twelfth, -w2);
    right = fmaf(fmaf(a0, e0p, fmaf(a1, e1m, a2 * e2m)), vrcp(a0 + a1 + a2), v2);
    left = fmaf(fmaf(l0, e2p, fmaf(a1, e1p, l2 * e0m)), vrcp(l0 + a1 + l2), v2);
}

// HLL flux along physical axis AX from the face states (primitives).
template <int AX, typename T>
__device__ __forceinline__ void hll_face(const T qL[NF], const T qR[NF], T gamma, T gx, T F[NF]) {
    using R = Rot<AX>;
    const T WL[NF] = {qL[0], qL[R::n], qL[R::t1], qL[R::t2], qL[4]};
    const T WR[NF] = {qR[0], qR[R::n], qR[R::t1], qR[R::t2], qR[4]};
    T Fn[NF];
    hll_normal(WL, WR, gamma, gx, Fn);
    F[0] = Fn[0];
    F[R::n] = Fn[1];
    F[R::t1] = Fn[2];
    F[R::t2] = Fn[3];
    F[4] = Fn[4];
}

// Boundary map with three ghost layers: m in [-3, n+2] -> interior index
// (flip for a reflecting wall); indices beyond them (ragged tiles) clamp to a
// valid cell whose value feeds no used face.
__device__ __forceinline__ int bc_map3(int m, int n, int lo, int hi, bool& flip) {
    flip = false;
    if (m >= 0 && m < n) return m;
    if (m < -WENO_G || m > n + WENO_G - 1) return m < 0 ? 0 : n - 1;
    const int bc = m < 0 ? lo : hi;
    if (bc == 0) {
        const int r = m % n;
        return r < 0 ? r + n : r;
    }
    if (bc == 1) return m < 0 ? 0 : n - 1;
    flip = true;
    const int s = m < 0 ? -1 - m : 2 * n - 1 - m;
    return s < 0 ? 0 : (s >= n ? n - 1 : s);
}

template <typename T, int DIM, int PX, int PY>
__device__ __forceinline__ void load_prim3(const StageArgs<T>& A, int gx, int gy, int gz,
                                           T W[NF], bool& bad) {
    bool fx, fy = false, fz = false;
    const int sx = bc_map3(gx, A.n[0], A.bc_lo[0], A.bc_hi[0], fx);
    int sy = 0, sz = 0;
    if (DIM >= 2) sy = bc_map3(gy, A.n[1], A.bc_lo[1], A.bc_hi[1], fy);
    if (DIM >= 3) sz = bc_map3(gz, A.n[2], A.bc_lo[2], A.bc_hi[2], fz);
    const long long c = ((long long)sz * A.n[1] + sy) * A.n[0] + sx;
    T U[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) U[f] = __ldg(A.Uc + f * A.N + c);
    if (fx) U[1 + PX] = -U[1 + PX];
    if (DIM >= 2 && fy) U[1 + PY] = -U[1 + PY];
    if (DIM >= 3 && fz) U[3] = -U[3];
    cons_to_prim(U, A.gm1, W);
    bad |= nonphys(W);
}

template <typename T, int TX, int TY, int DIM>
struct WenoSmem {
    static constexpr int HX = TX + 2 * WENO_G;
    static constexpr int HY = DIM >= 2 ? TY + 2 * WENO_G : 1;
    static constexpr int NP = NF * HX * HY;
    static constexpr int NFX = NF * TY * (TX + 1);                 // one x-face array
    static constexpr int NFY = DIM >= 2 ? NF * (TY + 1) * TX : 0;  // one y-face array
    // two primitive planes (by plane parity); face states (left, right) of
    // the x and y faces
    static constexpr size_t bytes = sizeof(T) * (2 * NP + 2 * NFX + 2 * NFY);
};

template <typename T, int TX, int TY, int DIM, int PX, int PY>
__global__ void __launch_bounds__(TX * TY)
weno_stage_kernel(const StageArgs<T> A) {
    using S = WenoSmem<T, TX, TY, DIM>;
    constexpr int NT = TX * TY;
    constexpr int HX = S::HX, HY = S::HY;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red_tot[NT / 32][NF];
    __shared__ unsigned long long red_rate[NT / 32];
    T* Ps2 = reinterpret_cast<T*>(smem_raw);         // 2 x [NF][HY][HX]
    T* QLx = Ps2 + 2 * S::NP;                         // left states of the x faces [NF][TY][TX+1]
    T* QRx = QLx + S::NFX;                            // right states
    T* QLy = QRx + S::NFX;                            // of the y faces [NF][TY+1][TX]
    T* QRy = QLy + S::NFY;

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX;
    const int y0 = DIM >= 2 ? blockIdx.y * TY : 0;
    const int z0 = DIM == 3 ? blockIdx.z * A.zchunk : 0;
    const int z1 = DIM == 3 ? min(z0 + A.zchunk, A.n[2]) : 1;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = x < A.n[0] && (DIM < 2 || y < A.n[1]);
    const T dt = (T)(A.dt_dev ? *A.dt_dev : A.dt);
    const T gamma = A.gamma;
    // the HLL energy closure: 1/(gamma-1) in FP32, gamma-1 (a divisor) in FP64
    const T gx = sizeof(T) == 4 ? A.igm1 : A.gm1;
    bool bad = false;
    T rate_max = T(0);
    T tot[NF] = {T(0), T(0), T(0), T(0), T(0)};

    // z stencil of this thread's column: primitives of the last five planes,
    // the pending left state of the next z face, the previous z-face flux and
    // the x/y flux differences of three planes
    T w[5][NF], qLz[NF], Fzp[NF], Da[NF], Db[NF], Dc[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        qLz[f] = Fzp[f] = Da[f] = Db[f] = Dc[f] = T(0);
#pragma unroll
        for (int s = 0; s < 5; ++s) w[s][f] = T(0);
    }

    const int jbeg = DIM == 3 ? z0 - WENO_G : 0;
    const int jend = DIM == 3 ? z1 + WENO_G : 1;
    for (int j = jbeg; j < jend; ++j) {
        const bool xy = DIM < 3 || (j >= z0 && j < z1);
        T qj[NF], Dj[NF];
        // Two barriers per plane.  The primitive planes alternate by parity:
        // plane j's is last read (own cell) after the second barrier of plane
        // j-2, and every thread has passed the barriers of plane j-1 before
        // any thread writes plane j; the face states of plane j are written
        // after its first barrier, which no thread passes before every thread
        // has finished plane j-1.  Each thread takes the HLL fluxes of its
        // own cell's four x/y faces from the face states (an interior face is
        // evaluated by both of its cells, identically).
        T* Ps = Ps2 + ((j - jbeg) & 1) * S::NP;
        if (xy) {
            for (int e = tid; e < HX * HY; e += NT) {
                const int hx = e % HX, hy = e / HX;
                T W[NF];
                load_prim3<T, DIM, PX, PY>(A, x0 - WENO_G + hx, y0 - (DIM >= 2 ? WENO_G : 0) + hy,
                                           j, W, bad);
#pragma unroll
                for (int f = 0; f < NF; ++f) Ps[(f * HY + hy) * HX + hx] = W[f];
            }
            __syncthreads();
            // each cell's two face values per axis (halo cells -1 and TX / TY
            // included): x face fx (left of tile cell fx) takes its left state
            // from cell fx-1 and its right state from cell fx
            constexpr int NRX = (TX + 2) * TY, NRY = DIM >= 2 ? TX * (TY + 2) : 0;
            for (int e = tid; e < NRX + NRY; e += NT) {
                if (e < NRX) {
                    const int cx = e % (TX + 2) - 1, row = e / (TX + 2);
                    const int hy = DIM >= 2 ? row + WENO_G : 0;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const T* v = Ps + (f * HY + hy) * HX + cx + WENO_G;
                        T rv, lv;
                        weno5z_pair(v[-2], v[-1], v[0], v[1], v[2], rv, lv);
                        if (cx + 1 <= TX) QLx[(f * TY + row) * (TX + 1) + cx + 1] = rv;
                        if (cx >= 0) QRx[(f * TY + row) * (TX + 1) + cx] = lv;
                    }
                } else {
                    const int e2 = e - NRX;
                    const int col = e2 % TX, cy = e2 / TX - 1;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const T* v = Ps + (f * HY + cy + WENO_G) * HX + col + WENO_G;
                        T rv, lv;
                        weno5z_pair(v[-2 * HX], v[-HX], v[0], v[HX], v[2 * HX], rv, lv);
                        if (cy + 1 <= TY) QLy[(f * (TY + 1) + cy + 1) * TX + col] = rv;
                        if (cy >= 0) QRy[(f * (TY + 1) + cy) * TX + col] = lv;
                    }
                }
            }
            __syncthreads();
            const int hyc = DIM >= 2 ? ty + WENO_G : 0;
            {
                constexpr int NX = (TX + 1) * TY, NY = DIM >= 2 ? TX * (TY + 1) : 0;
                const int ex = ty * (TX + 1) + tx;    // the x face below this cell
                T qL[NF], qR[NF], Fl[NF], Fr[NF];
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    qL[f] = QLx[f * NX + ex];
                    qR[f] = QRx[f * NX + ex];
                }
                hll_face<PX>(qL, qR, gamma, gx, Fl);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    qL[f] = QLx[f * NX + ex + 1];
                    qR[f] = QRx[f * NX + ex + 1];
                }
                hll_face<PX>(qL, qR, gamma, gx, Fr);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    qj[f] = Ps[(f * HY + hyc) * HX + tx + WENO_G];
                    Dj[f] = sub_over_dx(T(0), Fr[f] - Fl[f], A.dxk[0]);
                }
                if (DIM >= 2) {
                    const int ey = ty * TX + tx;      // the y face below this cell
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        qL[f] = QLy[f * NY + ey];
                        qR[f] = QRy[f * NY + ey];
                    }
                    hll_face<PY>(qL, qR, gamma, gx, Fl);
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        qL[f] = QLy[f * NY + ey + TX];
                        qR[f] = QRy[f * NY + ey + TX];
                    }
                    hll_face<PY>(qL, qR, gamma, gx, Fr);
#pragma unroll
                    for (int f = 0; f < NF; ++f) Dj[f] = sub_over_dx(Dj[f], Fr[f] - Fl[f], A.dxk[1]);
                }
            }
        } else {
            // warm-up / look-ahead plane: only this column's primitives
            load_prim3<T, DIM, PX, PY>(A, min(x, A.n[0] - 1), min(y, A.n[1] - 1), j, qj, bad);
#pragma unroll
            for (int f = 0; f < NF; ++f) Dj[f] = T(0);
        }

        int k;                 // cell completed in this iteration (-1: none)
        T L[NF];
        if (DIM == 3) {
            const int cnt = j - jbeg;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
#pragma unroll
                for (int s = 0; s < 4; ++s) w[s][f] = w[s + 1][f];
                w[4][f] = qj[f];
            }
            // cell j-2 (planes j-4 .. j): its lower face value closes the face
            // between j-3 and j-2; its upper value waits for the next plane
            T Fz[NF];
            if (cnt >= 4) {
                T qR[NF], up[NF];
#pragma unroll
                for (int f = 0; f < NF; ++f) weno5z_pair(w[0][f], w[1][f], w[2][f], w[3][f], w[4][f], up[f], qR[f]);
                if (cnt >= 5) hll_face<2>(qLz, qR, gamma, gx, Fz);
#pragma unroll
                for (int f = 0; f < NF; ++f) qLz[f] = up[f];
            }
            k = cnt >= 6 ? j - WENO_G : -1;
            if (k >= 0) {
#pragma unroll
                for (int f = 0; f < NF; ++f) L[f] = sub_over_dx(Da[f], Fz[f] - Fzp[f], A.dxk[2]);
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                if (cnt >= 5) Fzp[f] = Fz[f];
                Da[f] = Db[f];
                Db[f] = Dc[f];
                Dc[f] = Dj[f];
            }
        } else {
            k = 0;
#pragma unroll
            for (int f = 0; f < NF; ++f) L[f] = Dj[f];
        }

        if (k >= 0 && own) {
            const long long c = ((long long)k * A.n[1] + y) * A.n[0] + x;
            T Uo[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const T uc = A.Uc[f * A.N + c];
                if (A.stage == 1) {
                    Uo[f] = madd(dt, L[f], uc);
                } else {
                    const T u0 = A.U0[f * A.N + c];
                    Uo[f] = madd(T(0.5), u0, T(0.5) * madd(dt, L[f], uc));
                }
                A.Uo[f * A.N + c] = Uo[f];
            }
            if (A.rate_slot) {
                T W[NF];
                cons_to_prim(Uo, A.gm1, W);
                const T r = cell_rate(W, gamma, A.act, A.rdx);
                rate_max = (r > rate_max || r != r) ? r : rate_max;
            }
            if (A.tot_partial) {
#pragma unroll
                for (int f = 0; f < NF; ++f) tot[f] += Uo[f];
            }
        }
    }

    // ---- epilogue: block reductions ----
    const int lane = tid & 31, warp = tid >> 5;
    if (A.rate_slot) {
        unsigned long long b = rate_bits(rate_max);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
            b = v > b ? v : b;
        }
        if (lane == 0) red_rate[warp] = b;
    }
    if (A.tot_partial) {
        double v[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f] = (double)tot[f];
        const double s = warp_sum5(v, lane);
        if (sum5_writer(lane)) red_tot[warp][sum5_field(lane)] = s;
    }
    const int any_bad = __syncthreads_or(bad);
    if (tid == 0) {
        if (any_bad) atomicOr(A.status, 1);
        if (A.rate_slot) {
            unsigned long long b = 0;
            for (int wi = 0; wi < NT / 32; ++wi) b = red_rate[wi] > b ? red_rate[wi] : b;
            atomicMax(A.rate_slot, b);
        }
    }
    if (A.tot_partial && tid < NF) {
        const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        double s = 0.0;
        for (int wi = 0; wi < NT / 32; ++wi) s += red_tot[wi][tid];
        A.tot_partial[blk * NF + tid] = s;
    }
}

}  // namespace hh

namespace hh {

// ----------------------------------------------------- radiation energy --
// Advection of the radiation energy density E by the fluid velocity (the
// d_j(E v^j) term of Eq. "radiation"), Sec. 2.2.2: WENO5-Z face states of E
// and of the normal velocity, the Rusanov flux
//   F = (E_L u_L + E_R u_R)/2 - max(|u_L|, |u_R|) (E_R - E_L)/2,
// and the Heun stage combine, with the fluid state U held fixed.  Same tiling
// as weno_stage_kernel, with a four-field plane (E and the three velocity
// components along the kernel axes) and a two-field z window (E, w).

template <typename T>
struct AdvectArgs {
    const T* U;          // fluid state [5][N] (velocities)
    const T* E0;         // stage 2: E^n
    const T* Ec;         // E the flux difference is taken of
    T* Eo;               // output
    long long N;
    int n[3];
    int bc_lo[3], bc_hi[3];
    T dxk[3];            // per kernel axis: dx (FP64) or 1/dx (FP32)
    double dt;
    int stage;
    int zchunk;
};

__device__ __forceinline__ double rusanov_e(double EL, double ER, double uL, double uR) {
    const double a = fmax(fabs(uL), fabs(uR));
    return 0.5 * (EL * uL + ER * uR) - 0.5 * a * (ER - EL);
}
__device__ __forceinline__ float rusanov_e(float EL, float ER, float uL, float uR) {
    const float a = fmaxf(fabsf(uL), fabsf(uR));
    return 0.5f * (EL * uL + ER * uR) - 0.5f * a * (ER - EL);
}

// E and the velocity along kernel axes (x', y', z') = physical (PX, PY, 2)
// of kernel cell (gx, gy, gz) through the three-layer boundary map
template <typename T, int DIM, int PX, int PY>
__device__ __forceinline__ void load_ev(const AdvectArgs<T>& A, int gx, int gy, int gz, T out[4]) {
    bool fx, fy = false, fz = false;
    const int sx = bc_map3(gx, A.n[0], A.bc_lo[0], A.bc_hi[0], fx);
    int sy = 0, sz = 0;
    if (DIM >= 2) sy = bc_map3(gy, A.n[1], A.bc_lo[1], A.bc_hi[1], fy);
    if (DIM >= 3) sz = bc_map3(gz, A.n[2], A.bc_lo[2], A.bc_hi[2], fz);
    const long long c = ((long long)sz * A.n[1] + sy) * A.n[0] + sx;
    const T rho = __ldg(A.U + c);
    T m[3] = {__ldg(A.U + A.N + c), __ldg(A.U + 2 * A.N + c), __ldg(A.U + 3 * A.N + c)};
    if (fx) m[PX] = -m[PX];
    if (DIM >= 2 && fy) m[PY] = -m[PY];
    if (DIM >= 3 && fz) m[2] = -m[2];
    out[0] = __ldg(A.Ec + c);
    out[1] = m[PX] / rho;
    out[2] = DIM >= 2 ? m[PY] / rho : T(0);
    out[3] = DIM >= 3 ? m[2] / rho : T(0);
}

// Shared memory of the advection kernel: E and the three velocities of the
// haloed plane, two planes by parity; the face states of the plane's x faces
// ([TY][TX+1]: E and u' on the left and right of each face) and y faces
// ([TY+1][TX]: E and v').
template <typename T, int TX, int TY, int DIM>
struct AdvectSmem {
    static constexpr int HX = TX + 2 * WENO_G, HY = DIM >= 2 ? TY + 2 * WENO_G : 1;
    static constexpr int NPF = HX * HY;
    static constexpr int NQX = (TX + 1) * TY;
    static constexpr int NQY = DIM >= 2 ? TX * (TY + 1) : 0;
    static constexpr size_t bytes = sizeof(T) * (2 * 4 * NPF + 4 * NQX + 4 * NQY);
};

// Per plane: every cell of the tile, and one halo cell on each side along the
// axis, evaluates the WENO5-Z pair of E and of the normal velocity along x and
// y (its upper value is the left state of the face above it, its lower value
// the right state of the face below).  After the second barrier each thread
// takes the Rusanov fluxes of its own cell's four faces from those states:
// an interior face is evaluated by both of its cells (identically), which
// keeps the block at two barriers per plane.  Along z the thread's own column
// takes one pair per plane and quantity and carries the upper value to the
// next face.  FP64 evaluates each value as weno5z of its stencil, exactly the
// face-by-face form.
template <typename T, int TX, int TY, int DIM, int PX, int PY>
__global__ void __launch_bounds__(TX * TY) weno_advect_kernel(const AdvectArgs<T> A) {
    using S = AdvectSmem<T, TX, TY, DIM>;
    constexpr int NT = TX * TY;
    constexpr int HX = S::HX, HY = S::HY, NPF = S::NPF, NQX = S::NQX, NQY = S::NQY;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* Ps2 = reinterpret_cast<T*>(smem_raw);         // E, u', v', w' planes, two by plane parity
    T* QxE = Ps2 + 2 * 4 * NPF;                       // [2][TY][TX+1]: left, right state of E
    T* QxU = QxE + 2 * NQX;                           // [2][TY][TX+1]: of u'
    T* QyE = QxU + 2 * NQX;                           // [2][TY+1][TX]: of E
    T* QyV = QyE + 2 * NQY;                           // [2][TY+1][TX]: of v'
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX;
    const int y0 = DIM >= 2 ? blockIdx.y * TY : 0;
    const int z0 = DIM == 3 ? blockIdx.z * A.zchunk : 0;
    const int z1 = DIM == 3 ? min(z0 + A.zchunk, A.n[2]) : 1;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = x < A.n[0] && (DIM < 2 || y < A.n[1]);
    const T dt = (T)A.dt;

    // z: E and w' of the last five planes, the pending left states of the
    // next z face, the previous z-face flux, the x/y flux differences
    T we[5], ww[5], eUp = T(0), wUp = T(0), Fzp = T(0), Da = T(0), Db = T(0), Dc = T(0);
#pragma unroll
    for (int s = 0; s < 5; ++s) we[s] = ww[s] = T(0);

    const int jbeg = DIM == 3 ? z0 - WENO_G : 0;
    const int jend = DIM == 3 ? z1 + WENO_G : 1;
    for (int j = jbeg; j < jend; ++j) {
        const bool xy = DIM < 3 || (j >= z0 && j < z1);
        T ej, wj, Dj;
        // two barriers per plane: the planes alternate by parity (plane j's is
        // last read after the second barrier of plane j-2); the face states
        // are written after the first barrier, which no thread passes before
        // every thread has finished the previous plane
        T* Ps = Ps2 + ((j - jbeg) & 1) * 4 * NPF;
        if (xy) {
            for (int e = tid; e < NPF; e += NT) {
                const int hx = e % HX, hy = e / HX;
                T v[4];
                load_ev<T, DIM, PX, PY>(A, x0 - WENO_G + hx, y0 - (DIM >= 2 ? WENO_G : 0) + hy, j, v);
#pragma unroll
                for (int f = 0; f < 4; ++f) Ps[f * NPF + e] = v[f];
            }
            __syncthreads();
            constexpr int NRX = (TX + 2) * TY, NRY = DIM >= 2 ? TX * (TY + 2) : 0;
            for (int e = tid; e < NRX + NRY; e += NT) {
                if (e < NRX) {
                    // cell cx of the row: face cx+1 above it, face cx below
                    const int cx = e % (TX + 2) - 1, row = e / (TX + 2);
                    const int hy = DIM >= 2 ? row + WENO_G : 0;
                    const T* ve = Ps + hy * HX + cx + WENO_G;
                    const T* vu = ve + NPF;
                    T er, el, ur, ul;
                    weno5z_pair(ve[-2], ve[-1], ve[0], ve[1], ve[2], er, el);
                    weno5z_pair(vu[-2], vu[-1], vu[0], vu[1], vu[2], ur, ul);
                    const int q = row * (TX + 1) + cx;
                    if (cx + 1 <= TX) {
                        QxE[q + 1] = er;
                        QxU[q + 1] = ur;
                    }
                    if (cx >= 0) {
                        QxE[NQX + q] = el;
                        QxU[NQX + q] = ul;
                    }
                } else {
                    const int e2 = e - NRX;
                    const int col = e2 % TX, cy = e2 / TX - 1;
                    const T* ve = Ps + (cy + WENO_G) * HX + col + WENO_G;
                    const T* vv = ve + 2 * NPF;
                    T er, el, vr, vl;
                    weno5z_pair(ve[-2 * HX], ve[-HX], ve[0], ve[HX], ve[2 * HX], er, el);
                    weno5z_pair(vv[-2 * HX], vv[-HX], vv[0], vv[HX], vv[2 * HX], vr, vl);
                    const int q = cy * TX + col;
                    if (cy + 1 <= TY) {
                        QyE[q + TX] = er;
                        QyV[q + TX] = vr;
                    }
                    if (cy >= 0) {
                        QyE[NQY + q] = el;
                        QyV[NQY + q] = vl;
                    }
                }
            }
            __syncthreads();
            const int fx = ty * (TX + 1) + tx;        // the x face below this cell
            const T Fxl = rusanov_e(QxE[fx], QxE[NQX + fx], QxU[fx], QxU[NQX + fx]);
            const T Fxr = rusanov_e(QxE[fx + 1], QxE[NQX + fx + 1], QxU[fx + 1], QxU[NQX + fx + 1]);
            Dj = sub_over_dx(T(0), Fxr - Fxl, A.dxk[0]);
            if (DIM >= 2) {
                const int fy = ty * TX + tx;          // the y face below this cell
                const T Fyl = rusanov_e(QyE[fy], QyE[NQY + fy], QyV[fy], QyV[NQY + fy]);
                const T Fyr = rusanov_e(QyE[fy + TX], QyE[NQY + fy + TX], QyV[fy + TX],
                                        QyV[NQY + fy + TX]);
                Dj = sub_over_dx(Dj, Fyr - Fyl, A.dxk[1]);
            }
            const int hyc = DIM >= 2 ? ty + WENO_G : 0;
            ej = Ps[0 * NPF + hyc * HX + tx + WENO_G];
            wj = Ps[3 * NPF + hyc * HX + tx + WENO_G];
        } else {
            T v[4];
            load_ev<T, DIM, PX, PY>(A, min(x, A.n[0] - 1), min(y, A.n[1] - 1), j, v);
            ej = v[0];
            wj = v[3];
            Dj = T(0);
        }
        int k;
        T L;
        if (DIM == 3) {
            const int cnt = j - jbeg;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                we[s] = we[s + 1];
                ww[s] = ww[s + 1];
            }
            we[4] = ej;
            ww[4] = wj;
            // cell j-2 (planes j-4 .. j): its lower values close the face
            // between j-3 and j-2; its upper values wait for the next plane
            T Fz = T(0);
            if (cnt >= 4) {
                T eu, el, wu, wl;
                weno5z_pair(we[0], we[1], we[2], we[3], we[4], eu, el);
                weno5z_pair(ww[0], ww[1], ww[2], ww[3], ww[4], wu, wl);
                if (cnt >= 5) Fz = rusanov_e(eUp, el, wUp, wl);
                eUp = eu;
                wUp = wu;
            }
            k = cnt >= 6 ? j - WENO_G : -1;
            L = sub_over_dx(Da, Fz - Fzp, A.dxk[2]);
            if (cnt >= 5) Fzp = Fz;
            Da = Db;
            Db = Dc;
            Dc = Dj;
        } else {
            k = 0;
            L = Dj;
        }
        if (k >= 0 && own) {
            const long long c = ((long long)k * A.n[1] + y) * A.n[0] + x;
            const T ec = A.Ec[c];
            A.Eo[c] = A.stage == 1 ? madd(dt, L, ec) : madd(T(0.5), A.E0[c], T(0.5) * madd(dt, L, ec));
        }
    }
}

}  // namespace hh
