// Radiative heating / cooling exchange (Eq. "heating-cooling"):
//   qdot = c kappa rho (E - a T^4),  de/dt = qdot,  dE/dt = -qdot,
// T = e / (rho c_v), e the fluid's internal energy density, E the radiation
// energy density.  One backward-Euler step of length dt per cell:
//   e' = e + dt k (E_tot - e' - a (e'/(rho c_v))^4),  k = c kappa rho,
//   E' = E + (e - e'),  E_tot = e + E,
// solved by Newton's method on f(x) = x - e - dt k (E_tot - x - a T(x)^4),
// increasing and convex for x > 0: started right of the root at
//   x0 = min(e + dt k max(E_tot - e - a T(e)^4, 0), E_tot, x_q),
//   x_q = rho c_v ((e + dt k E_tot) / (dt k a))^(1/4)
// (x_q is within a few Newton steps of the root when the T^4 term dominates)
// the iterates decrease monotonically onto it.  Stops when the step is at
// most tol x (1e-15 in FP64, 4e-7 in FP32), after at most 200 steps.
//
// Pointwise and bandwidth-bound: reads rho, the momenta, E_total and E,
// writes E_total and E (32 B per cell in FP32).  FP64 evaluates the formulas
// in the written order with IEEE division and square root (no contraction,
// --fmad=false); FP32 multiplies by approximate reciprocals.
#include <cmath>

#include "hard_hydro.h"
#include "launch.h"
#include "rad_launch.h"
#include "vec2.cuh"

namespace hh {
namespace {

constexpr int RAD_MAX_NEWTON = 200;

__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qdiv(float a, float b) { return a * vrcp(b); }
__device__ __forceinline__ double qsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float qsqrt(float a) { return vsqrt(a); }

template <typename T>
struct RadArgs {
    T* U;                 // [5][N]
    T* Er;                // [N]
    long long N;
    T c, kappa, arad, cv, dt;
    int* status;          // bit 0: a cell with rho <= 0, e <= 0 or no convergence
};

template <typename T>
__device__ __forceinline__ bool exchange_cell(T rho, T m1, T m2, T m3, T& Etotal, T& Erad,
                                              const RadArgs<T>& a) {
    const T kin = qdiv(T(0.5) * (m1 * m1 + m2 * m2 + m3 * m3), rho);
    const T e = Etotal - kin;
    if (!(rho > T(0)) || !(e > T(0)) || !(Erad >= T(0))) return false;
    const T Etot = e + Erad;
    const T k = a.c * a.kappa * rho;
    const T rcv = rho * a.cv;
    const T ircv = sizeof(T) == 8 ? T(1) : qdiv(T(1), rcv);     // FP32 only
    const T Te = sizeof(T) == 8 ? qdiv(e, rcv) : e * ircv;
    const T R0 = Etot - e - a.arad * (Te * Te) * (Te * Te);
    T x = e + a.dt * k * (R0 > T(0) ? R0 : T(0));
    if (x > Etot) x = Etot;
    const T xq = rcv * qsqrt(qsqrt(qdiv(e + a.dt * k * Etot, a.dt * k * a.arad)));
    if (xq < x) x = xq;
    const T tol = sizeof(T) == 8 ? T(1e-15) : T(4e-7);
    bool ok = false;
    for (int it = 0; it < RAD_MAX_NEWTON; ++it) {
        const T Tx = sizeof(T) == 8 ? qdiv(x, rcv) : x * ircv;
        const T aT4 = a.arad * (Tx * Tx) * (Tx * Tx);
        const T f = x - e - a.dt * k * (Etot - x - aT4);
        const T df = T(1) + a.dt * k * (T(1) + qdiv(T(4) * aT4, x));
        const T dx = qdiv(f, df);
        x = x - dx;
        if (fabs(dx) <= tol * x) {
            ok = true;
            break;
        }
    }
    Etotal = x + kin;
    Erad = Erad + (e - x);
    return ok;
}

template <typename T>
__global__ void __launch_bounds__(256) rad_exchange_kernel(const RadArgs<T> a) {
    const long long N = a.N;
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += stride) {
        const T rho = a.U[q], m1 = a.U[N + q], m2 = a.U[2 * N + q], m3 = a.U[3 * N + q];
        T Et = a.U[4 * N + q], Er = a.Er[q];
        if (exchange_cell(rho, m1, m2, m3, Et, Er, a)) {
            a.U[4 * N + q] = Et;
            a.Er[q] = Er;
        } else {
            bad = true;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.status, 1);
}

template <typename T>
cudaError_t run_exchange(const MeshDesc& m, void* U, void* Er, double dt, const double prm[4],
                         int* status, cudaStream_t s) {
    RadArgs<T> a;
    a.U = static_cast<T*>(U);
    a.Er = static_cast<T*>(Er);
    a.N = m.N;
    a.c = (T)prm[0];
    a.kappa = (T)prm[1];
    a.arad = (T)prm[2];
    a.cv = (T)prm[3];
    a.dt = (T)dt;
    a.status = status;
    long long blocks = (m.N + 255) / 256;
    const long long cap = 152LL * 8;          // eight 256-thread blocks per SM, grid-stride beyond
    if (blocks > cap) blocks = cap;
    rad_exchange_kernel<T><<<(int)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rad_exchange(const MeshDesc& m, int dtype, void* U, void* Er, double dt,
                                const double prm[4], int* status, cudaStream_t s) {
    return dtype == HARD_F64 ? run_exchange<double>(m, U, Er, dt, prm, status, s)
                             : run_exchange<float>(m, U, Er, dt, prm, status, s);
}

}  // namespace hh
