// WENO5-Z + HLL stage as directional sweeps (the second scheme of Sec. 2.2.2,
// the same arithmetic as weno_stage_kernel in weno.cuh).
//
// The flux difference L(U) = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d is built
// one kernel axis at a time, in the oracle's order (x', then y', then z'):
//
//   x sweep      L  = 0 - (F^x_{i+1/2} - F^x_{i-1/2}) / dx         (writes L)
//   y' march     L <- L - (F^y_{j+1/2} - F^y_{j-1/2}) / dy         (reads, writes L)
//   z' march     L <- L - (F^z_{k+1/2} - F^z_{k-1/2}) / dz, then the RK stage
//                combine and the rate / totals epilogue             (reads L)
//
// The sweeps serve 3D meshes (1D and 2D meshes, small enough to be bound by
// launch latency, keep the fused kernel).  Each sweep reconstructs the two
// face values of every cell once (weno5z_pair) and evaluates every face's
// HLL flux once.  The x sweep gives each warp a 62-cell segment of a row:
// lane l holds cells x_s - 1 + 2l and x_s + 2l, the window of their
// five-cell stencils sits in shared memory, and the face between two lanes
// takes its left state from the lower lane by a shuffle.  The marches give each lane one x column and
// walk the march axis with the five-cell stencil, the pending face state and
// the last face flux in registers: no block barrier and no shared plane.
// Against the fused kernel this moves L through HBM between the sweeps
// (about three times the state traffic) to cut the instructions per cell:
// the fused kernel is bound by instruction issue, not by memory.
#pragma once
#include "weno.cuh"
#include "weno_launch.h"

namespace hh {

constexpr int WX_SEG = 62;                    // cells per warp in the x sweeps (two per lane)
constexpr int WX_WIN = WX_SEG + 6;            // their stencil window
constexpr int SWEEP_THREADS = WENO_SWEEP_THREADS;

// Conserved -> primitive of cell m along kernel axis AX (extent nA, element
// stride `stride` from `base`), through the three-layer boundary map of that
// axis; the other coordinates are interior.  PA: momentum slot normal to AX.
template <typename T, int AX, int PA>
__device__ __forceinline__ void sweep_load(const StageArgs<T>& A, long long base, int m, int nA,
                                           long long stride, T W[NF], bool& bad) {
    bool flip;
    const int s = bc_map3(m, nA, A.bc_lo[AX], A.bc_hi[AX], flip);
    const long long c = base + (long long)s * stride;
    T U[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) U[f] = __ldg(A.Uc + f * A.N + c);
    if (flip) U[1 + PA] = -U[1 + PA];
    cons_to_prim(U, A.gm1, W);
    bad |= nonphys(W);
}

// Block epilogue of the combining sweep: nonphysical flag, rate maximum and
// the block's row of the totals partial array (every thread calls it).
template <typename T>
__device__ __forceinline__ void sweep_epilogue(const StageArgs<T>& A, bool bad, T rate_max,
                                               const T tot[NF], long long blk) {
    __shared__ double red_tot[SWEEP_THREADS / 32][NF];
    __shared__ unsigned long long red_rate[SWEEP_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    if (threadIdx.x == 0) {
        if (any_bad) atomicOr(A.status, 1);
        if (A.rate_slot) {
            unsigned long long b = 0;
            for (int w = 0; w < SWEEP_THREADS / 32; ++w) b = red_rate[w] > b ? red_rate[w] : b;
            atomicMax(A.rate_slot, b);
        }
    }
    if (A.tot_partial && threadIdx.x < NF) {
        double s = 0.0;
        for (int w = 0; w < SWEEP_THREADS / 32; ++w) s += red_tot[w][threadIdx.x];
        A.tot_partial[blk * NF + threadIdx.x] = s;
    }
}

// x sweep: one warp per 62-cell segment of a row (y', z' fixed), two cells
// per lane; a block takes one segment of four consecutive rows.  Writes L.
template <typename T, int PX>
__global__ void __launch_bounds__(SWEEP_THREADS)
weno_x_kernel(const StageArgs<T> A, T* __restrict__ L) {
    __shared__ T win[SWEEP_THREADS / 32][NF][WX_WIN];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int n0 = A.n[0], n1 = A.n[1];
    // segment blockIdx.x of rows y' = 4 blockIdx.y + warp, z' = blockIdx.z
    const int yr = blockIdx.y * (SWEEP_THREADS / 32) + wq;
    const bool active = yr < n1;                       // warp-uniform
    const long long base = ((long long)blockIdx.z * n1 + (active ? yr : 0)) * n0;
    const int xs = blockIdx.x * WX_SEG;
    const T gamma = A.gamma;
    const T gx = sizeof(T) == 4 ? A.igm1 : A.gm1;     // the HLL energy closure
    bool bad = false;                                  // reported by the combining sweep

    // the window: cells xs-3 .. xs+64 (lane l loads cells xs-3+l and
    // xs+29+l, and lanes 0..3 also cell xs+61+l)
    {
        T W[NF];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            sweep_load<T, 0, PX>(A, base, xs - 3 + 32 * h + lane, n0, 1, W, bad);
#pragma unroll
            for (int f = 0; f < NF; ++f) win[wq][f][32 * h + lane] = W[f];
        }
        if (lane < WX_WIN - 64) {
            sweep_load<T, 0, PX>(A, base, xs + 61 + lane, n0, 1, W, bad);
#pragma unroll
            for (int f = 0; f < NF; ++f) win[wq][f][64 + lane] = W[f];
        }
    }
    __syncwarp();
    // lane l: cells c0 = xs-1+2l and c1 = c0+1, their stencils win[2l .. 2l+4]
    // and win[2l+1 .. 2l+5]; the face left of c0 takes its left state from
    // c1 of lane l-1, the face right of c1 is lane l+1's face left of its c0
    T rv0[NF], lv0[NF], rv1[NF], lv1[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const T* v = &win[wq][f][2 * lane];
        weno5z_pair(v[0], v[1], v[2], v[3], v[4], rv0[f], lv0[f]);
        weno5z_pair(v[1], v[2], v[3], v[4], v[5], rv1[f], lv1[f]);
    }
    T qL[NF], Fl[NF], Fm[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) qL[f] = __shfl_up_sync(0xffffffffu, rv1[f], 1);
    hll_face<PX>(qL, lv0, gamma, gx, Fl);              // face c0 - 1/2
    hll_face<PX>(rv0, lv1, gamma, gx, Fm);             // face c0 + 1/2
    T D0[NF], D1[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const T Fr = __shfl_down_sync(0xffffffffu, Fl[f], 1);   // face c1 + 1/2
        D0[f] = sub_over_dx(T(0), Fm[f] - Fl[f], A.dxk[0]);
        D1[f] = sub_over_dx(T(0), Fr - Fm[f], A.dxk[0]);
    }
    // cells xs .. xs+61: c1 of lanes 0..30, c0 of lanes 1..31
    const int x0 = xs - 1 + 2 * lane;
    if (active && lane >= 1 && x0 < n0) {
#pragma unroll
        for (int f = 0; f < NF; ++f) L[f * A.N + base + x0] = D0[f];
    }
    if (active && lane <= 30 && x0 + 1 < n0) {
#pragma unroll
        for (int f = 0; f < NF; ++f) L[f * A.N + base + x0 + 1] = D1[f];
    }
}

// March along kernel axis AX (1: y', 2: z'): lane = x', one block row of
// SWEEP_THREADS columns, the other transverse coordinate blockIdx.y, a chunk
// of A.zchunk cells of the march axis per blockIdx.z.  Adds this axis' flux
// difference to L; LAST: then the combine.  Every global load is issued one
// step before its value is used (the next cell's state; the flux difference,
// state and U^n of the cell that completes at the next step), so a step's
// arithmetic covers the memory latency.  At least four blocks per SM (at
// most 128 registers a thread): 16 warps hide more latency than the 11 the
// unbounded 138-168 registers allow.
#ifndef HH_WENO_MINB
#define HH_WENO_MINB 4
#endif
template <typename T, int AX, int PA, bool LAST>
__global__ void __launch_bounds__(SWEEP_THREADS, HH_WENO_MINB)
weno_march_kernel(const StageArgs<T> A, T* __restrict__ L) {
    static_assert(AX == 1 || AX == 2, "the x' axis is the x sweep's");
    const int n0 = A.n[0], n1 = A.n[1];
    const int nA = A.n[AX];
    const int x = blockIdx.x * SWEEP_THREADS + threadIdx.x;
    const bool xin = x < n0;
    const int xl = xin ? x : n0 - 1;                   // lanes past the row load a valid cell
    const int o = blockIdx.y;                          // z' (AX = 1) or y' (AX = 2)
    const long long stride = AX == 1 ? (long long)n0 : (long long)n0 * n1;
    const long long base = (AX == 1 ? (long long)o * n1 * n0 : (long long)o * n0) + xl;
    const long long N = A.N;
    const int a0 = blockIdx.z * A.zchunk;
    const int a1 = min(a0 + A.zchunk, nA);
    const T gamma = A.gamma;
    const T gx = sizeof(T) == 4 ? A.igm1 : A.gm1;
    const T dt = (T)(A.dt_dev ? *A.dt_dev : A.dt);
    const bool two = A.stage == 2;
    bool bad = false;
    T rate_max = T(0);
    T tot[NF] = {T(0), T(0), T(0), T(0), T(0)};

    // the conserved state of cell m through the axis' boundary map (raw:
    // the reflecting flip is applied when the value is used)
    auto fetch = [&](int m, T U[NF], bool& flip) {
        const int sidx = bc_map3(m, nA, A.bc_lo[AX], A.bc_hi[AX], flip);
        const long long c = base + (long long)sidx * stride;
#pragma unroll
        for (int f = 0; f < NF; ++f) U[f] = __ldg(A.Uc + f * N + c);
    };
    // the operands of interior cell k's update: its flux difference so far
    // and, when this sweep combines, its state and U^n
    auto fetch_cell = [&](int k, T Lk[NF], T Uk[NF], T U0k[NF]) {
        const long long c = base + (long long)k * stride;
#pragma unroll
        for (int f = 0; f < NF; ++f) Lk[f] = L[f * N + c];
        if constexpr (LAST) {
#pragma unroll
            for (int f = 0; f < NF; ++f) Uk[f] = __ldg(A.Uc + f * N + c);
            if (two) {
#pragma unroll
                for (int f = 0; f < NF; ++f) U0k[f] = A.U0[f * N + c];
            }
        }
    };

    // cells a0-3 .. a1+2 are loaded; the window w holds the primitives of
    // the last five, rvp the right-face value of the cell below the newest
    // pair, Fp the flux of the face below that cell
    T w[5][NF], rvp[NF], Fp[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        rvp[f] = Fp[f] = T(0);
#pragma unroll
        for (int q = 0; q < 5; ++q) w[q][f] = T(0);
    }
    T Un[NF], Lk[NF], Uk[NF], U0k[NF];
    bool fn;
    fetch(a0 - 3, Un, fn);
#pragma unroll
    for (int f = 0; f < NF; ++f) Lk[f] = Uk[f] = U0k[f] = T(0);
#pragma unroll 2       // by two: 17.5 -> 17.7 G; by five: 16.6 G under the register cap
    for (int j = a0 - 3; j <= a1 + 2; ++j) {
        const int cnt = j - (a0 - 3);
        T U[NF];
        const bool fl = fn;
#pragma unroll
        for (int f = 0; f < NF; ++f) U[f] = Un[f];
        if (j < a1 + 2) fetch(j + 1, Un, fn);
        // cell j-3 completes at this step (cnt >= 6): its operands were
        // fetched one step earlier
        T Lc[NF], Uc_[NF], U0c[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            Lc[f] = Lk[f];
            Uc_[f] = Uk[f];
            U0c[f] = U0k[f];
        }
        if (cnt >= 5 && j < a1 + 2) fetch_cell(j - 2, Lk, Uk, U0k);
        if (fl) U[1 + PA] = -U[1 + PA];
        T W[NF];
        cons_to_prim(U, A.gm1, W);
        bad |= nonphys(W);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q][f] = w[q + 1][f];
            w[4][f] = W[f];
        }
        if (cnt >= 4) {
            // the pair of cell j-2, the face between j-3 and j-2, cell j-3
            T rv[NF], lv[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f)
                weno5z_pair(w[0][f], w[1][f], w[2][f], w[3][f], w[4][f], rv[f], lv[f]);
            if (cnt >= 5) {
                T F[NF];
                hll_face<PA>(rvp, lv, gamma, gx, F);
                if (cnt >= 6 && xin) {
                    const long long c = base + (long long)(j - 3) * stride;
                    T D[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) D[f] = sub_over_dx(Lc[f], F[f] - Fp[f], A.dxk[AX]);
                    if constexpr (LAST) {
                        T Uo[NF];
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            Uo[f] = two ? madd(T(0.5), U0c[f], T(0.5) * madd(dt, D[f], Uc_[f]))
                                        : madd(dt, D[f], Uc_[f]);
                            A.Uo[f * N + c] = Uo[f];
                        }
                        if (A.rate_slot) {
                            T Wo[NF];
                            cons_to_prim(Uo, A.gm1, Wo);
                            const T r = cell_rate(Wo, gamma, A.act, A.rdx);
                            rate_max = (r > rate_max || r != r) ? r : rate_max;
                        }
                        if (A.tot_partial) {
#pragma unroll
                            for (int f = 0; f < NF; ++f) tot[f] += Uo[f];
                        }
                    } else {
#pragma unroll
                        for (int f = 0; f < NF; ++f) L[f * N + c] = D[f];
                    }
                }
#pragma unroll
                for (int f = 0; f < NF; ++f) Fp[f] = F[f];
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) rvp[f] = rv[f];
        }
    }
    if constexpr (LAST) {
        const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        sweep_epilogue(A, bad, rate_max, tot, blk);
    }
}

// ---------------------------------------------------- radiation energy --
// The advection of E (weno_advect_kernel's scheme: WENO5-Z states of E and of
// the normal velocity, the Rusanov flux) as the same three sweeps on 3D
// meshes: the x sweep writes L, the y' march adds to it, the z' march adds
// its part and forms the Heun stage.  L is one field.

// m / rho: IEEE division in FP64 (the oracle's rounding); FP32 multiplies by
// the approximate reciprocal, as its conversion to primitives does.
__device__ __forceinline__ double sweep_ratio(double m, double rho) { return m / rho; }
__device__ __forceinline__ float sweep_ratio(float m, float rho) { return m * vrcp(rho); }

// E and the velocity along kernel axis AX (momentum slot 1+PA) of cell m of
// the line, through the axis' boundary map.
template <typename T, int AX, int PA>
__device__ __forceinline__ void sweep_ev(const AdvectArgs<T>& A, long long base, int m, int nA,
                                         long long stride, T& e, T& u) {
    bool flip;
    const int sidx = bc_map3(m, nA, A.bc_lo[AX], A.bc_hi[AX], flip);
    const long long c = base + (long long)sidx * stride;
    const T rho = __ldg(A.U + c);
    T mom = __ldg(A.U + (1 + PA) * A.N + c);
    if (flip) mom = -mom;
    e = __ldg(A.Ec + c);
    u = sweep_ratio(mom, rho);
}

template <typename T, int PX>
__global__ void __launch_bounds__(SWEEP_THREADS)
advect_x_kernel(const AdvectArgs<T> A, T* __restrict__ L) {
    __shared__ T win[SWEEP_THREADS / 32][2][WX_WIN];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int n0 = A.n[0], n1 = A.n[1];
    const int yr = blockIdx.y * (SWEEP_THREADS / 32) + wq;     // as in weno_x_kernel
    const bool active = yr < n1;
    const long long base = ((long long)blockIdx.z * n1 + (active ? yr : 0)) * n0;
    const int xs = blockIdx.x * WX_SEG;
    {
        T e, u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            sweep_ev<T, 0, PX>(A, base, xs - 3 + 32 * h + lane, n0, 1, e, u);
            win[wq][0][32 * h + lane] = e;
            win[wq][1][32 * h + lane] = u;
        }
        if (lane < WX_WIN - 64) {
            sweep_ev<T, 0, PX>(A, base, xs + 61 + lane, n0, 1, e, u);
            win[wq][0][64 + lane] = e;
            win[wq][1][64 + lane] = u;
        }
    }
    __syncwarp();
    // two cells per lane, as in weno_x_kernel
    const T* ve = &win[wq][0][2 * lane];
    const T* vu = &win[wq][1][2 * lane];
    T er0, el0, ur0, ul0, er1, el1, ur1, ul1;
    weno5z_pair(ve[0], ve[1], ve[2], ve[3], ve[4], er0, el0);
    weno5z_pair(vu[0], vu[1], vu[2], vu[3], vu[4], ur0, ul0);
    weno5z_pair(ve[1], ve[2], ve[3], ve[4], ve[5], er1, el1);
    weno5z_pair(vu[1], vu[2], vu[3], vu[4], vu[5], ur1, ul1);
    const T eL = __shfl_up_sync(0xffffffffu, er1, 1), uL = __shfl_up_sync(0xffffffffu, ur1, 1);
    const T Fl = rusanov_e(eL, el0, uL, ul0);                   // face c0 - 1/2
    const T Fm = rusanov_e(er0, el1, ur0, ul1);                 // face c0 + 1/2
    const T Fr = __shfl_down_sync(0xffffffffu, Fl, 1);          // face c1 + 1/2
    const int x0 = xs - 1 + 2 * lane;
    if (active && lane >= 1 && x0 < n0) L[base + x0] = sub_over_dx(T(0), Fm - Fl, A.dxk[0]);
    if (active && lane <= 30 && x0 + 1 < n0)
        L[base + x0 + 1] = sub_over_dx(T(0), Fr - Fm, A.dxk[0]);
}

template <typename T, int AX, int PA, bool LAST>
__global__ void __launch_bounds__(SWEEP_THREADS)
advect_march_kernel(const AdvectArgs<T> A, T* __restrict__ L) {
    static_assert(AX == 1 || AX == 2, "the x' axis is the x sweep's");
    const int n0 = A.n[0], n1 = A.n[1];
    const int nA = A.n[AX];
    const int x = blockIdx.x * SWEEP_THREADS + threadIdx.x;
    const bool xin = x < n0;
    const int xl = xin ? x : n0 - 1;
    const int o = blockIdx.y;
    const long long stride = AX == 1 ? (long long)n0 : (long long)n0 * n1;
    const long long base = (AX == 1 ? (long long)o * n1 * n0 : (long long)o * n0) + xl;
    const int a0 = blockIdx.z * A.zchunk;
    const int a1 = min(a0 + A.zchunk, nA);
    const T dt = (T)A.dt;
    const bool two = A.stage == 2;
    // E and u of the last five cells, the upper values of the newest pair's
    // lower neighbour, the last face flux; the next cell and the operands of
    // the cell completing at the next step are fetched one step ahead
    T we[5], wu[5], eUp = T(0), uUp = T(0), Fp = T(0);
#pragma unroll
    for (int q = 0; q < 5; ++q) we[q] = wu[q] = T(0);
    // the next cell's raw values (density, normal momentum, E, wall flip):
    // the velocity is formed when the cell enters the window, so the loads
    // have a whole step to arrive
    auto fetch = [&](int m, T& r, T& mo, T& e, bool& flip) {
        const int sidx = bc_map3(m, nA, A.bc_lo[AX], A.bc_hi[AX], flip);
        const long long c = base + (long long)sidx * stride;
        r = __ldg(A.U + c);
        mo = __ldg(A.U + (1 + PA) * A.N + c);
        e = __ldg(A.Ec + c);
    };
    T rn, mn, en, Lk = T(0), E0k = T(0);
    bool fn;
    fetch(a0 - 3, rn, mn, en, fn);
#pragma unroll 5       // the window's five registers rotate by renaming (0.86 -> 0.82 ms per step)
    for (int j = a0 - 3; j <= a1 + 2; ++j) {
        const int cnt = j - (a0 - 3);
        const T rj = rn, ej = en;
        const T mj = fn ? -mn : mn;
        if (j < a1 + 2) fetch(j + 1, rn, mn, en, fn);
        const T uj = sweep_ratio(mj, rj);
        const T Lc = Lk, E0c = E0k;
        if (cnt >= 5 && j < a1 + 2) {
            const long long ck = base + (long long)(j - 2) * stride;
            Lk = L[ck];
            if (LAST && two) E0k = A.E0[ck];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            we[q] = we[q + 1];
            wu[q] = wu[q + 1];
        }
        we[4] = ej;
        wu[4] = uj;
        if (cnt >= 4) {
            T eu, el, uu, ul;
            weno5z_pair(we[0], we[1], we[2], we[3], we[4], eu, el);
            weno5z_pair(wu[0], wu[1], wu[2], wu[3], wu[4], uu, ul);
            if (cnt >= 5) {
                const T F = rusanov_e(eUp, el, uUp, ul);
                if (cnt >= 6 && xin) {
                    // cell j-3, whose E is we[1]
                    const long long c = base + (long long)(j - 3) * stride;
                    const T D = sub_over_dx(Lc, F - Fp, A.dxk[AX]);
                    if constexpr (LAST) {
                        const T ec = we[1];
                        A.Eo[c] = two ? madd(T(0.5), E0c, T(0.5) * madd(dt, D, ec)) : madd(dt, D, ec);
                    } else {
                        L[c] = D;
                    }
                }
                Fp = F;
            }
            eUp = eu;
            uUp = uu;
        }
    }
}

}  // namespace hh
