// Batched persistent stage kernel: many independent 1D and 2D problems of
// uneven size in one launch.
//
// Every block is persistent: it takes the next problem from a queue (one
// atomic counter over a largest-first order, so no block ever waits) and runs
// all of that problem's steps by itself:
//     r = block max of the signal rate of U          (first step only)
//     repeat nsteps times:
//         dt = cfl / r                                 (FP64)
//         stage 1 over the problem's tiles: U -> W
//         stage 2 over the problem's tiles: (U, W) -> U, signal rate fused
//         r = block max of that rate;  t += dt         (FP64)
// The tiles are evaluated by the same stage_tile code as the single-problem
// kernel, so a problem advanced here matches the same problem advanced alone
// bit for bit.  State is read through the coherent cache path because the
// block rewrites it within the launch.  A block never waits on another block:
// problems are disjoint and the rate reduction is block-local.
#pragma once
#include "launch.h"
#include "stage_kernel.cuh"

namespace hh {

template <typename T>
struct BatchArgs {
    T* U;                              // packed states, updated in place
    T* W;                              // packed intermediate stage (same layout)
    const BatchProblem* probs;
    const int* order;                  // queue order (largest problems first)
    int nprob;
    int nsteps;
    double cfl;
    double* t;                         // per-problem time, FP64, advanced in place
    int* counter;                      // queue head, zeroed before the launch
    int* status;
};

template <typename T>
__device__ __forceinline__ StageArgs<T> batch_stage_args(const BatchProblem& P, T* U, T* W,
                                                        int stage, double dt) {
    StageArgs<T> A;
    const bool two_d = P.ny > 1;
    A.U0 = U;
    A.Uc = stage == 1 ? U : W;
    A.Uo = stage == 1 ? W : U;
    A.N = (long long)P.nx * P.ny;
    A.n[0] = P.nx;
    A.n[1] = P.ny;
    A.n[2] = 1;
    for (int a = 0; a < 3; ++a) {
        A.bc_lo[a] = P.bc;
        A.bc_hi[a] = P.bc;
    }
    const double dx = 1.0 / P.nx, dy = 1.0 / P.ny;
    A.gamma = (T)P.gamma;
    A.gm1 = (T)(P.gamma - 1.0);
    A.igm1 = (T)(1.0 / (P.gamma - 1.0));
    const bool f64 = sizeof(T) == 8;
    A.dxk[0] = f64 ? (T)dx : (T)(1.0 / dx);
    A.dxk[1] = f64 ? (T)dy : (T)(1.0 / dy);
    A.dxk[2] = T(1);
    A.rdx[0] = A.dxk[0];
    A.rdx[1] = A.dxk[1];
    A.rdx[2] = T(1);
    A.act[0] = true;
    A.act[1] = two_d;
    A.act[2] = false;
    A.dt = dt;
    A.dt_dev = nullptr;
    A.stage = stage;
    A.zchunk = 1;
    A.zlo = 0;
    A.zhi = 1;
    A.rate_slot = nullptr;
    A.tot_partial = nullptr;
    A.status = nullptr;
    A.tmap = nullptr;
    return A;
}

// Block-wide maximum of a non-negative rate (NaN propagates), as a double.
template <typename T, int NT>
__device__ __forceinline__ double block_rate_max(T r, unsigned long long* red) {
    unsigned long long b = rate_bits(r);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
        b = v > b ? v : b;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();                    // red[] free from any earlier use
    if (lane == 0) red[warp] = b;
    __syncthreads();
    unsigned long long m = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) m = red[w] > m ? red[w] : m;
    return __longlong_as_double((long long)m);
}

// TX1: tile width of 1D problems; TX2 x TY2: tile of 2D problems.  Both use
// the same block of TX1 == TX2 * TY2 threads.
template <typename T, int TX1, int TX2, int TY2>
__global__ void __launch_bounds__(TX1) batched_kernel(const BatchArgs<T> B) {
    static_assert(TX1 == TX2 * TY2, "1D and 2D tiles share one block size");
    constexpr int NT = TX1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ unsigned long long red[NT / 32];
    __shared__ int s_next;
    const int tid = threadIdx.x;
    bool bad = false;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_next = atomicAdd(B.counter, 1);
        __syncthreads();
        const int qi = s_next;
        if (qi >= B.nprob) break;
        const BatchProblem P = B.probs[B.order[qi]];
        T* U = B.U + P.off;
        T* W = B.W + P.off;
        const bool two_d = P.ny > 1;
        const long long N = (long long)P.nx * P.ny;

        // signal rate of the initial state
        StageArgs<T> A1 = batch_stage_args<T>(P, U, W, 1, 0.0);
        T r0 = T(0);
        for (long long c = tid; c < N; c += NT) {
            T Uc[NF], Wp[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) Uc[f] = U[f * N + c];
            cons_to_prim(Uc, A1.gm1, Wp);
            bad |= nonphys(Wp);
            const T r = cell_rate(Wp, A1.gamma, A1.act, A1.rdx);
            r0 = (r > r0 || r != r) ? r : r0;
        }
        double rate = block_rate_max<T, NT>(r0, red);
        double t = B.t[B.order[qi]];

        for (int step = 0; step < B.nsteps; ++step) {
            double dt;
            if (!(rate > 0.0) || isinf(rate)) {
                dt = 0.0;
                bad = true;
            } else {
                dt = B.cfl / rate;
            }
            TileAcc<T> acc;
            acc.rate_max = T(0);
            acc.bad = false;
#pragma unroll
            for (int f = 0; f < NF; ++f) acc.tot[f] = T(0);
            int tile = 0;                   // tile count: the parity of stage_tile's plane
            for (int stage = 1; stage <= 2; ++stage) {
                StageArgs<T> A = batch_stage_args<T>(P, U, W, stage, dt);
                // non-null: stage_tile folds the signal rate of the new state
                // into acc (it never writes through the pointer)
                A.rate_slot = stage == 2 ? red : nullptr;
                if (two_d) {
                    for (int y0 = 0; y0 < P.ny; y0 += TY2)
                        for (int x0 = 0; x0 < P.nx; x0 += TX2)
                            stage_tile<T, TX2, TY2, 2, 0, 1, false>(A, smem_raw, x0, y0, 0, 1, acc,
                                                                    tile++);
                } else {
                    for (int x0 = 0; x0 < P.nx; x0 += TX1)
                        stage_tile<T, TX1, 1, 1, 0, 0, false>(A, smem_raw, x0, 0, 0, 1, acc,
                                                              tile++);
                }
                __syncthreads();            // every cell of this stage written
            }
            bad |= acc.bad;
            rate = block_rate_max<T, NT>(acc.rate_max, red);
            t = t + dt;
        }
        if (tid == 0) B.t[B.order[qi]] = t;
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(B.status, 1);
}

}  // namespace hh
