// Per-element-type launchers of the WENO5-Z + HLL stage kernel.  Included by
// exactly one translation unit per type with HH_T (float or double) and
// HH_SUFFIX (f32 or f64) defined.
#pragma once
#include "devattr.h"
#include "weno.cuh"
#include "weno_launch.h"
#include "weno_sweep.cuh"

#define HH_WCAT2(a, b) a##b
#define HH_WCAT(a, b) HH_WCAT2(a, b)

namespace hh {
namespace {

using T = HH_T;

template <typename V> inline V wcdiv(V a, V b) { return (a + b - 1) / b; }

inline T width_param_w(double dx) { return sizeof(T) == 8 ? (T)dx : (T)(1.0 / dx); }

// The kernel arguments of one stage (the same fields the PLM kernels get).
StageArgs<T> weno_args(const MeshDesc& m, int zchunk, const StageCall& c) {
    StageArgs<T> A{};
    A.U0 = static_cast<const T*>(c.U0);
    A.Uc = static_cast<const T*>(c.Uc);
    A.Uo = static_cast<T*>(c.Uo);
    A.N = m.N;
    for (int a = 0; a < 3; ++a) {
        A.n[a] = m.n[a];
        A.bc_lo[a] = m.bc_lo[a];
        A.bc_hi[a] = m.bc_hi[a];
        A.dxk[a] = width_param_w(m.dxk[a]);
        A.rdx[a] = width_param_w(m.dx[a]);
        A.act[a] = m.act[a];
    }
    A.gamma = (T)m.gamma;
    A.gm1 = (T)(m.gamma - 1.0);
    A.igm1 = (T)(1.0 / (m.gamma - 1.0));
    A.dt = c.dt;
    A.dt_dev = c.dt_dev;
    A.stage = c.stage;
    A.zchunk = zchunk > 0 ? zchunk : 1;
    A.rate_slot = c.rate_slot;
    A.tot_partial = c.tot_partial;
    A.status = c.status;
    A.tmap = nullptr;
    return A;
}

template <int TX, int TY, int DIM, int PX, int PY>
cudaError_t run_weno(const MeshDesc& m, const StageCall& c, cudaStream_t s) {
    const TileDesc td = tile_desc(DIM, 0);
    static_assert(DIM < 2 || TY > 1, "2D/3D tiles have rows");
    const StageArgs<T> A = weno_args(m, td.zc, c);
    const dim3 grid(wcdiv(m.n[0], TX), DIM >= 2 ? wcdiv(m.n[1], TY) : 1,
                    DIM == 3 ? wcdiv(m.n[2], A.zchunk) : 1);
    constexpr size_t smem = WenoSmem<T, TX, TY, DIM>::bytes;
    auto kern = weno_stage_kernel<T, TX, TY, DIM, PX, PY>;
    static std::atomic<unsigned long long> attr{0};
    const cudaError_t e = smem_attr_once(kern, smem, attr);
    if (e != cudaSuccess) return e;
    kern<<<grid, TX * TY, smem, s>>>(A);
    return cudaGetLastError();
}

// The three sweeps of one stage on a 3D mesh (weno_sweep.cuh).
cudaError_t run_weno_sweeps(const MeshDesc& m, const StageCall& c, cudaStream_t s) {
    const StageArgs<T> A = weno_args(m, WENO_SWEEP_CHUNK, c);
    T* L = static_cast<T*>(c.scratch);
    if (m.n[1] > 65535 || m.n[2] > 65535) return cudaErrorInvalidValue;
    const dim3 gx(wcdiv(m.n[0], WX_SEG), wcdiv(m.n[1], SWEEP_THREADS / 32), m.n[2]);
    weno_x_kernel<T, 0><<<gx, SWEEP_THREADS, 0, s>>>(A, L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 gy(wcdiv(m.n[0], SWEEP_THREADS), m.n[2], wcdiv(m.n[1], WENO_SWEEP_CHUNK));
    weno_march_kernel<T, 1, 1, false><<<gy, SWEEP_THREADS, 0, s>>>(A, L);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 gz(wcdiv(m.n[0], SWEEP_THREADS), m.n[1], wcdiv(m.n[2], WENO_SWEEP_CHUNK));
    weno_march_kernel<T, 2, 2, true><<<gz, SWEEP_THREADS, 0, s>>>(A, L);
    return cudaGetLastError();
}

template <int TX, int TY, int DIM, int PX, int PY>
cudaError_t run_advect(const MeshDesc& m, const AdvectArgs<T>& A, cudaStream_t s) {
    const dim3 grid(wcdiv(m.n[0], TX), DIM >= 2 ? wcdiv(m.n[1], TY) : 1,
                    DIM == 3 ? wcdiv(m.n[2], A.zchunk) : 1);
    constexpr size_t smem = AdvectSmem<T, TX, TY, DIM>::bytes;
    auto kern = weno_advect_kernel<T, TX, TY, DIM, PX, PY>;
    static std::atomic<unsigned long long> attr{0};
    const cudaError_t e = smem_attr_once(kern, smem, attr);
    if (e != cudaSuccess) return e;
    kern<<<grid, TX * TY, smem, s>>>(A);
    return cudaGetLastError();
}

// The three sweeps of one advection stage on a 3D mesh (weno_sweep.cuh).
cudaError_t run_advect_sweeps(const MeshDesc& m, const AdvectArgs<T>& A, T* L, cudaStream_t s) {
    if (m.n[1] > 65535 || m.n[2] > 65535) return cudaErrorInvalidValue;
    const dim3 gx(wcdiv(m.n[0], WX_SEG), wcdiv(m.n[1], SWEEP_THREADS / 32), m.n[2]);
    advect_x_kernel<T, 0><<<gx, SWEEP_THREADS, 0, s>>>(A, L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 gy(wcdiv(m.n[0], SWEEP_THREADS), m.n[2], wcdiv(m.n[1], WENO_SWEEP_CHUNK));
    advect_march_kernel<T, 1, 1, false><<<gy, SWEEP_THREADS, 0, s>>>(A, L);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 gz(wcdiv(m.n[0], SWEEP_THREADS), m.n[1], wcdiv(m.n[2], WENO_SWEEP_CHUNK));
    advect_march_kernel<T, 2, 2, true><<<gz, SWEEP_THREADS, 0, s>>>(A, L);
    return cudaGetLastError();
}

}  // namespace

cudaError_t HH_WCAT(launch_advect_E_stage_, HH_SUFFIX)(const MeshDesc& m, int stage, const void* U,
                                                       const void* E0, const void* Ec, void* Eo,
                                                       double dt, void* scratch, cudaStream_t s) {
    for (int a = 0; a < 3; ++a)
        if (m.n[a] > 1 && m.n[a] < WENO_G) return cudaErrorInvalidValue;
    AdvectArgs<T> A{};
    A.U = static_cast<const T*>(U);
    A.E0 = static_cast<const T*>(E0);
    A.Ec = static_cast<const T*>(Ec);
    A.Eo = static_cast<T*>(Eo);
    A.N = m.N;
    for (int a = 0; a < 3; ++a) {
        A.n[a] = m.n[a];
        A.bc_lo[a] = m.bc_lo[a];
        A.bc_hi[a] = m.bc_hi[a];
        A.dxk[a] = width_param_w(m.dxk[a]);
    }
    A.dt = dt;
    A.stage = stage;
    A.zchunk = tile_desc(3, 0).zc;
    if (m.dim == 3 && scratch) {
        A.zchunk = WENO_SWEEP_CHUNK;
        return run_advect_sweeps(m, A, static_cast<T*>(scratch), s);
    }
    if (m.dim == 3) return run_advect<32, 8, 3, 0, 1>(m, A, s);
    if (m.dim == 2) {
        if (m.px == 0 && m.py == 1) return run_advect<32, 8, 2, 0, 1>(m, A, s);
        if (m.px == 0 && m.py == 2) return run_advect<32, 8, 2, 0, 2>(m, A, s);
        return run_advect<32, 8, 2, 1, 2>(m, A, s);
    }
    if (m.dim == 1) {
        if (m.px == 0) return run_advect<128, 1, 1, 0, 0>(m, A, s);
        if (m.px == 1) return run_advect<128, 1, 1, 1, 0>(m, A, s);
        return run_advect<128, 1, 1, 2, 0>(m, A, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t HH_WCAT(launch_weno_stage_, HH_SUFFIX)(const MeshDesc& m, const StageCall& c,
                                                   cudaStream_t s) {
    // the tile of each dimension is entry 0 of its table: 32 x 8 (z-chunk 32), 32 x 8, 128 x 1
    static_assert(TILES3[0].tx == 32 && TILES3[0].ty == 8 && TILES2[0].tx == 32 &&
                      TILES2[0].ty == 8 && TILES1[0].tx == 128,
                  "the WENO launcher runs tile 0 of each table");
    for (int a = 0; a < 3; ++a)
        if (m.n[a] > 1 && m.n[a] < WENO_G) return cudaErrorInvalidValue;
    if (m.dim == 3) return c.scratch ? run_weno_sweeps(m, c, s) : run_weno<32, 8, 3, 0, 1>(m, c, s);
    if (m.dim == 2) {
        if (m.px == 0 && m.py == 1) return run_weno<32, 8, 2, 0, 1>(m, c, s);
        if (m.px == 0 && m.py == 2) return run_weno<32, 8, 2, 0, 2>(m, c, s);
        return run_weno<32, 8, 2, 1, 2>(m, c, s);
    }
    if (m.dim == 1) {
        if (m.px == 0) return run_weno<128, 1, 1, 0, 0>(m, c, s);
        if (m.px == 1) return run_weno<128, 1, 1, 1, 0>(m, c, s);
        return run_weno<128, 1, 1, 2, 0>(m, c, s);
    }
    return cudaErrorInvalidValue;               // no active axis: the PLM launcher handles it
}

}  // namespace hh
