// Per-element-type instantiation of the stage, rate and totals kernels and
// their launchers.  Included by exactly one translation unit per type with
// HH_T defined (float or double) and HH_SUFFIX (f32 or f64).
#pragma once
#include <cstdlib>
#include <cstring>
#include <utility>

#include "adjoint.cuh"
#include "batched.cuh"
#include "devattr.h"
#include "launch.h"
#include "stage_kernel.cuh"
#include "stage_tma.cuh"
#ifdef HH_WS
#include "stage_ws.cuh"
#endif

namespace hh {

namespace {

using T = HH_T;

template <typename V> __host__ __device__ inline V cdiv(V a, V b) { return (a + b - 1) / b; }

inline T width_param(double dx) {
    // FP64 kernels divide by dx; FP32 kernels multiply by 1/dx
    return sizeof(T) == 8 ? (T)dx : (T)(1.0 / dx);
}

StageArgs<T> make_args(const MeshDesc& m, const TileDesc& td, const StageCall& c) {
    StageArgs<T> A;
    A.U0 = static_cast<const T*>(c.U0);
    A.Uc = static_cast<const T*>(c.Uc);
    A.Uo = static_cast<T*>(c.Uo);
    A.N = m.N;
    for (int a = 0; a < 3; ++a) {
        A.n[a] = m.n[a];
        A.bc_lo[a] = m.bc_lo[a];
        A.bc_hi[a] = m.bc_hi[a];
        A.dxk[a] = width_param(m.dxk[a]);
        A.rdx[a] = width_param(m.dx[a]);
        A.act[a] = m.act[a];
    }
    A.gamma = (T)m.gamma;
    A.gm1 = (T)(m.gamma - 1.0);
    A.igm1 = (T)(1.0 / (m.gamma - 1.0));
    A.dt = c.dt;
    A.dt_dev = c.dt_dev;
    A.stage = c.stage;
    A.zchunk = td.zc > 0 ? td.zc : 1;
    A.zlo = m.dim == 3 ? c.zlo : 0;
    A.zhi = m.dim == 3 ? (c.zhi < 0 ? m.n[2] : c.zhi) : 1;
    A.rate_slot = c.rate_slot;
    A.tot_partial = c.tot_partial;
    A.status = c.status;
    A.tmap = nullptr;
    A.starve_tma = false;
    A.zg[0] = static_cast<const T*>(c.zg[0]);
    A.zg[1] = static_cast<const T*>(c.zg[1]);
    return A;
}

template <int TX, int TY, int DIM, int PX, int PY>
cudaError_t run_stage(const MeshDesc& m, const TileDesc& td, const StageCall& c, cudaStream_t s) {
    StageArgs<T> A = make_args(m, td, c);
    dim3 grid(cdiv(m.n[0], TX), DIM >= 2 ? cdiv(m.n[1], TY) : 1,
              DIM == 3 ? cdiv(A.zhi - A.zlo, A.zchunk) : 1);
    const size_t smem = StageSmem<T, TX, TY, DIM>::bytes;
    auto kern = stage_kernel<T, TX, TY, DIM, PX, PY, false>;
    static std::atomic<unsigned long long> attr{0};
    cudaError_t e = smem_attr_once(kern, smem, attr);
    if (e != cudaSuccess) return e;
    kern<<<grid, TX * TY, smem, s>>>(A);
    return cudaGetLastError();
}

// ---- TMA path (3D meshes whose rows are 16-byte multiples) ----

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor map of U as a 4D tensor (x, y, z, field) with box (bx, by, 1, 5).
bool encode_state_map(CUtensorMap* map, const void* base, const MeshDesc& m, int bx, int by) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t es = sizeof(T);
    const cuuint64_t dims[4] = {(cuuint64_t)m.n[0], (cuuint64_t)m.n[1], (cuuint64_t)m.n[2], 5};
    const cuuint64_t strides[3] = {m.n[0] * es, (cuuint64_t)m.n[0] * m.n[1] * es,
                                   (cuuint64_t)m.N * es};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 5};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = fn(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                          4, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Tensor map of a ghost-plane buffer [5][2][ny][nx] (x, y, plane, field) with
// box (bx, by, 1, 5).
bool encode_ghost_map(CUtensorMap* map, const void* base, const MeshDesc& m, int bx, int by) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t es = sizeof(T);
    const cuuint64_t dims[4] = {(cuuint64_t)m.n[0], (cuuint64_t)m.n[1], 2, 5};
    const cuuint64_t strides[3] = {m.n[0] * es, (cuuint64_t)m.n[0] * m.n[1] * es,
                                   2 * (cuuint64_t)m.n[0] * m.n[1] * es};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 5};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = fn(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                          4, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Ghost-plane maps of the BC_HALO z faces (boxes of the main box and the two
// strips); faces of other kinds keep zeroed maps that no load uses.
template <class Maps>
bool encode_ghost_maps(Maps& maps, const MeshDesc& m, const StageCall& c, int bx, int by) {
    for (int s = 0; s < 2; ++s) {
        std::memset(&maps.gmain[s], 0, sizeof(CUtensorMap));
        std::memset(&maps.gxstrip[s], 0, sizeof(CUtensorMap));
        std::memset(&maps.gystrip[s], 0, sizeof(CUtensorMap));
        const bool halo = (s == 0 ? m.bc_lo[2] : m.bc_hi[2]) == BC_HALO;
        if (!halo) continue;
        if (!c.zg[s] || (reinterpret_cast<uintptr_t>(c.zg[s]) & 15u) != 0) return false;
        if (!encode_ghost_map(&maps.gmain[s], c.zg[s], m, bx, by) ||
            !encode_ghost_map(&maps.gxstrip[s], c.zg[s], m, 4, by) ||
            !encode_ghost_map(&maps.gystrip[s], c.zg[s], m, bx, 2))
            return false;
    }
    return true;
}

// The TMA kernel needs 3 active axes, rows (and so every stride) a multiple of
// 16 bytes, at least 4 cells along x (the periodic x strip), a 16-byte
// aligned base and element indices of all five fields below 2^32; otherwise
// the plain kernel runs.
bool tma_eligible(const MeshDesc& m, const void* Uc) {
    const int per16 = 16 / (int)sizeof(T);
    return m.dim == 3 && m.n[0] % per16 == 0 && m.n[0] >= 4 && 5 * m.N < (1ll << 32) &&
           (reinterpret_cast<uintptr_t>(Uc) & 15u) == 0 && encode_fn() != nullptr;
}

constexpr size_t SMEM_LIMIT = 232448;     // 227 KB opt-in per block

template <int TX, int TY>
cudaError_t run_stage_tma(const MeshDesc& m, const TileDesc& td, const StageCall& c,
                          cudaStream_t s, bool& used) {
    using L = TmaLayout<T, TX, TY, 2>;                 // the larger of the two stages
    used = false;
    if constexpr (L::bytes > SMEM_LIMIT) {
        return cudaSuccess;
    } else {
        TmaMaps maps;
        if (!encode_state_map(&maps.main, c.Uc, m, TX + 8, TY + 4) ||
            !encode_state_map(&maps.xstrip, c.Uc, m, 4, TY + 4) ||
            !encode_state_map(&maps.ystrip, c.Uc, m, TX + 8, 2) ||
            !encode_state_map(&maps.u0, c.stage == 2 ? c.U0 : c.Uc, m, TX, TY) ||
            !encode_ghost_maps(maps, m, c, TX + 8, TY + 4))
            return cudaSuccess;
        StageArgs<T> A = make_args(m, td, c);
        // failure-path test: HARD_HYDRO_STARVE_TMA=1 makes the ring's waits
        // run out (the stage then reports HARD_ETIMEOUT and leaves Uout unset)
        const char* starve = std::getenv("HARD_HYDRO_STARVE_TMA");
        A.starve_tma = starve && starve[0] == '1';
        dim3 grid(cdiv(m.n[0], TX), cdiv(m.n[1], TY), cdiv(A.zhi - A.zlo, A.zchunk));
        auto kern = c.stage == 1 ? stage_tma_kernel<T, TX, TY, 1> : stage_tma_kernel<T, TX, TY, 2>;
        constexpr size_t b1 = TmaLayout<T, TX, TY, 1>::bytes, b2 = L::bytes;
        static std::atomic<unsigned long long> attr1{0}, attr2{0};
        cudaError_t e = c.stage == 1 ? smem_attr_once(stage_tma_kernel<T, TX, TY, 1>, b1, attr1)
                                     : smem_attr_once(stage_tma_kernel<T, TX, TY, 2>, b2, attr2);
        if (e != cudaSuccess) return e;
        kern<<<grid, TX * TY, c.stage == 1 ? b1 : b2, s>>>(A, maps);
        used = true;
        return cudaGetLastError();
    }
}

#ifdef HH_WS
// Warp-specialised FP32 kernel (stage_ws.cuh): tiles 32 x TY with NCW
// converter warps and RPW tile rows per face warp; blocks per SM by tile
// height.
#ifndef HH_WS_NCW8
#define HH_WS_NCW8 2
#endif
#ifndef HH_WS_NCW16
#define HH_WS_NCW16 3
#endif
#ifndef HH_WS_RPW8
#define HH_WS_RPW8 1
#endif
template <int TY> struct WsConf {
    static constexpr int NCW = TY >= 16 ? HH_WS_NCW16 : (TY >= 8 ? HH_WS_NCW8 : 1);
    static constexpr int RPW = TY == 8 ? HH_WS_RPW8 : 1;
};

template <int TY>
cudaError_t run_stage_ws(const MeshDesc& m, const TileDesc& td, const StageCall& c,
                         cudaStream_t s, bool& used) {
    constexpr int NCW = WsConf<TY>::NCW, RPW = WsConf<TY>::RPW;
    using L1 = WsLayout<32, TY, NCW, 1, RPW>;
    using L2 = WsLayout<32, TY, NCW, 2, RPW>;
    used = false;
    if constexpr (L2::bytes > SMEM_LIMIT) {
        return cudaSuccess;
    } else {
        if ((reinterpret_cast<uintptr_t>(c.Uo) & 15u) != 0 ||
            (c.stage == 2 && (reinterpret_cast<uintptr_t>(c.U0) & 15u) != 0))
            return cudaSuccess;
        WsMaps maps;
        if (!encode_state_map(&maps.main, c.Uc, m, L1::HXC, L1::HYC) ||
            !encode_state_map(&maps.xstrip, c.Uc, m, 4, L1::HYC) ||
            !encode_state_map(&maps.ystrip, c.Uc, m, L1::HXC, 2) ||
            !encode_state_map(&maps.u0, c.stage == 2 ? c.U0 : c.Uc, m, 32, TY) ||
            !encode_state_map(&maps.out, c.Uo, m, 32, TY) ||
            !encode_ghost_maps(maps, m, c, L1::HXC, L1::HYC))
            return cudaSuccess;
        StageArgs<T> A = make_args(m, td, c);
        // failure-path test: HARD_HYDRO_STARVE_TMA=1 makes the ring's waits
        // run out (the stage then reports HARD_ETIMEOUT and leaves Uout unset)
        const char* starve = std::getenv("HARD_HYDRO_STARVE_TMA");
        A.starve_tma = starve && starve[0] == '1';
        dim3 grid(cdiv(m.n[0], 32), cdiv(m.n[1], TY), cdiv(A.zhi - A.zlo, A.zchunk));
        static std::atomic<unsigned long long> attr1{0}, attr2{0};
        cudaError_t e;
        if (c.stage == 1) {
            e = smem_attr_once(stage_ws_kernel<32, TY, NCW, 1, RPW>, L1::bytes, attr1);
            if (e != cudaSuccess) return e;
            stage_ws_kernel<32, TY, NCW, 1, RPW><<<grid, L1::NT, L1::bytes, s>>>(A, maps);
        } else {
            e = smem_attr_once(stage_ws_kernel<32, TY, NCW, 2, RPW>, L2::bytes, attr2);
            if (e != cudaSuccess) return e;
            stage_ws_kernel<32, TY, NCW, 2, RPW><<<grid, L2::NT, L2::bytes, s>>>(A, maps);
        }
        used = true;
        return cudaGetLastError();
    }
}
#endif

// No active axis: L(U) = 0, the stage combine alone.
__global__ void pointwise_stage_kernel(const T* U0, const T* Uc, T* Uo, long long n5, double dt,
                                       const double* dt_dev, int stage) {
    const T d = (T)(dt_dev ? *dt_dev : dt);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n5;
         q += (long long)gridDim.x * blockDim.x) {
        const T L = T(0);
        Uo[q] = stage == 1 ? madd(d, L, Uc[q]) : madd(T(0.5), U0[q], T(0.5) * madd(d, L, Uc[q]));
    }
}

__global__ void rate_kernel(const T* __restrict__ U, long long N, T gamma, T gm1, bool a0,
                            bool a1, bool a2, T r0, T r1, T r2, unsigned long long* slot,
                            int* status) {
    const bool act[3] = {a0, a1, a2};
    const T rdx[3] = {r0, r1, r2};
    T rmax = T(0);
    bool bad = false;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        T Uc[NF], W[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) Uc[f] = __ldg(U + f * N + c);
        cons_to_prim(Uc, gm1, W);
        bad |= nonphys(W);
        T r = cell_rate(W, gamma, act, rdx);
        rmax = (r > rmax || r != r) ? r : rmax;
    }
    __shared__ unsigned long long red[32];
    unsigned long long b = rate_bits(rmax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
        b = v > b ? v : b;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = b;
    const int any_bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = red[w] > b ? red[w] : b;
        b = red[0] > b ? red[0] : b;
        atomicMax(slot, b);
        if (any_bad) atomicOr(status, 1);
    }
}

constexpr int TOT_BLOCKS = TOTALS_BLOCKS;
constexpr int TOT_THREADS = 256;

__global__ void totals_kernel(const T* __restrict__ U, long long N, double* partial) {
    double s[NF] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int f = 0; f < NF; ++f) s[f] += (double)__ldg(U + f * N + c);
    }
    __shared__ double red[TOT_THREADS / 32][NF];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        double v = s[f];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][f] = v;
    }
    __syncthreads();
    if (threadIdx.x < NF) {
        double v = 0.0;
        for (int w = 0; w < TOT_THREADS / 32; ++w) v += red[w][threadIdx.x];
        partial[blockIdx.x * NF + threadIdx.x] = v;
    }
}

template <int DIM, int PX, int PY>
cudaError_t dispatch_tile(const MeshDesc& m, int kernel, int tile, const StageCall& c,
                          cudaStream_t s) {
    const TileDesc td = tile_desc(DIM, tile);
    if constexpr (DIM == 3) {
        // the TMA kernel carries the rate / totals epilogue for stage 2 only
        const bool epi_ok = c.stage == 2 || (!c.rate_slot && !c.tot_partial);
        if (kernel == 0 && epi_ok && tma_eligible(m, c.Uc)) {
            bool used = false;
            cudaError_t e;
#ifdef HH_WS
            switch (tile) {
                case 0: case 1: e = run_stage_ws<8>(m, td, c, s, used); break;
                case 2: case 5: e = run_stage_ws<16>(m, td, c, s, used); break;
                case 3: e = cudaSuccess; break;            // 64-wide tiles: no warp-per-row form
                default: e = run_stage_ws<4>(m, td, c, s, used); break;
            }
#else
            switch (tile) {
                case 0: case 1: e = run_stage_tma<32, 8>(m, td, c, s, used); break;
                case 2: case 5: e = run_stage_tma<32, 16>(m, td, c, s, used); break;
                case 3: e = run_stage_tma<64, 8>(m, td, c, s, used); break;
                default: e = run_stage_tma<32, 4>(m, td, c, s, used); break;
            }
#endif
            if (used || e != cudaSuccess) return e;
        }
        switch (tile) {
            case 0: case 1: return run_stage<32, 8, 3, 0, 1>(m, td, c, s);
            case 2: case 5: return run_stage<32, 16, 3, 0, 1>(m, td, c, s);
            case 3: return run_stage<64, 8, 3, 0, 1>(m, td, c, s);
            default: return run_stage<32, 4, 3, 0, 1>(m, td, c, s);
        }
    } else if constexpr (DIM == 2) {
        if constexpr (PX != 0 || PY != 1) {
            return run_stage<32, 8, 2, PX, PY>(m, tile_desc(2, 0), c, s);
        } else {
            switch (tile) {
                case 0: return run_stage<32, 8, 2, 0, 1>(m, td, c, s);
                case 1: return run_stage<32, 16, 2, 0, 1>(m, td, c, s);
                default: return run_stage<64, 8, 2, 0, 1>(m, td, c, s);
            }
        }
    } else {
        if constexpr (PX != 0) {
            return run_stage<128, 1, 1, PX, 0>(m, tile_desc(1, 0), c, s);
        } else {
            if (tile == 0) return run_stage<128, 1, 1, 0, 0>(m, td, c, s);
            return run_stage<256, 1, 1, 0, 0>(m, td, c, s);
        }
    }
}

template <int TX1, int TX2, int TY2>
cudaError_t run_batched(const BatchCall& c, cudaStream_t s) {
    constexpr size_t s1 = StageSmem<T, TX1, 1, 1>::bytes, s2 = StageSmem<T, TX2, TY2, 2>::bytes;
    constexpr size_t smem = s1 > s2 ? s1 : s2;
    auto kern = batched_kernel<T, TX1, TX2, TY2>;
    static PerDeviceInt grids;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int grid = grids.get(dev);
    if (grid == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int sms = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX1, smem);
        if (e != cudaSuccess) return e;
        grid = sms * (per_sm > 0 ? per_sm : 1);
        grids.set(dev, grid);
    }
    BatchArgs<T> B;
    B.U = static_cast<T*>(c.U);
    B.W = static_cast<T*>(c.W);
    B.probs = c.probs;
    B.order = c.order;
    B.nprob = c.nprob;
    B.nsteps = c.nsteps;
    B.cfl = c.cfl;
    B.t = c.t;
    B.counter = c.counter;
    B.status = c.status;
    const int blocks = grid < c.nprob ? grid : c.nprob;
    kern<<<blocks, TX1, smem, s>>>(B);
    return cudaGetLastError();
}

AdjArgs<T> make_adj(const MeshDesc& m, const AdjointCall& c) {
    AdjArgs<T> A;
    A.Uc = static_cast<const T*>(c.Uc);
    A.gout = static_cast<const T*>(c.G);
    A.lam = (T)c.lam;
    A.gW = static_cast<T*>(c.gW);
    A.g_gamma = c.g_gamma;
    A.N = m.N;
    for (int k = 0; k < 3; ++k) {
        A.n[k] = m.n[k];
        A.bc_lo[k] = m.bc_lo[k];
        A.bc_hi[k] = m.bc_hi[k];
        A.dxk[k] = width_param(m.dxk[k]);
    }
    A.gamma = (T)m.gamma;
    A.gm1 = (T)(m.gamma - 1.0);
    for (int k = 0; k < 2; ++k) {
        A.zg[k] = static_cast<const T*>(c.zg[k]);
        A.gwg[k] = static_cast<T*>(c.gwg[k]);
    }
    return A;
}

template <int DIM, int PX, int PY>
cudaError_t run_faces_vjp(const AdjArgs<T>& A, int dim, cudaStream_t s) {
    long long total = (long long)DIM * (A.n[0] + 1) * (dim >= 2 ? A.n[1] + 1 : 1) *
                      (dim >= 3 ? A.n[2] + 1 : 1);     // one thread per face
    if (total >= (1ll << 31)) return cudaErrorInvalidValue;   // 32-bit face indices
    long long blocks = (total + FACES_VJP_THREADS - 1) / FACES_VJP_THREADS;
    if (blocks > 152 * 32) blocks = 152 * 32;
    return launch_pdl(faces_vjp_kernel<T, DIM, PX, PY>, dim3((unsigned)blocks),
                      dim3(FACES_VJP_THREADS), 0, s, A);
}

}  // namespace

#define HH_CAT2(a, b) a##b
#define HH_CAT(a, b) HH_CAT2(a, b)

cudaError_t HH_CAT(launch_stage_, HH_SUFFIX)(const MeshDesc& m, int kernel, int tile,
                                              const StageCall& c, cudaStream_t s) {
    if (m.dim == 0) {
        long long n5 = 5 * m.N;
        int blocks = (int)((n5 + 255) / 256 < 4096 ? (n5 + 255) / 256 : 4096);
        pointwise_stage_kernel<<<blocks, 256, 0, s>>>(
            static_cast<const T*>(c.U0), static_cast<const T*>(c.Uc), static_cast<T*>(c.Uo), n5,
            c.dt, c.dt_dev, c.stage);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess || !c.rate_slot) return e;
        return HH_CAT(launch_rate_, HH_SUFFIX)(m, c.Uo, c.rate_slot, c.status, s);
    }
    if (m.dim == 3) return dispatch_tile<3, 0, 1>(m, kernel, tile, c, s);
    if (m.dim == 2) {
        if (m.px == 0 && m.py == 1) return dispatch_tile<2, 0, 1>(m, kernel, tile, c, s);
        if (m.px == 0 && m.py == 2) return dispatch_tile<2, 0, 2>(m, kernel, tile, c, s);
        return dispatch_tile<2, 1, 2>(m, kernel, tile, c, s);
    }
    if (m.px == 0) return dispatch_tile<1, 0, 0>(m, kernel, tile, c, s);
    if (m.px == 1) return dispatch_tile<1, 1, 0>(m, kernel, tile, c, s);
    return dispatch_tile<1, 2, 0>(m, kernel, tile, c, s);
}

cudaError_t HH_CAT(launch_rate_, HH_SUFFIX)(const MeshDesc& m, const void* U,
                                             unsigned long long* rate_slot, int* status,
                                             cudaStream_t s) {
    long long blocks = (m.N + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    rate_kernel<<<(int)blocks, 256, 0, s>>>(
        static_cast<const T*>(U), m.N, (T)m.gamma, (T)(m.gamma - 1.0), m.act[0], m.act[1],
        m.act[2], width_param(m.dx[0]), width_param(m.dx[1]), width_param(m.dx[2]), rate_slot,
        status);
    return cudaGetLastError();
}

cudaError_t HH_CAT(launch_totals_, HH_SUFFIX)(const MeshDesc& m, const void* U, double* partial,
                                               cudaStream_t s) {
    totals_kernel<<<TOT_BLOCKS, TOT_THREADS, 0, s>>>(static_cast<const T*>(U), m.N, partial);
    return cudaGetLastError();
}

}  // namespace hh

namespace hh {
cudaError_t HH_CAT(launch_batched_, HH_SUFFIX)(const BatchCall& c, int tile, cudaStream_t s) {
    switch (tile) {
        case 1: return run_batched<128, 32, 4>(c, s);
        case 2: return run_batched<512, 64, 8>(c, s);
        default: return run_batched<256, 32, 8>(c, s);
    }
}
}  // namespace hh

namespace hh {
cudaError_t HH_CAT(launch_adjoint_stage_, HH_SUFFIX)(const MeshDesc& m, const AdjointCall& c,
                                                     cudaStream_t s) {
    const AdjArgs<T> A = make_adj(m, c);
    cudaError_t e = cudaSuccess;
    if (c.passes & 1) {
        if (m.dim == 3) e = run_faces_vjp<3, 0, 1>(A, 3, s);
        else if (m.dim == 2)
            e = m.px == 0 ? (m.py == 1 ? run_faces_vjp<2, 0, 1>(A, 2, s)
                                       : run_faces_vjp<2, 0, 2>(A, 2, s))
                          : run_faces_vjp<2, 1, 2>(A, 2, s);
        else if (m.dim == 1)
            e = m.px == 0 ? run_faces_vjp<1, 0, 0>(A, 1, s)
                          : (m.px == 1 ? run_faces_vjp<1, 1, 0>(A, 1, s)
                                       : run_faces_vjp<1, 2, 0>(A, 1, s));
        if (e != cudaSuccess) return e;
    }
    if (!(c.passes & 2)) return cudaSuccess;
    long long blocks = (m.N + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    return launch_pdl(cell_vjp_kernel<T>, dim3((unsigned)blocks), dim3(256), 0, s,
                      static_cast<const T*>(c.Uc), static_cast<T*>(c.gW),
                      static_cast<const T*>(c.G), (T)c.b, (T)c.a, static_cast<T*>(c.out_c),
                      c.accumulate, static_cast<T*>(c.out0), m.N, (T)m.gamma, c.g_gamma,
                      c.clear_gW);
}

cudaError_t HH_CAT(launch_add_ghost_cotangent_, HH_SUFFIX)(const MeshDesc& m, void* gW,
                                                           const void* from, int k0,
                                                           cudaStream_t s) {
    const long long plane = (long long)m.n[0] * m.n[1];
    long long blocks = (2 * plane * GW_STRIDE + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    add_ghost_cotangent_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(
        static_cast<T*>(gW), static_cast<const T*>(from), plane, k0);
    return cudaGetLastError();
}
}  // namespace hh
