// Fused stage kernel: ghost fill -> conserved-to-primitive -> PLM/minmod face
// states -> HLLC -> flux difference -> RK stage combine, one launch per stage,
// with the signal-rate max and the conserved totals fused into the epilogue.
//
// Tiling (2.5D z-march).  A CTA owns a TX x TY column of the mesh and marches
// its z-chunk plane by plane.  For each plane it stages the haloed
// (TX+4) x (TY+4) primitive plane in shared memory, evaluates every x and y
// face flux once into shared memory and forms the x/y part of the flux
// difference.  The z direction needs no shared memory: each thread keeps its
// own column's z stencil (last primitive, last difference, pending left face
// state, previous z-face flux) in registers and completes cell k when plane
// k+2 arrives.
//
// Kernel axes vs physical axes.  The layout U[5][nz][ny][nx] is reinterpreted
// so that the active axes become kernel axes x', y', z' in the same order
// (e.g. nx = 1 makes physical y the kernel x').  PX / PY name the physical
// axis of kernel x' / y' (kernel z' is always physical z), which fixes the
// normal momentum component of each sweep.
#pragma once
#include "hydro_math.cuh"
#include "tma.cuh"

namespace hh {

template <typename T>
struct StageArgs {
    const T* U0;                  // Un (stage 2), may alias Uo
    const T* Uc;                  // state the flux difference is taken of
    T* Uo;                        // output
    long long N;                  // cells = field stride
    int n[3];                     // kernel-axis extents
    int bc_lo[3], bc_hi[3];       // boundary kind per kernel axis
    T gamma, gm1;
    T igm1;                       // 1/(gamma-1), rounded once on the host (FP32 path)
    T dxk[3];                     // per kernel axis: dx (FP64) or 1/dx (FP32)
    T rdx[3];                     // per physical axis, same convention
    bool act[3];                  // per physical axis: active
    double dt;                    // used when dt_dev == nullptr
    const double* dt_dev;
    int stage;                    // 1 or 2
    int zchunk;
    int zlo, zhi;                 // 3D: kernel-z cells [zlo, zhi) of this launch (zlo a multiple of zchunk)
    unsigned long long* rate_slot;    // epilogue max-rate (nullptr = off)
    double* tot_partial;              // epilogue totals [nblocks][5] (nullptr = off)
    int* status;                      // non-physical flag
    const CUtensorMap* tmap;          // TMA descriptor of Uc (fused variant)
    bool starve_tma;                  // test switch: arm the ring's barriers, issue no copies
    // z faces of kind BC_HALO: the two ghost planes below z = 0 (zg[0]) and
    // above z = nz - 1 (zg[1]), each [5][2][ny][nx] (plane 0 of zg[0] is
    // z = -2, plane 0 of zg[1] is z = nz)
    const T* zg[2];
};

// Boundary kind of a z face whose ghost planes come from a caller buffer
// (a neighbouring z slab of a decomposed mesh).
constexpr int BC_HALO = 3;

// Boundary map of one kernel axis: m in [-2, n+1] -> interior index, flip set
// for a reflecting wall.  Indices beyond the ghost layers (ragged tiles only)
// clamp to any valid cell; their values feed faces nobody uses.
__device__ __forceinline__ int bc_map(int m, int n, int lo, int hi, bool& flip) {
    flip = false;
    if (m >= 0 && m < n) return m;
    if (m < -2 || m > n + 1) return m < 0 ? 0 : n - 1;
    int bc = m < 0 ? lo : hi;
    if (bc == 0) {
        int r = m % n;
        return r < 0 ? r + n : r;
    }
    if (bc == 1) return m < 0 ? 0 : n - 1;
    flip = true;
    int s = m < 0 ? -1 - m : 2 * n - 1 - m;
    return s < 0 ? 0 : (s >= n ? n - 1 : s);
}

template <typename T, int TX, int TY, int DIM>
struct StageSmem {
    static constexpr int HX = TX + 4;
    static constexpr int HY = DIM >= 2 ? TY + 4 : 1;
    static constexpr int NP = NF * HX * HY;                       // primitive plane
    static constexpr int NFX = NF * TY * (TX + 1);                // x-face fluxes
    static constexpr int NFY = DIM >= 2 ? NF * (TY + 1) * TX : 0; // y-face fluxes
    // two primitive planes (by plane parity, or by tile parity when a block
    // evaluates one tile after another), one plane of x and y face fluxes
    static constexpr size_t bytes = sizeof(T) * (2 * NP + NFX + NFY);
};

// Load the conserved values of kernel cell (gx, gy, gz) with the boundary map
// applied along the active kernel axes, as primitives.
// NC: the state is not written during this launch, so the read-only
// (non-coherent) cache path may serve it.  A kernel that rewrites its input
// within the launch (the batched time loop) must read with NC = false.
template <typename T, int DIM, int PX, int PY, bool NC>
__device__ __forceinline__ void load_prim(const StageArgs<T>& A, int gx, int gy, int gz, T W[NF],
                                          bool& bad) {
    bool fx, fy = false, fz = false;
    int sx = bc_map(gx, A.n[0], A.bc_lo[0], A.bc_hi[0], fx);
    int sy = 0, sz = 0;
    if (DIM >= 2) sy = bc_map(gy, A.n[1], A.bc_lo[1], A.bc_hi[1], fy);
    const T* src = A.Uc;
    long long fstride = A.N;
    if (DIM >= 3) {
        const bool hlo = gz < 0 && A.bc_lo[2] == BC_HALO;
        const bool hhi = gz >= A.n[2] && A.bc_hi[2] == BC_HALO;
        if (hlo || hhi) {
            // ghost plane from the neighbouring slab (planes -2, -1 / nz, nz+1)
            const int k = hlo ? gz + 2 : gz - A.n[2];
            sz = k < 0 ? 0 : (k > 1 ? 1 : k);
            src = A.zg[hlo ? 0 : 1];
            fstride = 2ll * A.n[1] * A.n[0];
        } else {
            sz = bc_map(gz, A.n[2], A.bc_lo[2], A.bc_hi[2], fz);
        }
    }
    long long c = ((long long)sz * A.n[1] + sy) * A.n[0] + sx;
    T U[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) U[f] = NC ? __ldg(src + f * fstride + c) : src[f * fstride + c];
    if (fx) U[1 + PX] = -U[1 + PX];
    if (DIM >= 2 && fy) U[1 + PY] = -U[1 + PY];
    if (DIM >= 3 && fz) U[3] = -U[3];
    cons_to_prim(U, A.gm1, W);
    bad |= nonphys(W);
}

// What a block accumulates over the cells it completes: the largest signal
// rate, the conserved totals and the non-physical flag.
template <typename T>
struct TileAcc {
    T rate_max;
    T tot[NF];
    bool bad;
};

// Warp sum of the five per-lane FP64 totals as a reduce-scatter butterfly:
// over the first three levels the lanes split the fields between them, so
// each lane takes 8 shuffles and 8 additions instead of 25 of each (FP64
// runs at a small fraction of the FP32 rate on this part).  Returns the
// warp's total of field sum5_field(lane) in the lanes where sum5_writer(lane)
// holds: field 0 in lane 0, 1 in lane 4, 2 in lane 8, 3 in lane 16, 4 in
// lane 24.  The order of the additions is fixed, so the sum is deterministic.
__device__ __forceinline__ double warp_sum5(const double v[NF], int lane) {
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    // offset 16: lanes 0-15 keep fields 0, 1, 2; lanes 16-31 keep 3, 4
    double a0 = h16 ? v[3] : v[0];
    double a1 = h16 ? v[4] : v[1];
    double a2 = h16 ? 0.0 : v[2];
    const double s0 = h16 ? v[0] : v[3];
    const double s1 = h16 ? v[1] : v[4];
    const double s2 = h16 ? v[2] : 0.0;
    a0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    a1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    a2 += __shfl_xor_sync(0xffffffffu, s2, 16);
    // offset 8: lanes 0-7 keep fields 0, 1; 8-15 field 2; 16-23 field 3;
    // 24-31 field 4
    double c0, c1, t0, t1;
    if (!h16) {
        c0 = h8 ? a2 : a0;
        c1 = h8 ? 0.0 : a1;
        t0 = h8 ? a0 : a2;
        t1 = h8 ? a1 : 0.0;
    } else {
        c0 = h8 ? a1 : a0;
        c1 = 0.0;
        t0 = h8 ? a0 : a1;
        t1 = 0.0;
    }
    c0 += __shfl_xor_sync(0xffffffffu, t0, 8);
    c1 += __shfl_xor_sync(0xffffffffu, t1, 8);
    // offset 4: lanes 0-3 keep field 0, 4-7 field 1; every other lane holds
    // one field already and adds its partner's share of it
    const bool two = !h16 && !h8;
    double k = (two && h4) ? c1 : c0;
    const double t = two ? (h4 ? c0 : c1) : c0;
    k += __shfl_xor_sync(0xffffffffu, t, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    return k;
}
__device__ __forceinline__ int sum5_field(int lane) {
    return (lane & 16) ? ((lane & 8) ? 4 : 3) : ((lane & 8) ? 2 : ((lane & 4) ? 1 : 0));
}
__device__ __forceinline__ bool sum5_writer(int lane) {
    return lane == 0 || lane == 4 || lane == 8 || lane == 16 || lane == 24;
}

// One tile of one stage: the TX x TY column at (x0, y0), z-planes [z0, z1)
// (DIM == 3; a single plane otherwise).  Writes the completed cells of the
// tile to A.Uo and folds them into `acc`.  All threads of the block call it.
// A block that evaluates tiles one after another numbers them in `tile`: the
// primitive plane alternates by that parity (by plane parity along z), so a
// tile's loads never overwrite the plane that the previous tile's cells are
// still reading, and no barrier is needed before them.
template <typename T, int TX, int TY, int DIM, int PX, int PY, bool NC>
__device__ __forceinline__ void stage_tile(const StageArgs<T>& A, unsigned char* smem_raw, int x0,
                                           int y0, int z0, int z1, TileAcc<T>& acc,
                                           int tile = 0) {
    using S = StageSmem<T, TX, TY, DIM>;
    constexpr int NT = TX * TY;
    constexpr int HX = S::HX, HY = S::HY;
    T* Ps2 = reinterpret_cast<T*>(smem_raw);         // 2 x [NF][HY][HX]
    T* Fx = Ps2 + 2 * S::NP;                          // [NF][TY][TX+1]
    T* Fy = Fx + S::NFX;                              // [NF][TY+1][TX]

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = x < A.n[0] && (DIM < 2 || y < A.n[1]);
    const T dt = (T)(A.dt_dev ? *A.dt_dev : A.dt);
    const T gamma = A.gamma, gm1 = A.gm1, igm1 = A.igm1;
    bool bad = false;
    T rate_max = acc.rate_max;

    // z stencil state of this thread's column
    T qm1[NF], dprev[NF], qLp[NF], Fzp[NF], Da[NF], Db[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        qm1[f] = dprev[f] = qLp[f] = Fzp[f] = Da[f] = Db[f] = T(0);
    }

    const int jbeg = DIM == 3 ? z0 - 2 : 0;
    const int jend = DIM == 3 ? z1 + 2 : 1;
    for (int j = jbeg; j < jend; ++j) {
        const bool xy = DIM < 3 || (j >= z0 && j < z1);
        T qj[NF];
        T Dj[NF];
        T* Ps = Ps2 + (((DIM == 3 ? j : tile) & 1) * S::NP);
        if (xy) {
            // Ps of the previous plane (tile) stays untouched; the fluxes are
            // written after the next barrier, which no thread passes before
            // every thread has finished reading the previous ones
            for (int e = tid; e < HX * HY; e += NT) {
                int hx = e % HX, hy = e / HX;
                T W[NF];
                load_prim<T, DIM, PX, PY, NC>(A, x0 - 2 + hx, y0 - 2 + hy, j, W, bad);
#pragma unroll
                for (int f = 0; f < NF; ++f) Ps[(f * HY + hy) * HX + hx] = W[f];
            }
            __syncthreads();
            // x faces: (TX+1) per row; face fx sits left of tile cell fx
            for (int e = tid; e < (TX + 1) * TY; e += NT) {
                int fx = e % (TX + 1), row = e / (TX + 1);
                int hy = DIM >= 2 ? row + 2 : 0;
                T q[4][NF];
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int f = 0; f < NF; ++f) q[s][f] = Ps[(f * HY + hy) * HX + fx + s];
                T F[NF];
                face_flux4<PX>(q[0], q[1], q[2], q[3], gamma, gm1, igm1, F);
#pragma unroll
                for (int f = 0; f < NF; ++f) Fx[(f * TY + row) * (TX + 1) + fx] = F[f];
            }
            if (DIM >= 2) {
                for (int e = tid; e < TX * (TY + 1); e += NT) {
                    int col = e % TX, fy = e / TX;
                    T q[4][NF];
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int f = 0; f < NF; ++f) q[s][f] = Ps[(f * HY + fy + s) * HX + col + 2];
                    T F[NF];
                    face_flux4<PY>(q[0], q[1], q[2], q[3], gamma, gm1, igm1, F);
#pragma unroll
                    for (int f = 0; f < NF; ++f) Fy[(f * (TY + 1) + fy) * TX + col] = F[f];
                }
            }
            __syncthreads();
            const int hyc = DIM >= 2 ? ty + 2 : 0;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                qj[f] = Ps[(f * HY + hyc) * HX + tx + 2];
                T a = Fx[(f * TY + ty) * (TX + 1) + tx + 1] - Fx[(f * TY + ty) * (TX + 1) + tx];
                Dj[f] = sub_over_dx(T(0), a, A.dxk[0]);
                if (DIM >= 2) {
                    T b = Fy[(f * (TY + 1) + ty + 1) * TX + tx] - Fy[(f * (TY + 1) + ty) * TX + tx];
                    Dj[f] = sub_over_dx(Dj[f], b, A.dxk[1]);
                }
            }
        } else {
            // warm-up / look-ahead plane: only this column's primitives
            load_prim<T, DIM, PX, PY, NC>(A, min(x, A.n[0] - 1), min(y, A.n[1] - 1), j, qj, bad);
#pragma unroll
            for (int f = 0; f < NF; ++f) Dj[f] = T(0);
        }

        int k;                 // cell completed in this iteration (-1: none)
        T L[NF];
        if (DIM == 3) {
            const int cnt = j - jbeg;
            T dcur[NF], Fz[NF];
            if (cnt >= 2) {
                T qL[NF], qR[NF];
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    dcur[f] = qj[f] - qm1[f];
                    T d = minmod(dprev[f], dcur[f]);
                    qR[f] = madd(T(-0.5), d, qm1[f]);
                    qL[f] = madd(T(0.5), d, qm1[f]);
                }
                if (cnt >= 3) hllc_axis<2>(qLp, qR, gamma, gm1, igm1, Fz);   // face j-3/2
#pragma unroll
                for (int f = 0; f < NF; ++f) qLp[f] = qL[f];
            } else {
#pragma unroll
                for (int f = 0; f < NF; ++f) dcur[f] = qj[f] - qm1[f];
            }
            k = cnt >= 4 ? j - 2 : -1;
            if (k >= 0) {
#pragma unroll
                for (int f = 0; f < NF; ++f) L[f] = sub_over_dx(Da[f], Fz[f] - Fzp[f], A.dxk[2]);
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                if (cnt >= 3) Fzp[f] = Fz[f];
                dprev[f] = dcur[f];
                qm1[f] = qj[f];
                Da[f] = Db[f];
                Db[f] = Dj[f];
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
                T uc = A.Uc[f * A.N + c];
                if (A.stage == 1) {
                    Uo[f] = madd(dt, L[f], uc);
                } else {
                    T u0 = A.U0[f * A.N + c];
                    Uo[f] = madd(T(0.5), u0, T(0.5) * madd(dt, L[f], uc));
                }
                A.Uo[f * A.N + c] = Uo[f];
            }
            if (A.rate_slot) {
                T W[NF];
                cons_to_prim(Uo, gm1, W);
                T r = cell_rate(W, gamma, A.act, A.rdx);
                rate_max = (r > rate_max || r != r) ? r : rate_max;
            }
            if (A.tot_partial) {
#pragma unroll
                for (int f = 0; f < NF; ++f) acc.tot[f] += Uo[f];
            }
        }
    }

    acc.rate_max = rate_max;
    acc.bad |= bad;
}

template <typename T, int TX, int TY, int DIM, int PX, int PY, bool TMA>
__global__ void __launch_bounds__(TX * TY)
stage_kernel(const StageArgs<T> A) {
    constexpr int NT = TX * TY;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red_tot[NT / 32][NF];
    __shared__ unsigned long long red_rate[NT / 32];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX;
    const int y0 = DIM >= 2 ? blockIdx.y * TY : 0;
    const int z0 = DIM == 3 ? A.zlo + blockIdx.z * A.zchunk : 0;
    const int z1 = DIM == 3 ? min(z0 + A.zchunk, A.zhi) : 1;
    TileAcc<T> acc;
    acc.rate_max = T(0);
    acc.bad = false;
#pragma unroll
    for (int f = 0; f < NF; ++f) acc.tot[f] = T(0);
    stage_tile<T, TX, TY, DIM, PX, PY, true>(A, smem_raw, x0, y0, z0, z1, acc);
    const T rate_max = acc.rate_max;
    const bool bad = acc.bad;
    T tot[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) tot[f] = acc.tot[f];

    // ---- epilogue: block reductions ----
    const int lane = tid & 31, warp = tid >> 5;
    if (A.rate_slot) {
        unsigned long long b = rate_bits(rate_max);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
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
            for (int w = 0; w < NT / 32; ++w) b = red_rate[w] > b ? red_rate[w] : b;
            atomicMax(A.rate_slot, b);
        }
    }
    if (A.tot_partial && tid < NF) {
        const long long bz = DIM == 3 ? A.zlo / A.zchunk + blockIdx.z : blockIdx.z;
        const long long blk = (bz * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += red_tot[w][tid];
        A.tot_partial[blk * NF + tid] = s;
    }
}

}  // namespace hh
