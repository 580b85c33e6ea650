// TMA-fed fused stage kernel for FP64 3D meshes (the FP32 path is the
// warp-specialised kernel of stage_ws.cuh).
//
// Same arithmetic as stage_kernel (each face flux evaluated once, in the same
// operation order), different data movement:
//   * one elected thread streams the haloed conserved plane of the CTA's
//     column, box (TX+8) x (TY+4) x 5 fields, with one 4D bulk tensor load per
//     plane into a 4-slot shared-memory ring, one plane ahead, completing on
//     one mbarrier per slot;
//   * periodic x/y ghosts of boundary tiles arrive as narrow extra boxes of
//     the wrapped columns / rows on the same mbarrier; outflow and reflecting
//     ghosts are read from the tile's own interior;
//   * the conserved value of a cell, needed by the RK combine two planes
//     later, is read back from the ring instead of from HBM.
// The x start of every box is x0 - 4 (x0 a multiple of TX): 16-byte aligned
// for 4- and 8-byte elements.
#pragma once
#include "stage_kernel.cuh"
#include "tma.cuh"

namespace hh {

struct TmaMaps {
    CUtensorMap main;    // box (TX+8, TY+4, 1, 5) of Uc
    CUtensorMap xstrip;  // box (4, TY+4, 1, 5) of Uc
    CUtensorMap ystrip;  // box (TX+8, 2, 1, 5) of Uc
    CUtensorMap u0;      // box (TX, TY, 1, 5) of U0 (stage 2)
    // the ghost planes of BC_HALO z faces ([0] below z = 0, [1] above z = nz-1,
    // each [5][2][ny][nx]), with the boxes of main / xstrip / ystrip
    CUtensorMap gmain[2], gxstrip[2], gystrip[2];
};

template <typename T, int TX, int TY, int STAGE = 1>
struct TmaLayout {
    static constexpr int D = 4;                         // ring slots
    static constexpr int P = 1;                         // planes loaded ahead
    static constexpr int HXC = TX + 8, HYC = TY + 4;    // conserved box
    // every TMA destination starts on a 128-byte boundary
    static constexpr int A128 = 128 / (int)sizeof(T);
    static constexpr int pad(int n) { return (n + A128 - 1) / A128 * A128; }
    static constexpr int MAIN = pad(NF * HYC * HXC);
    static constexpr int XS = pad(NF * HYC * 4);        // x strip box
    static constexpr int YS = pad(NF * 2 * HXC);        // y strip box
    static constexpr int XLO = MAIN, XHI = MAIN + XS, YLO = MAIN + 2 * XS, YHI = YLO + YS;
    static constexpr int SLOT = MAIN + 2 * XS + 2 * YS; // elements per slot
    // stage 2: the tile's U0 plane of the update, two slots by iteration parity
    static constexpr int U0S = pad(NF * TY * TX);
    static constexpr int NU0 = STAGE == 2 ? 2 : 0;
    static constexpr uint32_t U0_BYTES = sizeof(T) * NF * TY * TX;
    static constexpr int HXP = TX + 4, HYP = TY + 4;    // primitive plane
    static constexpr int NP = NF * HYP * HXP;           // one primitive plane
    static constexpr int NFX = NF * TY * (TX + 1);      // one plane of x-face fluxes
    static constexpr int NFY = NF * (TY + 1) * TX;      // one plane of y-face fluxes
    // one primitive plane and one plane of x / y face fluxes (see the barrier
    // comment in the kernel for why one of each suffices)
    static constexpr size_t BAR_BYTES = 128;            // D mbarriers, then the ring
    static constexpr size_t RED_BYTES = (TX * TY / 32) * (NF + 1) * 8;
    static constexpr size_t data_bytes =
        BAR_BYTES + sizeof(T) * (size_t(D) * SLOT + NU0 * U0S + NP + NFX + NFY) + RED_BYTES;
    static constexpr size_t bytes = data_bytes + 128;   // slack to align the base by hand
    static constexpr uint32_t MAIN_BYTES = sizeof(T) * NF * HYC * HXC;
    static constexpr uint32_t XS_BYTES = sizeof(T) * NF * HYC * 4;
    static constexpr uint32_t YS_BYTES = sizeof(T) * NF * 2 * HXC;
    static constexpr size_t RED_OFF =
        BAR_BYTES + sizeof(T) * (size_t(D) * SLOT + NU0 * U0S + NP + NFX + NFY);
    static_assert((U0S * sizeof(T)) % 128 == 0, "U0 slots must start on 128-byte boundaries");
    static_assert((SLOT * sizeof(T)) % 128 == 0 && (XLO * sizeof(T)) % 128 == 0 &&
                  (XHI * sizeof(T)) % 128 == 0 && (YLO * sizeof(T)) % 128 == 0 &&
                  (YHI * sizeof(T)) % 128 == 0 && BAR_BYTES % 128 == 0,
                  "every TMA destination must start on a 128-byte boundary");
    static_assert(RED_OFF % 8 == 0, "reduction scratch must be 8-byte aligned");
    // A slot is read until two iterations after its own, and the load for
    // iteration it + P is issued after the first barrier of iteration it.
    static_assert(P <= D - 3, "ring too shallow for the prefetch distance");
};

// FP32 blocks of up to 256 threads run two per SM (register cap 128 per
// thread); FP64 rings fill an SM's shared memory with one block.
// STAGE (1 or 2) is a template parameter: the stage-2 combine and its U0
// stream, and the signal-rate and totals epilogue (which the time loop asks
// of stage 2 only; the launcher sends any other such call to the plain
// kernel), compile away from stage 1.
template <typename T, int TX, int TY, int STAGE>
__global__ void __launch_bounds__(TX * TY, (sizeof(T) == 4 && TX * TY <= 256) ? 2 : 1)
stage_tma_kernel(const __grid_constant__ StageArgs<T> A, const __grid_constant__ TmaMaps M) {
    using L = TmaLayout<T, TX, TY, STAGE>;
    constexpr int NT = TX * TY;
    constexpr bool EPI = STAGE == 2;
    constexpr int D = L::D, P = L::P;
    constexpr int HXC = L::HXC, HYC = L::HYC, HXP = L::HXP, HYP = L::HYP;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // all shared memory is dynamic; the base is rounded up to 128 bytes here
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t* bars = reinterpret_cast<uint64_t*>(base);
    // abort flags by plane parity: a thread one plane ahead (past barrier A of a
    // column-only plane) must not change the flag that a slower thread reads
    int* s_abort = reinterpret_cast<int*>(base + 8 * D);
    static_assert(8 * D + 2 * sizeof(int) <= L::BAR_BYTES, "barrier block too small");
    T* ring = reinterpret_cast<T*>(base + L::BAR_BYTES);
    T* u0s = ring + D * L::SLOT;                      // NU0 x [NF][TY][TX]
    T* Ps = u0s + L::NU0 * L::U0S;                    // [NF][HYP][HXP]
    T* Fx = Ps + L::NP;                               // [NF][TY][TX+1]
    T* Fy = Fx + L::NFX;                              // [NF][TY+1][TX]
    double (*red_tot)[NF] = reinterpret_cast<double (*)[NF]>(Fy + L::NFY);
    unsigned long long* red_rate =
        reinterpret_cast<unsigned long long*>(reinterpret_cast<double*>(red_tot) + (NT / 32) * NF);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = x < nx && y < ny;
    const int z0 = A.zlo + blockIdx.z * A.zchunk;
    const int z1 = min(z0 + A.zchunk, A.zhi);
    const int jbeg = z0 - 2;
    const int niter = (z1 + 2) - jbeg;
    // boundary tiles and their periodic strips (uniform over the CTA)
    const bool xlo = x0 == 0, xhi = x0 + TX + 2 > nx;
    const bool ylo = y0 == 0, yhi = y0 + TY + 2 > ny;
    const bool px_lo = xlo && A.bc_lo[0] == 0, px_hi = xhi && A.bc_hi[0] == 0;
    const bool py_lo = ylo && A.bc_lo[1] == 0, py_hi = yhi && A.bc_hi[1] == 0;
    const bool edge = xlo || xhi || ylo || yhi;
    const uint32_t tx_bytes = L::MAIN_BYTES + (px_lo ? L::XS_BYTES : 0) +
                              (px_hi ? L::XS_BYTES : 0) + (py_lo ? L::YS_BYTES : 0) +
                              (py_hi ? L::YS_BYTES : 0);

    const T dt = (T)(A.dt_dev ? *A.dt_dev : A.dt);
    const T gamma = A.gamma, gm1 = A.gm1, igm1 = A.igm1;
    constexpr int NPF = HXP * HYP;                    // one field of the primitive plane
    // Work split per plane.  The first EW warps evaluate the TX+TY faces on
    // the tile's top and right edges beside their own x and y faces, and
    // their z face after barrier B; the other NC threads evaluate their z
    // face before barrier B and convert the primitive plane.  Each warp then
    // evaluates three faces between the barriers, and the edge warps' z face
    // stands against the conversion after barrier B.
    constexpr int EW = (TX + TY + 31) / 32;           // edge warps
    constexpr int NC = NT - 32 * EW;                  // converting threads
    static_assert(NC >= 32, "tile too small for the edge-warp split");
    constexpr int MAXE = (NPF + NC - 1) / NC;         // plane cells converted per thread
    const bool edge_warp = tid < 32 * EW;             // warp-uniform
    const int ct = tid - 32 * EW;                     // conversion thread index

    auto slot_main = [&](int it) { return ring + (it % D) * L::SLOT; };
    auto issue = [&](int it) {
        T* s = slot_main(it);
        uint64_t* bar = bars + (it % D);
        bool fz;
        const int pz = jbeg + it;
        const bool hlo = pz < 0 && A.bc_lo[2] == BC_HALO, hhi = pz >= nz && A.bc_hi[2] == BC_HALO;
        const int side = hlo ? 0 : 1;
        const int jj = hlo ? pz + 2 : (hhi ? pz - nz : bc_map(pz, nz, A.bc_lo[2], A.bc_hi[2], fz));
        const CUtensorMap* mm = hlo || hhi ? &M.gmain[side] : &M.main;
        const CUtensorMap* mx = hlo || hhi ? &M.gxstrip[side] : &M.xstrip;
        const CUtensorMap* my = hlo || hhi ? &M.gystrip[side] : &M.ystrip;
        // stage 2, update iterations: the U0 plane of the cell completed then
        const bool with_u0 = STAGE == 2 && it >= 4;
        mbar_arrive_expect_tx(bar, tx_bytes + (with_u0 ? L::U0_BYTES : 0u));
        // test switch: the barrier expects bytes that never come, so every
        // wait on it runs to its limit (no copy is ever in flight)
        if (A.starve_tma) return;
        if (with_u0) tma_load_4d(u0s + (it & 1) * L::U0S, &M.u0, x0, y0, jbeg + it - 2, 0, bar);
        tma_load_4d(s, mm, x0 - 4, y0 - 2, jj, 0, bar);
        if (px_lo) tma_load_4d(s + L::XLO, mx, nx - 4, y0 - 2, jj, 0, bar);
        if (px_hi) tma_load_4d(s + L::XHI, mx, 0, y0 - 2, jj, 0, bar);
        if (py_lo) tma_load_4d(s + L::YLO, my, x0 - 4, ny - 2, jj, 0, bar);
        if (py_hi) tma_load_4d(s + L::YHI, my, x0 - 4, 0, jj, 0, bar);
    };

    if (tid == 0) {
        for (int s = 0; s < D; ++s) mbar_init(bars + s, 1);
        mbar_fence_init();
        s_abort[0] = s_abort[1] = 0;
        prefetch_tmap(&M.main);
    }
    __syncthreads();
    if (tid == 0)
        for (int it = 0; it < P && it < niter; ++it) issue(it);

    bool bad = false;
    T rate_max = T(0);
    T tot[NF] = {T(0), T(0), T(0), T(0), T(0)};
    T qm1[NF], dprev[NF], qLp[NF], Fzp[NF], Da[NF], Db[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) qm1[f] = dprev[f] = qLp[f] = Fzp[f] = Da[f] = Db[f] = T(0);

    // Where each plane cell this thread converts comes from inside a ring slot:
    // the same for every plane of the column, so worked out once and packed in
    // one word per cell: bits 0-15 the slot offset of field 0 (0xFFFF: a cell
    // no face reads), bits 16-27 the field stride, bit 28 / bit 29 negate
    // rho*u / rho*v (reflecting walls).
    static_assert(L::SLOT < 0xFFFF && HYC * HXC < 4096, "conversion map field widths");
    int cv[MAXE];
#pragma unroll
    for (int q = 0; q < MAXE; ++q) {
        const int e = edge_warp ? 0 : ct + q * NC;
        const int cx = e % HXP - 2, cy = e / HXP - 2;
        int src = (cy + 2) * HXC + cx + 4, fs = HYC * HXC, flip = 0;
        if (edge) {
            const int gx = x0 + cx, gy = y0 + cy;
            const bool gxo = gx < 0 || gx >= nx, gyo = gy < 0 || gy >= ny;
            if ((gxo && gyo) || gx > nx + 1 || gy > ny + 1) {
                src = -1;                             // tile corner / beyond a ragged edge
            } else if (gxo) {
                const int bc = gx < 0 ? A.bc_lo[0] : A.bc_hi[0];
                if (bc == 0) {
                    src = (gx < 0 ? L::XLO : L::XHI) + (cy + 2) * 4 + (gx < 0 ? gx + 4 : gx - nx);
                    fs = HYC * 4;
                } else if (bc == 1) {
                    src = (cy + 2) * HXC + (gx < 0 ? 0 : nx - 1) - x0 + 4;
                } else {
                    src = (cy + 2) * HXC + (gx < 0 ? -1 - gx : 2 * nx - 1 - gx) - x0 + 4;
                    flip = 1;
                }
            } else if (gyo) {
                const int bc = gy < 0 ? A.bc_lo[1] : A.bc_hi[1];
                if (bc == 0) {
                    src = (gy < 0 ? L::YLO : L::YHI) + (gy < 0 ? gy + 2 : gy - ny) * HXC + cx + 4;
                    fs = 2 * HXC;
                } else if (bc == 1) {
                    src = ((gy < 0 ? 0 : ny - 1) - y0 + 2) * HXC + cx + 4;
                } else {
                    src = ((gy < 0 ? -1 - gy : 2 * ny - 1 - gy) - y0 + 2) * HXC + cx + 4;
                    flip = 2;
                }
            }
        }
        // interior tiles: the bare slot offset (constant field stride, no flips)
        cv[q] = edge ? ((src < 0 ? 0xFFFF : src) | (fs << 16) | (flip << 28)) : src;
    }

    // 32-bit element indices (the launcher guarantees 5 N < 2^32): this
    // thread's cell in the next plane to complete, one plane per update
    const uint32_t Nu = (uint32_t)A.N, plane = (uint32_t)ny * (uint32_t)nx;
    uint32_t cell = (uint32_t)z0 * plane + (uint32_t)y * (uint32_t)nx + (uint32_t)x;

    // Barriers: two per plane.  Barrier A (the plane's primitives are in shared
    // memory) also marks every thread done with iteration it-1, which frees
    // the ring slot that the next load overwrites.  One primitive plane and
    // one flux plane suffice: the primitives of a plane are read only between
    // its barriers A and B, and a thread writes the next plane's primitives
    // after barrier B; the fluxes are read after barrier B, and the next
    // plane's are written after the next barrier A, which no thread passes
    // before every thread has finished reading them.
    int it = 0;
    for (; it < niter; ++it) {
        const int j = jbeg + it;
        const bool upd = it >= 4 && own;              // completes cell j - 2 (z0 at it = 4)
        if (!mbar_wait(bars + (it % D), (uint32_t)((it / D) & 1))) {
            atomicOr(A.status, 4);
            s_abort[it & 1] = 1;
        }
        const T* S = slot_main(it);
        const bool xy = j >= z0 && j < z1;
        T qj[NF], Dj[NF], Fown_x[NF], Fown_y[NF];
        // z direction: streaming stencil of this column.  It needs only this
        // cell's primitives (the work split above says where it runs).
        T Fz[NF] = {T(0), T(0), T(0), T(0), T(0)};
        T dcur[NF];
        auto zstep = [&]() {
#pragma unroll
            for (int f = 0; f < NF; ++f) dcur[f] = qj[f] - qm1[f];
            if (it >= 2) {
                T qL[NF], qR[NF];
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const T d = minmod(dprev[f], dcur[f]);
                    qR[f] = madd(T(-0.5), d, qm1[f]);
                    qL[f] = madd(T(0.5), d, qm1[f]);
                }
                if (it >= 3) hllc_axis<2>(qLp, qR, gamma, gm1, igm1, Fz);  // face j-3/2
#pragma unroll
                for (int f = 0; f < NF; ++f) qLp[f] = qL[f];
            }
        };
        if (xy) {
            // conserved -> primitive over the haloed (TX+4) x (TY+4) plane
            if (!edge) {
                // interior tile: every plane cell is in the main box
#pragma unroll
                for (int q = 0; q < MAXE; ++q) {
                    const int e = ct + q * NC;
                    if (edge_warp || e >= NPF) break;
                    T U[NF], W[NF];
                    const T* src = S + cv[q];
#pragma unroll
                    for (int f = 0; f < NF; ++f) U[f] = src[f * (HYC * HXC)];
                    cons_to_prim(U, gm1, W);
#pragma unroll
                    for (int f = 0; f < NF; ++f) Ps[f * NPF + e] = W[f];
                }
            } else {
#pragma unroll
                for (int q = 0; q < MAXE; ++q) {
                    const int e = ct + q * NC;
                    if (edge_warp || e >= NPF) break;
                    T U[NF], W[NF];
                    const int off = cv[q] & 0xFFFF, fs = (cv[q] >> 16) & 0xFFF;
                    if (off != 0xFFFF) {
                        const T* src = S + off;
#pragma unroll
                        for (int f = 0; f < NF; ++f) U[f] = src[f * fs];
                        if (cv[q] & (1 << 28)) U[1] = -U[1];
                        if (cv[q] & (1 << 29)) U[2] = -U[2];
                    } else {
                        U[0] = T(1); U[1] = U[2] = U[3] = T(0); U[4] = T(1);
                    }
                    cons_to_prim(U, gm1, W);
#pragma unroll
                    for (int f = 0; f < NF; ++f) Ps[f * NPF + e] = W[f];
                }
            }
            __syncthreads();                          // barrier A
            if (s_abort[it & 1]) break;
            if (tid == 0 && it + P < niter) issue(it + P);
            // this thread's own cell: shared by its x face, its y face and the z stencil
#pragma unroll
            for (int f = 0; f < NF; ++f) qj[f] = Ps[(f * HYP + ty + 2) * HXP + tx + 2];
            if (!edge_warp) zstep();
            // the x face left of the cell and the y face below it
            T q[4][NF], F[NF];
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    q[s4][f] = s4 == 2 ? qj[f] : Ps[(f * HYP + ty + 2) * HXP + tx + s4];
            face_flux4<0>(q[0], q[1], q[2], q[3], gamma, gm1, igm1, Fown_x);
#pragma unroll
            for (int f = 0; f < NF; ++f) Fx[(f * TY + ty) * (TX + 1) + tx] = Fown_x[f];
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    q[s4][f] = s4 == 2 ? qj[f] : Ps[(f * HYP + ty + s4) * HXP + tx + 2];
            face_flux4<1>(q[0], q[1], q[2], q[3], gamma, gm1, igm1, Fown_y);
#pragma unroll
            for (int f = 0; f < NF; ++f) Fy[(f * (TY + 1) + ty) * TX + tx] = Fown_y[f];
            // the TX faces above the top row and the TY faces right of the last column
            auto edge_face = [&](int e) {
                if (e < TX) {
#pragma unroll
                    for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
                        for (int f = 0; f < NF; ++f)
                            q[s4][f] = Ps[(f * HYP + TY + s4) * HXP + e + 2];
                    face_flux4<1>(q[0], q[1], q[2], q[3], gamma, gm1, igm1, F);
#pragma unroll
                    for (int f = 0; f < NF; ++f) Fy[(f * (TY + 1) + TY) * TX + e] = F[f];
                } else if (e < TX + TY) {
                    const int row = e - TX;
#pragma unroll
                    for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
                        for (int f = 0; f < NF; ++f)
                            q[s4][f] = Ps[(f * HYP + row + 2) * HXP + TX + s4];
                    face_flux4<0>(q[0], q[1], q[2], q[3], gamma, gm1, igm1, F);
#pragma unroll
                    for (int f = 0; f < NF; ++f) Fx[(f * TY + row) * (TX + 1) + TX] = F[f];
                }
            };
            if (tid < TX + TY) edge_face(tid);
            __syncthreads();                          // barrier B: every face of the plane
            if (edge_warp) zstep();
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const T a = Fx[(f * TY + ty) * (TX + 1) + tx + 1] - Fown_x[f];
                const T b = Fy[(f * (TY + 1) + ty + 1) * TX + tx] - Fown_y[f];
                Dj[f] = sub_over_dx(T(0), a, A.dxk[0]);
                Dj[f] = sub_over_dx(Dj[f], b, A.dxk[1]);
            }
            if (own) bad |= nonphys(qj);
        } else {
            // warm-up / look-ahead plane: this column only
            T U[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) U[f] = S[(f * HYC + ty + 2) * HXC + tx + 4];
            bool fz = false;
            if (!((j < 0 && A.bc_lo[2] == BC_HALO) || (j >= nz && A.bc_hi[2] == BC_HALO)))
                bc_map(j, nz, A.bc_lo[2], A.bc_hi[2], fz);
            if (fz) U[3] = -U[3];
            cons_to_prim(U, gm1, qj);
#pragma unroll
            for (int f = 0; f < NF; ++f) Dj[f] = T(0);
            __syncthreads();                          // barrier A of a column-only plane
            if (s_abort[it & 1]) break;
            if (tid == 0 && it + P < niter) issue(it + P);
            zstep();
        }

        if (upd) {
            const T* Sk = slot_main(it - 2);
            T Uo[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const T Lf = sub_over_dx(Da[f], Fz[f] - Fzp[f], A.dxk[2]);
                const T uc = Sk[(f * HYC + ty + 2) * HXC + tx + 4];
                Uo[f] = STAGE == 1
                            ? madd(dt, Lf, uc)
                            : madd(T(0.5), u0s[(it & 1) * L::U0S + (f * TY + ty) * TX + tx],
                                   T(0.5) * madd(dt, Lf, uc));
                A.Uo[f * Nu + cell] = Uo[f];
            }
            cell += plane;
            if (EPI && A.rate_slot) {
                T W[NF];
                cons_to_prim(Uo, gm1, W);
                const T r = cell_rate(W, gamma, A.act, A.rdx);
                rate_max = (r > rate_max || r != r) ? r : rate_max;
            }
            if (EPI && A.tot_partial) {
#pragma unroll
                for (int f = 0; f < NF; ++f) tot[f] += Uo[f];
            }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (it >= 3) Fzp[f] = Fz[f];
            dprev[f] = dcur[f];
            qm1[f] = qj[f];
            Da[f] = Db[f];
            Db[f] = Dj[f];
        }
    }
    if (it < niter) {
        // a transfer never completed (every thread left at the same barrier A):
        // wait (bounded) for the loads still in flight so none lands after this
        // block has left, then return; the failed wait was iteration it and
        // loads were issued up to it-1+P
        if (tid == 0)
            for (int r = it; r < niter && r <= it - 1 + P; ++r)
                mbar_wait(bars + (r % D), (uint32_t)((r / D) & 1));
        __syncthreads();
        return;
    }

    // ---- epilogue: block reductions ----
    const int lane = tid & 31, warp = tid >> 5;
    if (EPI && A.rate_slot) {
        unsigned long long b = rate_bits(rate_max);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
            b = v > b ? v : b;
        }
        if (lane == 0) red_rate[warp] = b;
    }
    if (EPI && A.tot_partial) {
        double v[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f] = (double)tot[f];
        const double s = warp_sum5(v, lane);
        if (sum5_writer(lane)) red_tot[warp][sum5_field(lane)] = s;
    }
    const int any_bad = __syncthreads_or(bad);
    if (tid == 0) {
        if (any_bad) atomicOr(A.status, 1);
        if (EPI && A.rate_slot) {
            unsigned long long b = 0;
            for (int w = 0; w < NT / 32; ++w) b = red_rate[w] > b ? red_rate[w] : b;
            atomicMax(A.rate_slot, b);
        }
    }
    if (EPI && A.tot_partial && tid < NF) {
        const long long bz = A.zlo / A.zchunk + blockIdx.z;
        const long long blk = (bz * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += red_tot[w][tid];
        A.tot_partial[blk * NF + tid] = s;
    }
}

}  // namespace hh
