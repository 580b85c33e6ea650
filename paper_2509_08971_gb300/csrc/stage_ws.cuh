// Warp-specialised TMA stage kernel for FP32 3D meshes (the bench path).
//
// Same scheme as stage_kernel (a1-a6: ghost map, conserved -> primitive,
// minmod PLM, HLLC, flux difference, RK stage combine; the a7/a8 epilogue in
// stage 2), with the work of a 32 x TY column tile split between two kinds
// of warps and one block barrier per z plane:
//
//   * face warps, one per tile row: lane = x.  In the iteration of plane p a
//     face warp evaluates the x face left of its cell (the left state of the
//     face comes from the neighbouring lane by a shuffle) and the y face
//     below it, then converts its own cell of plane p+1, then closes cell
//     p-1: the z face p-1/2 from the column's register stencil and the RK
//     combine with the x and y fluxes of plane p-1 read from shared memory.
//   * converter warps: they issue the TMA loads, convert the halo ring of
//     plane p+1 and evaluate the tile's edge faces of plane p (the y faces
//     above the top row, the x faces left of the first and right of the last
//     column), whose fluxes the face warps read one plane later.
//
// The finished plane of the tile is staged in shared memory and written by
// one TMA tile store.  Primitive planes, y-face fluxes, edge fluxes and the
// output staging are double-buffered by plane parity, so the barrier after each plane is the only block barrier:
// everything written in the iteration of plane p is read in the iteration of
// plane p+1, and rewritten in that of plane p+2.  Primitives and fluxes are
// stored as a float4 (rho, u, v, w) array beside a float array (p), so that
// a cell's primitive state is two shared-memory loads.
//
// The conserved haloed plane (TX+8) x (TY+4) x 5 fields arrives by one 4D
// bulk tensor load per plane into a 4-slot ring, two planes ahead; periodic
// x/y ghosts of boundary tiles come as narrow strip boxes on the same
// mbarrier.  The conserved value of a cell, needed by the RK combine, is read
// back from the ring; stage 2's U^n plane arrives by TMA on the same barrier.
#pragma once
#include "stage_kernel.cuh"
#include "stage_tma.cuh"
#include "tma.cuh"

namespace hh {

struct WsMaps {
    CUtensorMap main;    // box (TX+8, TY+4, 1, 5) of Uc
    CUtensorMap xstrip;  // box (4, TY+4, 1, 5) of Uc
    CUtensorMap ystrip;  // box (TX+8, 2, 1, 5) of Uc
    CUtensorMap u0;      // box (TX, TY, 1, 5) of U0 (stage 2)
    CUtensorMap out;     // box (TX, TY, 1, 5) of Uo (TMA store)
    // the ghost planes of BC_HALO z faces ([0] below z = 0, [1] above z = nz-1,
    // each [5][2][ny][nx]), with the boxes of main / xstrip / ystrip
    CUtensorMap gmain[2], gxstrip[2], gystrip[2];
};

template <int TX, int TY, int NCW, int STAGE, int RPW>
struct WsLayout {
    static_assert(TX == 32, "lane = x in the face warps");
    static_assert(2 * TY <= 32, "one converter lane per x edge face");
    static_assert(TY % RPW == 0, "whole tile rows per face warp");
    static constexpr int NFW = TY / RPW;                // face warps, RPW tile rows each
    static constexpr int NW = NFW + NCW;
    static constexpr int NT = 32 * NW;
    static constexpr int D = 4;                         // conserved ring slots (a power of 2)
    static constexpr int HXC = TX + 8, HYC = TY + 4;    // conserved box
    static constexpr int HXP = TX + 4, HYP = TY + 4;    // primitive plane
    static constexpr int NPC = HXP * HYP;               // cells of a primitive plane
    static constexpr int pad32(int n) { return (n + 31) / 32 * 32; }   // floats -> 128 B
    static constexpr int MAIN = pad32(NF * HYC * HXC);
    static constexpr int XS = pad32(NF * HYC * 4);      // x strip box
    static constexpr int YS = pad32(NF * 2 * HXC);      // y strip box
    static constexpr int XLO = 0, XHI = XS, YLO = 2 * XS, YHI = 2 * XS + YS;
    static constexpr int STRIP = 2 * XS + 2 * YS;
    static constexpr int U0S = pad32(NF * TY * TX);
    static constexpr int NU0 = STAGE == 2 ? 2 : 0;
    static constexpr int PQ = pad32(5 * NPC);           // float4 part, then p
    static constexpr int FYR = TY + 1;                  // y-face rows
    static constexpr int FQ = pad32(5 * FYR * TX);      // float4 part, then the energy flux
    static constexpr int FXR = TX + 1;                  // x faces per tile row
    static constexpr int FX = pad32(5 * TY * FXR);      // x-face fluxes: float4 part, then energy
    static constexpr int OST = pad32(NF * TY * TX);     // output plane staged for the TMA store
    // offsets in floats from the end of the barrier block
    static constexpr int O_STRIP = D * MAIN;
    static constexpr int O_U0 = O_STRIP + 2 * STRIP;
    static constexpr int O_P = O_U0 + NU0 * U0S;
    static constexpr int O_FY = O_P + 2 * PQ;
    static constexpr int O_FX = O_FY + 2 * FQ;
    static constexpr int O_OST = O_FX + 2 * FX;
    static constexpr int O_MAP = O_OST + 2 * OST;       // halo conversion map (ints)
    static constexpr int O_END = O_MAP + pad32(4 * TX + 4 * TY);
    static constexpr size_t BAR_BYTES = 128;            // D mbarriers, abort flags
    static constexpr size_t RED_BYTES = (size_t)NFW * (NF + 1) * 8;
    static constexpr size_t data_bytes = BAR_BYTES + 4 * (size_t)O_END + RED_BYTES;
    static constexpr size_t bytes = data_bytes + 128;   // slack to align the base by hand
    static constexpr uint32_t MAIN_BYTES = 4u * NF * HYC * HXC;
    static constexpr uint32_t XS_BYTES = 4u * NF * HYC * 4;
    static constexpr uint32_t YS_BYTES = 4u * NF * 2 * HXC;
    static constexpr uint32_t U0_BYTES = 4u * NF * TY * TX;
    // halo ring of the primitive plane (corners excluded), spread over the
    // converter lanes
    static constexpr int NHALO = 4 * TX + 4 * TY;
    static constexpr int HPL = (NHALO + 32 * NCW - 1) / (32 * NCW);
};

// Halo cell e (0 .. NHALO-1) of the primitive plane -> plane coordinates
// (cx, cy) relative to the tile origin: two rows below, two rows above
// (x = 0 .. TX-1), then two columns left and two right (y = 0 .. TY-1).
template <int TX, int TY>
__device__ __forceinline__ void halo_cell(int e, int& cx, int& cy) {
    if (e < 4 * TX) {
        const int r = e / TX;                           // 0, 1: rows -2, -1; 2, 3: TY, TY+1
        cx = e % TX;
        cy = r < 2 ? r - 2 : TY + r - 2;
    } else {
        const int k = e - 4 * TX;
        const int c = k / TY;                           // 0, 1: cols -2, -1; 2, 3: TX, TX+1
        cy = k % TY;
        cx = c < 2 ? c - 2 : TX + c - 2;
    }
}

// Where plane cell (cx, cy) of the tile at (x0, y0) comes from inside a ring
// slot: bits 0-15 the offset of field 0 (0xFFFF: a cell no face reads),
// bits 16-27 the field stride, bit 28 / bit 29 negate rho*u / rho*v
// (reflecting walls), bit 30 set: the offset is into the strip block.
template <int TX, int TY, int HXC, int HYC, int XLO, int XHI, int YLO, int YHI>
__device__ __forceinline__ int ws_source(int cx, int cy, int x0, int y0, int nx, int ny,
                                         const int* bc_lo, const int* bc_hi) {
    const int gx = x0 + cx, gy = y0 + cy;
    const bool gxo = gx < 0 || gx >= nx, gyo = gy < 0 || gy >= ny;
    int src = (cy + 2) * HXC + cx + 4, fs = HYC * HXC, flags = 0;
    if ((gxo && gyo) || gx > nx + 1 || gy > ny + 1) return 0xFFFF;   // corner / beyond a ragged edge
    if (gxo) {
        const int bc = gx < 0 ? bc_lo[0] : bc_hi[0];
        if (bc == 0) {
            src = (gx < 0 ? XLO : XHI) + (cy + 2) * 4 + (gx < 0 ? gx + 4 : gx - nx);
            fs = HYC * 4;
            flags = 4;
        } else if (bc == 1) {
            src = (cy + 2) * HXC + (gx < 0 ? 0 : nx - 1) - x0 + 4;
        } else {
            src = (cy + 2) * HXC + (gx < 0 ? -1 - gx : 2 * nx - 1 - gx) - x0 + 4;
            flags = 1;
        }
    } else if (gyo) {
        const int bc = gy < 0 ? bc_lo[1] : bc_hi[1];
        if (bc == 0) {
            src = (gy < 0 ? YLO : YHI) + (gy < 0 ? gy + 2 : gy - ny) * HXC + cx + 4;
            fs = 2 * HXC;
            flags = 4;
        } else if (bc == 1) {
            src = ((gy < 0 ? 0 : ny - 1) - y0 + 2) * HXC + cx + 4;
        } else {
            src = ((gy < 0 ? -1 - gy : 2 * ny - 1 - gy) - y0 + 2) * HXC + cx + 4;
            flags = 2;
        }
    }
    return src | (fs << 16) | (flags << 28);
}

// Conserved state of a plane cell from its source word (see ws_source).
__device__ __forceinline__ void ws_gather(int cv, const float* slot, const float* strip,
                                          float U[NF]) {
    const int off = cv & 0xFFFF;
    if (off == 0xFFFF) {
        U[0] = 1.f; U[1] = U[2] = U[3] = 0.f; U[4] = 1.f;   // benign filler
        return;
    }
    const int fs = (cv >> 16) & 0xFFF;
    const float* src = ((cv >> 30) & 1 ? strip : slot) + off;
#pragma unroll
    for (int f = 0; f < NF; ++f) U[f] = src[f * fs];
    if (cv & (1 << 28)) U[1] = -U[1];
    if (cv & (1 << 29)) U[2] = -U[2];
}

__device__ __forceinline__ void ws_put(float4* P4, float* Pp, int i, const float W[NF]) {
    P4[i] = make_float4(W[0], W[1], W[2], W[3]);
    Pp[i] = W[4];
}
__device__ __forceinline__ void ws_get(const float4* P4, const float* Pp, int i, float W[NF]) {
    const float4 a = P4[i];
    W[0] = a.x; W[1] = a.y; W[2] = a.z; W[3] = a.w;
    W[4] = Pp[i];
}


// Signal rate of a conserved state on a 3D mesh: cons_to_prim followed by
// cell_rate with every axis active, the density's reciprocal taken once (the
// same operations, so the same value).
__device__ __forceinline__ float ws_rate(const float U[NF], float gamma, float gm1,
                                         const float rdx[3]) {
    const float ir = vrcp(U[0]);
    const float u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
    const float kin = 0.5f * fmaf(U[1], u, fmaf(U[2], v, U[3] * w));
    const float p = gm1 * (U[4] - kin);
    const float cs = vsqrt(gamma * p * ir);
    float r = fmaf(fabsf(u) + cs, rdx[0], 0.0f);
    r = fmaf(fabsf(v) + cs, rdx[1], r);
    return fmaf(fabsf(w) + cs, rdx[2], r);
}

// Iteration schedule of a block's z chunk [z0, z1): the iteration of plane
// p = z0 - 2 + it converts plane p+1, evaluates the x/y faces of plane p when
// z0 <= p < z1, and closes cell p-1 when z0 <= p-1 < z1.  The z stencil takes
// its first slope in iteration 1 and its first face in iteration 2.  One copy
// of the iteration body: copies specialised per iteration kind (measured)
// ran slower, from instruction-cache misses.  A face warp owns RPW
// consecutive tile rows: with two, the y slope of a row is shared by the two
// y faces around it and the iteration's control work is spread over two
// cells per thread.
template <int TX, int TY, int NCW, int STAGE, int RPW>
__global__ void __launch_bounds__(32 * (TY / RPW + NCW), TY >= 16 ? 1 : (TY >= 8 ? 2 : 3))
stage_ws_kernel(const __grid_constant__ StageArgs<float> A, const __grid_constant__ WsMaps M) {
    using L = WsLayout<TX, TY, NCW, STAGE, RPW>;
    constexpr int D = L::D, HXC = L::HXC, HYC = L::HYC, HXP = L::HXP, NPC = L::NPC;
    constexpr int FYR = L::FYR, NCT = 32 * NCW, NFW = L::NFW;
    constexpr bool EPI = STAGE == 2;
    static_assert(D == 4, "the wait parity below divides by 4");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the base stays a pointer into the shared array (not an integer round
    // trip), so every access below compiles to a shared-memory instruction
    unsigned char* base =
        smem_raw + ((128u - ((uint32_t)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base);
    int* s_abort = reinterpret_cast<int*>(base + 8 * D);      // by iteration parity
    static_assert(8 * D + 2 * sizeof(int) <= L::BAR_BYTES, "barrier block too small");
    float* sm = reinterpret_cast<float*>(base + L::BAR_BYTES);
    float* ring = sm;
    float* strips = sm + L::O_STRIP;
    float* u0s = sm + L::O_U0;
    float* Pbase = sm + L::O_P;
    float* Fybase = sm + L::O_FY;
    float* Fxbase = sm + L::O_FX;
    float* Ost = sm + L::O_OST;
    int* hmap = reinterpret_cast<int*>(sm + L::O_MAP);
    double (*red_tot)[NF] = reinterpret_cast<double (*)[NF]>(sm + L::O_END);
    unsigned long long* red_rate =
        reinterpret_cast<unsigned long long*>(reinterpret_cast<double*>(red_tot) + L::NFW * NF);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool facew = warp < NFW;                      // warp-uniform
    const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = A.zlo + blockIdx.z * A.zchunk;
    const int z1 = min(z0 + A.zchunk, A.zhi);
    const int jbeg = z0 - 2;
    const int niter = z1 - jbeg + 1;                    // planes p = jbeg .. z1; p+1 converted
    const bool xlo = x0 == 0, xhi = x0 + TX + 2 > nx;
    const bool ylo = y0 == 0, yhi = y0 + TY + 2 > ny;
    const bool px_lo = xlo && A.bc_lo[0] == 0, px_hi = xhi && A.bc_hi[0] == 0;
    const bool py_lo = ylo && A.bc_lo[1] == 0, py_hi = yhi && A.bc_hi[1] == 0;
    const bool edge = xlo || xhi || ylo || yhi;
    const bool zr_lo = A.bc_lo[2] == 2, zr_hi = A.bc_hi[2] == 2;
    const uint32_t tx_bytes = L::MAIN_BYTES + (px_lo ? L::XS_BYTES : 0) +
                              (px_hi ? L::XS_BYTES : 0) + (py_lo ? L::YS_BYTES : 0) +
                              (py_hi ? L::YS_BYTES : 0);
    const int issuer = 32 * NFW;                        // lane 0 of the first converter warp

    // Ring plane of iteration index q (plane jbeg + q) with its strips; in
    // stage 2 also the U^n plane jbeg + q - 2 that the RK combine of
    // iteration q - 1 needs (it completes on the same barrier).
    auto issue = [&](int q) {
        uint64_t* bar = bars + (q & (D - 1));
        bool fz;
        const int pz = jbeg + q;
        const bool hlo = pz < 0 && A.bc_lo[2] == BC_HALO, hhi = pz >= nz && A.bc_hi[2] == BC_HALO;
        const int side = hlo ? 0 : 1;
        const int jj = hlo ? pz + 2 : (hhi ? pz - nz : bc_map(pz, nz, A.bc_lo[2], A.bc_hi[2], fz));
        const CUtensorMap* mm = hlo || hhi ? &M.gmain[side] : &M.main;
        const CUtensorMap* mx = hlo || hhi ? &M.gxstrip[side] : &M.xstrip;
        const CUtensorMap* my = hlo || hhi ? &M.gystrip[side] : &M.ystrip;
        const int pu = jbeg + q - 2;
        const bool with_u0 = STAGE == 2 && pu >= z0 && pu < z1;
        mbar_arrive_expect_tx(bar, tx_bytes + (with_u0 ? L::U0_BYTES : 0u));
        if (A.starve_tma) return;          // test switch: the waits run out, no copy in flight
        float* s = ring + (q & (D - 1)) * L::MAIN;
        float* st = strips + (q & 1) * L::STRIP;
        if (with_u0) tma_load_4d(u0s + (q & 1) * L::U0S, &M.u0, x0, y0, pu, 0, bar);
        tma_load_4d(s, mm, x0 - 4, y0 - 2, jj, 0, bar);
        if (px_lo) tma_load_4d(st + L::XLO, mx, nx - 4, y0 - 2, jj, 0, bar);
        if (px_hi) tma_load_4d(st + L::XHI, mx, 0, y0 - 2, jj, 0, bar);
        if (py_lo) tma_load_4d(st + L::YLO, my, x0 - 4, ny - 2, jj, 0, bar);
        if (py_hi) tma_load_4d(st + L::YHI, my, x0 - 4, 0, jj, 0, bar);
    };
    // reflecting wall across z: the ghost plane's rho*w changes sign
    auto zflip = [&](int pz) { return (pz < 0 && zr_lo) || (pz >= nz && zr_hi); };

    // conversion maps of edge tiles: the face warps' own cells in registers,
    // the halo ring in shared memory (written by the converter lanes, read
    // after the barrier); interior tiles read the main box at fixed offsets
    const int yr0 = warp * RPW;                         // first tile row of a face warp
    int cv_own[RPW];
#pragma unroll
    for (int r = 0; r < RPW; ++r) cv_own[r] = 0;
    if (edge) {
        if (facew) {
#pragma unroll
            for (int r = 0; r < RPW; ++r)
                cv_own[r] = ws_source<TX, TY, HXC, HYC, L::XLO, L::XHI, L::YLO, L::YHI>(
                    lane, yr0 + r, x0, y0, nx, ny, A.bc_lo, A.bc_hi);
        } else {
            for (int e = tid - 32 * NFW; e < L::NHALO; e += NCT) {
                int cx, cy;
                halo_cell<TX, TY>(e, cx, cy);
                hmap[e] = ws_source<TX, TY, HXC, HYC, L::XLO, L::XHI, L::YLO, L::YHI>(
                    cx, cy, x0, y0, nx, ny, A.bc_lo, A.bc_hi);
            }
        }
    }
    int issued = -1;                                    // last iteration index loaded (issuer)
    if (tid == issuer) {
        for (int s = 0; s < D; ++s) mbar_init(bars + s, 1);
        mbar_fence_init();
        s_abort[0] = s_abort[1] = 0;
        prefetch_tmap(&M.main);
    }
    __syncthreads();
    if (tid == issuer) {
        issue(0);
        issue(1);                                       // niter >= 4: z1 > z0
        issued = 1;
    }

    const float gamma = A.gamma, gm1 = A.gm1, igm1 = A.igm1;
    const float idx = A.dxk[0], idy = A.dxk[1], idz = A.dxk[2];
    const float dt = (float)(A.dt_dev ? *A.dt_dev : A.dt);
    // the face warps' cells: tile row yr0 + r, column lane
    bool own[RPW];
#pragma unroll
    for (int r = 0; r < RPW; ++r) own[r] = facew && x0 + lane < nx && y0 + yr0 + r < ny;
    const int pown0 = (yr0 + 2) * HXP + lane + 2;       // row yr0 in a primitive plane
    const int rown0 = (yr0 + 2) * HXC + lane + 4;       // row yr0 in a ring slot

    // conserved -> primitive of the own cells of the plane of iteration index q
    auto convert_own = [&](int q, float (&W)[RPW][NF]) {
        const float* slot = ring + (q & (D - 1)) * L::MAIN;
        const bool fz = zflip(jbeg + q);
        float* Pq = Pbase + (q & 1) * L::PQ;
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
            float U[NF];
            if (!edge) {
#pragma unroll
                for (int f = 0; f < NF; ++f) U[f] = slot[rown0 + r * HXC + f * (HYC * HXC)];
            } else {
                ws_gather(cv_own[r], slot, strips + (q & 1) * L::STRIP, U);
            }
            if (fz) U[3] = -U[3];
            cons_to_prim(U, gm1, W[r]);
            ws_put(reinterpret_cast<float4*>(Pq), Pq + 4 * NPC, pown0 + r * HXP, W[r]);
        }
    };

    // z-column register stencil of the face warps, per own row
    float qn[RPW][NF], dn[RPW][NF], qLz[RPW][NF], Fzb[RPW][NF];
#pragma unroll
    for (int r = 0; r < RPW; ++r)
#pragma unroll
        for (int f = 0; f < NF; ++f) qn[r][f] = dn[r][f] = qLz[r][f] = Fzb[r][f] = 0.f;
    bool bad = false;
    float rate_max = 0.f;
    float tot[NF] = {0.f, 0.f, 0.f, 0.f, 0.f};

    // One iteration (see the schedule above); returns true when a bounded
    // wait ran out somewhere in the block (every thread returns the same).
    auto body = [&](int it) -> bool {
        const int p = jbeg + it;
        const bool XY = p >= z0 && p < z1;               // faces of plane p wanted
        const bool FIN = p - 1 >= z0 && p - 1 < z1;      // cells p-1 complete
        const int cb = it & 1, pb = cb ^ 1;              // buffers of plane p and of plane p+-1
        const uint32_t wpar = (uint32_t)((it + 1) >> 2) & 1u;      // D = 4
        uint64_t* wbar = bars + ((it + 1) & (D - 1));
        if (facew) {
            if (XY) {
                const float4* P4 = reinterpret_cast<const float4*>(Pbase + cb * L::PQ);
                const float* Pp = Pbase + cb * L::PQ + 4 * NPC;
                // the column's rows yr0 - 2 .. yr0 + RPW: Y[k] is row yr0 - 2 + k
                float Y[RPW + 3][NF];
#pragma unroll
                for (int r = 0; r < RPW; ++r) {
                    float* q = Y[2 + r];
                    float qm[NF], qp[NF];
                    ws_get(P4, Pp, pown0 + r * HXP, q);
                    ws_get(P4, Pp, pown0 + r * HXP - 1, qm);
                    ws_get(P4, Pp, pown0 + r * HXP + 1, qp);
                    // x: slope of the own cell; its right state goes to the
                    // next lane, which evaluates the face between them.  Lane
                    // 0's left face is the tile's edge face (a converter
                    // warp's), so its result is not stored.
                    float qRx[NF], qLl[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const float s = vminmod(q[f] - qm[f], qp[f] - q[f]);
                        qRx[f] = fmaf(-0.5f, s, q[f]);
                        qLl[f] = __shfl_up_sync(0xffffffffu, fmaf(0.5f, s, q[f]), 1);
                    }
                    float Fl[NF];
                    hllc_axis<0>(qLl, qRx, gamma, gm1, igm1, Fl);
                    if (lane != 0) {
                        float* Fx = Fxbase + cb * L::FX;
                        ws_put(reinterpret_cast<float4*>(Fx), Fx + 4 * TY * L::FXR,
                               (yr0 + r) * L::FXR + lane, Fl);
                    }
                }
                // y: the face below each own row.  The slope of row k, from
                // rows k-1, k, k+1, serves the faces below and above it.
                ws_get(P4, Pp, pown0 - 2 * HXP, Y[0]);
                ws_get(P4, Pp, pown0 - HXP, Y[1]);
                ws_get(P4, Pp, pown0 + RPW * HXP, Y[RPW + 2]);
                float sl[RPW + 1][NF];                   // slope of row yr0 - 1 + j
#pragma unroll
                for (int j = 0; j <= RPW; ++j)
#pragma unroll
                    for (int f = 0; f < NF; ++f)
                        sl[j][f] = vminmod(Y[1 + j][f] - Y[j][f], Y[2 + j][f] - Y[1 + j][f]);
                float* Fq = Fybase + cb * L::FQ;
#pragma unroll
                for (int r = 0; r < RPW; ++r) {
                    float qLy[NF], qRy[NF], Fb[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        qLy[f] = fmaf(0.5f, sl[r][f], Y[1 + r][f]);
                        qRy[f] = fmaf(-0.5f, sl[r + 1][f], Y[2 + r][f]);
                    }
                    hllc_axis<1>(qLy, qRy, gamma, gm1, igm1, Fb);
                    ws_put(reinterpret_cast<float4*>(Fq), Fq + 4 * FYR * TX, (yr0 + r) * TX + lane,
                           Fb);
                }
            }
            // own cells of plane p+1
            float q1[RPW][NF];
            if (!mbar_wait(wbar, wpar)) {
                atomicOr(A.status, 4);
                s_abort[cb] = 1;
#pragma unroll
                for (int r = 0; r < RPW; ++r)
#pragma unroll
                    for (int f = 0; f < NF; ++f) q1[r][f] = qn[r][f];
            } else {
                convert_own(it + 1, q1);
            }
            if (p + 1 >= z0 && p + 1 < z1) {
#pragma unroll
                for (int r = 0; r < RPW; ++r)
                    if (own[r]) bad |= nonphys(q1[r]);
            }
            // z, per own row: slope of plane p, face p-1/2, then cell p-1
            if (it >= 1) {
                const float* Fq = Fybase + pb * L::FQ;
                const float* Fx = Fxbase + pb * L::FX;
                float yb[NF];                             // y flux below the row
#pragma unroll
                for (int r = 0; r < RPW; ++r) {
                    float qRz[NF], qLn[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const float d1 = q1[r][f] - qn[r][f];
                        const float s = vminmod(dn[r][f], d1);
                        qRz[f] = fmaf(-0.5f, s, qn[r][f]);
                        qLn[f] = fmaf(0.5f, s, qn[r][f]);
                        dn[r][f] = d1;
                    }
                    if (it >= 2) {
                        float Fz[NF];
                        hllc_axis<2>(qLz[r], qRz, gamma, gm1, igm1, Fz);
                        if (FIN) {
                            // the x/y divergence of plane p-1 from the fluxes
                            // written in the last iteration
                            float yt[NF], xl[NF], xr[NF];
                            if (r == 0)
                                ws_get(reinterpret_cast<const float4*>(Fq), Fq + 4 * FYR * TX,
                                       yr0 * TX + lane, yb);
                            ws_get(reinterpret_cast<const float4*>(Fq), Fq + 4 * FYR * TX,
                                   (yr0 + r + 1) * TX + lane, yt);
                            ws_get(reinterpret_cast<const float4*>(Fx), Fx + 4 * TY * L::FXR,
                                   (yr0 + r) * L::FXR + lane, xl);
                            ws_get(reinterpret_cast<const float4*>(Fx), Fx + 4 * TY * L::FXR,
                                   (yr0 + r) * L::FXR + lane + 1, xr);
                            const float* Sk =
                                ring + ((it - 1) & (D - 1)) * L::MAIN + rown0 + r * HXC;
                            const float* U0k = u0s + pb * L::U0S + (yr0 + r) * TX + lane;
                            float* Ok = Ost + cb * L::OST + (yr0 + r) * TX + lane;
                            float Uo[NF];
#pragma unroll
                            for (int f = 0; f < NF; ++f) {
                                const float Lf = fmaf(Fzb[r][f] - Fz[f], idz,
                                                      fmaf(yb[f] - yt[f], idy, (xl[f] - xr[f]) * idx));
                                const float uc = Sk[f * (HYC * HXC)];
                                if constexpr (STAGE == 1) {
                                    Uo[f] = fmaf(dt, Lf, uc);
                                } else {
                                    Uo[f] = fmaf(0.5f, U0k[f * (TY * TX)], 0.5f * fmaf(dt, Lf, uc));
                                }
                                Ok[f * (TY * TX)] = Uo[f];
                                yb[f] = yt[f];
                            }
                            if (EPI && A.rate_slot) {
                                const float rr = ws_rate(Uo, gamma, gm1, A.rdx);
                                const bool up = own[r] && (rr > rate_max || rr != rr);
                                rate_max = up ? rr : rate_max;
                            }
                            if (EPI && A.tot_partial) {
#pragma unroll
                                for (int f = 0; f < NF; ++f) tot[f] += own[r] ? Uo[f] : 0.f;
                            }
                        }
#pragma unroll
                        for (int f = 0; f < NF; ++f) Fzb[r][f] = Fz[f];
                    }
#pragma unroll
                    for (int f = 0; f < NF; ++f) qLz[r][f] = qLn[f];
                }
                if (FIN && it >= 2) fence_proxy_async_smem();   // the staged plane is read by TMA
            } else {
#pragma unroll
                for (int r = 0; r < RPW; ++r)
#pragma unroll
                    for (int f = 0; f < NF; ++f) dn[r][f] = q1[r][f] - qn[r][f];
            }
#pragma unroll
            for (int r = 0; r < RPW; ++r)
#pragma unroll
                for (int f = 0; f < NF; ++f) qn[r][f] = q1[r][f];
        } else {
            // ---- converter warps ----
            if (tid == issuer) {
                // the plane the face warps staged in the last iteration
                if (p - 2 >= z0 && p - 2 < z1) {
                    tma_store_4d(&M.out, Ost + pb * L::OST, x0, y0, p - 2, 0);
                    bulk_commit();
                }
                if (it + 2 <= niter) {
                    issue(it + 2);
                    issued = it + 2;
                }
            }
            if (XY) {
                const float4* P4 = reinterpret_cast<const float4*>(Pbase + cb * L::PQ);
                const float* Pp = Pbase + cb * L::PQ + 4 * NPC;
                const int cw = warp - NFW;               // converter warp index
                float q0[NF], q1[NF], q2[NF], q3[NF], F[NF];
                if (cw == 0) {
                    // y faces above the top row (one per column)
                    const int c = (TY + 2) * HXP + lane + 2;   // plane row TY
                    ws_get(P4, Pp, c - 2 * HXP, q0);
                    ws_get(P4, Pp, c - HXP, q1);
                    ws_get(P4, Pp, c, q2);
                    ws_get(P4, Pp, c + HXP, q3);
                    face_flux4<1>(q0, q1, q2, q3, gamma, gm1, igm1, F);
                    float* Fq = Fybase + cb * L::FQ;
                    ws_put(reinterpret_cast<float4*>(Fq), Fq + 4 * FYR * TX, TY * TX + lane, F);
                }
                if (cw == NCW - 1 && lane < 2 * TY) {
                    // the x faces at the tile's left and right edges (one per
                    // row and side): lanes 0 .. TY-1 left, TY .. 2TY-1 right
                    const int row = lane < TY ? lane : lane - TY;
                    const int col = lane < TY ? 0 : TX;
                    const int c = (row + 2) * HXP + col + 2;
                    ws_get(P4, Pp, c - 2, q0);
                    ws_get(P4, Pp, c - 1, q1);
                    ws_get(P4, Pp, c, q2);
                    ws_get(P4, Pp, c + 1, q3);
                    face_flux4<0>(q0, q1, q2, q3, gamma, gm1, igm1, F);
                    float* Fx = Fxbase + cb * L::FX;
                    ws_put(reinterpret_cast<float4*>(Fx), Fx + 4 * TY * L::FXR, row * L::FXR + col,
                           F);
                }
            }
            if (!mbar_wait(wbar, wpar)) {
                atomicOr(A.status, 4);
                s_abort[cb] = 1;
            } else if (p + 1 >= z0 && p + 1 < z1) {
                // halo ring of plane p+1
                const int q = it + 1;
                const float* slot = ring + (q & (D - 1)) * L::MAIN;
                const float* strip = strips + pb * L::STRIP;
                float* Pq = Pbase + pb * L::PQ;
                const bool fz = zflip(p + 1);
                for (int e = tid - 32 * NFW; e < L::NHALO; e += NCT) {
                    int cx, cy;
                    halo_cell<TX, TY>(e, cx, cy);
                    float U[NF], W[NF];
                    if (!edge) {
                        const float* src = slot + (cy + 2) * HXC + cx + 4;
#pragma unroll
                        for (int f = 0; f < NF; ++f) U[f] = src[f * (HYC * HXC)];
                    } else {
                        ws_gather(hmap[e], slot, strip, U);
                    }
                    if (fz) U[3] = -U[3];
                    cons_to_prim(U, gm1, W);
                    ws_put(reinterpret_cast<float4*>(Pq), Pq + 4 * NPC, (cy + 2) * HXP + cx + 2, W);
                }
            }
            // the store issued above has read its buffer before the face
            // warps stage the next plane but one into it
            if (tid == issuer) bulk_wait_read_all();
        }
        __syncthreads();
        return s_abort[cb] != 0;
    };

    // ---- prologue: plane jbeg, own column only ----
    if (!mbar_wait(bars + 0, 0u)) {
        atomicOr(A.status, 4);
        s_abort[1] = 1;
    } else if (facew) {
        convert_own(0, qn);
    }
    __syncthreads();
    const bool prologue_failed = s_abort[1] != 0;
    bool aborted = prologue_failed;
    int it = 0;                                         // the iteration that ran last / failed
    if (!aborted) {
#pragma unroll 1
        for (; it < niter; ++it) {
            if (body(it)) {
                aborted = true;
                break;
            }
        }
    }
    if (aborted) {
        // a transfer never completed: wait (bounded) for the loads still in
        // flight, so that none lands after this block has left, then return.
        // The failed wait was that of iteration index 0 (prologue) or it + 1;
        // loads were issued up to `issued`.
        if (tid == issuer) {
            const int first = prologue_failed ? 0 : it + 1;
            for (int r = first; r <= issued; ++r) mbar_wait(bars + (r % D), (uint32_t)((r / D) & 1));
            bulk_wait_all();
        }
        __syncthreads();
        return;
    }
    if (tid == issuer) {
        // the last plane: cell z1 - 1, staged in iteration niter - 1
        tma_store_4d(&M.out, Ost + ((niter - 1) & 1) * L::OST, x0, y0, z1 - 1, 0);
        bulk_commit();
        bulk_wait_all();
    }

    // ---- epilogue: block reductions over the face warps ----
    if (EPI && A.rate_slot && facew) {
        unsigned long long b = rate_bits(rate_max);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
            b = v > b ? v : b;
        }
        if (lane == 0) red_rate[warp] = b;
    }
    if (EPI && A.tot_partial && facew) {
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
            for (int w = 0; w < NFW; ++w) b = red_rate[w] > b ? red_rate[w] : b;
            atomicMax(A.rate_slot, b);
        }
    }
    if (EPI && A.tot_partial && tid < NF) {
        const long long bz = A.zlo / A.zchunk + blockIdx.z;
        const long long blk = (bz * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        double s = 0.0;
        for (int w = 0; w < NFW; ++w) s += red_tot[w][tid];
        A.tot_partial[blk * NF + tid] = s;
    }
}

}  // namespace hh
