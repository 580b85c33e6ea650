// Flux-limited radiation diffusion (Sec. 2.2.1-2.2.2): one backward-Euler
// step of dE/dt = div(D grad E) with D = c lambda(R) / (kappa rho) frozen at
// the old state,
//   lambda = (2 + R) / (6 + 3R + R^2),  R = |grad E| / (rho kappa E),
// on the cell-centred mesh: the linear system (Eq. "linear_equation")
//   E' (1 + sum_f w_f) - sum_f w_f E'_nb = E,   w_f = dt (D_i + D_nb) / (2 dx^2),
// over the faces f of each cell (periodic faces wrap; outflow and reflecting
// faces carry no flux), solved by geometric multigrid V-cycles (the paper's
// GMG, Sec. 2.2.2):
//   * levels: every active axis of even length >= 4 halves (cell-centred
//     coarsening, 2 children per coarsened axis), D of a coarse cell is the
//     mean of its children, dx doubles on coarsened axes (re-discretised
//     coarse operators);
//   * smoother: red-black Gauss-Seidel, two sweeps before and after the
//     coarse correction, 50 on the coarsest level;
//   * restriction: the mean of the children's residuals; prolongation:
//     the coarse correction added to every child (piecewise constant).
// grad E of R: central differences, the edge cell repeated at a non-periodic
// boundary.  Everything is bandwidth-bound stencil work over the levels.
#include <cmath>
#include <new>

#include "devattr.h"
#include "fld_launch.h"
#include "pdl.h"
#include "hard_hydro.h"

namespace hh {

constexpr int FLD_MAX_LEVELS = 16;
constexpr int FLD_PRE = 2, FLD_POST = 2, FLD_COARSE = 50;

struct FldLevel {
    int n[3];
    double dx[3];
    long long N;
    bool coarsened[3];       // this level's axes halved into the next level
    void* x;                 // solution / correction (level 0: the caller's Er)
    void* b;                 // right-hand side
    void* D;                 // cell coefficient
};

struct FldHierarchy {
    int dtype;
    int nl;
    int n0[3];
    int bc_lo[3], bc_hi[3];
    FldLevel L[FLD_MAX_LEVELS];
    double* norms;           // device: sum r^2, sum b^2
};

namespace {

template <typename T>
struct LvlArgs {
    T* x;
    const T* b;
    const T* D;
    int n[3];
    T wk[3];                 // dt / (2 dx^2) per axis (0: inactive): face weight (D_c + D_n) wk
    bool per[3];
    long long N;
    T dt;
};

__device__ __forceinline__ void cell_ijk(long long q, const int n[3], int& i, int& j, int& k) {
    i = (int)(q % n[0]);
    const long long t = q / n[0];
    j = (int)(t % n[1]);
    k = (int)(t / n[1]);
}

// The cell's stencil: diagonal 1 + sum w and sum w x_nb (32-bit cell
// indices: a level has fewer than 2^31 cells), in two steps so that a kernel
// can issue the loads of several cells before any of their arithmetic.  The
// neighbour indices are selects (across the wrap on a periodic axis; at a
// wall the cell itself, with weight 0: a wall carries no flux).
template <typename T>
struct StencilVals {
    T Dc;
    T Dn[6], xn[6];           // neighbours (axis, side): 2 ax + (s > 0)
    int face;                 // bit 2 ax + (s > 0): that face carries a flux
};

// Neighbour offsets of a cell along one axis (coordinate c of n cells, the
// axis' element stride): lo / hi are added to the cell's index (across the
// wrap on a periodic axis; 0 at a wall, whose face carries no flux), face
// bit 0 / 1 set when the low / high face carries a flux.
struct AxisNb {
    int lo, hi, face;
};

__device__ __forceinline__ AxisNb axis_nb(int c, int n, bool per, int stride) {
    const bool inl = c > 0, inh = c + 1 < n;
    AxisNb b;
    b.lo = inl ? -stride : (per ? (n - 1) * stride : 0);
    b.hi = inh ? stride : (per ? -(n - 1) * stride : 0);
    b.face = (inl || per ? 1 : 0) | (inh || per ? 2 : 0);
    return b;
}

// The loads of cell q with the z-axis neighbours given (nbz: the same for
// every cell of a plane, so a kernel that takes several rows of one plane
// per thread computes it once).
template <typename T>
__device__ __forceinline__ void stencil_load_z(const LvlArgs<T>& a, int i, int j, int q,
                                               const AxisNb& nbz, StencilVals<T>& v) {
    v.Dc = a.D[q];
    v.face = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int n = a.n[ax];
        if (n <= 1) continue;                       // inactive axis: the same for every thread
        const AxisNb b = ax == 2 ? nbz : axis_nb(ax == 0 ? i : j, n, a.per[ax], ax == 0 ? 1 : a.n[0]);
        v.Dn[2 * ax] = a.D[q + b.lo];
        v.xn[2 * ax] = a.x[q + b.lo];
        v.Dn[2 * ax + 1] = a.D[q + b.hi];
        v.xn[2 * ax + 1] = a.x[q + b.hi];
        v.face |= b.face << (2 * ax);
    }
}

template <typename T>
__device__ __forceinline__ AxisNb plane_nb(const LvlArgs<T>& a, int k) {
    return axis_nb(k, a.n[2], a.per[2], a.n[0] * a.n[1]);
}

template <typename T>
__device__ __forceinline__ void stencil_load(const LvlArgs<T>& a, int i, int j, int k, int q,
                                             StencilVals<T>& v) {
    stencil_load_z(a, i, j, q, plane_nb(a, k), v);
}

template <typename T>
__device__ __forceinline__ void stencil_eval(const LvlArgs<T>& a, const StencilVals<T>& v,
                                             T& diag, T& off) {
    diag = T(1);
    off = T(0);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int n = a.n[ax];
        if (n <= 1) continue;
#pragma unroll
        for (int s = -1; s <= 1; s += 2) {
            const bool use = (v.face >> (2 * ax + (s > 0))) & 1;
            const T Dn = v.Dn[2 * ax + (s > 0)], xn = v.xn[2 * ax + (s > 0)];
            const T w = use ? (v.Dc + Dn) * a.wk[ax] : T(0);
            diag += w;
            off += w * xn;
        }
    }
}

template <typename T>
__device__ __forceinline__ void stencil(const LvlArgs<T>& a, int i, int j, int k, int q, T& diag,
                                        T& off) {
    StencilVals<T> v;
    stencil_load(a, i, j, k, q, v);
    stencil_eval(a, v, diag, off);
}

// Launch shape of the level kernels: x along threads (and blockIdx.x), one
// row j per blockIdx.y (SMOOTH_ROWS rows for the smoother), one plane k per
// blockIdx.z: no index division.
//
// The smoother gives each thread its colour's cell in SMOOTH_ROWS consecutive
// rows.  The rows' stencil loads are independent, so several are in flight
// per thread (with one cell per thread the kernel waited on load latency),
// and the rows share their y neighbours through L1.  A half-sweep writes only
// cells of its colour and reads only the other colour's x, so all of a
// thread's stores can wait until its loads are done.
constexpr int SMOOTH_ROWS = 4;
#ifndef HH_FLD_COARSE_ROWS
#define HH_FLD_COARSE_ROWS 2
#endif
constexpr int FLD_COARSE_ROWS = HH_FLD_COARSE_ROWS;   // the smoother's rows per thread below level 0
#ifndef HH_FLD_FINE_ROWS
#define HH_FLD_FINE_ROWS 4
#endif
constexpr int FLD_FINE_ROWS = HH_FLD_FINE_ROWS;       // and on level 0

// SR rows per thread (FLD_FINE_ROWS on the finest level; fewer on the coarser,
// L2-resident levels, for more blocks).  lg: log2 of the threads per row.
// Rows whose colour has at least 128 cells take whole blocks along x
// (lg = 7); a shorter row takes 2^lg threads and a block serves 2^(7-lg)
// groups of SR rows, so that the coarse levels keep every thread busy.
template <typename T, int SR>
__global__ void __launch_bounds__(128) smooth_kernel(const LvlArgs<T> a, int color, int lg) {
    griddep_wait();
    const int k = blockIdx.z;
    const int p = blockIdx.x * (1 << lg) + (threadIdx.x & ((1 << lg) - 1));
    const int j0 = (blockIdx.y * (128 >> lg) + (threadIdx.x >> lg)) * SR;
    StencilVals<T> v[SR];
    T bq[SR];
    int qs[SR];
    bool on[SR];
    const AxisNb nbz = plane_nb(a, k);
    // all rows' loads first (a row outside the level evaluates cell (0, 0, k)
    // and is not stored), then the arithmetic, then the stores
#pragma unroll
    for (int r = 0; r < SR; ++r) {
        const int j = j0 + r;
        // the cells of this colour in the row: i = 2p + ((j + k + color) & 1)
        const int i = 2 * p + ((j + k + color) & 1);
        on[r] = j < a.n[1] && i < a.n[0];
        const int ii = on[r] ? i : 0, jj = on[r] ? j : 0;
        qs[r] = (k * a.n[1] + jj) * a.n[0] + ii;
        stencil_load_z(a, ii, jj, qs[r], nbz, v[r]);
        bq[r] = a.b[qs[r]];
    }
#pragma unroll
    for (int r = 0; r < SR; ++r) {
        T diag, off;
        stencil_eval(a, v[r], diag, off);
        bq[r] = (bq[r] + off) / diag;
    }
#pragma unroll
    for (int r = 0; r < SR; ++r)
        if (on[r]) a.x[qs[r]] = bq[r];
    griddep_launch_dependents();
}

// Residual of level l restricted to level l+1 in one pass: one thread per
// coarse cell computes its children's residuals and writes their mean to the
// coarse right-hand side, and zeroes the coarse correction.
// H2: every axis coarsened by 2 (the children of each child plane loaded
// together, then evaluated, so their loads overlap); otherwise the factors
// h0, h1, h2 are read at run time.  The children are summed in the same order
// (z, then y, then x) either way.
// RED: only the colour-0 children are evaluated.  After a half-sweep of
// colour 1 each colour-1 cell solves its own equation, so its residual is
// zero up to rounding (see residual_norm_color_kernel) and it adds nothing to
// the mean; used when the pre-smoothing ends with colour 1 and no periodic
// axis of the level has odd length.
template <typename T, bool H2, bool RED = false>
__global__ void __launch_bounds__(128) residual_restrict_kernel(const LvlArgs<T> a, T* bc, T* xc,
                                                                int nc0, int nc1, int h0, int h1,
                                                                int h2) {
    griddep_wait();
    const int J = blockIdx.y, K = blockIdx.z;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc0) return;
    T sum = T(0);
    if (H2) {
        h0 = h1 = h2 = 2;
        // per child plane: the four children's loads, then their residuals
#pragma unroll
        for (int cz = 0; cz < 2; ++cz) {
            // child c = cx + 2 cy of the plane; colour 0: cx + cy + cz even
            constexpr int NC = RED ? 2 : 4;
            StencilVals<T> v[NC];
            T bq[NC], xq[NC];
            const int k = 2 * K + cz;
            const AxisNb nbz = plane_nb(a, k);
#pragma unroll
            for (int n = 0; n < NC; ++n) {
                const int c = RED ? (cz == 0 ? 3 * n : 1 + n) : n;
                const int i = 2 * I + (c & 1), j = 2 * J + (c >> 1);
                const int q = (k * a.n[1] + j) * a.n[0] + i;
                stencil_load_z(a, i, j, q, nbz, v[n]);
                bq[n] = a.b[q];
                xq[n] = a.x[q];
            }
#pragma unroll
            for (int n = 0; n < NC; ++n) {
                T diag, off;
                stencil_eval(a, v[n], diag, off);
                sum += bq[n] - (diag * xq[n] - off);
            }
        }
    } else {
        for (int cz = 0; cz < h2; ++cz)
            for (int cy = 0; cy < h1; ++cy)
                for (int cx = 0; cx < h0; ++cx) {
                    const int i = I * h0 + cx, j = J * h1 + cy, k = K * h2 + cz;
                    const int q = (k * a.n[1] + j) * a.n[0] + i;
                    T diag, off;
                    stencil(a, i, j, k, q, diag, off);
                    sum += a.b[q] - (diag * a.x[q] - off);
                }
    }
    const int Q = (K * nc1 + J) * nc0 + I;
    bc[Q] = sum / T(h0 * h1 * h2);
    xc[Q] = T(0);
    griddep_launch_dependents();
}

// Convergence check of the fine level: sum r^2 and sum b^2 (r = b - A x) into
// norms[0..1], without storing r.  A work item is SMOOTH_ROWS consecutive
// rows of one 128-cell x segment of a plane; each thread takes its x cell in
// those rows with every load issued before the arithmetic (one cell at a time
// left each thread waiting on load latency), and blocks take items in a
// grid-stride loop, one pair of atomics per block.  Each thread sums its
// rows' terms in the element type and adds them to FP64 per item (at most
// SMOOTH_ROWS FP32 terms: exact to ~1e-7 relative, far inside what a
// convergence test of the residual needs); FP64 sums every term in FP64.
template <typename T>
__global__ void __launch_bounds__(128) residual_norms_kernel(const LvlArgs<T> a, double* norms) {
    griddep_wait();
    __shared__ double sr[4], sb[4];
    double rr = 0.0, bb = 0.0;
    const int segs = (a.n[0] + 127) / 128;
    const int groups = (a.n[1] + SMOOTH_ROWS - 1) / SMOOTH_ROWS;
    const long long items = (long long)segs * groups * a.n[2];
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int seg = (int)(it % segs);
        const long long t = it / segs;
        const int grp = (int)(t % groups), k = (int)(t / groups);
        const int i = seg * 128 + threadIdx.x;
        StencilVals<T> v[SMOOTH_ROWS];
        T bq[SMOOTH_ROWS], xq[SMOOTH_ROWS];
        bool on[SMOOTH_ROWS];
        const AxisNb nbz = plane_nb(a, k);
#pragma unroll
        for (int r = 0; r < SMOOTH_ROWS; ++r) {
            const int j = grp * SMOOTH_ROWS + r;
            on[r] = j < a.n[1] && i < a.n[0];
            const int ii = on[r] ? i : 0, jj = on[r] ? j : 0;
            const int q = (k * a.n[1] + jj) * a.n[0] + ii;
            stencil_load_z(a, ii, jj, q, nbz, v[r]);
            bq[r] = a.b[q];
            xq[r] = a.x[q];
        }
        T pr = T(0), pb = T(0);
#pragma unroll
        for (int r = 0; r < SMOOTH_ROWS; ++r) {
            T diag, off;
            stencil_eval(a, v[r], diag, off);
            const T res = bq[r] - (diag * xq[r] - off);
            if (on[r]) {
                if (sizeof(T) == 8) {
                    rr += (double)res * (double)res;
                    bb += (double)bq[r] * (double)bq[r];
                } else {
                    pr = fma(res, res, pr);
                    pb = fma(bq[r], bq[r], pb);
                }
            }
        }
        rr += (double)pr;
        bb += (double)pb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
        bb += __shfl_xor_sync(0xffffffffu, bb, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sr[w] = rr;
        sb[w] = bb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, tb = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            tr += sr[k];
            tb += sb[k];
        }
        atomicAdd(norms, tr);
        atomicAdd(norms + 1, tb);
    }
    griddep_launch_dependents();
}

// The same check once the fine level's post-smoothing has ended with a
// half-sweep of colour 1: each colour-1 cell then solves its own equation
// with its (colour-0) neighbours as they stand, so its residual is zero up
// to rounding and sum r^2 is the sum over the colour-0 cells, which this
// kernel takes (half the stencils of residual_norms_kernel, in the
// smoother's launch shape) into norms[0].  Only for a proper two-colouring:
// no periodic axis of odd length.
template <typename T>
__global__ void __launch_bounds__(128) residual_norm_color_kernel(const LvlArgs<T> a, int color,
                                                                  double* norms) {
    griddep_wait();
    const int k = blockIdx.z;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    StencilVals<T> v[SMOOTH_ROWS];
    T bq[SMOOTH_ROWS], xq[SMOOTH_ROWS];
    bool on[SMOOTH_ROWS];
    const AxisNb nbz = plane_nb(a, k);
#pragma unroll
    for (int r = 0; r < SMOOTH_ROWS; ++r) {
        const int j = blockIdx.y * SMOOTH_ROWS + r;
        const int i = 2 * p + ((j + k + color) & 1);
        on[r] = j < a.n[1] && i < a.n[0];
        const int ii = on[r] ? i : 0, jj = on[r] ? j : 0;
        const int q = (k * a.n[1] + jj) * a.n[0] + ii;
        stencil_load_z(a, ii, jj, q, nbz, v[r]);
        bq[r] = a.b[q];
        xq[r] = a.x[q];
    }
    T pr = T(0);
    double rr = 0.0;
#pragma unroll
    for (int r = 0; r < SMOOTH_ROWS; ++r) {
        T diag, off;
        stencil_eval(a, v[r], diag, off);
        const T res = bq[r] - (diag * xq[r] - off);
        if (on[r]) {
            if (sizeof(T) == 8) rr += (double)res * (double)res;
            else pr = fma(res, res, pr);
        }
    }
    if (sizeof(T) == 8) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
    } else {
        // the warp's sum in FP32, then one conversion per warp (the FP64
        // pipe is narrow; 128 terms in FP32 change the relative residual
        // by ~1e-6 of itself)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pr += __shfl_xor_sync(0xffffffffu, pr, o);
        rr = (double)pr;
    }
    __shared__ double sr[4];
    if ((threadIdx.x & 31) == 0) sr[threadIdx.x >> 5] = rr;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double t = sr[0] + sr[1] + sr[2] + sr[3];
        if (t != 0.0) atomicAdd(norms, t);
    }
    griddep_launch_dependents();
}

// sum b^2 of the fine level into *out (once per solve; b does not change).
template <typename T>
__global__ void __launch_bounds__(256) sumsq_kernel(const T* b, long long n, double* out) {
    // a thread's values in grid-stride order, eight loads issued at a time
    constexpr int UN = 8;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double acc = 0.0;
    for (; i + (UN - 1) * stride < n; i += UN * stride) {
        T v[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) v[u] = b[i + u * stride];
        // the group's sum in the element type, then one FP64 addition (the
        // FP64 pipe of this GPU is narrow; the sum normalises a convergence
        // check, to which FP32 partial sums of eight terms add ~1e-7)
        T part = T(0);
#pragma unroll
        for (int u = 0; u < UN; ++u) part = fma(v[u], v[u], part);
        acc += (double)part;
    }
    for (; i < n; i += stride) acc += (double)b[i] * (double)b[i];
    __shared__ double sr[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sr[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sr[w];
        atomicAdd(out, t);
    }
}

// The small levels of the V-cycle (each at most FLD_SMALL_CELLS cells, at
// most FLD_SMALL_MAX of them: the bottom of the hierarchy) in one block, in
// shared memory: the same smoothing, residual restriction, coarsest-level
// sweeps and prolongation as the level kernels, with block barriers between
// them instead of launches.  In: level 0 of the set's x and b (global: its
// x is the current iterate or the zeroed correction, its b the restricted
// residual or the right-hand side) and every level's D.  Out: level 0's x.
constexpr int FLD_SMALL_CELLS = 4096;
constexpr int FLD_SMALL_MAX = 8;
#ifndef HH_FLD_SMALL_THREADS
#define HH_FLD_SMALL_THREADS 1024
#endif
constexpr int FLD_SMALL_THREADS = HH_FLD_SMALL_THREADS;   // the block of the small-level kernel

template <typename T>
struct SmallLevels {
    int count;                       // levels of the set, finest first
    LvlArgs<T> lv[FLD_SMALL_MAX];    // global arrays (x, b of the first; D of all), extents, weights
    int h[FLD_SMALL_MAX][3];         // coarsening factors of level i into level i+1
    int off[FLD_SMALL_MAX];          // element offset of level i's x, b, D in shared memory
    // division by n[0], n[1] and n[0] / 2 of level i as a multiply-high:
    // q / d = umulhi(q, floor(2^32 / d) + 1), exact for q < 2^16 and d <= 2^16
    // (the error q (m - 2^32/d) / 2^32 stays below 1/d); d = 1 passes q
    unsigned mg[FLD_SMALL_MAX][3];
    int pre, post, coarse;           // sweeps
};

__device__ __forceinline__ int small_div(int q, unsigned m, int d) {
    return d == 1 ? q : (int)__umulhi((unsigned)q, m);
}

// Level l of the set with its arrays in shared memory, built from the kernel
// parameter (read in place) rather than kept in a local array.
template <typename T>
__device__ __forceinline__ LvlArgs<T> small_level(const SmallLevels<T>& S, T* sm, int l) {
    LvlArgs<T> a = S.lv[l];
    T* base = sm + S.off[l];
    const int N = (int)a.N;
    a.x = base;
    a.b = base + N;
    a.D = base + 2 * N;
    return a;
}

// One red-black half-sweep of a level held in shared memory: with an even
// row length the threads run over the colour's cells only (row r = j + n1 k
// holds them at i = 2 i2 + ((j + k + colour) & 1)), else over every cell.
template <typename T>
__device__ __forceinline__ void small_half_sweep(const LvlArgs<T>& s, unsigned m0, unsigned m1,
                                                 unsigned mh, int color) {
    const int n0 = s.n[0], n1 = s.n[1], N = (int)s.N;
    if ((n0 & 1) == 0) {
        const int h = n0 >> 1;
#pragma unroll 1
        for (int q2 = threadIdx.x; q2 < (N >> 1); q2 += blockDim.x) {
            const int r = small_div(q2, mh, h);
            const int k = small_div(r, m1, n1), j = r - k * n1;
            const int i = 2 * (q2 - r * h) + ((j + k + color) & 1);
            const int q = r * n0 + i;
            T diag, off;
            stencil(s, i, j, k, q, diag, off);
            s.x[q] = (s.b[q] + off) / diag;
        }
    } else {
#pragma unroll 1
        for (int q = threadIdx.x; q < N; q += blockDim.x) {
            const int t = small_div(q, m0, n0), i = q - t * n0;
            const int k = small_div(t, m1, n1), j = t - k * n1;
            if (((i + j + k) & 1) != color) continue;
            T diag, off;
            stencil(s, i, j, k, q, diag, off);
            s.x[q] = (s.b[q] + off) / diag;
        }
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(FLD_SMALL_THREADS)
small_vcycle_kernel(const __grid_constant__ SmallLevels<T> S) {
    griddep_wait();
    extern __shared__ __align__(16) unsigned char fld_smem[];
    T* sm = reinterpret_cast<T*>(fld_smem);
    for (int l = 0; l < S.count; ++l) {
        const int N = (int)S.lv[l].N;
        T* base = sm + S.off[l];
        const T* Dg = S.lv[l].D;
        for (int q = threadIdx.x; q < N; q += blockDim.x) base[2 * N + q] = Dg[q];
        if (l == 0) {
            for (int q = threadIdx.x; q < N; q += blockDim.x) {
                base[q] = S.lv[0].x[q];
                base[N + q] = S.lv[0].b[q];
            }
        }
    }
    __syncthreads();
    // down: smooth, then the children's mean residual as the next b, x = 0
    for (int l = 0; l + 1 < S.count; ++l) {
        const LvlArgs<T> F = small_level(S, sm, l);
        for (int it = 0; it < S.pre; ++it) {
            small_half_sweep(F, S.mg[l][0], S.mg[l][1], S.mg[l][2], 0);
            small_half_sweep(F, S.mg[l][0], S.mg[l][1], S.mg[l][2], 1);
        }
        const LvlArgs<T> C = small_level(S, sm, l + 1);
        const int h0 = S.h[l][0], h1 = S.h[l][1], h2 = S.h[l][2];
        const int c0 = C.n[0], c1 = C.n[1];
        T* cb = const_cast<T*>(C.b);
        for (int Q = threadIdx.x; Q < (int)C.N; Q += blockDim.x) {
            const int t = small_div(Q, S.mg[l + 1][0], c0), I = Q - t * c0;
            const int K = small_div(t, S.mg[l + 1][1], c1), J = t - K * c1;
            T sum = T(0);
            for (int cz = 0; cz < h2; ++cz)
                for (int cy = 0; cy < h1; ++cy)
                    for (int cx = 0; cx < h0; ++cx) {
                        const int i = I * h0 + cx, j = J * h1 + cy, k = K * h2 + cz;
                        const int q = (k * F.n[1] + j) * F.n[0] + i;
                        T diag, off;
                        stencil(F, i, j, k, q, diag, off);
                        sum += F.b[q] - (diag * F.x[q] - off);
                    }
            cb[Q] = sum / T(h0 * h1 * h2);
            C.x[Q] = T(0);
        }
        __syncthreads();
    }
    // the coarsest level: red-black sweeps until a sweep changes nothing
    // (every later sweep would return the same values) or `coarse` sweeps
    {
        __shared__ int changed[2];
        const int lc = S.count - 1;
        const LvlArgs<T> s = small_level(S, sm, lc);
        const int N = (int)s.N, n0 = s.n[0], n1 = s.n[1];
        if (threadIdx.x == 0) changed[0] = 0;
        __syncthreads();
        for (int it = 0; it < S.coarse; ++it) {
            for (int color = 0; color < 2; ++color) {
                if (color == 1 && threadIdx.x == 0) changed[(it + 1) & 1] = 0;
                for (int q = threadIdx.x; q < N; q += blockDim.x) {
                    const int t = small_div(q, S.mg[lc][0], n0), i = q - t * n0;
                    const int k = small_div(t, S.mg[lc][1], n1), j = t - k * n1;
                    if (((i + j + k) & 1) != color) continue;
                    T diag, off;
                    stencil(s, i, j, k, q, diag, off);
                    const T nx = (s.b[q] + off) / diag;
                    if (!(nx == s.x[q])) changed[it & 1] = 1;    // also NaN: keep sweeping
                    s.x[q] = nx;
                }
                __syncthreads();
            }
            if (!changed[it & 1]) break;          // the same value in every thread
        }
    }
    // up: add the coarse correction to the children, smooth
    for (int l = S.count - 2; l >= 0; --l) {
        const LvlArgs<T> F = small_level(S, sm, l);
        const LvlArgs<T> C = small_level(S, sm, l + 1);
        const int h0 = S.h[l][0], h1 = S.h[l][1], h2 = S.h[l][2];
        const int n0 = F.n[0], n1 = F.n[1];
        for (int q = threadIdx.x; q < (int)F.N; q += blockDim.x) {
            const int t = small_div(q, S.mg[l][0], n0), i = q - t * n0;
            const int k = small_div(t, S.mg[l][1], n1), j = t - k * n1;
            F.x[q] += C.x[((k / h2) * C.n[1] + j / h1) * C.n[0] + i / h0];
        }
        __syncthreads();
        for (int it = 0; it < S.post; ++it) {
            small_half_sweep(F, S.mg[l][0], S.mg[l][1], S.mg[l][2], 0);
            small_half_sweep(F, S.mg[l][0], S.mg[l][1], S.mg[l][2], 1);
        }
    }
    {
        const int N = (int)S.lv[0].N;
        for (int q = threadIdx.x; q < N; q += blockDim.x) S.lv[0].x[q] = sm[S.off[0] + q];
    }
    griddep_launch_dependents();
}

// coarse[I] = mean of the children fine[...] (restriction of D): one thread
// per coarse x cell, a coarse row per blockIdx.y, a coarse plane per blockIdx.z
template <typename T>
__global__ void __launch_bounds__(128) restrict_kernel(const T* fine, T* coarse, int nf0, int nf1,
                                                       int nc0, int nc1, int h0, int h1, int h2) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y, K = blockIdx.z;
    if (I >= nc0) return;
    const T inv = T(1) / T(h0 * h1 * h2);
    T s = T(0);
    for (int c = 0; c < h2; ++c)
        for (int b = 0; b < h1; ++b)
            for (int a = 0; a < h0; ++a)
                s += fine[((long long)(K * h2 + c) * nf1 + (J * h1 + b)) * nf0 + (I * h0 + a)];
    coarse[((long long)K * nc1 + J) * nc0 + I] = s * inv;
}

// fine[i] += coarse[parent(i)]
// fine += the coarse correction of the parent cell (piecewise constant).  Each
// thread takes its x cell in SMOOTH_ROWS consecutive rows, loads first.
template <typename T>
__global__ void __launch_bounds__(128) prolong_kernel(T* fine, const T* coarse, int nf0, int nf1,
                                                      int nc0, int nc1, int h0, int h1, int h2) {
    griddep_wait();
    const int k = blockIdx.z;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf0) return;
    const int ic = i / h0;
    const int kc = (k / h2) * nc1;                     // levels have fewer than 2^31 cells
    T f[SMOOTH_ROWS], c[SMOOTH_ROWS];
    int qs[SMOOTH_ROWS];
    bool on[SMOOTH_ROWS];
#pragma unroll
    for (int r = 0; r < SMOOTH_ROWS; ++r) {
        const int j = blockIdx.y * SMOOTH_ROWS + r;
        on[r] = j < nf1;
        const int jj = on[r] ? j : 0;
        qs[r] = (k * nf1 + jj) * nf0 + i;
        f[r] = fine[qs[r]];
        c[r] = coarse[(kc + jj / h1) * nc0 + ic];
    }
#pragma unroll
    for (int r = 0; r < SMOOTH_ROWS; ++r)
        if (on[r]) fine[qs[r]] = f[r] + c[r];
    griddep_launch_dependents();
}

// D = c lambda(R) / (kappa rho), R = |grad E| / (rho kappa E), on level 0:
// each thread takes its x cell in SMOOTH_ROWS consecutive rows of a plane
// (x along threads, a row group per blockIdx.y, a plane per blockIdx.z), the
// rows' loads issued before their arithmetic; neighbours across a periodic
// wrap or, at a wall, the cell itself.  h0, h1, h2: 1 / (2 dx) per axis; the
// limiter's quotient and the last one are taken together,
// D = c (2 + R) / ((6 + 3R + R^2) kappa rho).
template <typename T>
__global__ void __launch_bounds__(128) coeff_kernel(const T* U, const T* E, T* D, LvlArgs<T> a,
                                                    T c, T kappa, T h0, T h1, T h2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.z;
    if (i >= a.n[0]) return;
    const T hx[3] = {h0, h1, h2};
    T Eu[SMOOTH_ROWS][3], Ed[SMOOTH_ROWS][3], Ec[SMOOTH_ROWS], rho[SMOOTH_ROWS];
    int qs[SMOOTH_ROWS];                              // the level has fewer than 2^31 cells
    bool on[SMOOTH_ROWS];
    // the wall neighbour is the cell itself (the edge cell repeated), the
    // periodic one across the wrap: the offsets of axis_nb
    const AxisNb nbz = plane_nb(a, k);
#pragma unroll
    for (int r = 0; r < SMOOTH_ROWS; ++r) {
        const int j = blockIdx.y * SMOOTH_ROWS + r;
        on[r] = j < a.n[1];
        const int jj = on[r] ? j : 0;                // a row outside the level is not stored
        const int q = (k * a.n[1] + jj) * a.n[0] + i;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const int n = a.n[ax];
            Eu[r][ax] = Ed[r][ax] = T(0);
            if (n <= 1) continue;
            const AxisNb b =
                ax == 2 ? nbz : axis_nb(ax == 0 ? i : jj, n, a.per[ax], ax == 0 ? 1 : a.n[0]);
            Eu[r][ax] = E[q + b.hi];
            Ed[r][ax] = E[q + b.lo];
        }
        Ec[r] = E[q];
        rho[r] = U[q];
        qs[r] = q;
    }
#pragma unroll
    for (int r = 0; r < SMOOTH_ROWS; ++r) {
        T grad2 = T(0);
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            if (a.n[ax] <= 1) continue;
            const T g = (Eu[r][ax] - Ed[r][ax]) * hx[ax];
            grad2 += g * g;
        }
        const T R = sqrt(grad2) / (rho[r] * kappa * Ec[r]);
        const T den = (T(6) + T(3) * R + R * R) * (kappa * rho[r]);
        if (on[r]) D[qs[r]] = c * (T(2) + R) / den;
    }
}

int grid_for(long long N) {
    long long b = (N + 255) / 256;
    return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

// one thread per x cell (or per x pair), a row per blockIdx.y, a plane per blockIdx.z
dim3 rows_grid(const FldLevel& L, int per_thread) {
    const int nx = (L.n[0] + per_thread - 1) / per_thread;
    return dim3((unsigned)((nx + 127) / 128), (unsigned)L.n[1], (unsigned)L.n[2]);
}

template <typename T>
LvlArgs<T> level_args(const FldHierarchy* H, int l, double dt) {
    const FldLevel& L = H->L[l];
    LvlArgs<T> a;
    a.x = static_cast<T*>(L.x);
    a.b = static_cast<const T*>(L.b);
    a.D = static_cast<const T*>(L.D);
    for (int ax = 0; ax < 3; ++ax) {
        a.n[ax] = L.n[ax];
        a.wk[ax] = L.n[ax] > 1 ? (T)(0.5 * dt / (L.dx[ax] * L.dx[ax])) : T(0);
        a.per[ax] = H->bc_lo[ax] == 0 && H->bc_hi[ax] == 0;
    }
    a.N = L.N;
    a.dt = (T)dt;
    return a;
}

template <typename T>
cudaError_t smooth(const FldHierarchy* H, int l, double dt, int sweeps, cudaStream_t s) {
    const LvlArgs<T> a = level_args<T>(H, l, dt);
    const FldLevel& L = H->L[l];
    const int hx = (L.n[0] + 1) / 2;                  // cells of a colour in a row (at most)
    int lg = 0;
    while (lg < 7 && (1 << lg) < hx) ++lg;
    const int sr = l == 0 ? FLD_FINE_ROWS : FLD_COARSE_ROWS;
    const int rows = (128 >> lg) * sr;                // rows of a block
    const dim3 g(lg == 7 ? (unsigned)((hx + 127) / 128) : 1u, (unsigned)((L.n[1] + rows - 1) / rows),
                 (unsigned)L.n[2]);
    auto kern = l == 0 ? smooth_kernel<T, FLD_FINE_ROWS> : smooth_kernel<T, FLD_COARSE_ROWS>;
    for (int it = 0; it < sweeps; ++it)
        for (int color = 0; color < 2; ++color) {
            const cudaError_t e = launch_pdl(kern, g, dim3(128), 0, s, a, color, lg);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

template <typename T>
void restrict_to(const FldHierarchy* H, int l, const void* fine, void* coarse, cudaStream_t s) {
    const FldLevel& F = H->L[l];
    const FldLevel& C = H->L[l + 1];
    restrict_kernel<T><<<rows_grid(C, 1), 128, 0, s>>>(
        static_cast<const T*>(fine), static_cast<T*>(coarse), F.n[0], F.n[1], C.n[0], C.n[1],
        F.coarsened[0] ? 2 : 1, F.coarsened[1] ? 2 : 1, F.coarsened[2] ? 2 : 1);
}

template <typename T>
cudaError_t solve_t(FldHierarchy* H, const MeshDesc& m, const void* U, void* Er, double dt,
                    double c, double kappa, double rtol, int max_cycles, int* cycles,
                    double* rel_resid, cudaStream_t s) {
    FldLevel& L0 = H->L[0];
    L0.x = Er;
    cudaError_t e = cudaMemcpyAsync(L0.b, Er, sizeof(T) * L0.N, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    {
        const LvlArgs<T> a = level_args<T>(H, 0, dt);
        dim3 g = rows_grid(L0, 1);
        g.y = (g.y + SMOOTH_ROWS - 1) / SMOOTH_ROWS;
        coeff_kernel<T><<<g, 128, 0, s>>>(
            static_cast<const T*>(U), static_cast<const T*>(L0.b), static_cast<T*>(L0.D), a,
            (T)c, (T)kappa, (T)(0.5 / m.dxk[0]), (T)(0.5 / m.dxk[1]), (T)(0.5 / m.dxk[2]));
    }
    for (int l = 0; l + 1 < H->nl; ++l) restrict_to<T>(H, l, H->L[l].D, H->L[l + 1].D, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    // the small levels at the bottom run in one block per cycle
    int ls = H->nl;
    while (ls > 0 && H->L[ls - 1].N <= FLD_SMALL_CELLS && H->nl - (ls - 1) <= FLD_SMALL_MAX) --ls;
    SmallLevels<T> S;
    size_t small_bytes = 0;
    if (ls < H->nl) {
        S.count = H->nl - ls;
        S.pre = FLD_PRE;
        S.post = FLD_POST;
        S.coarse = FLD_COARSE;
        int off = 0;
        for (int i = 0; i < S.count; ++i) {
            const FldLevel& F = H->L[ls + i];
            S.lv[i] = level_args<T>(H, ls + i, dt);
            for (int a = 0; a < 3; ++a) S.h[i][a] = F.coarsened[a] ? 2 : 1;
            const int dv[3] = {F.n[0], F.n[1], F.n[0] / 2 > 0 ? F.n[0] / 2 : 1};
            for (int a = 0; a < 3; ++a)
                S.mg[i][a] = dv[a] > 1 ? (unsigned)((1ull << 32) / (unsigned)dv[a] + 1) : 0u;
            S.off[i] = off;
            off += 3 * (int)F.N;
        }
        small_bytes = sizeof(T) * (size_t)off;
        // the limit is raised once per device to the largest set there can
        // be: levels of at most FLD_SMALL_CELLS cells, each at most half the
        // one above, three arrays each
        static std::atomic<unsigned long long> attr{0};
        if ((e = smem_attr_once(small_vcycle_kernel<T>, sizeof(T) * 3 * 2 * FLD_SMALL_CELLS,
                                attr)) != cudaSuccess)
            return e;
    }

    // the convergence check over colour 0 alone (see residual_norm_color_kernel)
    // when the fine level is smoothed by the level kernels and the colouring
    // is proper; sum b^2 then once
    bool color_check = ls > 0 && H->nl > 1;
    for (int ax = 0; ax < 3; ++ax)
        if (L0.n[ax] > 1 && m.bc_lo[ax] == HARD_BC_PERIODIC && (L0.n[ax] & 1)) color_check = false;
    if (rtol > 0.0 && color_check) {
        if ((e = cudaMemsetAsync(H->norms, 0, 2 * sizeof(double), s)) != cudaSuccess) return e;
        sumsq_kernel<T><<<grid_for(L0.N) < 152 * 8 ? grid_for(L0.N) : 152 * 8, 256, 0, s>>>(
            static_cast<const T*>(L0.b), L0.N, H->norms + 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }

    int done = 0;
    double rel = -1.0;
    for (int cyc = 0; cyc < max_cycles; ++cyc) {
        // down: smooth, residual, restrict (the large levels)
        for (int l = 0; l < ls; ++l) {
            if (l + 1 >= H->nl) break;
            if ((e = smooth<T>(H, l, dt, FLD_PRE, s)) != cudaSuccess) return e;
            const FldLevel& F = H->L[l];
            const FldLevel& C = H->L[l + 1];
            const bool h2 = F.coarsened[0] && F.coarsened[1] && F.coarsened[2];
            bool proper = true;                      // red-black is a two-colouring of level l
            for (int ax = 0; ax < 3; ++ax)
                if (F.n[ax] > 1 && m.bc_lo[ax] == HARD_BC_PERIODIC && (F.n[ax] & 1)) proper = false;
            auto rr = h2 ? (proper ? residual_restrict_kernel<T, true, true>
                                   : residual_restrict_kernel<T, true, false>)
                         : residual_restrict_kernel<T, false>;
            e = launch_pdl(rr, rows_grid(C, 1), dim3(128), 0, s, level_args<T>(H, l, dt),
                           static_cast<T*>(C.b), static_cast<T*>(C.x), C.n[0], C.n[1],
                           F.coarsened[0] ? 2 : 1, F.coarsened[1] ? 2 : 1,
                           F.coarsened[2] ? 2 : 1);
            if (e != cudaSuccess) return e;
        }
        if (ls < H->nl) {
            e = launch_pdl(small_vcycle_kernel<T>, dim3(1), dim3(FLD_SMALL_THREADS), small_bytes, s,
                           S);
            if (e != cudaSuccess) return e;
        } else if ((e = smooth<T>(H, H->nl - 1, dt, FLD_COARSE, s)) != cudaSuccess) {
            return e;                                // a coarsest level too large for one block
        }
        // up: prolong the correction, smooth (the large levels)
        for (int l = ls - 1; l >= 0; --l) {
            if (l + 1 >= H->nl) continue;
            const FldLevel& F = H->L[l];
            const FldLevel& C = H->L[l + 1];
            dim3 gp = rows_grid(F, 1);
            gp.y = (gp.y + SMOOTH_ROWS - 1) / SMOOTH_ROWS;
            e = launch_pdl(prolong_kernel<T>, gp, dim3(128), 0, s, static_cast<T*>(F.x),
                           static_cast<const T*>(C.x), F.n[0], F.n[1], C.n[0], C.n[1],
                           F.coarsened[0] ? 2 : 1, F.coarsened[1] ? 2 : 1,
                           F.coarsened[2] ? 2 : 1);
            if (e != cudaSuccess) return e;
            if ((e = smooth<T>(H, l, dt, FLD_POST, s)) != cudaSuccess) return e;
        }
        done = cyc + 1;
        if (rtol > 0.0 && color_check) {
            if ((e = cudaMemsetAsync(H->norms, 0, sizeof(double), s)) != cudaSuccess) return e;
            dim3 g = rows_grid(L0, 2);
            g.y = (g.y + SMOOTH_ROWS - 1) / SMOOTH_ROWS;
            e = launch_pdl(residual_norm_color_kernel<T>, g, dim3(128), 0, s,
                           level_args<T>(H, 0, dt), 0, H->norms);
            if (e != cudaSuccess) return e;
        } else if (rtol > 0.0) {
            if ((e = cudaMemsetAsync(H->norms, 0, 2 * sizeof(double), s)) != cudaSuccess) return e;
            const long long items = (long long)((L0.n[0] + 127) / 128) *
                                    ((L0.n[1] + SMOOTH_ROWS - 1) / SMOOTH_ROWS) * L0.n[2];
            e = launch_pdl(residual_norms_kernel<T>,
                           dim3((unsigned)(items < 152 * 16 ? items : 152 * 16)), dim3(128), 0, s,
                           level_args<T>(H, 0, dt), H->norms);
            if (e != cudaSuccess) return e;
        }
        if (rtol > 0.0) {
            double nr[2];
            if ((e = cudaMemcpyAsync(nr, H->norms, sizeof(nr), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            rel = nr[1] > 0.0 ? std::sqrt(nr[0] / nr[1]) : 0.0;
            if (!(rel > rtol)) break;             // converged (or NaN: stop and report it)
        }
    }
    if (cycles) *cycles = done;
    if (rel_resid) *rel_resid = rel;
    return cudaGetLastError();
}

}  // namespace

FldHierarchy* fld_create(const MeshDesc& m, int dtype) {
    FldHierarchy* H = new (std::nothrow) FldHierarchy();
    if (!H) return nullptr;
    H->dtype = dtype;
    const size_t es = dtype == HARD_F64 ? 8 : 4;
    for (int a = 0; a < 3; ++a) {
        H->n0[a] = m.n[a];
        H->bc_lo[a] = m.bc_lo[a];
        H->bc_hi[a] = m.bc_hi[a];
    }
    int n[3] = {m.n[0], m.n[1], m.n[2]};
    double dx[3] = {m.dxk[0], m.dxk[1], m.dxk[2]};
    int nl = 0;
    bool ok = true;
    if ((long long)n[0] * n[1] * n[2] >= (1ll << 31)) {      // 32-bit cell indices
        delete H;
        return nullptr;
    }
    while (nl < FLD_MAX_LEVELS) {
        FldLevel& L = H->L[nl];
        L.N = (long long)n[0] * n[1] * n[2];
        for (int a = 0; a < 3; ++a) {
            L.n[a] = n[a];
            L.dx[a] = dx[a];
        }
        L.x = nullptr;
        if (nl > 0 && cudaMalloc(&L.x, es * L.N) != cudaSuccess) ok = false;
        if (cudaMalloc(&L.b, es * L.N) != cudaSuccess) ok = false;
        if (cudaMalloc(&L.D, es * L.N) != cudaSuccess) ok = false;
        ++nl;
        if (!ok) break;
        bool any = false;
        for (int a = 0; a < 3; ++a) {
            L.coarsened[a] = n[a] >= 4 && n[a] % 2 == 0;
            any |= L.coarsened[a];
        }
        if (!any || L.N <= 64) {
            for (int a = 0; a < 3; ++a) L.coarsened[a] = false;
            break;
        }
        for (int a = 0; a < 3; ++a)
            if (L.coarsened[a]) {
                n[a] /= 2;
                dx[a] *= 2.0;
            }
    }
    H->nl = nl;
    if (ok && cudaMalloc(&H->norms, 2 * sizeof(double)) != cudaSuccess) ok = false;
    if (!ok) {
        fld_destroy(H);
        cudaGetLastError();
        return nullptr;
    }
    return H;
}

void fld_destroy(FldHierarchy* H) {
    if (!H) return;
    for (int l = 0; l < H->nl; ++l) {
        if (l > 0) cudaFree(H->L[l].x);
        cudaFree(H->L[l].b);
        cudaFree(H->L[l].D);
    }
    cudaFree(H->norms);
    delete H;
}

bool fld_matches(const FldHierarchy* H, const MeshDesc& m, int dtype) {
    if (!H || H->dtype != dtype) return false;
    for (int a = 0; a < 3; ++a)
        if (H->n0[a] != m.n[a] || H->bc_lo[a] != m.bc_lo[a] || H->bc_hi[a] != m.bc_hi[a] ||
            H->L[0].dx[a] != m.dxk[a])
            return false;
    return true;
}

int fld_levels(const FldHierarchy* H) { return H ? H->nl : 0; }

cudaError_t fld_solve(FldHierarchy* H, const MeshDesc& m, const void* U, void* Er, double dt,
                      double c, double kappa, double rtol, int max_cycles, int* cycles,
                      double* rel_resid, cudaStream_t s) {
    return H->dtype == HARD_F64
               ? solve_t<double>(H, m, U, Er, dt, c, kappa, rtol, max_cycles, cycles, rel_resid, s)
               : solve_t<float>(H, m, U, Er, dt, c, kappa, rtol, max_cycles, cycles, rel_resid, s);
}

}  // namespace hh
