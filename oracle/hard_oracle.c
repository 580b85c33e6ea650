/*
 * Plain FP64 CPU oracle for the explicit finite-volume hydro stage update.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; it exists so that tests, the smoke check and the bench's
 * CPU-baseline leg can compare the CUDA path against an independent,
 * obviously-correct restatement of the method.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * What it computes (paper: "HARD", arXiv 2509.08971):
 *   - Eq. "conservative form" with S = 0:  d_t U + d_j F^j = 0,
 *     U = [rho, rho v^i, e + rho v^2/2]  (radiation energy E dropped),
 *     F^j from Eq. "fluxes", ideal-gas closure p = (gamma-1) e
 *     (the ideal EoS of the temperature-induced shock test, Sec. 3.4).
 *   - Sec. 2.2.2: cell-centred uniform Cartesian mesh, flux difference
 *     (F*_{i+1/2} - F*_{i-1/2}) / dx_i summed over the active axes.
 *   - Face states: piecewise-linear, minmod-limited reconstruction of the
 *     primitives (rho, v, p).  The paper uses WENO5-Z here; this scheme is
 *     the documented deviation (see the minmod and plm_faces comments).
 *   - Face flux: HLLC (three-wave) with Davis wave-speed bounds.  The paper
 *     uses HLL; HLLC is its contact-restoring extension (Toro, "Riemann
 *     Solvers and Numerical Methods for Fluid Dynamics", ch. 10).
 *   - Time advance: Heun's method, Table "Butcher tableau for Heun's
 *     method", evaluated in the Shu-Osher form; the Heun form is kept as a
 *     separate entry point for the cross-check.
 *   - Time step: unsplit CFL rule dt = C / max_cells sum_d (|v_d| + c)/dx_d
 *     (Sec. 3.1 and Sec. 3.5 use a CFL-limited step but print no formula).
 *   - Exact Riemann solver for the 1D ideal-gas Euler equations (Toro ch. 4),
 *     used to build the reference solution of the L1 metric, Eq. "l1_error".
 *   - Radiation energy advection, d_j(E v^j) of Eq. "radiation": WENO5-Z
 *     states and the Rusanov flux, Heun in time with U held fixed.
 *   - Radiative heating / cooling, Eq. "heating-cooling": a pointwise
 *     backward-Euler exchange of fluid and radiation energy (orc_rad_exchange).
 *   - Second scheme (scheme = 1), the paper's own choice of Sec. 2.2.2:
 *     WENO5-Z face states of every primitive (Borges, Carmona, Costa, Don
 *     2008) and the HLL flux (Harten, Lax, van Leer 1983) with the same
 *     Davis wave-speed bounds; three ghost layers per active axis.
 *
 * Storage: structure of arrays U[5][nz][ny][nx], x fastest.  Field order
 * rho, rho*u, rho*v, rho*w, E_total.  Ghost cells are not stored; they are
 * produced by the boundary map of ghost_src().
 *
 * Compile with -ffp-contract=off: every + - * / and sqrt is a separately
 * rounded IEEE operation, on x86 and on Arm alike.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NF 5

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECT = 2 };

typedef struct {
    int n[3];        /* cells along x, y, z                          */
    double dx[3];    /* cell widths                                   */
    int bc[6];       /* x-, x+, y-, y+, z-, z+                        */
    double gamma;    /* ratio of specific heats                       */
    int scheme;      /* 0: PLM-minmod + HLLC;  1: WENO5-Z + HLL        */
} grid_t;

static size_t ncell(const grid_t* g) { return (size_t)g->n[0] * g->n[1] * g->n[2]; }

static size_t cell_index(const grid_t* g, int i, int j, int k) {
    return ((size_t)k * g->n[1] + j) * g->n[0] + i;
}

/* An axis takes part in the update only when it has more than one cell. */
static int axis_active(const grid_t* g, int d) { return g->n[d] > 1; }

/*
 * Boundary map for one axis.  Index m in [-3, n+2] (three ghost layers; the
 * PLM scheme uses two) is
 * mapped to an interior index; *flip is set to 1 when the normal momentum of
 * the source cell must change sign (reflecting wall).
 *   periodic: wrap around;  outflow: copy the nearest interior cell;
 *   reflect: mirror about the wall.
 */
static int ghost_src(int m, int n, int bc_lo, int bc_hi, int* flip) {
    *flip = 0;
    if (m >= 0 && m < n) return m;
    int bc = (m < 0) ? bc_lo : bc_hi;
    if (bc == BC_PERIODIC) {
        int r = m % n;
        return r < 0 ? r + n : r;
    }
    if (bc == BC_OUTFLOW) return m < 0 ? 0 : n - 1;
    /* reflect: ghost -1 <- 0, -2 <- 1, -3 <- 2;  ghost n <- n-1, n+1 <- n-2, ... */
    *flip = 1;
    return m < 0 ? -1 - m : 2 * n - 1 - m;
}

/* Conserved state of cell (i,j,k) displaced by m cells along axis d, with
 * the boundary map applied along that axis only. */
static void fetch_cons(const grid_t* g, const double* U, int d, int i, int j, int k,
                       int m, double out[NF]) {
    int idx[3] = {i, j, k};
    int flip = 0;
    idx[d] = ghost_src(idx[d] + m, g->n[d], g->bc[2 * d], g->bc[2 * d + 1], &flip);
    size_t c = cell_index(g, idx[0], idx[1], idx[2]);
    size_t N = ncell(g);
    for (int f = 0; f < NF; ++f) out[f] = U[f * N + c];
    if (flip) out[1 + d] = -out[1 + d];
}

/* Eq. "fluxes" with the ideal-gas closure: conserved -> primitive
 * W = (rho, u, v, w, p),  p = (gamma-1)(E - rho |v|^2 / 2). */
static void cons_to_prim(const double U[NF], double gamma, double W[NF]) {
    double rho = U[0];
    double u = U[1] / rho;
    double v = U[2] / rho;
    double w = U[3] / rho;
    double kin = 0.5 * rho * (u * u + v * v + w * w);
    W[0] = rho;
    W[1] = u;
    W[2] = v;
    W[3] = w;
    W[4] = (gamma - 1.0) * (U[4] - kin);
}

/*
 * minmod limiter.  Zero unless both slopes have the same strict sign (a sign
 * test, not a product, so tiny slopes do not underflow to a false zero);
 * otherwise the one of smaller magnitude, taking a on a tie.
 */
double orc_minmod(double a, double b) {
    if (a > 0.0 && b > 0.0) return (a <= b) ? a : b;
    if (a < 0.0 && b < 0.0) return (-a <= -b) ? a : b;
    return 0.0;
}

/* Physical flux along the normal of a rotated primitive state
 * Wn = (rho, un, vt1, vt2, p): Eq. "fluxes" for the normal direction. */
static void normal_flux(const double Wn[NF], double gamma, double Un[NF], double F[NF]) {
    double rho = Wn[0], un = Wn[1], t1 = Wn[2], t2 = Wn[3], p = Wn[4];
    double E = p / (gamma - 1.0) + 0.5 * rho * (un * un + t1 * t1 + t2 * t2);
    Un[0] = rho;
    Un[1] = rho * un;
    Un[2] = rho * t1;
    Un[3] = rho * t2;
    Un[4] = E;
    F[0] = rho * un;
    F[1] = rho * un * un + p;
    F[2] = rho * un * t1;
    F[3] = rho * un * t2;
    F[4] = (E + p) * un;
}

/*
 * HLLC flux for two rotated primitive states (normal along component 1).
 *   sound speeds      c_K = sqrt(gamma p_K / rho_K)
 *   Davis bounds      S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R)
 *   contact speed     S* = [p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R)]
 *                          / [rho_L (S_L - u_L) - rho_R (S_R - u_R)]
 *   star state        U*_K = rho_K (S_K - u_K)/(S_K - S*) *
 *                        [1, S*, t1_K, t2_K, E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))]
 *   flux              F_L            if 0 <= S_L
 *                     F_L + S_L (U*_L - U_L)   if S_L < 0 <= S*
 *                     F_R + S_R (U*_R - U_R)   if S* < 0 <  S_R
 *                     F_R            if S_R <= 0
 */
static void hllc_normal(const double WL[NF], const double WR[NF], double gamma, double F[NF]) {
    double UL[NF], FL[NF], UR[NF], FR[NF];
    normal_flux(WL, gamma, UL, FL);
    normal_flux(WR, gamma, UR, FR);
    double rL = WL[0], uL = WL[1], pL = WL[4];
    double rR = WR[0], uR = WR[1], pR = WR[4];
    double cL = sqrt(gamma * pL / rL);
    double cR = sqrt(gamma * pR / rR);
    double SL = fmin(uL - cL, uR - cR);
    double SR = fmax(uL + cL, uR + cR);
    double Sstar = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR))
                 / (rL * (SL - uL) - rR * (SR - uR));
    if (0.0 <= SL) {
        for (int f = 0; f < NF; ++f) F[f] = FL[f];
        return;
    }
    if (SR <= 0.0) {
        for (int f = 0; f < NF; ++f) F[f] = FR[f];
        return;
    }
    const double* W = (Sstar >= 0.0) ? WL : WR;
    const double* UK = (Sstar >= 0.0) ? UL : UR;
    const double* FK = (Sstar >= 0.0) ? FL : FR;
    double SK = (Sstar >= 0.0) ? SL : SR;
    double r = W[0], u = W[1], p = W[4];
    double fac = r * (SK - u) / (SK - Sstar);
    double Us[NF];
    Us[0] = fac;
    Us[1] = fac * Sstar;
    Us[2] = fac * W[2];
    Us[3] = fac * W[3];
    Us[4] = fac * (UK[4] / r + (Sstar - u) * (Sstar + p / (r * (SK - u))));
    for (int f = 0; f < NF; ++f) F[f] = FK[f] + SK * (Us[f] - UK[f]);
}

/* Exposed for unit tests: x-normal HLLC on primitive states (rho,u,v,w,p). */
void orc_hllc(const double* WL, const double* WR, double gamma, double* F) {
    hllc_normal(WL, WR, gamma, F);
}

/*
 * HLL flux (Harten, Lax, van Leer 1983) for two rotated primitive states,
 * with the Davis bounds S_L, S_R of hllc_normal:
 *   F = F_L                                              if 0 <= S_L
 *       (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L)   if S_L < 0 < S_R
 *       F_R                                              if S_R <= 0
 * (the flux of the single averaged state between the two outer waves).
 */
static void hll_normal(const double WL[NF], const double WR[NF], double gamma, double F[NF]) {
    double UL[NF], FL[NF], UR[NF], FR[NF];
    normal_flux(WL, gamma, UL, FL);
    normal_flux(WR, gamma, UR, FR);
    double cL = sqrt(gamma * WL[4] / WL[0]);
    double cR = sqrt(gamma * WR[4] / WR[0]);
    double SL = fmin(WL[1] - cL, WR[1] - cR);
    double SR = fmax(WL[1] + cL, WR[1] + cR);
    if (0.0 <= SL) {
        for (int f = 0; f < NF; ++f) F[f] = FL[f];
        return;
    }
    if (SR <= 0.0) {
        for (int f = 0; f < NF; ++f) F[f] = FR[f];
        return;
    }
    for (int f = 0; f < NF; ++f)
        F[f] = (SR * FL[f] - SL * FR[f] + SL * SR * (UR[f] - UL[f])) / (SR - SL);
}

/* Exposed for unit tests: x-normal HLL on primitive states (rho,u,v,w,p). */
void orc_hll(const double* WL, const double* WR, double gamma, double* F) {
    hll_normal(WL, WR, gamma, F);
}

/*
 * WENO5-Z reconstruction (Borges, Carmona, Costa, Don 2008) of the value at
 * the right face of the middle cell of v[0..4] = v_{i-2} .. v_{i+2} (cell
 * averages).  Three third-order candidates on the stencils {i-2,i-1,i},
 * {i-1,i,i+1}, {i,i+1,i+2}:
 *   p0 = ( 2 v_{i-2} - 7 v_{i-1} + 11 v_i    ) / 6
 *   p1 = (  -v_{i-1} + 5 v_i     +  2 v_{i+1}) / 6
 *   p2 = ( 2 v_i     + 5 v_{i+1} -    v_{i+2}) / 6
 * Jiang-Shu smoothness indicators
 *   b0 = 13/12 (v_{i-2} - 2 v_{i-1} + v_i)^2     + 1/4 (v_{i-2} - 4 v_{i-1} + 3 v_i)^2
 *   b1 = 13/12 (v_{i-1} - 2 v_i + v_{i+1})^2     + 1/4 (v_{i-1} - v_{i+1})^2
 *   b2 = 13/12 (v_i - 2 v_{i+1} + v_{i+2})^2     + 1/4 (3 v_i - 4 v_{i+1} + v_{i+2})^2
 * global indicator tau5 = |b0 - b2| and the Z weights
 *   a_k = d_k (1 + tau5 / (b_k + eps)),  (d0, d1, d2) = (1/10, 6/10, 3/10),
 *   value = sum a_k p_k / sum a_k.
 * The exponent on tau5 / (b_k + eps) is 1 (the original WENO-Z) and
 * eps = 1e-30; the paper fixes neither.  The right state of a face is the
 * same function of the mirrored stencil.
 */
#define WENO_EPS 1e-30
double orc_weno5z(const double* v) {
    double p0 = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) / 6.0;
    double p1 = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;
    double p2 = (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0;
    double s0 = v[0] - 2.0 * v[1] + v[2], t0 = v[0] - 4.0 * v[1] + 3.0 * v[2];
    double s1 = v[1] - 2.0 * v[2] + v[3], t1 = v[1] - v[3];
    double s2 = v[2] - 2.0 * v[3] + v[4], t2 = 3.0 * v[2] - 4.0 * v[3] + v[4];
    double b0 = 13.0 / 12.0 * s0 * s0 + 0.25 * t0 * t0;
    double b1 = 13.0 / 12.0 * s1 * s1 + 0.25 * t1 * t1;
    double b2 = 13.0 / 12.0 * s2 * s2 + 0.25 * t2 * t2;
    double tau = fabs(b0 - b2);
    double a0 = 0.1 * (1.0 + tau / (b0 + WENO_EPS));
    double a1 = 0.6 * (1.0 + tau / (b1 + WENO_EPS));
    double a2 = 0.3 * (1.0 + tau / (b2 + WENO_EPS));
    return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2);
}

/* Component order of the rotated frame for axis d: normal, tangent 1, tangent 2
 * (indices into the momentum/velocity slots 1..3). */
static const int ROT[3][3] = {{1, 2, 3}, {2, 1, 3}, {3, 1, 2}};

/*
 * Numerical flux through the face between cell (i,j,k) and its +1 neighbour
 * along axis d.  PLM with minmod on the primitives:
 *   dq_m   = minmod(q_m - q_{m-1}, q_{m+1} - q_m)
 *   q_L    = q_i     + dq_i / 2          (left state at i+1/2)
 *   q_R    = q_{i+1} - dq_{i+1} / 2      (right state at i+1/2)
 * then HLLC in the frame whose normal is axis d.
 */
static void face_flux_weno(const grid_t* g, const double* U, int d, int i, int j, int k,
                           double F[NF]);

static void face_flux(const grid_t* g, const double* U, int d, int i, int j, int k,
                      double F[NF]) {
    if (g->scheme == 1) {
        face_flux_weno(g, U, d, i, j, k, F);
        return;
    }
    double W[4][NF];                   /* cells i-1, i, i+1, i+2 along d */
    for (int s = 0; s < 4; ++s) {
        double Uc[NF];
        fetch_cons(g, U, d, i, j, k, s - 1, Uc);
        cons_to_prim(Uc, g->gamma, W[s]);
    }
    double qL[NF], qR[NF];
    for (int f = 0; f < NF; ++f) {
        double dqi = orc_minmod(W[1][f] - W[0][f], W[2][f] - W[1][f]);
        double dqi1 = orc_minmod(W[2][f] - W[1][f], W[3][f] - W[2][f]);
        qL[f] = W[1][f] + 0.5 * dqi;
        qR[f] = W[2][f] - 0.5 * dqi1;
    }
    double WLn[NF] = {qL[0], qL[ROT[d][0]], qL[ROT[d][1]], qL[ROT[d][2]], qL[4]};
    double WRn[NF] = {qR[0], qR[ROT[d][0]], qR[ROT[d][1]], qR[ROT[d][2]], qR[4]};
    double Fn[NF];
    hllc_normal(WLn, WRn, g->gamma, Fn);
    F[0] = Fn[0];
    F[ROT[d][0]] = Fn[1];
    F[ROT[d][1]] = Fn[2];
    F[ROT[d][2]] = Fn[3];
    F[4] = Fn[4];
}

/*
 * Numerical flux of scheme 1 through the face between cell (i,j,k) and its
 * +1 neighbour along axis d: WENO5-Z states of the primitives from the six
 * cells i-2 .. i+3,
 *   q_L = weno5z(q_{i-2}, q_{i-1}, q_i, q_{i+1}, q_{i+2})
 *   q_R = weno5z(q_{i+3}, q_{i+2}, q_{i+1}, q_i, q_{i-1})   (mirrored)
 * then HLL in the frame whose normal is axis d.
 */
static void face_flux_weno(const grid_t* g, const double* U, int d, int i, int j, int k,
                           double F[NF]) {
    double W[6][NF];                   /* cells i-2 .. i+3 along d */
    for (int s = 0; s < 6; ++s) {
        double Uc[NF];
        fetch_cons(g, U, d, i, j, k, s - 2, Uc);
        cons_to_prim(Uc, g->gamma, W[s]);
    }
    double qL[NF], qR[NF];
    for (int f = 0; f < NF; ++f) {
        double l[5] = {W[0][f], W[1][f], W[2][f], W[3][f], W[4][f]};
        double r[5] = {W[5][f], W[4][f], W[3][f], W[2][f], W[1][f]};
        qL[f] = orc_weno5z(l);
        qR[f] = orc_weno5z(r);
    }
    double WLn[NF] = {qL[0], qL[ROT[d][0]], qL[ROT[d][1]], qL[ROT[d][2]], qL[4]};
    double WRn[NF] = {qR[0], qR[ROT[d][0]], qR[ROT[d][1]], qR[ROT[d][2]], qR[4]};
    double Fn[NF];
    hll_normal(WLn, WRn, g->gamma, Fn);
    F[0] = Fn[0];
    F[ROT[d][0]] = Fn[1];
    F[ROT[d][1]] = Fn[2];
    F[ROT[d][2]] = Fn[3];
    F[4] = Fn[4];
}

/* scheme 1 needs three cells along every active axis (three ghost layers
 * mirror into the interior of a reflecting wall) */
static int make_grid_s(grid_t* g, int scheme, int nx, int ny, int nz, const double* dxyz,
                       const int* bc6, double gamma) {
    if (nx < 1 || ny < 1 || nz < 1 || (scheme != 0 && scheme != 1)) return -1;
    g->n[0] = nx; g->n[1] = ny; g->n[2] = nz;
    for (int d = 0; d < 3; ++d) g->dx[d] = dxyz[d];
    for (int f = 0; f < 6; ++f) g->bc[f] = bc6[f];
    g->gamma = gamma;
    g->scheme = scheme;
    if (scheme == 1)
        for (int d = 0; d < 3; ++d)
            if (g->n[d] > 1 && g->n[d] < 3) return -1;
    return 0;
}

static int make_grid(grid_t* g, int nx, int ny, int nz, const double* dxyz, const int* bc6,
                     double gamma) {
    return make_grid_s(g, 0, nx, ny, nz, dxyz, bc6, gamma);
}

/*
 * Right-hand side of the semi-discrete system (Sec. 2.2.2):
 *   L(U)_i = - sum_{d active, in order x, y, z} (F*_{i+1/2} - F*_{i-1/2}) / dx_d
 * The face flux is a function of the face alone; each face is evaluated once
 * per call and used by both of its cells.
 */
static void rhs(const grid_t* g, const double* U, double* L) {
    size_t N = ncell(g);
    memset(L, 0, sizeof(double) * NF * N);
    for (int d = 0; d < 3; ++d) {
        if (!axis_active(g, d)) continue;
        int nf[3] = {g->n[0], g->n[1], g->n[2]};
        nf[d] += 1;                                   /* faces along d */
        size_t nfaces = (size_t)nf[0] * nf[1] * nf[2];
        double* Ff = (double*)malloc(sizeof(double) * NF * nfaces);
        /* face index m along d sits between cells m-1 and m */
#pragma omp parallel for schedule(static)
        for (int kk = 0; kk < nf[2]; ++kk)
            for (int jj = 0; jj < nf[1]; ++jj)
                for (int ii = 0; ii < nf[0]; ++ii) {
                    int c[3] = {ii, jj, kk};
                    c[d] -= 1;                        /* left cell of the face */
                    double F[NF];
                    face_flux(g, U, d, c[0], c[1], c[2], F);
                    size_t fi = ((size_t)kk * nf[1] + jj) * nf[0] + ii;
                    for (int f = 0; f < NF; ++f) Ff[f * nfaces + fi] = F[f];
                }
#pragma omp parallel for schedule(static)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                    hi[d] += 1;
                    size_t flo = ((size_t)lo[2] * nf[1] + lo[1]) * nf[0] + lo[0];
                    size_t fhi = ((size_t)hi[2] * nf[1] + hi[1]) * nf[0] + hi[0];
                    size_t c = cell_index(g, i, j, k);
                    for (int f = 0; f < NF; ++f)
                        L[f * N + c] -= (Ff[f * nfaces + fhi] - Ff[f * nfaces + flo]) / g->dx[d];
                }
        free(Ff);
    }
}

int orc_rhs_s(int scheme, int nx, int ny, int nz, const double* dxyz, const int* bc6,
              double gamma, const double* U, double* L) {
    grid_t g;
    if (make_grid_s(&g, scheme, nx, ny, nz, dxyz, bc6, gamma)) return -1;
    rhs(&g, U, L);
    return 0;
}

int orc_rhs(int nx, int ny, int nz, const double* dxyz, const int* bc6, double gamma,
            const double* U, double* L) {
    return orc_rhs_s(0, nx, ny, nz, dxyz, bc6, gamma, U, L);
}

/*
 * One RK stage in Shu-Osher form (Table "Butcher tableau for Heun's method"):
 *   stage 1:  U1      = Un + dt L(Un)
 *   stage 2:  U^{n+1} = Un/2 + (U1 + dt L(U1))/2
 * stage = 1 reads Ucur = Un; stage = 2 reads Ucur = U1 and U0 = Un.
 */
int orc_stage_s(int scheme, int nx, int ny, int nz, const double* dxyz, const int* bc6,
                double gamma, int stage, const double* U0, const double* Ucur, double* Uout,
                double dt) {
    grid_t g;
    if (make_grid_s(&g, scheme, nx, ny, nz, dxyz, bc6, gamma)) return -1;
    size_t n = NF * ncell(&g);
    double* L = (double*)malloc(sizeof(double) * n);
    rhs(&g, Ucur, L);
    for (size_t q = 0; q < n; ++q) {
        if (stage == 1)
            Uout[q] = Ucur[q] + dt * L[q];
        else
            Uout[q] = 0.5 * U0[q] + 0.5 * (Ucur[q] + dt * L[q]);
    }
    free(L);
    return 0;
}

int orc_stage(int nx, int ny, int nz, const double* dxyz, const int* bc6, double gamma,
              int stage, const double* U0, const double* Ucur, double* Uout, double dt) {
    return orc_stage_s(0, nx, ny, nz, dxyz, bc6, gamma, stage, U0, Ucur, Uout, dt);
}

/* One full step, Shu-Osher form. */
int orc_step_s(int scheme, int nx, int ny, int nz, const double* dxyz, const int* bc6,
               double gamma, const double* Un, double* Unew, double dt) {
    size_t n = (size_t)NF * nx * ny * nz;
    double* U1 = (double*)malloc(sizeof(double) * n);
    int rc = orc_stage_s(scheme, nx, ny, nz, dxyz, bc6, gamma, 1, Un, Un, U1, dt);
    if (!rc) rc = orc_stage_s(scheme, nx, ny, nz, dxyz, bc6, gamma, 2, Un, U1, Unew, dt);
    free(U1);
    return rc;
}

int orc_step(int nx, int ny, int nz, const double* dxyz, const int* bc6, double gamma,
             const double* Un, double* Unew, double dt) {
    return orc_step_s(0, nx, ny, nz, dxyz, bc6, gamma, Un, Unew, dt);
}

/* One full step in the Butcher form of Heun's method (cross-check only):
 *   k1 = L(Un), k2 = L(Un + dt k1), U^{n+1} = Un + dt (k1/2 + k2/2). */
int orc_step_heun(int nx, int ny, int nz, const double* dxyz, const int* bc6, double gamma,
                  const double* Un, double* Unew, double dt) {
    grid_t g;
    if (make_grid(&g, nx, ny, nz, dxyz, bc6, gamma)) return -1;
    size_t n = NF * ncell(&g);
    double* k1 = (double*)malloc(sizeof(double) * n);
    double* k2 = (double*)malloc(sizeof(double) * n);
    double* Y = (double*)malloc(sizeof(double) * n);
    rhs(&g, Un, k1);
    for (size_t q = 0; q < n; ++q) Y[q] = Un[q] + dt * k1[q];
    rhs(&g, Y, k2);
    for (size_t q = 0; q < n; ++q) Unew[q] = Un[q] + dt * (0.5 * k1[q] + 0.5 * k2[q]);
    free(k1); free(k2); free(Y);
    return 0;
}

/* Largest signal rate over the cells: r = max sum_{d active} (|v_d| + c) / dx_d,
 * c = sqrt(gamma p / rho).  dt = C / r is the unsplit CFL step. */
double orc_max_rate(int nx, int ny, int nz, const double* dxyz, const int* bc6, double gamma,
                    const double* U) {
    grid_t g;
    if (make_grid(&g, nx, ny, nz, dxyz, bc6, gamma)) return -1.0;
    size_t N = ncell(&g);
    double rmax = 0.0;
    for (size_t c = 0; c < N; ++c) {
        double Uc[NF], W[NF];
        for (int f = 0; f < NF; ++f) Uc[f] = U[f * N + c];
        cons_to_prim(Uc, gamma, W);
        double cs = sqrt(gamma * W[4] / W[0]);
        double r = 0.0;
        for (int d = 0; d < 3; ++d)
            if (axis_active(&g, d)) r += (fabs(W[1 + d]) + cs) / g.dx[d];
        if (r > rmax || r != r) rmax = r;         /* a NaN rate propagates */
    }
    return rmax;
}

/*
 * Time loop: for each of nsteps steps, dt = cfl / r(U^n), clipped so that
 * t + dt <= t_end when t_end > 0, then one Shu-Osher step.  Stops early when
 * t reaches t_end.  *t is advanced in place; dt_log (may be NULL) receives
 * each dt.  Returns the number of steps taken, or -1 on a bad rate.
 */
int orc_run_s(int scheme, int nx, int ny, int nz, const double* dxyz, const int* bc6,
              double gamma, double* U, int nsteps, double cfl, double t_end, double* t,
              double* dt_log) {
    size_t n = (size_t)NF * nx * ny * nz;
    double* Unew = (double*)malloc(sizeof(double) * n);
    int s = 0;
    for (; s < nsteps; ++s) {
        if (t_end > 0.0 && *t >= t_end) break;
        double r = orc_max_rate(nx, ny, nz, dxyz, bc6, gamma, U);
        if (!(r > 0.0) || !isfinite(r)) { free(Unew); return -1; }
        double dt = cfl / r;
        if (t_end > 0.0 && *t + dt > t_end) dt = t_end - *t;
        if (orc_step_s(scheme, nx, ny, nz, dxyz, bc6, gamma, U, Unew, dt)) {
            free(Unew);
            return -1;
        }
        memcpy(U, Unew, sizeof(double) * n);
        *t += dt;
        if (dt_log) dt_log[s] = dt;
    }
    free(Unew);
    return s;
}

int orc_run(int nx, int ny, int nz, const double* dxyz, const int* bc6, double gamma,
            double* U, int nsteps, double cfl, double t_end, double* t, double* dt_log) {
    return orc_run_s(0, nx, ny, nz, dxyz, bc6, gamma, U, nsteps, cfl, t_end, t, dt_log);
}

/* Same loop on a recorded dt schedule (no CFL evaluation). */
int orc_run_fixed_s(int scheme, int nx, int ny, int nz, const double* dxyz, const int* bc6,
                    double gamma, double* U, int nsteps, const double* dts) {
    size_t n = (size_t)NF * nx * ny * nz;
    double* Unew = (double*)malloc(sizeof(double) * n);
    for (int s = 0; s < nsteps; ++s) {
        if (orc_step_s(scheme, nx, ny, nz, dxyz, bc6, gamma, U, Unew, dts[s])) {
            free(Unew);
            return -1;
        }
        memcpy(U, Unew, sizeof(double) * n);
    }
    free(Unew);
    return nsteps;
}

int orc_run_fixed(int nx, int ny, int nz, const double* dxyz, const int* bc6, double gamma,
                  double* U, int nsteps, const double* dts) {
    return orc_run_fixed_s(0, nx, ny, nz, dxyz, bc6, gamma, U, nsteps, dts);
}

/* Conserved totals sum_cells U_f dV with Neumaier compensated summation. */
void orc_totals(int nx, int ny, int nz, const double* dxyz, const double* U, double* out5) {
    size_t N = (size_t)nx * ny * nz;
    double dV = dxyz[0] * dxyz[1] * dxyz[2];
    for (int f = 0; f < NF; ++f) {
        double s = 0.0, comp = 0.0;
        for (size_t c = 0; c < N; ++c) {
            double x = U[f * N + c];
            double t = s + x;
            if (fabs(s) >= fabs(x)) comp += (s - t) + x;
            else comp += (x - t) + s;
            s = t;
        }
        out5[f] = (s + comp) * dV;
    }
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Radiation energy advection (the d_j(E v^j) term of Eq. "radiation").       */
/* ------------------------------------------------------------------------ */

/* The Rusanov flux of E u from face states (E_L, u_L), (E_R, u_R). */
double orc_rusanov_E(double EL, double ER, double uL, double uR) {
    double a = fmax(fabs(uL), fabs(uR));
    return 0.5 * (EL * uL + ER * uR) - 0.5 * a * (ER - EL);
}

/* E of cell (i,j,k) displaced by m cells along axis d (the ghost map of
 * fetch_cons; E is a scalar, so a reflecting wall does not flip it). */
static double fetch_scalar(const grid_t* g, const double* E, int d, int i, int j, int k, int m) {
    int idx[3] = {i, j, k};
    int flip = 0;
    idx[d] = ghost_src(idx[d] + m, g->n[d], g->bc[2 * d], g->bc[2 * d + 1], &flip);
    return E[cell_index(g, idx[0], idx[1], idx[2])];
}

/*
 * Rusanov (local Lax-Friedrichs) flux of E v through the face between cell
 * (i,j,k) and its +1 neighbour along d (Sec. 2.2.2: WENO5-Z states of every
 * variable, Rusanov for the radiation energy density): WENO5-Z states E_L,
 * E_R of E and u_L, u_R of the normal velocity (a primitive of U) from the
 * six cells i-2 .. i+3, then
 *   F = (E_L u_L + E_R u_R) / 2 - a (E_R - E_L) / 2,  a = max(|u_L|, |u_R|).
 */
static double rusanov_E(const grid_t* g, const double* U, const double* E, int d, int i, int j,
                        int k) {
    double e[6], u[6];
    for (int s = 0; s < 6; ++s) {
        double Uc[NF], W[NF];
        fetch_cons(g, U, d, i, j, k, s - 2, Uc);
        cons_to_prim(Uc, g->gamma, W);
        u[s] = W[1 + d];
        e[s] = fetch_scalar(g, E, d, i, j, k, s - 2);
    }
    double el[5] = {e[0], e[1], e[2], e[3], e[4]}, er[5] = {e[5], e[4], e[3], e[2], e[1]};
    double ul[5] = {u[0], u[1], u[2], u[3], u[4]}, ur[5] = {u[5], u[4], u[3], u[2], u[1]};
    return orc_rusanov_E(orc_weno5z(el), orc_weno5z(er), orc_weno5z(ul), orc_weno5z(ur));
}

/* L_E(E; U) = - sum_{d active} (F_{i+1/2} - F_{i-1/2}) / dx_d. */
static void rhs_E(const grid_t* g, const double* U, const double* E, double* L) {
    size_t N = ncell(g);
    memset(L, 0, sizeof(double) * N);
    for (int d = 0; d < 3; ++d) {
        if (!axis_active(g, d)) continue;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    int lo[3] = {i, j, k};
                    lo[d] -= 1;
                    double Fhi = rusanov_E(g, U, E, d, i, j, k);
                    double Flo = rusanov_E(g, U, E, d, lo[0], lo[1], lo[2]);
                    L[cell_index(g, i, j, k)] -= (Fhi - Flo) / g->dx[d];
                }
    }
}

/*
 * One Heun step (Shu-Osher form, the Butcher tableau of Sec. 2.2.2) of the
 * radiation energy advection with the velocity field of U held fixed:
 *   E1 = E + dt L_E(E),  E' = E/2 + (E1 + dt L_E(E1))/2.
 * Needs three cells along every active axis.  Updates E in place.
 */
int orc_advect_E_step(int nx, int ny, int nz, const double* dxyz, const int* bc6, double gamma,
                      const double* U, double* E, double dt) {
    grid_t g;
    if (make_grid_s(&g, 1, nx, ny, nz, dxyz, bc6, gamma)) return -1;
    size_t N = ncell(&g);
    double* L = (double*)malloc(sizeof(double) * N);
    double* E1 = (double*)malloc(sizeof(double) * N);
    rhs_E(&g, U, E, L);
    for (size_t q = 0; q < N; ++q) E1[q] = E[q] + dt * L[q];
    rhs_E(&g, U, E1, L);
    for (size_t q = 0; q < N; ++q) E[q] = 0.5 * E[q] + 0.5 * (E1[q] + dt * L[q]);
    free(L);
    free(E1);
    return 0;
}

/* Exposed for unit tests: the flux-difference operator L_E alone. */
int orc_rhs_E(int nx, int ny, int nz, const double* dxyz, const int* bc6, double gamma,
              const double* U, const double* E, double* L) {
    grid_t g;
    if (make_grid_s(&g, 1, nx, ny, nz, dxyz, bc6, gamma)) return -1;
    rhs_E(&g, U, E, L);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Radiative heating / cooling (the q-dot source, Sec. 2.2.1 and Sec. 3.2).   */
/* ------------------------------------------------------------------------ */

/*
 * The heating rate of Eq. "heating-cooling", qdot = c kappa rho (E - a T^4),
 * adds to the fluid energy and takes from the radiation energy density E
 * (the sources of Eq. "conservative form" with no radiation flux and no
 * fluid velocity coupling), so e + E is conserved pointwise.  The fluid
 * temperature is T = e / (rho c_v), c_v the specific heat per mass (for the
 * ideal gas c_v = k_B / ((gamma - 1) mu m_u)).
 *
 * One backward-Euler step of length dt:
 *   e' = e + dt k (E_tot - e' - a (e' / (rho c_v))^4),   k = c kappa rho,
 *   E' = E_tot - e',   E_tot = e + E,
 * solved for e' by Newton's method on
 *   f(x) = x - e - dt k (E_tot - x - a (x / (rho c_v))^4),
 * which is increasing and convex for x > 0, so Newton started right of the
 * root decreases monotonically onto it.  The start
 *   x0 = min(e + dt k max(E_tot - e - a T(e)^4, 0), E_tot, x_q),
 *   x_q = rho c_v ((e + dt k E_tot) / (dt k a))^(1/4),
 * has f(x0) >= 0: each of the three has (the root lies in (0, E_tot), since
 * E' = E_tot - e' >= 0, and f(x) >= (1 + dt k) x + dt k a T(x)^4 - e - dt k E_tot,
 * which is >= 0 at x_q).  x_q is the close start when the T^4 term dominates
 * (stiff cooling).  Iteration stops when the step is at most 1e-15 x (at most
 * 200 steps).  The fluid's kinetic energy is left as it is: the update
 * changes U[4] by e' - e and E by e - e'.
 * prm = {c, kappa, a, c_v}.  Returns the largest Newton step count.
 */
int orc_rad_exchange(int ncell, const double* prm, double dt, double* U, double* Er) {
    const double c = prm[0], kappa = prm[1], arad = prm[2], cv = prm[3];
    int worst = 0;
    size_t N = (size_t)ncell;
    for (size_t q = 0; q < N; ++q) {
        double rho = U[q];
        double m1 = U[N + q], m2 = U[2 * N + q], m3 = U[3 * N + q];
        double kin = 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) / rho;
        double e = U[4 * N + q] - kin;
        double Etot = e + Er[q];
        double k = c * kappa * rho;
        double rcv = rho * cv;
        double Te = e / rcv;
        double R0 = Etot - e - arad * (Te * Te) * (Te * Te);
        double x = e + dt * k * (R0 > 0.0 ? R0 : 0.0);
        if (x > Etot) x = Etot;                    /* the root lies below E_tot */
        double xq = rcv * sqrt(sqrt((e + dt * k * Etot) / (dt * k * arad)));
        if (xq < x) x = xq;
        int it = 0;
        for (; it < 200; ++it) {
            double T = x / rcv;
            double aT4 = arad * (T * T) * (T * T);
            double f = x - e - dt * k * (Etot - x - aT4);
            double df = 1.0 + dt * k * (1.0 + 4.0 * aT4 / x);
            double dx = f / df;
            x = x - dx;
            if (fabs(dx) <= 1e-15 * x) { ++it; break; }
        }
        if (it > worst) worst = it;
        U[4 * N + q] = x + kin;
        Er[q] = Er[q] + (e - x);
    }
    return worst;
}

/* ------------------------------------------------------------------------ */
/* Exact Riemann solver for the 1D ideal-gas Euler equations (Toro ch. 4).   */
/* ------------------------------------------------------------------------ */

/*
 * Pressure function of one side K and its derivative:
 *   shock (p > p_K):       f = (p - p_K) sqrt(A_K / (p + B_K)),
 *                          A_K = 2 / ((gamma+1) rho_K),  B_K = (gamma-1)/(gamma+1) p_K
 *   rarefaction (p <= p_K): f = 2 c_K/(gamma-1) [ (p/p_K)^((gamma-1)/(2 gamma)) - 1 ]
 */
static void pressure_fn(double p, double rK, double pK, double gamma, double* f, double* df) {
    double cK = sqrt(gamma * pK / rK);
    if (p > pK) {
        double A = 2.0 / ((gamma + 1.0) * rK);
        double B = (gamma - 1.0) / (gamma + 1.0) * pK;
        double q = sqrt(A / (p + B));
        *f = (p - pK) * q;
        *df = q * (1.0 - 0.5 * (p - pK) / (B + p));
    } else {
        double e = (gamma - 1.0) / (2.0 * gamma);
        *f = 2.0 * cK / (gamma - 1.0) * (pow(p / pK, e) - 1.0);
        *df = 1.0 / (rK * cK) * pow(p / pK, -(gamma + 1.0) / (2.0 * gamma));
    }
}

/*
 * Star-region pressure and velocity: root of f_L(p) + f_R(p) + (u_R - u_L) = 0
 * by Newton iteration from the two-rarefaction guess, then
 * u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2.  Returns 0, or -1 when the data
 * generate vacuum (2(c_L + c_R)/(gamma-1) <= u_R - u_L) or Newton fails.
 */
int orc_riemann_star(double rL, double uL, double pL, double rR, double uR, double pR,
                     double gamma, double* pstar, double* ustar) {
    double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
    if (2.0 * (cL + cR) / (gamma - 1.0) <= uR - uL) return -1;
    double z = (gamma - 1.0) / (2.0 * gamma);
    double p = pow((cL + cR - 0.5 * (gamma - 1.0) * (uR - uL))
                       / (cL / pow(pL, z) + cR / pow(pR, z)), 1.0 / z);
    if (!(p > 0.0)) p = 1e-8 * fmin(pL, pR);
    for (int it = 0; it < 200; ++it) {
        double fL, dL, fR, dR;
        pressure_fn(p, rL, pL, gamma, &fL, &dL);
        pressure_fn(p, rR, pR, gamma, &fR, &dR);
        double pn = p - (fL + fR + uR - uL) / (dL + dR);
        if (pn < 0.0) pn = 0.5 * p;
        double change = 2.0 * fabs(pn - p) / (pn + p);
        p = pn;
        if (change < 1e-15) {
            pressure_fn(p, rL, pL, gamma, &fL, &dL);
            pressure_fn(p, rR, pR, gamma, &fR, &dR);
            *pstar = p;
            *ustar = 0.5 * (uL + uR) + 0.5 * (fR - fL);
            return 0;
        }
    }
    return -1;
}

/*
 * Sample the self-similar solution at xi = (x - x0)/t.  Writes (rho, u, p).
 * Left/right shocks move at u_K -/+ c_K sqrt((gamma+1)/(2 gamma) p_star/p_K + (gamma-1)/(2 gamma));
 * rarefaction fans span [u_K -/+ c_K, u_star -/+ c_star_K] with the isentropic fan state.
 */
int orc_riemann_sample(double rL, double uL, double pL, double rR, double uR, double pR,
                       double gamma, double xi, double* W3) {
    double ps, us;
    if (orc_riemann_star(rL, uL, pL, rR, uR, pR, gamma, &ps, &us)) return -1;
    double g = gamma;
    double gm = (g - 1.0) / (g + 1.0);
    if (xi <= us) {                                    /* left of the contact */
        double cL = sqrt(g * pL / rL);
        if (ps > pL) {                                 /* left shock */
            double SL = uL - cL * sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g));
            if (xi <= SL) { W3[0] = rL; W3[1] = uL; W3[2] = pL; }
            else {
                W3[0] = rL * (ps / pL + gm) / (gm * ps / pL + 1.0);
                W3[1] = us; W3[2] = ps;
            }
        } else {                                       /* left rarefaction */
            double rs = rL * pow(ps / pL, 1.0 / g);
            double cs = cL * pow(ps / pL, (g - 1.0) / (2.0 * g));
            double head = uL - cL, tail = us - cs;
            if (xi <= head) { W3[0] = rL; W3[1] = uL; W3[2] = pL; }
            else if (xi >= tail) { W3[0] = rs; W3[1] = us; W3[2] = ps; }
            else {
                double c = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (uL - xi));
                W3[0] = rL * pow(c / cL, 2.0 / (g - 1.0));
                W3[1] = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + xi);
                W3[2] = pL * pow(c / cL, 2.0 * g / (g - 1.0));
            }
        }
    } else {                                           /* right of the contact */
        double cR = sqrt(g * pR / rR);
        if (ps > pR) {                                 /* right shock */
            double SR = uR + cR * sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g));
            if (xi >= SR) { W3[0] = rR; W3[1] = uR; W3[2] = pR; }
            else {
                W3[0] = rR * (ps / pR + gm) / (gm * ps / pR + 1.0);
                W3[1] = us; W3[2] = ps;
            }
        } else {                                       /* right rarefaction */
            double rs = rR * pow(ps / pR, 1.0 / g);
            double cs = cR * pow(ps / pR, (g - 1.0) / (2.0 * g));
            double head = uR + cR, tail = us + cs;
            if (xi >= head) { W3[0] = rR; W3[1] = uR; W3[2] = pR; }
            else if (xi <= tail) { W3[0] = rs; W3[1] = us; W3[2] = ps; }
            else {
                double c = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (uR - xi));
                W3[0] = rR * pow(c / cR, 2.0 / (g - 1.0));
                W3[1] = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + xi);
                W3[2] = pR * pow(c / cR, 2.0 * g / (g - 1.0));
            }
        }
    }
    return 0;
}

/* Outermost wave speeds of the exact solution (left-going minimum, right-going
 * maximum), used to keep a problem's waves inside the domain. */
int orc_riemann_extent(double rL, double uL, double pL, double rR, double uR, double pR,
                       double gamma, double* smin, double* smax) {
    double ps, us, g = gamma;
    if (orc_riemann_star(rL, uL, pL, rR, uR, pR, gamma, &ps, &us)) return -1;
    double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    *smin = (ps > pL) ? uL - cL * sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g))
                      : uL - cL;
    *smax = (ps > pR) ? uR + cR * sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g))
                      : uR + cR;
    return 0;
}
