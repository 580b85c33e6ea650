/*
 * hard_hydro.h -- C ABI of the GB300 (sm_103a) explicit finite-volume hydro
 * stage update.
 *
 * The library advances the ideal-gas Euler equations, the hydrodynamic rows of
 * the conservation law of the HARD paper (arXiv 2509.08971), Eq. "conservative
 * form" with S = 0 and the fluxes of Eq. "fluxes":
 *     d_t U + d_j F^j = 0,   U = [rho, rho v^i, e + rho v^2/2],  p = (gamma-1) e,
 * on a uniform Cartesian mesh of cell-centred values (Sec. 2.2.2).  One stage
 * is the fused chain
 *     ghost fill -> conserved-to-primitive -> minmod-limited piecewise-linear
 *     face states -> HLLC face flux -> flux difference (F*_{i+1/2}-F*_{i-1/2})/dx
 *     -> Runge-Kutta stage combine,
 * and a step is the two stages of Heun's method (Table "Butcher tableau for
 * Heun's method"), evaluated in Shu-Osher form:
 *     U1 = Un + dt L(Un),   U^{n+1} = Un/2 + (U1 + dt L(U1))/2.
 * The time step is dt = cfl / max_cells sum_d (|v_d| + c)/dx_d, c = sqrt(gamma p/rho).
 *
 * Conventions shared by every call
 *   Layout    U is a structure of arrays U[5][nz][ny][nx], x fastest, fields
 *             (rho, rho*u, rho*v, rho*w, E_total), contiguous, element type
 *             float (HARD_F32) or double (HARD_F64) as set on the handle.
 *             Ghost cells are not stored.  An axis with one cell is inactive.
 *   Memory    U pointers are DEVICE pointers owned by the caller (e.g. torch
 *             tensors), 16-byte aligned, unless the name says _host.  The
 *             handle owns its scratch (the intermediate stage U1, reduction
 *             slots, the status flag) and frees it in hard_hydro_destroy.
 *   Streams   `stream` is a cudaStream_t passed as void* (NULL = legacy
 *             default stream).  Calls are asynchronous on it unless stated.
 *   Errors    Every int-returning call returns HARD_OK (0) or a negative
 *             HARD_E* code and never aborts, exits or traps.  Argument errors
 *             are returned at once.  A non-physical state met on the device
 *             (rho <= 0, p <= 0 or NaN) raises a device flag that the next
 *             synchronising call (cfl_dt, totals, *_host) returns as
 *             HARD_ENONPHYS, or that hard_hydro_get_error reads and clears.
 *   Threads   A handle is not thread-safe; distinct handles are independent.
 */
#ifndef HARD_HYDRO_H
#define HARD_HYDRO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hard_hydro_s* hard_hydro_t;

/* boundary kinds (per face): periodic wrap, outflow (zero gradient: the two
 * ghost layers repeat the edge cell), reflecting wall (mirror image with the
 * normal momentum negated); HARD_BC_HALO (z faces only): the two ghost planes
 * are read from a caller buffer (hard_hydro_set_zghost), the planes of the
 * neighbouring slab of a mesh decomposed along z (the ghost entities of the
 * N-Array layout of Sec. 2.1) */
enum { HARD_BC_PERIODIC = 0, HARD_BC_OUTFLOW = 1, HARD_BC_REFLECT = 2, HARD_BC_HALO = 3 };

/* element type of U */
enum { HARD_F32 = 0, HARD_F64 = 1 };

/* stage kernel variant: TMA-staged fused z-march, or the same kernel fed by
 * plain per-thread loads */
enum { HARD_KERNEL_FUSED = 0, HARD_KERNEL_PLAIN = 1 };

/* face reconstruction and flux (Sec. 2.2.2): minmod-limited PLM states with
 * the HLLC flux (the default), or the paper's own WENO5-Z states (Borges et
 * al. 2008) with the HLL flux, three ghost layers */
enum { HARD_SCHEME_PLM_HLLC = 0, HARD_SCHEME_WENO5Z_HLL = 1 };

enum {
    HARD_OK = 0,
    HARD_EINVAL = -1,        /* bad argument                                  */
    HARD_ENOMEM = -2,        /* device allocation failed                      */
    HARD_ECUDA = -3,         /* a CUDA runtime call failed                    */
    HARD_ENONPHYS = -4,      /* non-physical state met on the device          */
    HARD_ETIMEOUT = -5,      /* a bounded device wait ran out                 */
    HARD_EUNSUPPORTED = -6   /* valid request the library does not support   */
};

/* Create a handle for an nx x ny x nz mesh (each >= 1) on the unit box with
 * ratio of specific heats gamma > 1 and the boundary kind `bc` on all six
 * faces.  Defaults: HARD_F32, HARD_KERNEL_FUSED.  Allocates nothing on the
 * device yet.  Returns NULL on a bad argument or host allocation failure. */
hard_hydro_t hard_hydro_create(int nx, int ny, int nz, double gamma, int bc);

/* Set the element type, the domain extents (cell width = extent / cells) and
 * the boundary kind of each face, ordered x-, x+, y-, y+, z-, z+ (NULL keeps
 * the current kinds).  Periodic must be set on both faces of an axis or on
 * neither.  HARD_BC_HALO is accepted on the z faces of a mesh with at least
 * two cells along every axis (HARD_EINVAL otherwise).  Frees scratch of a
 * previous element type. */
int hard_hydro_set(hard_hydro_t h, int dtype, double lx, double ly, double lz,
                   const int bc_per_face[6]);

/* Set the cell widths directly (each > 0; the extents become width x cells).
 * A slab of a mesh decomposed along z uses the whole mesh's widths, which
 * extent / cells of the slab need not reproduce bit for bit. */
int hard_hydro_set_cells(hard_hydro_t h, double dx, double dy, double dz);

/* Choose the stage kernel variant and tile configuration (tile < 0 picks the
 * built-in default).  Tile ids index a table that depends on the number of
 * active axes of the handle's mesh: hard_hydro_tile_count returns its size
 * (or a negative error code) and hard_hydro_tile_info writes
 * {tile_x, tile_y, z_chunk, threads_per_block} of one entry. */
int hard_hydro_set_kernel(hard_hydro_t h, int kernel, int tile);
int hard_hydro_tile_count(hard_hydro_t h);
int hard_hydro_tile_info(hard_hydro_t h, int tile, int out4[4]);

/* Choose the scheme of every later stage, step and advance call:
 * HARD_SCHEME_PLM_HLLC (default) or HARD_SCHEME_WENO5Z_HLL.  The WENO5-Z
 * scheme needs at least three cells along every active axis (else
 * HARD_EINVAL), ignores the kernel and tile choice of hard_hydro_set_kernel
 * (which apply to the default scheme only), and has no adjoint:
 * hard_hydro_step_backward returns HARD_EUNSUPPORTED for it.  On a 3D mesh
 * a stage runs as three directional sweeps that keep the flux difference in
 * a state-sized buffer the handle allocates with its other scratch (the
 * results equal the fused kernel's, which 1D and 2D meshes and
 * hard_hydro_step_noalloc use).  The CFL rate and the totals are the same
 * for both schemes. */
int hard_hydro_set_scheme(hard_hydro_t h, int scheme);

/* One Runge-Kutta stage (Sec. 2.2.2 flux difference, Heun tableau):
 *   stage 1: Uout = Ucur + dt L(Ucur)                       (U0 ignored)
 *   stage 2: Uout = U0/2 + (Ucur + dt L(Ucur))/2
 * Uout must not alias Ucur; it may alias U0.  HARD_BC_HALO faces read their
 * ghost planes from the buffers set by hard_hydro_set_zghost (HARD_EINVAL
 * when a halo face has none; HARD_EUNSUPPORTED with the WENO5-Z scheme). */
int hard_hydro_stage(hard_hydro_t h, int stage, const void* U0, const void* Ucur, void* Uout,
                     double dt, void* stream);

/* hard_hydro_stage with the step taken from device memory and, for stage 2,
 * the signal rate of the result (the CFL reduction of Sec. 3.1 / Sec. 3.5,
 * max over the handle's cells of sum_d (|v_d| + c)/dx_d):
 *   dt_dev    device double read as dt (NULL: the host value dt is used);
 *   rate_dev  device double that receives the largest signal rate of Uout,
 *             in double (NULL: none; stage 1 with rate_dev is HARD_EINVAL).
 * The rate of each slab of a decomposed mesh is reduced over the slabs by
 * the caller (a max) and turned into the common dt by hard_hydro_finalize_dt.
 * Asynchronous. */
int hard_hydro_stage_ex(hard_hydro_t h, int stage, const void* U0, const void* Ucur, void* Uout,
                        double dt, const double* dt_dev, double* rate_dev, void* stream);

/* ---- z-slab decomposition (ghost exchange between slabs, Sec. 2.1) ----
 * A mesh decomposed along z gives each slab its own handle, whose z faces
 * towards a neighbouring slab are HARD_BC_HALO and whose cell widths are the
 * whole mesh's (hard_hydro_set_cells).  Before each stage the caller packs
 * the two bottom and the two top planes of the stage's input (Ucur) of every
 * slab, sends them to the neighbours and receives theirs into the ghost
 * buffers:
 *   ghost_lo  the two planes below z = 0 (the neighbour's top planes, lowest
 *             first), ghost_hi the two planes above z = nz - 1 (the
 *             neighbour's bottom planes); each [5][2][ny][nx] of the handle's
 *             element type, 16-byte aligned device memory owned by the caller
 *             and read by every later stage; NULL where the face is not a
 *             halo face.
 * hard_hydro_pack_zhalo copies planes 0, 1 of U into send_lo and planes
 * nz-2, nz-1 into send_hi (each [5][2][ny][nx]; either may be NULL) with
 * device copies on `stream`, so the buffers can go straight to a
 * send/receive.  A step is then: exchange U^n, stage 1, exchange U1,
 * stage 2 with the rate, a max of the rates over the slabs, and
 * hard_hydro_finalize_dt.  hard_hydro_step, hard_hydro_advance(_host),
 * hard_hydro_step_backward, the radiation advection and diffusion and the
 * no-allocation step return HARD_EUNSUPPORTED on a handle with a halo face
 * (the ghosts change between the two stages of a step); the adjoint of a
 * slab runs through the split calls below. */
int hard_hydro_set_zghost(hard_hydro_t h, const void* ghost_lo, const void* ghost_hi);
int hard_hydro_pack_zhalo(hard_hydro_t h, const void* U, void* send_lo, void* send_hi,
                          void* stream);

/* ---- the adjoint of a slab (the ghost exchange reversed) ----
 * The paper has no counterpart (it computes no derivatives).  A stage's VJP
 * (see hard_hydro_step_backward; lambda = b dt G with b = 1 in stage 1 and
 * 1/2 in stage 2) is split around an exchange of cotangents:
 *   hard_hydro_stage_vjp_faces  every face of the slab (the faces on its
 *       z boundaries included, with the lambda of the neighbour's cells
 *       taken as zero: the neighbour evaluates the same face with this
 *       slab's lambda as zero, and the two halves sum to the face's VJP)
 *       runs its flux backwards onto the primitive cotangents of its four
 *       stencil cells: this slab's cells into the handle's accumulator, the
 *       ghost cells into the caller's accumulators set by
 *       hard_hydro_set_zghost_adjoint (gw_lo for the two planes below,
 *       gw_hi above; each [2][ny][nx] records of 8 elements of the
 *       handle's type, 16-byte aligned, zeroed by this call first).  Uc's
 *       ghost planes come from hard_hydro_set_zghost.  Adds the faces'
 *       d/dgamma to *g_gamma.
 *   the caller sends gw_lo to the slab below and gw_hi to the slab above;
 *   hard_hydro_add_zghost_cotangent adds what the slab below sent (its
 *       gw_hi: this slab's planes 0, 1) and what the slab above sent (its
 *       gw_lo: planes nz-2, nz-1) into the accumulator (either may be NULL);
 *   hard_hydro_stage_vjp_cells  per cell, the transpose of the
 *       conserved-to-primitive map of the accumulator (which it clears)
 *       plus the combine: gUc (=|+=, accumulate) b G + J^T, and in stage 2
 *       gU0 = G / 2 when gU0 is not NULL (stage 1: must be NULL); adds the
 *       pressure's d/dgamma to *g_gamma.
 * A backward step of a slab: exchange U^n, stage 1 (forward) to U1,
 * exchange U1; stage 2: faces(U1, G), exchange, cells(U1, G, gU1, 0, gU);
 * exchange U^n; stage 1: faces(U^n, gU1), exchange, cells(U^n, gU1, gU, 1,
 * NULL); the *g_gamma of the slabs summed by the caller.  HARD_EUNSUPPORTED
 * for the second scheme.  Asynchronous. */
int hard_hydro_set_zghost_adjoint(hard_hydro_t h, void* gw_lo, void* gw_hi);
int hard_hydro_stage_vjp_faces(hard_hydro_t h, int stage, const void* Uc, const void* G,
                               double dt, double* g_gamma, void* stream);
int hard_hydro_add_zghost_cotangent(hard_hydro_t h, const void* from_lo, const void* from_hi,
                                    void* stream);
int hard_hydro_stage_vjp_cells(hard_hydro_t h, int stage, const void* Uc, const void* G,
                               void* gUc, int accumulate, void* gU0, double* g_gamma,
                               void* stream);

/* Largest signal rate of U over the handle's cells into the device double
 * *rate_dev (the reduction of hard_hydro_cfl_dt without the division).
 * Asynchronous. */
int hard_hydro_local_rate(hard_hydro_t h, const void* U, double* rate_dev, void* stream);

/* dt = cfl / *rate_dev (device doubles), clipped so that t + dt <= t_end when
 * t_end > 0, then *t_dev += dt (t_dev may be NULL when t_end == 0); the rule
 * of hard_hydro_advance.  A zero, infinite or NaN rate gives dt = 0 and raises
 * the device flag (read by hard_hydro_get_error).  Asynchronous. */
int hard_hydro_finalize_dt(hard_hydro_t h, const double* rate_dev, double cfl, double t_end,
                           double* t_dev, double* dt_dev, void* stream);

/* One full step (both stages) with a fixed dt > 0.  U_out may alias U_in.
 * The intermediate stage lives in handle-owned scratch. */
int hard_hydro_step(hard_hydro_t h, const void* U_in, void* U_out, double dt, void* stream);

/* CFL time step of U (Sec. 3.1: the Courant number of each test, e.g. 0.3;
 * Sec. 3.5: a CFL-limited step; the multi-axis sum rule is this library's
 * reading): dt = cfl / max_cells sum_d (|v_d| + c)/dx_d.  Computed
 * in the element type, returned in double.  _host synchronises the stream and
 * writes *dt_host; _dev writes the double at device address dt_dev and does
 * not synchronise. */
int hard_hydro_cfl_dt(hard_hydro_t h, const void* U, double cfl, double* dt_host, void* stream);
int hard_hydro_cfl_dt_dev(hard_hydro_t h, const void* U, double cfl, double* dt_dev, void* stream);

/* Device-resident time loop, in place on U: nsteps steps, each with
 * dt = cfl / r(U^n) clipped so that t + dt <= t_end when t_end > 0 (steps
 * after t reaches t_end leave U unchanged).  The signal rate of U^{n+1} is
 * reduced in the epilogue of each step's second stage, so a step reads the
 * state once per stage.  t_dev is a device double (read as the start time,
 * advanced in place, FP64); it may be NULL when t_end == 0 (then t starts at
 * 0 in handle scratch).  dt_log_dev, if not NULL, is a device array of nsteps
 * doubles receiving each dt.  totals_log_dev, if not NULL, is a device array
 * of 5*nsteps doubles receiving the conserved totals of U^{n+1} after each
 * step, summed in FP64 in the second stage's epilogue.  Asynchronous. */
int hard_hydro_advance(hard_hydro_t h, void* U, int nsteps, double cfl, double t_end,
                       double* t_dev, double* dt_log_dev, double* totals_log_dev, void* stream);

/* The same loop from and to HOST memory: copies U_host_in to a handle-owned
 * device buffer, advances, copies the result to U_host_out (may alias) and
 * writes the final time to *t_host (read as the start time).  Synchronises
 * the stream.  Pinned host memory gives the full copy bandwidth. */
int hard_hydro_advance_host(hard_hydro_t h, const void* U_host_in, void* U_host_out, int nsteps,
                            double cfl, double t_end, double* t_host, void* stream);

/* Conserved totals sum_cells U_f dV for the 5 fields, summed in FP64 from the
 * warp level up in a fixed order (deterministic).  Synchronises the stream.
 * The paper has no counterpart: a diagnostic of the conservation that the
 * flux form of Sec. 2.2.2 guarantees, kept in FP64 beside an FP32 state. */
int hard_hydro_totals(hard_hydro_t h, const void* U, double out5[5], void* stream);

/* ---- batched persistent launch (many independent 1D/2D problems) ----
 * The paper has no counterpart (it runs one mesh per run): these calls serve
 * throughput on many small problems.
 * A batch is a set of independent problems of uneven size, each a uniform
 * mesh of nx x ny cells (nz must be 1; ny = 1 makes it 1D along x; nx >= 2)
 * on the unit square, with its own gamma and one boundary kind on all faces.
 * The packed state holds problem p's U[5][ny][nx] (same field order as
 * above) at element offset hard_batch_offset(b, p); hard_batch_elements is
 * the packed length.  One hard_hydro_step_batched call advances every problem
 * by nsteps Heun steps, each with its own CFL step dt_p = cfl / r_p(U_p), in a
 * single persistent launch: blocks take problems largest-first from an atomic
 * queue head (no block ever waits on another) and run all steps of a problem
 * with block-local reductions.  A problem advanced in a batch equals the same
 * problem advanced alone by hard_hydro_advance (t_end = 0), bit for bit.
 * The call allocates nothing and issues one memset and one kernel on
 * `stream`, so it can be captured in a CUDA graph.  t_dev: device array of
 * nprob doubles, read as each problem's start time and advanced in place.
 * hard_batch_create returns NULL on a bad argument or allocation failure; it
 * owns the problem table, the queue order and the packed intermediate stage.
 * Non-physical states raise the batch's status word (hard_batch_get_error). */
typedef struct hard_batch_s* hard_batch_t;
hard_batch_t hard_batch_create(int nprob, const int* nx, const int* ny, const int* nz,
                               const double* gamma, const int* bc, int dtype);
long long hard_batch_offset(hard_batch_t b, int p);
long long hard_batch_elements(hard_batch_t b);
int hard_batch_tile_count(void);
/* tile id: {1D tile width, 2D tile} = 0: {256, 32x8}, 1: {128, 32x4}, 2: {512, 64x8} */
int hard_batch_set_tile(hard_batch_t b, int tile);
int hard_hydro_step_batched(hard_batch_t b, void* U_packed, int nsteps, double cfl, double* t_dev,
                            void* stream);
/* HARD_OK or HARD_ENONPHYS (and clears it); synchronises the last stream. */
int hard_batch_get_error(hard_batch_t b);
void hard_batch_destroy(hard_batch_t b);

/* hard_hydro_step with no device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc when they
 * step (code running during CUDA-graph stream capture, hosts whose device
 * memory is pre-reserved by another allocator or runtime).  A handle with a
 * HARD_BC_HALO face returns HARD_EUNSUPPORTED.  It computes
 * exactly what hard_hydro_step computes with the handle's element type,
 * kernel and tile, but keeps the intermediate stage in a fixed 64 MiB
 * (HARD_NOALLOC_SCRATCH_BYTES) device array that the library holds on every
 * GPU that loads it until process exit, and touches no handle scratch.
 *   - Meshes whose state (5 * cells * element size) exceeds the array return
 *     HARD_EUNSUPPORTED (FP32: 3,355,443 cells; FP64: 1,677,721 cells).
 *   - The first call on a device, with that device current, looks up the
 *     array's device address; make that first call before any stream capture.
 *   - All calls share the array: calls that overlap on the GPU (other streams
 *     or host threads) race.  Its status word is cleared at the start of each
 *     call; hard_hydro_noalloc_get_error reads it.
 *   - U_out may alias U_in; U pointers are device pointers, 16-byte aligned. */
#define HARD_NOALLOC_SCRATCH_BYTES (64ull * 1024ull * 1024ull)
int hard_hydro_step_noalloc(hard_hydro_t h, const void* U_in, void* U_out, double dt,
                            void* stream);

/* Status word of the no-allocation step on the current device: HARD_OK,
 * HARD_ENONPHYS or HARD_ETIMEOUT (then cleared), or HARD_ECUDA.  It reflects
 * the calls that have finished on the device: synchronise their stream
 * first.  A handle's own flag (hard_hydro_get_error) does not see these
 * calls. */
int hard_hydro_noalloc_get_error(void);

/* Radiative heating / cooling (Eq. "heating-cooling"): one backward-Euler
 * step of length dt > 0 of the pointwise exchange
 *   de/dt = c kappa rho (E - a T^4),  dE/dt = -(same),  T = e / (rho c_v),
 * between the fluid's internal energy density e = E_total - rho |v|^2 / 2 and
 * the radiation energy density E (e + E is conserved; rho and the momenta are
 * not touched).  U is the handle's state [5][nz][ny][nx]; Er the radiation
 * energy density [nz][ny][nx]; both device buffers of the handle's element
 * type, 16-byte aligned, caller-owned, updated in place.  prm = {c, kappa, a,
 * c_v} (host array, all > 0, consistent units).  Each cell solves its implicit
 * update by Newton's method to 1e-15 (FP64) / 4e-7 (FP32) relative.  A cell
 * with rho <= 0, e <= 0 or E < 0 (or no convergence) is left unchanged and
 * raises the non-physical flag, read by hard_hydro_get_error.  Asynchronous
 * on `stream`; allocates nothing beyond the handle's status slot. */
int hard_hydro_rad_exchange(hard_hydro_t h, void* U, void* Er, double dt, const double prm[4],
                            void* stream);

/* Radiation energy advection (the d_j(E v^j) term of Eq. "radiation",
 * Sec. 2.2.2): one Heun step (the two stages of hard_hydro_step) of
 * dE/dt + div(E v) = 0 with the fluid velocity of U held fixed: WENO5-Z face
 * states of E and of the normal velocity, the Rusanov flux
 * (E_L u_L + E_R u_R)/2 - max(|u_L|, |u_R|)(E_R - E_L)/2, the handle's mesh
 * and boundary kinds (E mirrors without a sign change at a reflecting wall).
 * U: the handle's state (read); Er: the radiation energy density
 * [nz][ny][nx], updated in place.  Device buffers of the handle's element
 * type, 16-byte aligned, caller-owned; the intermediate stage (and, on a 3D
 * mesh, the flux difference passed between the directional sweeps) uses the
 * handle's scratch.  Every active axis needs at least three cells
 * (HARD_EINVAL otherwise).  The caller chooses dt (a CFL limit is
 * max |v_d| dt / dx_d <= 1 summed over the axes).  Asynchronous. */
int hard_hydro_advect_E(hard_hydro_t h, const void* U, void* Er, double dt, void* stream);

/* Flux-limited radiation diffusion (Sec. 2.2.1-2.2.2): one backward-Euler
 * step of dE/dt = div(D grad E), D = c lambda(R) / (kappa rho) with the
 * Levermore limiter lambda = (2 + R)/(6 + 3R + R^2), R = |grad E|/(rho kappa E),
 * D frozen at the old E, on the handle's mesh (face coefficient: the mean of
 * its two cells; periodic faces wrap, outflow and reflecting faces carry no
 * flux).  The linear system is solved by geometric-multigrid V-cycles
 * (red-black Gauss-Seidel, cell-centred coarsening of every even axis of
 * length >= 4) until the 2-norm of the residual is at most rtol times that of
 * the right-hand side, or max_cycles >= 1 cycles ran; rtol <= 0 runs exactly
 * max_cycles cycles without synchronising.  U: the handle's state (its
 * density field is read); Er: the radiation energy density [nz][ny][nx],
 * updated in place.  Both device buffers of the handle's element type,
 * 16-byte aligned, caller-owned.  c, kappa > 0 in consistent units.
 * *cycles_out and *resid_out (may be NULL) receive the cycles run and the last
 * relative residual (-1 when rtol <= 0).  The handle allocates its multigrid
 * levels on first use (freed by hard_hydro_set of another element type and by
 * hard_hydro_destroy).  With rtol > 0 the call synchronises `stream` once per
 * cycle.  A mesh with no active axis, with 2^31 cells or more, or with more
 * than 65535 cells along y or z returns HARD_EUNSUPPORTED. */
int hard_hydro_fld_step(hard_hydro_t h, const void* U, void* Er, double dt, double c,
                        double kappa, double rtol, int max_cycles, int* cycles_out,
                        double* resid_out, void* stream);

/* The paper has no counterpart (it computes no derivatives): the adjoint
 * serves gradient-based fitting of initial states and of gamma.
 * Adjoint of one full step with dt held constant (a vector-Jacobian product):
 * given the cotangent gU_out of U^{n+1} = step(U_in), writes
 * gU_in = (dU^{n+1}/dU_in)^T gU_out and adds (dU^{n+1}/dgamma)^T gU_out to the
 * device double *g_gamma.  The intermediate stage is recomputed from U_in.
 * Each face runs its flux backwards in the region the forward pass took;
 * minmod and the Davis min/max pass the cotangent to the argument they
 * selected (subgradients).  gU_in may alias gU_out.  Summation into the
 * cotangents uses device atomics, so results agree to rounding, not bitwise,
 * from run to run.  Device pointers, 16-byte aligned; asynchronous.  Faces
 * are indexed in 32 bits: a mesh with (number of active axes) x
 * prod_d (n_d + 1) >= 2^31 (about 7e8 cells in 3D) returns
 * HARD_EUNSUPPORTED. */
int hard_hydro_step_backward(hard_hydro_t h, const void* U_in, const void* gU_out, void* gU_in,
                             double dt, double* g_gamma, void* stream);

/* Device status flag: returns HARD_OK, HARD_ENONPHYS (a non-physical state
 * was met) or HARD_ETIMEOUT (a bounded wait of a TMA-fed stage ran out and
 * that stage left its output incomplete), and clears the flag.  Synchronises
 * the handle's last stream. */
int hard_hydro_get_error(hard_hydro_t h);

/* Static description of an error code. */
const char* hard_hydro_strerror(int code);

void hard_hydro_destroy(hard_hydro_t h);

#ifdef __cplusplus
}
#endif

#endif /* HARD_HYDRO_H */
