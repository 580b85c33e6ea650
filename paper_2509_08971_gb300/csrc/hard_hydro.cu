// C ABI of the hydro stage update: handles, argument checks, scratch
// ownership, the device-resident time loop and the small finalize kernels.
// The declarations and their contracts are in include/hard_hydro.h.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "hard_hydro.h"
#include "launch.h"
#include "fld_launch.h"
#include "rad_launch.h"
#include "weno_launch.h"

using hh::MeshDesc;
using hh::StageCall;

struct hard_hydro_s {
    int n[3];
    double gamma;
    int bc[6];
    double ext[3];
    double cell[3];                  // cell widths (ext / n unless set directly)
    const void* zg[2] = {nullptr, nullptr};  // ghost planes of BC_HALO z faces (caller-owned)
    void* zgw[2] = {nullptr, nullptr};       // their cotangent accumulators (caller-owned)
    int dtype = HARD_F32;
    int kernel = HARD_KERNEL_FUSED;
    int tile = -1;
    int scheme = HARD_SCHEME_PLM_HLLC;
    MeshDesc mesh;
    // device scratch, allocated on first use
    void* U1 = nullptr;              // intermediate stage
    size_t U1_bytes = 0;
    void* Udev = nullptr;            // state buffer of advance_host
    size_t Udev_bytes = 0;
    unsigned char* slots = nullptr;  // rate | dt | t | status | totals[5]
    double* tot_partial = nullptr;
    long long tot_rows = 0;
    void* wL = nullptr;              // flux difference between the WENO sweeps (3D meshes)
    size_t wL_bytes = 0;
    void* adj = nullptr;             // adjoint scratch: primitive cotangent | stage-1 cotangent
    size_t adj_bytes = 0;
    hh::FldHierarchy* fld = nullptr; // radiation diffusion multigrid levels, on first use
    cudaStream_t last = nullptr;
};

namespace {

constexpr size_t SLOT_RATE = 0, SLOT_DT = 8, SLOT_T = 16, SLOT_STATUS = 24, SLOT_TOT = 32;
constexpr size_t SLOT_BYTES = 128;

int from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return HARD_OK;
    if (e == cudaErrorMemoryAllocation) return HARD_ENOMEM;
    return HARD_ECUDA;
}

bool alloc_fail_injected() {
    const char* v = std::getenv("HARD_HYDRO_FAIL_ALLOC");
    return v && v[0] == '1';
}

int dev_alloc(void** p, size_t bytes) {
    if (alloc_fail_injected()) return HARD_ENOMEM;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return from_cuda(e);
    }
    return HARD_OK;
}

size_t elem_size(const hard_hydro_s* h) { return h->dtype == HARD_F64 ? 8 : 4; }
size_t state_bytes(const hard_hydro_s* h) { return 5 * (size_t)h->mesh.N * elem_size(h); }

bool valid_bc(int b) { return b == HARD_BC_PERIODIC || b == HARD_BC_OUTFLOW || b == HARD_BC_REFLECT; }

// Active axes become kernel axes in order; see launch.h.
void build_mesh(hard_hydro_s* h) {
    MeshDesc& m = h->mesh;
    int a = 0;
    for (int d = 0; d < 3; ++d) {
        m.dx[d] = h->cell[d];
        m.act[d] = h->n[d] > 1;
    }
    m.px = 0;
    m.py = 1;
    for (int k = 0; k < 3; ++k) {
        m.n[k] = 1;
        m.bc_lo[k] = m.bc_hi[k] = HARD_BC_PERIODIC;
        m.dxk[k] = 1.0;
    }
    for (int d = 0; d < 3; ++d) {
        if (!m.act[d]) continue;
        m.n[a] = h->n[d];
        m.bc_lo[a] = h->bc[2 * d];
        m.bc_hi[a] = h->bc[2 * d + 1];
        m.dxk[a] = m.dx[d];
        if (a == 0) m.px = d;
        if (a == 1) m.py = d;
        ++a;
    }
    m.dim = a;
    m.gamma = h->gamma;
    m.N = (long long)h->n[0] * h->n[1] * h->n[2];
}

void free_scratch(hard_hydro_s* h) {
    hh::fld_destroy(h->fld);
    h->fld = nullptr;
    if (h->adj) cudaFree(h->adj);
    h->adj = nullptr;
    h->adj_bytes = 0;
    if (h->U1) cudaFree(h->U1);
    if (h->wL) cudaFree(h->wL);
    h->wL = nullptr;
    h->wL_bytes = 0;
    if (h->Udev) cudaFree(h->Udev);
    if (h->tot_partial) cudaFree(h->tot_partial);
    h->U1 = h->Udev = nullptr;
    h->tot_partial = nullptr;
    h->U1_bytes = h->Udev_bytes = 0;
    h->tot_rows = 0;
}

int ensure_slots(hard_hydro_s* h) {
    if (h->slots) return HARD_OK;
    int rc = dev_alloc(reinterpret_cast<void**>(&h->slots), SLOT_BYTES);
    if (rc) return rc;
    return from_cuda(cudaMemset(h->slots, 0, SLOT_BYTES));
}

// The WENO scheme on a 3D mesh runs as directional sweeps that pass the
// flux difference through a state-sized buffer.
int ensure_weno_scratch(hard_hydro_s* h) {
    if (!(h->scheme == HARD_SCHEME_WENO5Z_HLL && h->mesh.dim == 3)) return HARD_OK;
    const size_t need = state_bytes(h);
    if (h->wL && h->wL_bytes >= need) return HARD_OK;
    if (h->wL) cudaFree(h->wL);
    h->wL = nullptr;
    h->wL_bytes = 0;
    int rc = dev_alloc(&h->wL, need);
    if (rc) return rc;
    h->wL_bytes = need;
    return HARD_OK;
}

int ensure_U1(hard_hydro_s* h) {
    int rc = ensure_slots(h);
    if (rc) return rc;
    rc = ensure_weno_scratch(h);
    if (rc) return rc;
    size_t need = state_bytes(h);
    if (h->U1 && h->U1_bytes >= need) return HARD_OK;
    if (h->U1) cudaFree(h->U1);
    h->U1 = nullptr;
    h->U1_bytes = 0;
    rc = dev_alloc(&h->U1, need);
    if (rc) return rc;
    h->U1_bytes = need;
    return HARD_OK;
}

// Adjoint scratch: the primitive cotangent accumulator (8 slots per cell,
// zero between calls: zeroed here once, cleared by each cell pass) and the
// cotangent of the intermediate stage.
int ensure_adj(hard_hydro_s* h) {
    const size_t gw_bytes = 8 * (size_t)h->mesh.N * elem_size(h);
    const size_t need = gw_bytes + state_bytes(h);
    if (h->adj && h->adj_bytes >= need) return HARD_OK;
    if (h->adj) cudaFree(h->adj);
    h->adj = nullptr;
    h->adj_bytes = 0;
    int rc = dev_alloc(&h->adj, need);
    if (rc) return rc;
    h->adj_bytes = need;
    return cudaMemset(h->adj, 0, gw_bytes) == cudaSuccess ? HARD_OK : HARD_ECUDA;
}

int ensure_partial(hard_hydro_s* h, long long rows) {
    if (h->tot_partial && h->tot_rows >= rows) return HARD_OK;
    if (h->tot_partial) cudaFree(h->tot_partial);
    h->tot_partial = nullptr;
    h->tot_rows = 0;
    int rc = dev_alloc(reinterpret_cast<void**>(&h->tot_partial), (size_t)rows * 5 * sizeof(double));
    if (rc) return rc;
    h->tot_rows = rows;
    return HARD_OK;
}

unsigned long long* rate_slot(hard_hydro_s* h) {
    return reinterpret_cast<unsigned long long*>(h->slots + SLOT_RATE);
}
double* dt_slot(hard_hydro_s* h) { return reinterpret_cast<double*>(h->slots + SLOT_DT); }
double* t_slot(hard_hydro_s* h) { return reinterpret_cast<double*>(h->slots + SLOT_T); }
int* status_slot(hard_hydro_s* h) { return reinterpret_cast<int*>(h->slots + SLOT_STATUS); }
double* tot_slot(hard_hydro_s* h) { return reinterpret_cast<double*>(h->slots + SLOT_TOT); }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int tile_of(const hard_hydro_s* h) { return h->tile < 0 ? 0 : h->tile; }

bool weno(const hard_hydro_s* h) { return h->scheme == HARD_SCHEME_WENO5Z_HLL && h->mesh.dim > 0; }

bool has_halo(const hard_hydro_s* h) {
    return h->bc[4] == HARD_BC_HALO || h->bc[5] == HARD_BC_HALO;
}

// Every BC_HALO face has a 16-byte aligned ghost buffer.
bool halo_ready(const hard_hydro_s* h) {
    for (int s = 0; s < 2; ++s)
        if (h->bc[4 + s] == HARD_BC_HALO && (!h->zg[s] || !aligned16(h->zg[s]))) return false;
    return true;
}

// blocks of one stage launch (rows of the totals partial array)
long long launch_blocks(const hard_hydro_s* h) {
    if (weno(h)) return hh::weno_stage_blocks(h->mesh, h->mesh.dim == 3);
    return hh::stage_blocks(h->mesh, tile_of(h));
}

cudaError_t stage_launch(hard_hydro_s* h, const StageCall& call, cudaStream_t s) {
    StageCall c = call;
    c.zg[0] = h->zg[0];
    c.zg[1] = h->zg[1];
    if (weno(h)) {
        c.scratch = h->wL;           // set by ensure_weno_scratch before any 3D launch
        if (h->mesh.dim == 3 && !c.scratch) return cudaErrorInvalidValue;
        return h->dtype == HARD_F64 ? hh::launch_weno_stage_f64(h->mesh, c, s)
                                    : hh::launch_weno_stage_f32(h->mesh, c, s);
    }
    if (h->dtype == HARD_F64) return hh::launch_stage_f64(h->mesh, h->kernel, tile_of(h), c, s);
    return hh::launch_stage_f32(h->mesh, h->kernel, tile_of(h), c, s);
}

// Both stages of one step, each over the whole mesh.
cudaError_t two_stages(hard_hydro_s* h, StageCall c1, StageCall c2, cudaStream_t s) {
    cudaError_t e = stage_launch(h, c1, s);
    return e == cudaSuccess ? stage_launch(h, c2, s) : e;
}

cudaError_t rate_launch(hard_hydro_s* h, const void* U, cudaStream_t s) {
    if (h->dtype == HARD_F64) return hh::launch_rate_f64(h->mesh, U, rate_slot(h), status_slot(h), s);
    return hh::launch_rate_f32(h->mesh, U, rate_slot(h), status_slot(h), s);
}

int read_status(hard_hydro_s* h, cudaStream_t s) {
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, status_slot(h), sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    if (st) {
        e = cudaMemsetAsync(status_slot(h), 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return from_cuda(e);
        return (st & 4) ? HARD_ETIMEOUT : HARD_ENONPHYS;   // bit 4: a bounded wait ran out
    }
    return HARD_OK;
}

// ---- finalize kernels ----

// dt of a step from the largest signal rate of the state it starts from.
__device__ void finalize_dt(unsigned long long* slot, double cfl, double t_end, double* t,
                            double* dt_out, double* dt_log, int step, int* status) {
    const double r = __longlong_as_double((long long)*slot);
    *slot = 0ull;                                  // ready for this step's stage-2 epilogue
    double dt;
    if (!(r > 0.0) || isinf(r)) {                  // NaN, zero or infinite rate
        dt = 0.0;
        atomicOr(status, 2);
    } else {
        dt = cfl / r;
        if (t && t_end > 0.0) {
            const double tc = *t;
            if (tc >= t_end) dt = 0.0;
            else if (tc + dt > t_end) dt = t_end - tc;
        }
    }
    if (t) *t = *t + dt;
    *dt_out = dt;
    if (dt_log) dt_log[step] = dt;
}

__global__ void finalize_dt_kernel(unsigned long long* slot, double cfl, double t_end, double* t,
                                   double* dt_out, double* dt_log, int step, int* status) {
    finalize_dt(slot, cfl, t_end, t, dt_out, dt_log, step, status);
}

// The largest signal rate left in the slot by a rate reduction, as a double;
// the slot is cleared for the next reduction.
__global__ void rate_out_kernel(unsigned long long* slot, double* rate_out) {
    *rate_out = __longlong_as_double((long long)*slot);
    *slot = 0ull;
}

// dt from a rate given as a double (e.g. reduced over the slabs of a
// decomposed mesh), with the rules of finalize_dt.
__global__ void finalize_dt_from_kernel(const double* rate, double cfl, double t_end, double* t,
                                        double* dt_out, int* status) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(*rate);
    finalize_dt(&bits, cfl, t_end, t, dt_out, nullptr, 0, status);
}

// Fixed-order sum of the per-block partials: warp f sums field f, lane l the
// rows l, l+32, ..., then a fixed xor tree.  Deterministic for a fixed grid.
__device__ void finalize_totals(const double* partial, long long rows, double dV, double* out5) {
    const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double s = 0.0;
    for (long long r = lane; r < rows; r += 32) s += partial[r * 5 + f];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out5[f] = s * dV;
}

__global__ void finalize_totals_kernel(const double* partial, long long rows, double dV,
                                       double* out5) {
    if ((threadIdx.x >> 5) < 5) finalize_totals(partial, rows, dV, out5);
}

// The end of one step of the time loop in one launch: warps 0-4 sum that
// step's totals, lane 0 of warp 5 sets the dt of the step after it (from the
// rate that the step's stage 2 left in the slot) when next_step >= 0.
__global__ void finalize_step_kernel(const double* partial, long long rows, double dV,
                                     double* out5, unsigned long long* slot, double cfl,
                                     double t_end, double* t, double* dt_out, double* dt_log,
                                     int next_step, int* status) {
    if ((threadIdx.x >> 5) < 5) finalize_totals(partial, rows, dV, out5);
    else if (threadIdx.x == 160 && next_step >= 0)
        finalize_dt(slot, cfl, t_end, t, dt_out, dt_log, next_step, status);
}

}  // namespace

namespace hh {

cudaError_t launch_finalize_dt(unsigned long long* rs, double cfl, double t_end, double* t_dev,
                               double* dt_dev, double* dt_log, int step, int* status,
                               cudaStream_t s) {
    finalize_dt_kernel<<<1, 1, 0, s>>>(rs, cfl, t_end, t_dev, dt_dev, dt_log, step, status);
    return cudaGetLastError();
}

cudaError_t launch_finalize_totals(const double* partial, long long rows, double dV, double* out5,
                                   cudaStream_t s) {
    finalize_totals_kernel<<<1, 160, 0, s>>>(partial, rows, dV, out5);
    return cudaGetLastError();
}

// Totals of step `next_step - 1` and, when next_step >= 0, the dt of next_step.
cudaError_t launch_finalize_step(const double* partial, long long rows, double dV, double* out5,
                                 unsigned long long* rs, double cfl, double t_end, double* t_dev,
                                 double* dt_dev, double* dt_log, int next_step, int* status,
                                 cudaStream_t s) {
    finalize_step_kernel<<<1, 192, 0, s>>>(partial, rows, dV, out5, rs, cfl, t_end, t_dev, dt_dev,
                                           dt_log, next_step, status);
    return cudaGetLastError();
}

}  // namespace hh

// ============================================================== C ABI ====

extern "C" {

hard_hydro_t hard_hydro_create(int nx, int ny, int nz, double gamma, int bc) {
    if (nx < 1 || ny < 1 || nz < 1) return nullptr;
    if (!(gamma > 1.0) || !std::isfinite(gamma)) return nullptr;
    if (!valid_bc(bc)) return nullptr;
    if ((long long)nx * ny * nz > (1ll << 40)) return nullptr;
    hard_hydro_s* h = new (std::nothrow) hard_hydro_s();
    if (!h) return nullptr;
    h->n[0] = nx; h->n[1] = ny; h->n[2] = nz;
    h->gamma = gamma;
    for (int f = 0; f < 6; ++f) h->bc[f] = bc;
    h->ext[0] = h->ext[1] = h->ext[2] = 1.0;
    for (int d = 0; d < 3; ++d) h->cell[d] = h->ext[d] / h->n[d];
    build_mesh(h);
    return h;
}

int hard_hydro_set(hard_hydro_t h, int dtype, double lx, double ly, double lz,
                   const int bc_per_face[6]) {
    if (!h) return HARD_EINVAL;
    if (dtype != HARD_F32 && dtype != HARD_F64) return HARD_EINVAL;
    const double e[3] = {lx, ly, lz};
    for (int d = 0; d < 3; ++d)
        if (!(e[d] > 0.0) || !std::isfinite(e[d])) return HARD_EINVAL;
    int bc[6];
    for (int f = 0; f < 6; ++f) bc[f] = bc_per_face ? bc_per_face[f] : h->bc[f];
    for (int f = 0; f < 6; ++f)
        if (!valid_bc(bc[f]) && !(f >= 4 && bc[f] == HARD_BC_HALO)) return HARD_EINVAL;
    for (int d = 0; d < 3; ++d)
        if ((bc[2 * d] == HARD_BC_PERIODIC) != (bc[2 * d + 1] == HARD_BC_PERIODIC))
            return HARD_EINVAL;
    // ghost planes from a neighbouring slab: 3D meshes only (z is kernel axis 3)
    if ((bc[4] == HARD_BC_HALO || bc[5] == HARD_BC_HALO) &&
        (h->n[0] < 2 || h->n[1] < 2 || h->n[2] < 2))
        return HARD_EINVAL;
    if (dtype != h->dtype) free_scratch(h);
    h->dtype = dtype;
    for (int d = 0; d < 3; ++d) h->ext[d] = e[d];
    for (int d = 0; d < 3; ++d) h->cell[d] = e[d] / h->n[d];
    for (int f = 0; f < 6; ++f) h->bc[f] = bc[f];
    build_mesh(h);
    return HARD_OK;
}

int hard_hydro_set_kernel(hard_hydro_t h, int kernel, int tile) {
    if (!h) return HARD_EINVAL;
    if (kernel != HARD_KERNEL_FUSED && kernel != HARD_KERNEL_PLAIN) return HARD_EINVAL;
    if (tile >= hh::tile_count(h->mesh.dim)) return HARD_EINVAL;
    h->kernel = kernel;
    h->tile = tile;
    return HARD_OK;
}

int hard_hydro_set_scheme(hard_hydro_t h, int scheme) {
    if (!h) return HARD_EINVAL;
    if (scheme != HARD_SCHEME_PLM_HLLC && scheme != HARD_SCHEME_WENO5Z_HLL) return HARD_EINVAL;
    if (scheme == HARD_SCHEME_WENO5Z_HLL && has_halo(h)) return HARD_EUNSUPPORTED;
    if (scheme == HARD_SCHEME_WENO5Z_HLL)
        for (int a = 0; a < 3; ++a)
            if (h->n[a] > 1 && h->n[a] < 3) return HARD_EINVAL;
    h->scheme = scheme;
    return HARD_OK;
}

int hard_hydro_tile_count(hard_hydro_t h) {
    if (!h) return HARD_EINVAL;
    return hh::tile_count(h->mesh.dim);
}

int hard_hydro_tile_info(hard_hydro_t h, int tile, int out4[4]) {
    if (!h || !out4 || tile < 0 || tile >= hh::tile_count(h->mesh.dim)) return HARD_EINVAL;
    hh::TileDesc t = hh::tile_desc(h->mesh.dim, tile);
    out4[0] = t.tx;
    out4[1] = t.ty;
    out4[2] = t.zc;
    out4[3] = t.tx * t.ty;
    return HARD_OK;
}

int hard_hydro_stage(hard_hydro_t h, int stage, const void* U0, const void* Ucur, void* Uout,
                     double dt, void* stream) {
    return hard_hydro_stage_ex(h, stage, U0, Ucur, Uout, dt, nullptr, nullptr, stream);
}

int hard_hydro_stage_ex(hard_hydro_t h, int stage, const void* U0, const void* Ucur, void* Uout,
                        double dt, const double* dt_dev, double* rate_dev, void* stream) {
    if (!h || (stage != 1 && stage != 2)) return HARD_EINVAL;
    if (rate_dev && stage != 2) return HARD_EINVAL;
    if (has_halo(h) && weno(h)) return HARD_EUNSUPPORTED;
    if (!halo_ready(h)) return HARD_EINVAL;
    if (!Ucur || !Uout || (stage == 2 && !U0)) return HARD_EINVAL;
    if (!aligned16(Ucur) || !aligned16(Uout) || (stage == 2 && !aligned16(U0))) return HARD_EINVAL;
    if (Uout == Ucur) return HARD_EINVAL;
    if (!dt_dev && (!(dt > 0.0) || !std::isfinite(dt))) return HARD_EINVAL;
    int rc = ensure_slots(h);
    if (rc) return rc;
    rc = ensure_weno_scratch(h);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    StageCall c{stage, U0, Ucur, Uout, dt, dt_dev, nullptr, nullptr, status_slot(h)};
    cudaError_t e = cudaSuccess;
    if (rate_dev) {
        c.rate_slot = rate_slot(h);
        e = cudaMemsetAsync(rate_slot(h), 0, sizeof(unsigned long long), s);
    }
    if (e == cudaSuccess) e = stage_launch(h, c, s);
    if (e == cudaSuccess && rate_dev) {
        rate_out_kernel<<<1, 1, 0, s>>>(rate_slot(h), rate_dev);
        e = cudaGetLastError();
    }
    return from_cuda(e);
}

int hard_hydro_step(hard_hydro_t h, const void* U_in, void* U_out, double dt, void* stream) {
    if (!h || !U_in || !U_out) return HARD_EINVAL;
    if (has_halo(h)) return HARD_EUNSUPPORTED;      // ghosts change between the stages
    if (!aligned16(U_in) || !aligned16(U_out)) return HARD_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt)) return HARD_EINVAL;
    int rc = ensure_U1(h);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    StageCall c1{1, U_in, U_in, h->U1, dt, nullptr, nullptr, nullptr, status_slot(h)};
    StageCall c2{2, U_in, h->U1, U_out, dt, nullptr, nullptr, nullptr, status_slot(h)};
    return from_cuda(two_stages(h, c1, c2, s));
}

static int cfl_common(hard_hydro_t h, const void* U, double cfl, cudaStream_t s) {
    if (!h || !U || !aligned16(U)) return HARD_EINVAL;
    if (!(cfl > 0.0) || !std::isfinite(cfl)) return HARD_EINVAL;
    int rc = ensure_slots(h);
    if (rc) return rc;
    h->last = s;
    cudaError_t e = cudaMemsetAsync(rate_slot(h), 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = rate_launch(h, U, s);
    if (e == cudaSuccess)
        e = hh::launch_finalize_dt(rate_slot(h), cfl, 0.0, nullptr, dt_slot(h), nullptr, 0,
                                   status_slot(h), s);
    return from_cuda(e);
}

int hard_hydro_cfl_dt(hard_hydro_t h, const void* U, double cfl, double* dt_host, void* stream) {
    if (!dt_host) return HARD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = cfl_common(h, U, cfl, s);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(dt_host, dt_slot(h), sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return from_cuda(e);
    return read_status(h, s);
}

int hard_hydro_cfl_dt_dev(hard_hydro_t h, const void* U, double cfl, double* dt_dev, void* stream) {
    if (!dt_dev) return HARD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = cfl_common(h, U, cfl, s);
    if (rc) return rc;
    return from_cuda(cudaMemcpyAsync(dt_dev, dt_slot(h), sizeof(double), cudaMemcpyDeviceToDevice, s));
}

int hard_hydro_advance(hard_hydro_t h, void* U, int nsteps, double cfl, double t_end,
                       double* t_dev, double* dt_log_dev, double* totals_log_dev, void* stream) {
    if (!h || !U || !aligned16(U) || nsteps < 0) return HARD_EINVAL;
    if (has_halo(h)) return HARD_EUNSUPPORTED;      // ghosts change between the stages
    if (!(cfl > 0.0) || !std::isfinite(cfl) || !(t_end >= 0.0) || !std::isfinite(t_end))
        return HARD_EINVAL;
    if (t_end > 0.0 && !t_dev) return HARD_EINVAL;
    int rc = ensure_U1(h);
    if (rc) return rc;
    const long long rows = launch_blocks(h);
    if (totals_log_dev) {
        rc = ensure_partial(h, rows);
        if (rc) return rc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    double* t = t_dev;
    cudaError_t e = cudaSuccess;
    if (!t) {
        t = t_slot(h);
        e = cudaMemsetAsync(t, 0, sizeof(double), s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(rate_slot(h), 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = rate_launch(h, U, s);
    const double dV = h->mesh.dx[0] * h->mesh.dx[1] * h->mesh.dx[2];
    // launches per step: stage 1, stage 2, then one finalize kernel that
    // closes the step (its totals) and sets the next step's dt
    if (e == cudaSuccess && nsteps > 0)
        e = hh::launch_finalize_dt(rate_slot(h), cfl, t_end, t, dt_slot(h), dt_log_dev, 0,
                                   status_slot(h), s);
    for (int step = 0; step < nsteps && e == cudaSuccess; ++step) {
        StageCall c1{1, U, U, h->U1, 0.0, dt_slot(h), nullptr, nullptr, status_slot(h)};
        double* part = (totals_log_dev && h->mesh.dim > 0) ? h->tot_partial : nullptr;
        StageCall c2{2, U, h->U1, U, 0.0, dt_slot(h), rate_slot(h), part, status_slot(h)};
        e = two_stages(h, c1, c2, s);
        if (e != cudaSuccess) break;
        const int next = step + 1 < nsteps ? step + 1 : -1;
        if (!totals_log_dev) {
            if (next >= 0)
                e = hh::launch_finalize_dt(rate_slot(h), cfl, t_end, t, dt_slot(h), dt_log_dev,
                                           next, status_slot(h), s);
            continue;
        }
        long long prow = rows;
        if (!part) {
            // no active axis: the stage kernel has no totals epilogue
            rc = ensure_partial(h, hh::totals_blocks());
            if (rc) return rc;
            e = h->dtype == HARD_F64 ? hh::launch_totals_f64(h->mesh, U, h->tot_partial, s)
                                     : hh::launch_totals_f32(h->mesh, U, h->tot_partial, s);
            prow = hh::totals_blocks();
        }
        if (e == cudaSuccess)
            e = hh::launch_finalize_step(h->tot_partial, prow, dV, totals_log_dev + 5 * step,
                                         rate_slot(h), cfl, t_end, t, dt_slot(h), dt_log_dev,
                                         next, status_slot(h), s);
    }
    return from_cuda(e);
}

int hard_hydro_advance_host(hard_hydro_t h, const void* U_host_in, void* U_host_out, int nsteps,
                            double cfl, double t_end, double* t_host, void* stream) {
    if (!h || !U_host_in || !U_host_out || !t_host) return HARD_EINVAL;
    if (has_halo(h)) return HARD_EUNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = ensure_slots(h);
    if (rc) return rc;
    const size_t bytes = state_bytes(h);
    if (!h->Udev || h->Udev_bytes < bytes) {
        if (h->Udev) cudaFree(h->Udev);
        h->Udev = nullptr;
        h->Udev_bytes = 0;
        rc = dev_alloc(&h->Udev, bytes);
        if (rc) return rc;
        h->Udev_bytes = bytes;
    }
    cudaError_t e = cudaMemcpyAsync(h->Udev, U_host_in, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(t_slot(h), t_host, sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return from_cuda(e);
    rc = hard_hydro_advance(h, h->Udev, nsteps, cfl, t_end, t_slot(h), nullptr, nullptr, stream);
    if (rc) return rc;
    e = cudaMemcpyAsync(U_host_out, h->Udev, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(t_host, t_slot(h), sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return from_cuda(e);
    return read_status(h, s);
}

int hard_hydro_totals(hard_hydro_t h, const void* U, double out5[5], void* stream) {
    if (!h || !U || !out5 || !aligned16(U)) return HARD_EINVAL;
    int rc = ensure_slots(h);
    if (rc) return rc;
    rc = ensure_partial(h, hh::totals_blocks());
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    const double dV = h->mesh.dx[0] * h->mesh.dx[1] * h->mesh.dx[2];
    cudaError_t e = h->dtype == HARD_F64 ? hh::launch_totals_f64(h->mesh, U, h->tot_partial, s)
                                         : hh::launch_totals_f32(h->mesh, U, h->tot_partial, s);
    if (e == cudaSuccess)
        e = hh::launch_finalize_totals(h->tot_partial, hh::totals_blocks(), dV, tot_slot(h), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out5, tot_slot(h), 5 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return from_cuda(e);
    return read_status(h, s);
}

int hard_hydro_rad_exchange(hard_hydro_t h, void* U, void* Er, double dt, const double prm[4],
                            void* stream) {
    if (!h || !U || !Er || !prm || !aligned16(U) || !aligned16(Er)) return HARD_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt)) return HARD_EINVAL;
    for (int i = 0; i < 4; ++i)
        if (!(prm[i] > 0.0) || !std::isfinite(prm[i])) return HARD_EINVAL;
    int rc = ensure_slots(h);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    return from_cuda(hh::launch_rad_exchange(h->mesh, h->dtype, U, Er, dt, prm, status_slot(h), s));
}

int hard_hydro_advect_E(hard_hydro_t h, const void* U, void* Er, double dt, void* stream) {
    if (!h || !U || !Er || !aligned16(U) || !aligned16(Er)) return HARD_EINVAL;
    if (has_halo(h)) return HARD_EUNSUPPORTED;
    if (!(dt > 0.0) || !std::isfinite(dt)) return HARD_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (h->n[a] > 1 && h->n[a] < 3) return HARD_EINVAL;
    if (h->mesh.dim == 0) return HARD_OK;                     // nothing moves
    int rc = ensure_U1(h);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    const bool f64 = h->dtype == HARD_F64;
    auto stage = f64 ? hh::launch_advect_E_stage_f64 : hh::launch_advect_E_stage_f32;
    // U1 holds E1 in its first field and, on 3D meshes, the sweeps' flux
    // difference in its second
    void* L = h->mesh.dim == 3 ? static_cast<char*>(h->U1) + h->mesh.N * elem_size(h) : nullptr;
    cudaError_t e = stage(h->mesh, 1, U, nullptr, Er, h->U1, dt, L, s);
    if (e == cudaSuccess) e = stage(h->mesh, 2, U, Er, h->U1, Er, dt, L, s);
    return from_cuda(e);
}

int hard_hydro_fld_step(hard_hydro_t h, const void* U, void* Er, double dt, double c,
                        double kappa, double rtol, int max_cycles, int* cycles_out,
                        double* resid_out, void* stream) {
    if (!h || !U || !Er || !aligned16(U) || !aligned16(Er)) return HARD_EINVAL;
    if (has_halo(h)) return HARD_EUNSUPPORTED;
    if (!(dt > 0.0) || !std::isfinite(dt) || !(c > 0.0) || !std::isfinite(c) ||
        !(kappa > 0.0) || !std::isfinite(kappa) || max_cycles < 1 || !std::isfinite(rtol))
        return HARD_EINVAL;
    if (h->mesh.dim == 0) return HARD_EUNSUPPORTED;          // nothing to diffuse along
    if (h->mesh.N >= (1ll << 31)) return HARD_EUNSUPPORTED;  // 32-bit cell indices
    // the level kernels take a row per blockIdx.y and a plane per blockIdx.z
    if (h->mesh.n[1] > 65535 || h->mesh.n[2] > 65535) return HARD_EUNSUPPORTED;
    if (!hh::fld_matches(h->fld, h->mesh, h->dtype)) {
        hh::fld_destroy(h->fld);
        h->fld = hh::fld_create(h->mesh, h->dtype);
        if (!h->fld) return HARD_ENOMEM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    int cyc = 0;
    double rel = -1.0;
    const cudaError_t e = hh::fld_solve(h->fld, h->mesh, U, Er, dt, c, kappa, rtol, max_cycles,
                                        &cyc, &rel, s);
    if (cycles_out) *cycles_out = cyc;
    if (resid_out) *resid_out = rel;
    return from_cuda(e);
}

int hard_hydro_step_backward(hard_hydro_t h, const void* U_in, const void* gU_out, void* gU_in,
                             double dt, double* g_gamma, void* stream) {
    if (!h || !U_in || !gU_out || !gU_in || !g_gamma) return HARD_EINVAL;
    if (has_halo(h)) return HARD_EUNSUPPORTED;
    if (!aligned16(U_in) || !aligned16(gU_out) || !aligned16(gU_in)) return HARD_EINVAL;
    if (weno(h)) return HARD_EUNSUPPORTED;
    if (!(dt > 0.0) || !std::isfinite(dt)) return HARD_EINVAL;
    {
        // the face VJP kernel indexes faces in 32 bits
        long long faces = h->mesh.dim;
        for (int k = 0; k < 3; ++k) faces *= (long long)h->mesh.n[k] + (k < h->mesh.dim ? 1 : 0);
        if (faces >= (1ll << 31)) return HARD_EUNSUPPORTED;
    }
    int rc = ensure_U1(h);
    if (rc) return rc;
    // adjoint scratch: the primitive cotangent accumulator (8 slots per cell,
    // zero between calls: zeroed here once, cleared by each cell pass) and
    // the cotangent of the intermediate stage
    rc = ensure_adj(h);
    if (rc) return rc;
    const size_t gw_bytes = 8 * (size_t)h->mesh.N * elem_size(h);
    void* gW = h->adj;
    void* gU1 = static_cast<unsigned char*>(h->adj) + gw_bytes;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    // recompute the intermediate stage U1 = Un + dt L(Un)
    const StageCall c1{1, U_in, U_in, h->U1, dt, nullptr, nullptr, nullptr, status_slot(h)};
    cudaError_t e = stage_launch(h, c1, s);
    if (e != cudaSuccess) return from_cuda(e);
    // stage 2: U^{n+1} = Un/2 + (U1 + dt L(U1))/2
    const hh::AdjointCall a2{h->U1, gU_out, gW, gU1, false, gU_in, 0.5, 0.5, 0.5 * dt, g_gamma,
                             true};
    e = h->dtype == HARD_F64 ? hh::launch_adjoint_stage_f64(h->mesh, a2, s)
                             : hh::launch_adjoint_stage_f32(h->mesh, a2, s);
    if (e != cudaSuccess) return from_cuda(e);
    // stage 1: U1 = Un + dt L(Un)
    const hh::AdjointCall a1{U_in, gU1, gW, gU_in, true, nullptr, 1.0, 0.0, dt, g_gamma, true};
    e = h->dtype == HARD_F64 ? hh::launch_adjoint_stage_f64(h->mesh, a1, s)
                             : hh::launch_adjoint_stage_f32(h->mesh, a1, s);
    return from_cuda(e);
}

int hard_hydro_set_cells(hard_hydro_t h, double dx, double dy, double dz) {
    if (!h) return HARD_EINVAL;
    const double d[3] = {dx, dy, dz};
    for (int k = 0; k < 3; ++k)
        if (!(d[k] > 0.0) || !std::isfinite(d[k])) return HARD_EINVAL;
    for (int k = 0; k < 3; ++k) {
        h->cell[k] = d[k];
        h->ext[k] = d[k] * h->n[k];
    }
    build_mesh(h);
    return HARD_OK;
}

int hard_hydro_set_zghost(hard_hydro_t h, const void* ghost_lo, const void* ghost_hi) {
    if (!h) return HARD_EINVAL;
    if ((ghost_lo && !aligned16(ghost_lo)) || (ghost_hi && !aligned16(ghost_hi))) return HARD_EINVAL;
    h->zg[0] = ghost_lo;
    h->zg[1] = ghost_hi;
    return HARD_OK;
}

int hard_hydro_set_zghost_adjoint(hard_hydro_t h, void* gw_lo, void* gw_hi) {
    if (!h) return HARD_EINVAL;
    if ((gw_lo && !aligned16(gw_lo)) || (gw_hi && !aligned16(gw_hi))) return HARD_EINVAL;
    h->zgw[0] = gw_lo;
    h->zgw[1] = gw_hi;
    return HARD_OK;
}

namespace {

// Argument checks shared by the two halves of a stage's decomposed VJP (no
// device work).
int vjp_args(hard_hydro_t h, int stage, const void* Uc, const void* G) {
    if (!h || (stage != 1 && stage != 2) || !Uc || !G) return HARD_EINVAL;
    if (!aligned16(Uc) || !aligned16(G)) return HARD_EINVAL;
    if (weno(h)) return HARD_EUNSUPPORTED;
    long long faces = h->mesh.dim;        // the face VJP kernel indexes faces in 32 bits
    for (int k = 0; k < 3; ++k) faces *= (long long)h->mesh.n[k] + (k < h->mesh.dim ? 1 : 0);
    return faces >= (1ll << 31) ? HARD_EUNSUPPORTED : HARD_OK;
}

int vjp_scratch(hard_hydro_t h) {
    int rc = ensure_slots(h);
    return rc ? rc : ensure_adj(h);
}

}  // namespace

int hard_hydro_stage_vjp_faces(hard_hydro_t h, int stage, const void* Uc, const void* G,
                               double dt, double* g_gamma, void* stream) {
    int rc = vjp_args(h, stage, Uc, G);
    if (rc) return rc;
    if (!g_gamma || !(dt > 0.0) || !std::isfinite(dt)) return HARD_EINVAL;
    if (!halo_ready(h)) return HARD_EINVAL;
    for (int side = 0; side < 2; ++side)
        if (h->bc[4 + side] == HARD_BC_HALO && !h->zgw[side]) return HARD_EINVAL;
    if ((rc = vjp_scratch(h)) != HARD_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    const size_t acc = 2 * (size_t)h->n[0] * h->n[1] * 8 * elem_size(h);
    cudaError_t e = cudaSuccess;
    for (int side = 0; side < 2 && e == cudaSuccess; ++side)
        if (h->bc[4 + side] == HARD_BC_HALO) e = cudaMemsetAsync(h->zgw[side], 0, acc, s);
    if (e != cudaSuccess) return from_cuda(e);
    const double b = stage == 1 ? 1.0 : 0.5;
    hh::AdjointCall a{Uc, G, h->adj, nullptr, false, nullptr, b, 0.0, b * dt, g_gamma, false};
    a.passes = 1;
    for (int side = 0; side < 2; ++side) {
        a.zg[side] = h->zg[side];
        a.gwg[side] = h->zgw[side];
    }
    e = h->dtype == HARD_F64 ? hh::launch_adjoint_stage_f64(h->mesh, a, s)
                             : hh::launch_adjoint_stage_f32(h->mesh, a, s);
    return from_cuda(e);
}

int hard_hydro_add_zghost_cotangent(hard_hydro_t h, const void* from_lo, const void* from_hi,
                                    void* stream) {
    if (!h) return HARD_EINVAL;
    if ((from_lo && !aligned16(from_lo)) || (from_hi && !aligned16(from_hi))) return HARD_EINVAL;
    if (h->mesh.dim != 3 || h->n[2] < 2) return HARD_EINVAL;
    int rc = vjp_scratch(h);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    auto add = h->dtype == HARD_F64 ? hh::launch_add_ghost_cotangent_f64
                                    : hh::launch_add_ghost_cotangent_f32;
    cudaError_t e = cudaSuccess;
    if (from_lo) e = add(h->mesh, h->adj, from_lo, 0, s);
    if (e == cudaSuccess && from_hi) e = add(h->mesh, h->adj, from_hi, h->n[2] - 2, s);
    return from_cuda(e);
}

int hard_hydro_stage_vjp_cells(hard_hydro_t h, int stage, const void* Uc, const void* G,
                               void* gUc, int accumulate, void* gU0, double* g_gamma,
                               void* stream) {
    int rc = vjp_args(h, stage, Uc, G);
    if (rc) return rc;
    if (!gUc || !aligned16(gUc) || !g_gamma || (gU0 && !aligned16(gU0))) return HARD_EINVAL;
    if (stage == 1 && gU0) return HARD_EINVAL;       // stage 1 does not depend on U^n separately
    if ((rc = vjp_scratch(h)) != HARD_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    const double b = stage == 1 ? 1.0 : 0.5, a0 = stage == 1 ? 0.0 : 0.5;
    hh::AdjointCall a{Uc, G, h->adj, gUc, accumulate != 0, gU0, b, a0, 0.0, g_gamma, true};
    a.passes = 2;
    const cudaError_t e = h->dtype == HARD_F64 ? hh::launch_adjoint_stage_f64(h->mesh, a, s)
                                               : hh::launch_adjoint_stage_f32(h->mesh, a, s);
    return from_cuda(e);
}

int hard_hydro_pack_zhalo(hard_hydro_t h, const void* U, void* send_lo, void* send_hi,
                          void* stream) {
    if (!h || !U || !aligned16(U)) return HARD_EINVAL;
    if ((send_lo && !aligned16(send_lo)) || (send_hi && !aligned16(send_hi))) return HARD_EINVAL;
    if (h->n[2] < 2) return HARD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t es = elem_size(h);
    const size_t plane = (size_t)h->n[0] * h->n[1] * es;       // bytes of one z plane of a field
    const size_t field = plane * h->n[2];
    const unsigned char* u = static_cast<const unsigned char*>(U);
    cudaError_t e = cudaSuccess;
    // five rows (one per field) of two planes each, into [5][2][ny][nx]
    if (send_lo)
        e = cudaMemcpy2DAsync(send_lo, 2 * plane, u, field, 2 * plane, 5, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && send_hi)
        e = cudaMemcpy2DAsync(send_hi, 2 * plane, u + (h->n[2] - 2) * plane, field, 2 * plane, 5,
                              cudaMemcpyDeviceToDevice, s);
    return from_cuda(e);
}

int hard_hydro_local_rate(hard_hydro_t h, const void* U, double* rate_dev, void* stream) {
    if (!h || !U || !aligned16(U) || !rate_dev) return HARD_EINVAL;
    int rc = ensure_slots(h);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    cudaError_t e = cudaMemsetAsync(rate_slot(h), 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = rate_launch(h, U, s);
    if (e == cudaSuccess) {
        rate_out_kernel<<<1, 1, 0, s>>>(rate_slot(h), rate_dev);
        e = cudaGetLastError();
    }
    return from_cuda(e);
}

int hard_hydro_finalize_dt(hard_hydro_t h, const double* rate_dev, double cfl, double t_end,
                           double* t_dev, double* dt_dev, void* stream) {
    if (!h || !rate_dev || !dt_dev) return HARD_EINVAL;
    if (!(cfl > 0.0) || !std::isfinite(cfl) || !(t_end >= 0.0) || !std::isfinite(t_end))
        return HARD_EINVAL;
    if (t_end > 0.0 && !t_dev) return HARD_EINVAL;
    int rc = ensure_slots(h);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last = s;
    finalize_dt_from_kernel<<<1, 1, 0, s>>>(rate_dev, cfl, t_end, t_dev, dt_dev, status_slot(h));
    return from_cuda(cudaGetLastError());
}

int hard_hydro_get_error(hard_hydro_t h) {
    if (!h) return HARD_EINVAL;
    if (!h->slots) return HARD_OK;
    return read_status(h, h->last);
}

const char* hard_hydro_strerror(int code) {
    switch (code) {
        case HARD_OK: return "ok";
        case HARD_EINVAL: return "invalid argument";
        case HARD_ENOMEM: return "device allocation failed";
        case HARD_ECUDA: return "CUDA runtime error";
        case HARD_ENONPHYS: return "non-physical state (rho <= 0, p <= 0 or NaN) on the device";
        case HARD_ETIMEOUT: return "bounded device wait timed out";
        case HARD_EUNSUPPORTED: return "unsupported request";
        default: return "unknown error code";
    }
}

void hard_hydro_destroy(hard_hydro_t h) {
    if (!h) return;
    free_scratch(h);
    if (h->slots) cudaFree(h->slots);
    delete h;
}

}  // extern "C"

namespace hh {

// Read-only view of a handle for the library's other translation units.
int handle_scheme(const hard_hydro_s* h) { return h->scheme; }

bool handle_view(hard_hydro_t h, const MeshDesc** mesh, int* dtype, int* kernel, int* tile) {
    if (!h) return false;
    *mesh = &h->mesh;
    *dtype = h->dtype;
    *kernel = h->kernel;
    *tile = tile_of(h);
    return true;
}

}  // namespace hh
