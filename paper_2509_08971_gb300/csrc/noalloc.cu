// hard_hydro_step_noalloc: one full step that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they step the mesh:
// code running while a stream is being captured into a CUDA graph, a host
// that has handed the whole device pool to another allocator and must not
// grow its own footprint, or an embedding runtime whose memory is reserved up
// front.  For them the intermediate Runge-Kutta stage lives in a fixed
// file-scope device array instead of handle-owned scratch.  The array is part
// of the module, so every GPU that loads this library holds its 64 MiB until
// the process exits.
//
// In host code `g_scratch` names a host-side stand-in, not a device address:
// a kernel handed that name would fault or, where the GPU can reach host
// memory, silently use the wrong memory.  So the first call on each device
// (with that device current) asks the runtime for the array's device address
// with cudaGetSymbolAddress, checks the result, caches it per device and
// passes it to the kernels.  That set-up call should come before any stream
// capture begins.
//
// Every call shares the one array, which keeps the last call's contents.  The
// first stage overwrites every scratch cell before the second stage reads it,
// so only the status word is cleared per call; hard_hydro_noalloc_get_error
// reads it (after the device has finished the call).  Calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// the array.
#include <cmath>
#include <mutex>

#include "hard_hydro.h"
#include "launch.h"
#include "weno_launch.h"

namespace {

constexpr size_t SCRATCH_BYTES = (size_t)HARD_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];
static __device__ __align__(256) int g_status;

constexpr int MAX_DEVICES = 64;
struct DeviceScratch {
    void* scratch = nullptr;
    int* status = nullptr;
    bool ready = false;
};
std::mutex g_mutex;
DeviceScratch g_devices[MAX_DEVICES];

// Device addresses of the static arrays on the current device (set up once).
int scratch_for_current_device(DeviceScratch* out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return HARD_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceScratch& d = g_devices[dev];
    if (!d.ready) {
        void* scratch = nullptr;
        void* status = nullptr;
        e = cudaGetSymbolAddress(&scratch, g_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&status, g_status);
        if (e != cudaSuccess || !scratch || !status) {
            cudaGetLastError();
            return HARD_ECUDA;
        }
        d.scratch = scratch;
        d.status = static_cast<int*>(status);
        d.ready = true;
    }
    *out = d;
    return HARD_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int hard_hydro_step_noalloc(hard_hydro_t h, const void* U_in, void* U_out, double dt,
                                       void* stream) {
    const hh::MeshDesc* mesh = nullptr;
    int dtype = 0, kernel = 0, tile = 0;
    if (!hh::handle_view(h, &mesh, &dtype, &kernel, &tile)) return HARD_EINVAL;
    if (!U_in || !U_out || !aligned16(U_in) || !aligned16(U_out)) return HARD_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt)) return HARD_EINVAL;
    // ghost planes of a decomposed mesh change between the stages
    if (mesh->dim == 3 && (mesh->bc_lo[2] == HARD_BC_HALO || mesh->bc_hi[2] == HARD_BC_HALO))
        return HARD_EUNSUPPORTED;
    const size_t need = 5 * (size_t)mesh->N * (dtype == HARD_F64 ? 8 : 4);
    if (need > SCRATCH_BYTES) return HARD_EUNSUPPORTED;       // mesh too large for the array
    DeviceScratch d;
    int rc = scratch_for_current_device(&d);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(d.status, 0, sizeof(int), s);
    if (e != cudaSuccess) return HARD_ECUDA;
    const bool weno = hh::handle_scheme(h) == HARD_SCHEME_WENO5Z_HLL && mesh->dim > 0;
    auto launch = [&](const hh::StageCall& c) {
        if (weno)
            return dtype == HARD_F64 ? hh::launch_weno_stage_f64(*mesh, c, s)
                                     : hh::launch_weno_stage_f32(*mesh, c, s);
        return dtype == HARD_F64 ? hh::launch_stage_f64(*mesh, kernel, tile, c, s)
                                 : hh::launch_stage_f32(*mesh, kernel, tile, c, s);
    };
    const hh::StageCall c1{1, U_in, U_in, d.scratch, dt, nullptr, nullptr, nullptr, d.status};
    e = launch(c1);
    if (e != cudaSuccess) return HARD_ECUDA;
    const hh::StageCall c2{2, U_in, d.scratch, U_out, dt, nullptr, nullptr, nullptr, d.status};
    e = launch(c2);
    return e == cudaSuccess ? HARD_OK : HARD_ECUDA;
}

extern "C" int hard_hydro_noalloc_get_error(void) {
    DeviceScratch d;
    int rc = scratch_for_current_device(&d);
    if (rc) return rc;
    int st = 0;
    // the status word of the last hard_hydro_step_noalloc call on this device
    cudaError_t e = cudaMemcpy(&st, d.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return HARD_ECUDA;
    }
    if (!st) return HARD_OK;
    e = cudaMemset(d.status, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return HARD_ECUDA;
    }
    return (st & 4) ? HARD_ETIMEOUT : HARD_ENONPHYS;
}
