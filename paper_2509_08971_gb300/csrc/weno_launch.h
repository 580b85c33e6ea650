// Launch interface of the WENO5-Z + HLL stage kernels (weno.cuh), one
// translation unit per element type like the PLM-minmod + HLLC kernels.
#pragma once
#include "launch.h"

namespace hh {

// The directional sweeps of the scheme on 3D meshes (weno_sweep.cuh): blocks
// of WENO_SWEEP_THREADS columns along x', chunks of WENO_SWEEP_CHUNK cells
// along the march axis.
#ifndef HH_WENO_CHUNK
#define HH_WENO_CHUNK 64
#endif
inline constexpr int WENO_SWEEP_THREADS = 128;
inline constexpr int WENO_SWEEP_CHUNK = HH_WENO_CHUNK;

// Blocks of the launch that carries a WENO stage's epilogue (rows of the
// totals partial array): the combining z' march of the sweeps, or the fused
// kernel's grid (the first tile of the mesh's tile table).
inline long long weno_stage_blocks(const MeshDesc& m, bool sweeps) {
    if (m.dim == 3 && sweeps) {
        const long long bx = (m.n[0] + WENO_SWEEP_THREADS - 1) / WENO_SWEEP_THREADS;
        const long long bz = (m.n[2] + WENO_SWEEP_CHUNK - 1) / WENO_SWEEP_CHUNK;
        return bx * m.n[1] * bz;
    }
    return stage_blocks(m, 0);
}

// One stage of the second scheme on the mesh: on a 3D mesh with c.scratch
// set, three directional sweeps (c.scratch holds the flux difference
// between them, [5][N] elements, aliasing none of the state buffers);
// otherwise the fused kernel.  Every active axis needs at least three cells.
cudaError_t launch_weno_stage_f32(const MeshDesc& m, const StageCall& c, cudaStream_t s);
cudaError_t launch_weno_stage_f64(const MeshDesc& m, const StageCall& c, cudaStream_t s);

// One Heun stage of the radiation energy advection (WENO5-Z states, Rusanov
// flux) with the fluid state U [5][N] held fixed: stage 1 writes
// Eo = Ec + dt L(Ec), stage 2 Eo = E0/2 + (Ec + dt L(Ec))/2 (Eo may alias E0,
// not Ec).  On a 3D mesh with `scratch` set (N elements aliasing none of the
// other buffers) it runs as three directional sweeps, otherwise as the fused
// kernel.  Every active axis needs at least three cells.
cudaError_t launch_advect_E_stage_f32(const MeshDesc& m, int stage, const void* U, const void* E0,
                                      const void* Ec, void* Eo, double dt, void* scratch,
                                      cudaStream_t s);
cudaError_t launch_advect_E_stage_f64(const MeshDesc& m, int stage, const void* U, const void* E0,
                                      const void* Ec, void* Eo, double dt, void* scratch,
                                      cudaStream_t s);

// The scheme of a handle (hard_hydro.cu): HARD_SCHEME_PLM_HLLC or
// HARD_SCHEME_WENO5Z_HLL.
int handle_scheme(const hard_hydro_s* h);

}  // namespace hh
