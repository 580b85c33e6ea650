// Launch interface of the WENO5-Z + HLL stage kernels (weno.cuh), one
// translation unit per element type like the PLM-minmod + HLLC kernels.
#pragma once
#include "launch.h"

namespace hh {

// One stage of the second scheme on the mesh; the kernels run the first tile
// of the mesh's tile table (the totals partial array has stage_blocks(m, 0)
// rows).  Every active axis needs at least three cells.
cudaError_t launch_weno_stage_f32(const MeshDesc& m, const StageCall& c, cudaStream_t s);
cudaError_t launch_weno_stage_f64(const MeshDesc& m, const StageCall& c, cudaStream_t s);

// One Heun stage of the radiation energy advection (WENO5-Z states, Rusanov
// flux) with the fluid state U [5][N] held fixed: stage 1 writes
// Eo = Ec + dt L(Ec), stage 2 Eo = E0/2 + (Ec + dt L(Ec))/2 (Eo may alias E0,
// not Ec).  Every active axis needs at least three cells.
cudaError_t launch_advect_E_stage_f32(const MeshDesc& m, int stage, const void* U, const void* E0,
                                      const void* Ec, void* Eo, double dt, cudaStream_t s);
cudaError_t launch_advect_E_stage_f64(const MeshDesc& m, int stage, const void* U, const void* E0,
                                      const void* Ec, void* Eo, double dt, cudaStream_t s);

// The scheme of a handle (hard_hydro.cu): HARD_SCHEME_PLM_HLLC or
// HARD_SCHEME_WENO5Z_HLL.
int handle_scheme(const hard_hydro_s* h);

}  // namespace hh
