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

// The scheme of a handle (hard_hydro.cu): HARD_SCHEME_PLM_HLLC or
// HARD_SCHEME_WENO5Z_HLL.
int handle_scheme(const hard_hydro_s* h);

}  // namespace hh
