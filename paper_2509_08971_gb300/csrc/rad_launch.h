// Launch interface of the radiative heating / cooling exchange (rad.cu).
#pragma once
#include "launch.h"

namespace hh {

// One backward-Euler exchange step on every cell of the mesh: U [5][N] (its
// E_total field is updated) and the radiation energy density Er [N], both of
// the element type `dtype`; prm = {c, kappa, a, c_v}.  Cells with rho <= 0,
// e <= 0, E < 0, or a Newton solve that does not converge are left unchanged
// and set bit 0 of *status.
cudaError_t launch_rad_exchange(const MeshDesc& m, int dtype, void* U, void* Er, double dt,
                                const double prm[4], int* status, cudaStream_t s);

}  // namespace hh
