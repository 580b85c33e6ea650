// Interface of the flux-limited radiation diffusion solver (fld.cu): one
// backward-Euler step of dE/dt = div(D grad E), D = c lambda(R) / (kappa rho)
// frozen at the old state, solved by geometric-multigrid V-cycles.
#pragma once
#include "launch.h"

namespace hh {

struct FldHierarchy;      // grid levels and their device arrays (fld.cu)

// Levels of a mesh: every active axis of even length >= 4 halves, until no
// axis can (or the level has at most 64 cells).  Allocates the device arrays;
// returns nullptr on a failed allocation.
FldHierarchy* fld_create(const MeshDesc& m, int dtype);
void fld_destroy(FldHierarchy* H);
bool fld_matches(const FldHierarchy* H, const MeshDesc& m, int dtype);
int fld_levels(const FldHierarchy* H);

// One implicit step on Er (in place), the density taken from U[0].  Runs
// V-cycles until the 2-norm of the residual is at most rtol times that of the
// right-hand side (rtol <= 0: exactly max_cycles cycles, no host sync), or
// max_cycles ran.  *cycles and *rel_resid (may be null) receive the count and
// the last relative residual (-1 when not measured).
cudaError_t fld_solve(FldHierarchy* H, const MeshDesc& m, const void* U, void* Er, double dt,
                      double c, double kappa, double rtol, int max_cycles, int* cycles,
                      double* rel_resid, cudaStream_t s);

}  // namespace hh
