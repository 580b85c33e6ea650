// Tensor-memory-accelerator (TMA) and mbarrier helpers for sm_103a, written
// as inline PTX.  Bulk tensor loads move a haloed box of the conserved state
// from global into shared memory; an mbarrier with an expected transaction
// count tells the consumer warps when a box has landed.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
