// Internal launch interface between the C ABI (hard_hydro.cu) and the kernel
// translation units (one per element type, so that the FP64 one can be built
// without FMA contraction).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hh {

struct TileDesc {
    int tx, ty, zc;        // tile extents along kernel x', y' and the z chunk
};

// Mesh as the kernels see it: the active axes become kernel axes x', y', z'.
struct MeshDesc {
    int dim;               // number of active axes (0..3)
    int px, py;            // physical axis of kernel x', y'
    int n[3];              // kernel-axis extents (inactive: 1)
    int bc_lo[3], bc_hi[3];
    double dxk[3];         // cell width per kernel axis
    double dx[3];          // cell width per physical axis
    bool act[3];           // physical axis active
    double gamma;
    long long N;           // total cells
};

struct StageCall {
    int stage;                     // 1 or 2
    const void* U0;
    const void* Uc;
    void* Uo;
    double dt;                     // used when dt_dev == nullptr
    const double* dt_dev;
    unsigned long long* rate_slot; // nullptr = no rate epilogue
    double* tot_partial;           // nullptr = no totals epilogue
    int* status;
    int zlo = 0, zhi = -1;         // 3D: the kernel-z cells [zlo, zhi) to update (-1: to nz);
                                   // zlo a multiple of the tile's z-chunk
    const void* zg[2] = {nullptr, nullptr};  // ghost planes of BC_HALO z faces (below, above),
                                             // each [5][2][ny][nx]
    void* scratch = nullptr;       // WENO on 3D meshes: [5][N] flux-difference buffer of the
                                   // sweeps (nullptr: the fused kernel)
};

// Tile configurations per number of active axes (the autotuner's space).
inline constexpr TileDesc TILES3[] = {{32, 8, 32}, {32, 8, 64}, {32, 16, 64}, {64, 8, 64},
                                      {32, 4, 64}, {32, 16, 32}};
inline constexpr TileDesc TILES2[] = {{32, 8, 0}, {32, 16, 0}, {64, 8, 0}};
inline constexpr TileDesc TILES1[] = {{128, 1, 0}, {256, 1, 0}};

inline int tile_count(int dim) {
    return dim == 3 ? 6 : dim == 2 ? 3 : dim == 1 ? 2 : 1;
}
inline TileDesc tile_desc(int dim, int tile) {
    if (dim == 3) return TILES3[tile];
    if (dim == 2) return TILES2[tile];
    if (dim == 1) return TILES1[tile];
    return TileDesc{256, 1, 0};
}
// Blocks the stage kernel launches (rows of the totals partial array).
inline long long stage_blocks(const MeshDesc& m, int tile) {
    if (m.dim == 0) return 1;
    TileDesc t = tile_desc(m.dim, tile);
    long long gx = (m.n[0] + t.tx - 1) / t.tx;
    long long gy = m.dim >= 2 ? (m.n[1] + t.ty - 1) / t.ty : 1;
    long long gz = m.dim == 3 ? (m.n[2] + t.zc - 1) / t.zc : 1;
    return gx * gy * gz;
}

cudaError_t launch_stage_f32(const MeshDesc& m, int kernel, int tile, const StageCall& c,
                             cudaStream_t s);
cudaError_t launch_stage_f64(const MeshDesc& m, int kernel, int tile, const StageCall& c,
                             cudaStream_t s);
// Signal-rate max of U into *rate_slot (which must be zeroed first).
cudaError_t launch_rate_f32(const MeshDesc& m, const void* U, unsigned long long* rate_slot,
                            int* status, cudaStream_t s);
cudaError_t launch_rate_f64(const MeshDesc& m, const void* U, unsigned long long* rate_slot,
                            int* status, cudaStream_t s);
// Per-block partial sums of the 5 fields; returns the number of partial rows.
inline constexpr int TOTALS_BLOCKS = 608;
inline long long totals_blocks() { return TOTALS_BLOCKS; }
cudaError_t launch_totals_f32(const MeshDesc& m, const void* U, double* partial, cudaStream_t s);
cudaError_t launch_totals_f64(const MeshDesc& m, const void* U, double* partial, cudaStream_t s);

// One problem of a batch (see batched.cuh).
struct BatchProblem {
    long long off;        // element offset of the problem's U[5][ny][nx] in the packed buffer
    int nx, ny;           // cells (nz = 1); ny == 1 makes a 1D problem
    int bc;               // boundary kind on all faces
    int pad;
    double gamma;
};

struct BatchCall {
    void* U;
    void* W;
    const BatchProblem* probs;
    const int* order;
    int nprob;
    int nsteps;
    double cfl;
    double* t;
    int* counter;
    int* status;
};

// Batched tile configurations: {1D tile width, 2D tile x, 2D tile y}.
inline constexpr int BATCH_TILES[][3] = {{256, 32, 8}, {128, 32, 4}, {512, 64, 8}};
inline constexpr int BATCH_TILE_COUNT = 3;

cudaError_t launch_batched_f32(const BatchCall& c, int tile, cudaStream_t s);
cudaError_t launch_batched_f64(const BatchCall& c, int tile, cudaStream_t s);

// VJP of one stage (adjoint.cuh): gW, 8 slots per cell holding zeros on
// entry, is the primitive cotangent accumulator (cleared again on exit when
// clear_gW);
// out_c (=|+=) b G + J^T(lam G) term; out0 = a G when not null; d/dgamma
// added to *g_gamma.
struct AdjointCall {
    const void* Uc;
    const void* G;
    void* gW;
    void* out_c;
    bool accumulate;
    void* out0;
    double b, a, lam;
    double* g_gamma;
    bool clear_gW;
    int passes = 3;                                // bit 0: the face pass, bit 1: the cell pass
    const void* zg[2] = {nullptr, nullptr};        // BC_HALO z faces: ghost planes of Uc
    void* gwg[2] = {nullptr, nullptr};             // and their cotangent accumulators
};
cudaError_t launch_adjoint_stage_f32(const MeshDesc& m, const AdjointCall& c, cudaStream_t s);
cudaError_t launch_adjoint_stage_f64(const MeshDesc& m, const AdjointCall& c, cudaStream_t s);
// A neighbouring slab's ghost accumulator ([2][ny][nx] records) added into
// planes k0, k0+1 of the accumulator gW.
cudaError_t launch_add_ghost_cotangent_f32(const MeshDesc& m, void* gW, const void* from, int k0,
                                           cudaStream_t s);
cudaError_t launch_add_ghost_cotangent_f64(const MeshDesc& m, void* gW, const void* from, int k0,
                                           cudaStream_t s);

// Read-only view of a handle (hard_hydro.cu); false for a NULL handle.
}  // namespace hh
struct hard_hydro_s;
namespace hh {
bool handle_view(hard_hydro_s* h, const MeshDesc** mesh, int* dtype, int* kernel, int* tile);

// Shared helpers (hard_hydro.cu).
cudaError_t launch_finalize_dt(unsigned long long* rate_slot, double cfl, double t_end,
                               double* t_dev, double* dt_dev, double* dt_log, int step,
                               int* status, cudaStream_t s);
cudaError_t launch_finalize_totals(const double* partial, long long rows, double dV,
                                   double* out5, cudaStream_t s);

}  // namespace hh
