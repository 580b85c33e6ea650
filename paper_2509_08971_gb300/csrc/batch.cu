// C ABI of the batched persistent launch (include/hard_hydro.h): a batch
// owns the problem table, the largest-first queue order, the packed
// intermediate stage and its status word.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <new>
#include <numeric>
#include <vector>

#include "hard_hydro.h"
#include "launch.h"

struct hard_batch_s {
    int nprob = 0;
    int dtype = HARD_F32;
    int tile = 0;
    long long elements = 0;
    std::vector<hh::BatchProblem> probs;
    hh::BatchProblem* d_probs = nullptr;
    int* d_order = nullptr;
    void* W = nullptr;
    int* d_words = nullptr;              // [0] queue head, [1] status
    cudaStream_t last = nullptr;
};

namespace {

constexpr long long ALIGN_ELEMS = 32;     // each problem's block starts on 128 bytes (FP32)

bool valid_bc(int b) { return b == HARD_BC_PERIODIC || b == HARD_BC_OUTFLOW || b == HARD_BC_REFLECT; }

void release(hard_batch_s* b) {
    if (b->d_probs) cudaFree(b->d_probs);
    if (b->d_order) cudaFree(b->d_order);
    if (b->W) cudaFree(b->W);
    if (b->d_words) cudaFree(b->d_words);
    delete b;
}

bool alloc_fail_injected() {
    const char* v = std::getenv("HARD_HYDRO_FAIL_ALLOC");
    return v && v[0] == '1';
}

}  // namespace

extern "C" {

hard_batch_t hard_batch_create(int nprob, const int* nx, const int* ny, const int* nz,
                               const double* gamma, const int* bc, int dtype) {
    if (nprob < 1 || !nx || !ny || !gamma || !bc) return nullptr;
    if (dtype != HARD_F32 && dtype != HARD_F64) return nullptr;
    if (alloc_fail_injected()) return nullptr;
    hard_batch_s* b = new (std::nothrow) hard_batch_s();
    if (!b) return nullptr;
    b->nprob = nprob;
    b->dtype = dtype;
    b->probs.resize(nprob);
    long long off = 0;
    for (int p = 0; p < nprob; ++p) {
        const int z = nz ? nz[p] : 1;
        if (nx[p] < 2 || ny[p] < 1 || z != 1 || !(gamma[p] > 1.0) || !std::isfinite(gamma[p]) ||
            !valid_bc(bc[p])) {
            delete b;
            return nullptr;
        }
        hh::BatchProblem& P = b->probs[p];
        P.off = off;
        P.nx = nx[p];
        P.ny = ny[p];
        P.bc = bc[p];
        P.pad = 0;
        P.gamma = gamma[p];
        const long long n = 5ll * nx[p] * ny[p];
        off = (off + n + ALIGN_ELEMS - 1) / ALIGN_ELEMS * ALIGN_ELEMS;
    }
    b->elements = off;
    std::vector<int> order(nprob);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (long long)nx[a] * ny[a] > (long long)nx[c] * ny[c];
    });
    const size_t es = dtype == HARD_F64 ? 8 : 4;
    if (cudaMalloc(&b->d_probs, sizeof(hh::BatchProblem) * nprob) != cudaSuccess ||
        cudaMalloc(&b->d_order, sizeof(int) * nprob) != cudaSuccess ||
        cudaMalloc(&b->W, es * (size_t)b->elements) != cudaSuccess ||
        cudaMalloc(&b->d_words, 2 * sizeof(int)) != cudaSuccess ||
        cudaMemcpy(b->d_probs, b->probs.data(), sizeof(hh::BatchProblem) * nprob,
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_order, order.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(b->d_words, 0, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        release(b);
        return nullptr;
    }
    return b;
}

long long hard_batch_offset(hard_batch_t b, int p) {
    if (!b || p < 0 || p >= b->nprob) return HARD_EINVAL;
    return b->probs[p].off;
}

long long hard_batch_elements(hard_batch_t b) {
    if (!b) return HARD_EINVAL;
    return b->elements;
}

int hard_batch_tile_count(void) { return hh::BATCH_TILE_COUNT; }

int hard_batch_set_tile(hard_batch_t b, int tile) {
    if (!b || tile < 0 || tile >= hh::BATCH_TILE_COUNT) return HARD_EINVAL;
    b->tile = tile;
    return HARD_OK;
}

int hard_hydro_step_batched(hard_batch_t b, void* U_packed, int nsteps, double cfl, double* t_dev,
                            void* stream) {
    if (!b || !U_packed || !t_dev || nsteps < 0) return HARD_EINVAL;
    if ((reinterpret_cast<uintptr_t>(U_packed) & 15u) != 0) return HARD_EINVAL;
    if (!(cfl > 0.0) || !std::isfinite(cfl)) return HARD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    b->last = s;
    if (cudaMemsetAsync(b->d_words, 0, sizeof(int), s) != cudaSuccess) return HARD_ECUDA;
    const hh::BatchCall c{U_packed, b->W, b->d_probs, b->d_order, b->nprob, nsteps,
                          cfl, t_dev, b->d_words, b->d_words + 1};
    const cudaError_t e = b->dtype == HARD_F64 ? hh::launch_batched_f64(c, b->tile, s)
                                               : hh::launch_batched_f32(c, b->tile, s);
    return e == cudaSuccess ? HARD_OK : HARD_ECUDA;
}

int hard_batch_get_error(hard_batch_t b) {
    if (!b) return HARD_EINVAL;
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, b->d_words + 1, sizeof(int), cudaMemcpyDeviceToHost,
                                    b->last);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->last);
    if (e != cudaSuccess) return HARD_ECUDA;
    if (st) {
        if (cudaMemsetAsync(b->d_words + 1, 0, sizeof(int), b->last) != cudaSuccess ||
            cudaStreamSynchronize(b->last) != cudaSuccess)
            return HARD_ECUDA;
        return HARD_ENONPHYS;
    }
    return HARD_OK;
}

void hard_batch_destroy(hard_batch_t b) {
    if (b) release(b);
}

}  // extern "C"
