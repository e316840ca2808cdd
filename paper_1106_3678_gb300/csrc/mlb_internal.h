// Host-side declarations shared by the C-ABI layer (mlb_api.cu) and the
// kernel translation unit (mlb_kernels.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mlb_engine.cuh"

namespace mlb {

// Persistent solve kernel (one launch per solve).  grid == 1 uses a plain
// launch (CTA-wide barriers only); grid > 1 a cooperative launch.
template <typename T>
cudaError_t launch_solve(const SysView<T> &sys, const SolveCtl &ctl, int grid,
                         cudaStream_t st);
// CTAs of the solve kernel that fit on one SM.
template <typename T>
int solve_blocks_per_sm();

// Q (ld x n, column-major) from the counter-based SplitMix64 + Box-Muller
// generator; rows N..ld-1 are left untouched (zero).
cudaError_t launch_qgen(void *Q, int is_complex, int64_t N, int64_t ld, int n,
                        uint64_t seed, cudaStream_t st);

// F(:, s) = AH Q(:, s) for s < m, AH in CSR (values already conjugated).
template <typename T>
cudaError_t launch_ahq(const int64_t *rp, const int32_t *ci, const T *av,
                       int64_t N, int64_t ld, const T *Q, T *F, int m,
                       cudaStream_t st);

// Fused y = A x, d = Q^H y.  `partials` holds grid * kQdMaxN * 2 doubles;
// d (device) receives n values (2n doubles for complex).
constexpr int kQdMaxN = 64;
constexpr int kQdThreads = 256;
template <typename T>
cudaError_t launch_spmv_qdot(const SysView<T> &sys, const T *x, T *y,
                             double *partials, int grid, double *d,
                             cudaStream_t st);
template <typename T>
int spmv_qdot_grid();

// Failure-detection self-test of the grid barrier (see the C ABI).
cudaError_t launch_barrier_selftest(int grid, BarrierState *bs,
                                    uint64_t timeout_ns, cudaStream_t st);

}  // namespace mlb
