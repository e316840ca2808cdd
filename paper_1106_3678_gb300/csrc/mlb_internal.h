// Host-side declarations shared by the C-ABI layer (mlb_api.cu) and the
// kernel translation unit (mlb_kernels.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

#include "mlbicgstab.h"
#include "mlb_engine.cuh"
#include "mlb_refine.cuh"

namespace mlb {

// Persistent solve kernel (one launch per solve).  grid == 1 uses a plain
// launch (CTA-wide barriers only); grid > 1 a cooperative launch.
template <typename T>
cudaError_t launch_solve(const SysView<T> &sys, const SolveCtl &ctl, int grid,
                         cudaStream_t st);
// CTAs of the solve kernel that fit on one SM.
template <typename T>
int solve_blocks_per_sm();

// FP32-inner / FP64-refined persistent solve kernel.
template <typename T32, typename T64>
cudaError_t launch_refine(const SysView<T32> &sys, const RefView<T64> &rv, const SolveCtl &ctl,
                          const RefCtl &rc, int grid, cudaStream_t st);
template <typename T32, typename T64>
int refine_blocks_per_sm();
// dst[i] = (float)src[i] for `count` doubles.
cudaError_t launch_narrow(const double *src, float *dst, int64_t count, cudaStream_t st);

// x[i] = x[i] * d[i] (divide = false) or x[i] / d[i] (divide = true), i < n:
// the map between x and y = M x of a diagonal (Jacobi) preconditioner.
template <typename T>
cudaError_t launch_diag_apply(T *x, const T *d, int64_t n, bool divide, cudaStream_t st);

// One system of a batch (device copy of its views and controls).
template <typename T>
struct BatchItem {
    SysView<T> sys;
    SolveCtl ctl;   // tol, maxit, kappa, max_outer; res -> this system's record
};
template <typename T32, typename T64>
struct BatchItemR {
    SysView<T32> sys;
    RefView<T64> rv;
    SolveCtl ctl;
    RefCtl rc;
};
// Batch work plan parameters: a system goes to a team when it has at
// least kTeamMinRows rows per team CTA and its estimated work exceeds
// kTeamShare of the average work per CTA; teams have at most kMaxBatchTeam
// CTAs.
constexpr int kTeamMinRows = 2048;
constexpr double kTeamShare = 0.1;
constexpr int kMaxBatchTeam = 8;

// Work plan of a batch launch (device pointers into the batch workspace).
// The first teams * team CTAs form `teams` teams of `team` consecutive CTAs;
// each team takes the systems of order_big (a device queue, largest first)
// one at a time and solves each with all its CTAs (team barriers and
// reductions like a multi-CTA solve with grid = team).  Then every CTA,
// and from the start every CTA outside the teams, takes the systems of
// order_small (largest first) and solves each alone.  With teams the launch
// is cooperative (all CTAs co-resident), so a team's CTAs all run.
struct BatchPlan {
    const int *order_big;    // item indices solved by teams
    int count_big;
    const int *order_small;  // item indices solved by one CTA
    int count_small;
    int team;                // CTAs per team
    int teams;               // teams (0: none)
    unsigned *queue;         // [0]: next of order_small, [1]: next of order_big (zeroed)
    BarrierState *tbar;      // per team: barrier of the team's turns (zeroed)
    int *team_item;          // per team: 2 slots, the turn's position in order_big
    BarrierState *sbar;      // per position of order_big: the solve's barrier (zeroed)
    double *spart;           // per position of order_big: 2 * kMaxSums * team doubles
    uint64_t timeout_ns;     // limit of the waits between turns
};
// ilu: some item has an ILU(0) preconditioner (the kernel with those passes
// then runs every item, each by its own view).
template <typename T>
cudaError_t launch_batch(const BatchItem<T> *items, const BatchPlan &plan, int grid, bool ilu, cudaStream_t st);
template <typename T32, typename T64>
cudaError_t launch_batch_refine(const BatchItemR<T32, T64> *items, const BatchPlan &plan, int grid, bool ilu,
                                cudaStream_t st);
template <typename T>
int batch_blocks_per_sm();
template <typename T32, typename T64>
int batch_refine_blocks_per_sm();

// Q (ld x n, column-major) from the counter-based SplitMix64 + Box-Muller
// generator; rows N..ld-1 are left untouched (zero).  With `perm`, row r
// receives the entries of original row perm[r] (Q of a multicolour-ordered
// handle is the Q of the original row order, permuted).
cudaError_t launch_qgen(void *Q, int is_complex, int64_t N, int64_t ld, int n,
                        uint64_t seed, cudaStream_t st, const int32_t *perm = nullptr);

// F(:, s) = AH Q(:, s) for s < m, AH in CSR (values already conjugated).
template <typename T>
cudaError_t launch_ahq(const int64_t *rp, const int32_t *ci, const T *av,
                       int64_t N, int64_t ld, const T *Q, T *F, int m,
                       cudaStream_t st);

// Fused y = A x, d = Q^H y.  `partials` holds grid * kQdMaxN * 2 doubles.
constexpr int kQdMaxN = 64;
// One CTA of kThreads per SM (grid <= the handle's grid_max),
// dynamic shared memory kRingBytes.  The first `ne` columns (1, 2 or 4;
// at most n, and at most 2 for complex values) of Q are epilogue vectors
// of the SELL product, whose tiles hold `spt`
// slices (sized for that many epilogue vectors); the others take tile
// passes over y.  x: the caller's N values (SELL padding columns stay below
// N); y: a padded scratch vector of ld values; yout: the caller's N values.
// status: one int per CTA (written every launch, nonzero where a tile wait
// timed out); ticket: a counter that is 0 between launches (zero it once
// at allocation); d (device) receives the n inner products (2n doubles for
// complex) and then d[n * DS] = 1.0 if any CTA timed out, else 0.0.
// ev (optional) is recorded on st directly before the kernel launch.
// Default fused columns: 4 only when that is all of them (real n = 4): four
// epilogue vectors leave room for 12 slices per tile, so 3 of the 15
// consumer warps idle in the product, which costs more than a later pass
// over y for the remaining columns; complex values take at most 2 (4
// spill registers).  Real FP64 with n > 4 fuses 1: the product is bound by
// FP64 issue, and the later passes over y overlap their DFMAs with the
// loads better (128^3, n = 8: 86 us fusing 1, 92 us fusing 2, 107 us
// fusing 4; n = 16: 119 against 126 us).
inline int qd_fused_columns(int n, bool cplx, bool narrow) {
    if (n == 4 && !cplx) return 4;
    if (n > 4 && !cplx && !narrow) return 1;
    return n >= 2 ? 2 : 1;
}
// maxw: the widest slice (entries per row), which selects the pipelined
// width of the product.
template <typename T>
cudaError_t launch_spmv_qdot_tiled(const SysView<T> &sys, int ne, int64_t maxw, int spt, const T *x, T *y,
                                   T *yout, double *partials, int grid, int *status, unsigned *ticket, double *d,
                                   cudaEvent_t ev, cudaStream_t st);

// ILU(0) preconditioner, host side (mlb_ilu.cu).  Factors of A in A's
// pattern (columns increasing within each row, repeated entries merged):
// entries before row i's diagonal are L's (unit diagonal implied), the rest
// U's; dpos[i] = position of the diagonal relative to rp[i]; rows grouped
// into the level sets of the forward (L) and backward (U) solves.
// For the solves, each triangle also in level-position order: position q
// (row lrows[q] or urows[q]) has its entry count (lcnt/ucnt) and its first
// kIluEll entries at e * N + q (columns lell_c/uell_c, values
// lell_a/uell_a); udiag[q] is U's diagonal of row urows[q].  A row's
// loads are then independent of each other (only the row's right-hand
// side needs the row index).
constexpr int kIluEll = 4;
struct IluHost {
    std::vector<int64_t> rp;
    std::vector<int32_t> ci, dpos, lrows, lptr, urows, uptr;
    std::vector<char> lu;   // nnz values of the handle's dtype
    int64_t nnz = 0;
    int nlev_l = 0, nlev_u = 0;
    std::vector<int32_t> lcnt, ucnt, lell_c, uell_c;
    std::vector<char> lell_a, uell_a, udiag;
};
// MLB_OK, or MLB_ERR_ARG when a row has no stored diagonal or a pivot is
// zero or not finite.
int ilu0_build(const mlb_matrix *A, IluHost &out);
// v <- M^{-H} v for the N values at v (M = L U from `f`).
void ilu0_apply_h(const IluHost &f, bool cplx, void *v);
// Multicolour order of A (the multicolour ILU(0) preconditioner): greedy
// colouring of the symmetrised adjacency graph in natural order (each row
// takes the smallest colour no neighbour coloured before it has), rows
// then listed colour by colour, natural order within a colour.
// perm[new] = old.  Returns the number of colours.
int mc_order(const mlb_matrix *A, std::vector<int32_t> &perm);
// B = P A P^T: row r of B is row perm[r] of A with column c renamed
// iperm[c] (entries of a row in A's order); es = bytes per value.
void permute_csr(const mlb_matrix *A, const std::vector<int32_t> &perm, const std::vector<int32_t> &iperm,
                 size_t es, std::vector<int64_t> &rp, std::vector<int32_t> &ci, std::vector<char> &val);
// Gather (to_perm: dst[r] = src[perm[r]]) or scatter (dst[perm[r]] =
// src[r]) of N values of `es` bytes between the original and the
// multicolour row order.
cudaError_t launch_permute(const void *src, void *dst, const int32_t *perm, int64_t N, int es, bool to_perm,
                           cudaStream_t st);

// Failure-detection self-test of the grid barrier (see the C ABI).
cudaError_t launch_barrier_selftest(int grid, BarrierState *bs,
                                    uint64_t timeout_ns, cudaStream_t st);

}  // namespace mlb
