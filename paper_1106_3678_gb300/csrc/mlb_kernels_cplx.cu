// Complex128 solve and batch kernels, with and without the ILU(0) passes
// (see mlb_solve.cuh), in a translation unit of their own so that they
// compile in parallel with the rest of the library.
#include "mlb_solve.cuh"

namespace mlb {

template cudaError_t launch_solve_pc<cdouble, false>(const SysView<cdouble> &, const SolveCtl &, int,
                                                     cudaStream_t);
template cudaError_t launch_solve_pc<cdouble, true>(const SysView<cdouble> &, const SolveCtl &, int, cudaStream_t);
template int solve_blocks_per_sm_pc<cdouble, false>();
template int solve_blocks_per_sm_pc<cdouble, true>();
template cudaError_t launch_batch_pc<cdouble, false>(const BatchItem<cdouble> *, const BatchPlan &, int,
                                                     cudaStream_t);
template cudaError_t launch_batch_pc<cdouble, true>(const BatchItem<cdouble> *, const BatchPlan &, int,
                                                    cudaStream_t);
template int batch_blocks_per_sm_pc<cdouble, false>();
template int batch_blocks_per_sm_pc<cdouble, true>();

}  // namespace mlb
