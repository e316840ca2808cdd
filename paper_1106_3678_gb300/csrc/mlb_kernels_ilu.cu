// Real FP64 solve and batch kernels and the refined kernels with the ILU(0)
// preconditioner passes (see mlb_solve.cuh), in a translation unit of their
// own so that they compile in parallel with the rest of the library.
#include "mlb_solve.cuh"

namespace mlb {

template cudaError_t launch_solve_pc<double, true>(const SysView<double> &, const SolveCtl &, int, cudaStream_t);
template cudaError_t launch_batch_pc<double, true>(const BatchItem<double> *, const BatchPlan &, int, cudaStream_t);
template int solve_blocks_per_sm_pc<double, true>();
template int batch_blocks_per_sm_pc<double, true>();
template cudaError_t launch_refine_pc<float, double, true>(const SysView<float> &, const RefView<double> &,
                                                           const SolveCtl &, const RefCtl &, int, cudaStream_t);
template cudaError_t launch_refine_pc<cfloat, cdouble, true>(const SysView<cfloat> &, const RefView<cdouble> &,
                                                             const SolveCtl &, const RefCtl &, int, cudaStream_t);
template int refine_blocks_per_sm_pc<float, double, true>();
template int refine_blocks_per_sm_pc<cfloat, cdouble, true>();
template cudaError_t launch_batch_refine_pc<float, double, true>(const BatchItemR<float, double> *,
                                                                 const BatchPlan &, int, cudaStream_t);
template cudaError_t launch_batch_refine_pc<cfloat, cdouble, true>(const BatchItemR<cfloat, cdouble> *,
                                                                   const BatchPlan &, int, cudaStream_t);
template int batch_refine_blocks_per_sm_pc<float, double, true>();
template int batch_refine_blocks_per_sm_pc<cfloat, cdouble, true>();

}  // namespace mlb
