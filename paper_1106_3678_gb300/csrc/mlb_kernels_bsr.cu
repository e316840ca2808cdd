// Solve and refined kernels for matrices stored as 3x3 blocks (see
// sell_slice_sum3), with and without the ILU(0) passes, in a translation
// unit of their own so that they compile in parallel with the rest of the
// library.  Real values only.
#include "mlb_solve.cuh"

namespace mlb {

template cudaError_t launch_solve_pc<double, false, 3>(const SysView<double> &, const SolveCtl &, int, cudaStream_t);
template cudaError_t launch_solve_pc<double, true, 3>(const SysView<double> &, const SolveCtl &, int, cudaStream_t);
template int solve_blocks_per_sm_pc<double, false, 3>();
template int solve_blocks_per_sm_pc<double, true, 3>();
template cudaError_t launch_refine_pc<float, double, false, 3>(const SysView<float> &, const RefView<double> &,
                                                               const SolveCtl &, const RefCtl &, int, cudaStream_t);
template cudaError_t launch_refine_pc<float, double, true, 3>(const SysView<float> &, const RefView<double> &,
                                                              const SolveCtl &, const RefCtl &, int, cudaStream_t);
template int refine_blocks_per_sm_pc<float, double, false, 3>();
template int refine_blocks_per_sm_pc<float, double, true, 3>();

}  // namespace mlb
