// FP64 instantiations of the iteration kernels.
#include "iter_launch.cuh"

namespace dcv {
template cudaError_t launch_row<double>(const RowArgs<double> &, const LaunchCfg &, cudaStream_t);
template cudaError_t launch_col<double>(const ColArgs<double> &, const LaunchCfg &, cudaStream_t);
template cudaError_t prepare_row<double>(const LaunchCfg &);
template cudaError_t prepare_col<double>(const LaunchCfg &);
template cudaError_t launch_row_half<double>(const RowArgs<double> &, const LaunchCfg &, int, cudaStream_t);
}  // namespace dcv
