// zk_launch_col_f64.cu - every column-kernel instantiation of the F64 compute type.
#include "zk_launch_impl.cuh"

namespace zk {
template cudaError_t launch_col<double>(int, int, int, const ColArgs<double>&, const cx<double>*, cudaStream_t, int*);
}  // namespace zk
