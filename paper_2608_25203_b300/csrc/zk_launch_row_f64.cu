// zk_launch_row_f64.cu - every row-kernel instantiation of the F64 compute type.
#include "zk_launch_impl.cuh"

namespace zk {
template cudaError_t launch_row<double>(int, int, const RowArgs<double>&, const cx<double>*, int, cudaStream_t);
}  // namespace zk
