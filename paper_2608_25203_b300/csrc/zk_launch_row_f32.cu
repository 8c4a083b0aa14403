// zk_launch_row_f32.cu - every row-kernel instantiation of the F32 compute type.
#include "zk_launch_impl.cuh"

namespace zk {
template cudaError_t launch_row<float>(int, int, const RowArgs<float>&, const cx<float>*, int, cudaStream_t);
}  // namespace zk
