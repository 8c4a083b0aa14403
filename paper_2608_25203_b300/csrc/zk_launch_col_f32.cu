// zk_launch_col_f32.cu - every column-kernel instantiation of the F32 compute type.
#include "zk_launch_impl.cuh"

namespace zk {
template cudaError_t launch_col<float>(int, int, int, const ColArgs<float>&, const cx<float>*, cudaStream_t, int*);
}  // namespace zk
