// zk_launch.h - launch helpers of the right-hand-side kernels (internal to the library).
//
// The row and column kernels are instantiated for every padded line length,
// plan variant, precision and padding; their launch functions live in their
// own translation units (zk_launch_{row,col}_{f32,f64}.cu) so that the
// library's build compiles them in parallel.
#pragma once

#include <cstddef>

#include "zk_kernels2.cuh"

namespace zk {

// columns per column-kernel block: 4 for wide line groups, else enough for 128 (FP32) / 64 (FP64) threads
template <int NPZ, int ES, int V = 0> constexpr int col_cb() {
    return IPlan<NPZ, V>::TL >= 64 ? 4 : ((ES == 8 ? 128 : 64) / IPlan<NPZ, V>::TL);
}
// autotuner choice ci of columns per block: 0 = half, 1 = default, 2 = double
template <int NPZ, int ES, int V> constexpr int col_cb_pick(int ci) {
    return ci == 0 ? (col_cb<NPZ, ES, V>() > 1 ? col_cb<NPZ, ES, V>() / 2 : 1)
                   : (ci == 2 ? 2 * col_cb<NPZ, ES, V>() : col_cb<NPZ, ES, V>());
}

// Resident blocks per SM of a kernel shape, and the SM count (cached per shape).
void occupancy(const void* fn, int threads, size_t smem, int* per_sm, int* sms);
// Largest dynamic shared memory a block may opt in to on this device.
int smem_optin();
// Raise a kernel's dynamic shared-memory limit to `bytes` (once per kernel).
cudaError_t ensure_smem(const void* fn, size_t bytes);

// One row-kernel launch (persistent over the npz padded rows) on the plan
// variant v, or one column-kernel launch with the columns-per-block choice ci.
template <typename T>
cudaError_t launch_row(int npx, int v, const RowArgs<T>& a, const cx<T>* tw, int npz, cudaStream_t s);
template <typename T>
cudaError_t launch_col(int npz, int v, int ci, const ColArgs<T>& a, const cx<T>* tw, cudaStream_t s,
                       int* nblocks = nullptr);

extern template cudaError_t launch_row<float>(int, int, const RowArgs<float>&, const cx<float>*, int, cudaStream_t);
extern template cudaError_t launch_row<double>(int, int, const RowArgs<double>&, const cx<double>*, int, cudaStream_t);
extern template cudaError_t launch_col<float>(int, int, int, const ColArgs<float>&, const cx<float>*, cudaStream_t, int*);
extern template cudaError_t launch_col<double>(int, int, int, const ColArgs<double>&, const cx<double>*, cudaStream_t, int*);

}  // namespace zk
