// zk_net_internal.h - calls between the closure network (zk_net.cu) and the
// right-hand-side pipeline (zk_api.cu); not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>

#include "../../include/zk.h"

// Make the activation buffers hold `pixels` = batch * nz * nx values per
// channel, so that later inference launches allocate nothing (and can be
// captured into a graph).
zk_status zk_net_reserve(zk_net* n, size_t pixels);

// Forward pass on device input x [B][6][H][W] on stream s, without keeping
// anything for a backward pass; *y receives the network's own output buffer
// [B][2][H][W] (valid until its next pass). H and W: multiples of 16.
cudaError_t zk_net_infer(zk_net* n, const float* x, const float** y, int B, int H, int W, cudaStream_t s);
