// Per-tensor amax records of the FP8 precision: a kernel that writes an
// activation a later E4M3 GEMM reads folds max|value| of what it wrote into
// the tensor's slot (float bits; |values| are non-negative floats, whose bit
// patterns order like the floats, so an unsigned atomicMax is a float max).
#pragma once

#include <cuda_runtime.h>

namespace alg {

// max over the warp's active lanes, then one atomicMax per warp (slot may be null).
// The slot only grows, so a warp whose max does not exceed the value it reads there
// (an L2 read, cheap even when every warp of a launch reads the same word) can skip
// the atomic: the result is the same, and the atomics on one address, which the L2
// serialises, drop from one per warp to a few per launch.
__device__ __forceinline__ void record_amax(unsigned* slot, float v) {
  if (!slot) return;
  const unsigned mask = __activemask();
  const unsigned m = __reduce_max_sync(mask, __float_as_uint(fabsf(v)));
  if ((threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1) && m > __ldcg(slot)) atomicMax(slot, m);
}

}  // namespace alg
