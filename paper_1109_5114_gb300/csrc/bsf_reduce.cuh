// Block-wide reduction for the kernels that fold a whole field into one
// status word: one atomic per block instead of one per warp (atomics of many
// warps on one word serialise in L2).
#pragma once

// op-reduce v over the block; every thread of the block must call it (no
// thread may have returned); blockDim.x a multiple of 32, at most 1024.  The
// result is valid in thread 0.
template <typename V, typename Op>
__device__ __forceinline__ V bsf_block_reduce(V v, Op op) {
  __shared__ V s[32];
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int nw = (int)(blockDim.x >> 5);
  __syncthreads();  // an earlier call's values have been read
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < nw; ++w) v = op(v, s[w]);
  return v;
}
