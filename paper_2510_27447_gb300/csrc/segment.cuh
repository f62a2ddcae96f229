// segment.cuh -- batched launches: one launch over the concatenated rows of
// many independent systems.  Block b of a launch belongs to the system r with
// blk[r] <= b < blk[r+1] (a device prefix of per-system block counts) and
// works on that system with that system's parameters, copied into the block's
// shared memory from a device table.
#pragma once
#include <cuda_runtime.h>

namespace bd {

struct SegInfo {
  int r, lb, nb;               // system, block within the system, blocks of the system
};

__device__ __forceinline__ SegInfo seg_locate(const int* blk, int nseg) {
  __shared__ int sr;
  if (threadIdx.x == 0) {
    int lo = 0, hi = nseg - 1;
    const int b = int(blockIdx.x);
    while (lo < hi) {           // the last system whose first block is <= b
      const int mid = (lo + hi + 1) >> 1;
      if (blk[mid] <= b) lo = mid;
      else hi = mid - 1;
    }
    sr = lo;
  }
  __syncthreads();
  const int r = sr;
  return {r, int(blockIdx.x) - blk[r], blk[r + 1] - blk[r]};
}

// a block's copy of its system's parameters (shared memory)
template <class P>
__device__ __forceinline__ const P& stage(const P* tab, int r) {
  static_assert(sizeof(P) % 4 == 0, "parameter block size");
  __shared__ __align__(16) int buf[sizeof(P) / 4];
  const int* s = reinterpret_cast<const int*>(tab + r);
  for (int i = threadIdx.x; i < int(sizeof(P) / 4); i += blockDim.x) buf[i] = s[i];
  __syncthreads();
  return *reinterpret_cast<const P*>(buf);
}

}  // namespace bd
