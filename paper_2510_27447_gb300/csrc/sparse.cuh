// sparse.cuh -- device building blocks of the persistent solvers: a bounded
// device-wide barrier, deterministic block and grid reductions, and the row
// product of a SELL-32 operator (layout described in bd_internal.h).
#pragma once
#include <cuda_runtime.h>

#include "bd_internal.h"

namespace bd {

#ifndef BD_PCG_SLEEP_NS
#define BD_PCG_SLEEP_NS 0
#endif
// minimum resident 1024-thread blocks per SM the persistent solver kernels are
// compiled for (1: up to 64 registers per thread)
#ifndef BD_SOLVER_MIN_BLOCKS
#define BD_SOLVER_MIN_BLOCKS 1
#endif
#ifndef BD_SELL_CHUNK
#define BD_SELL_CHUNK 2
#endif
// bounded waits: a device-barrier wait gives up after kWaitLimitNs of device
// time (%globaltimer), with an iteration cap as a backstop
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
constexpr long long kSpinLimit = 1ll << 28;

__device__ __forceinline__ unsigned long long device_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Device-wide barrier on one arrival word: block 0 adds 2^31 - (nblocks - 1),
// every other block adds 1, so the word's top bit flips exactly when the last
// block of a round arrives and the low bits return to their old value (no
// reset step).  Arrival is a release RMW (publishes the block's writes), the
// wait an acquire load (sees every arriving block's writes).  The wait is
// bounded (two seconds): on timeout the kernel records ST_TIMEOUT and every
// block returns, leaving the context usable.
__device__ __forceinline__ unsigned bar_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned bar_add_acq_rel(unsigned* p, unsigned x) {
  unsigned v;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "r"(x) : "memory");
  return v;
}

// Single-cluster launches (bar == nullptr): the whole grid is one thread-block
// cluster, and the barrier is the cluster's hardware barrier (every thread
// arrives with release and waits with acquire semantics at cluster scope).
// Every solver kernel reaches its barriers in grid-uniform control flow.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* status) {
  if (bar == nullptr) {
    cluster_barrier();
    return true;
  }
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (nblocks - 1u) : 1u;
    const unsigned old = bar_add_acq_rel(bar, add);
    ok = 1;
    long long spins = 0;
    const unsigned long long t0 = device_ns();
    while (((old ^ bar_ld_acquire(bar)) & 0x80000000u) == 0u) {
      if (BD_PCG_SLEEP_NS > 0) __nanosleep(BD_PCG_SLEEP_NS);
      ++spins;
      if (((spins & 255) == 0 && device_ns() - t0 > kWaitLimitNs) || spins > kSpinLimit) {
        atomicOr(status, ST_TIMEOUT);
        ok = 0;
        break;
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

// can `kernel` run as one cluster of `size` blocks of `block` threads?
// (non-portable sizes above 8 are enabled on the kernel first)
template <class K>
inline bool solver_cluster_ok(K kernel, int block, int size) {
  if (size > 8 && cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(size));
  cfg.blockDim = dim3(unsigned(block));
  cudaLaunchAttribute a;
  a.id = cudaLaunchAttributeClusterDimension;
  a.val.clusterDim.x = unsigned(size);
  a.val.clusterDim.y = 1;
  a.val.clusterDim.z = 1;
  cfg.attrs = &a;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= 1;
}

// copy a trivially copyable descriptor (e.g. the AMG hierarchy) from global
// into the block's shared memory; level loops then index it at run time with
// shared-memory latency
template <class D>
__device__ __forceinline__ void load_descriptor(D& dst, const D* src) {
  static_assert(sizeof(D) % 4 == 0, "descriptor size");
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(&dst);
  for (int i = threadIdx.x; i < int(sizeof(D) / 4); i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

// block-wide sum of NV values; result valid in thread 0
template <int NV, class T = double>
__device__ __forceinline__ void block_sum(T (&v)[NV], T (*sh)[32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T x = lane < nw ? sh[k][lane] : T(0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[k] = x;
    }
  }
  __syncthreads();
}

// every block sums part[b*STRIDE + slot] over b = 0..nb-1 in the same order
template <int NV, class T = double, int STRIDE = 4>
__device__ __forceinline__ void grid_total(const T* part, const int (&slot)[NV], int nb, T (&out)[NV],
                                           T (*sh)[32]) {
  T v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = T(0);
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += __ldcg(part + b * STRIDE + slot[k]);
  block_sum<NV, T>(v, sh);
  __shared__ T bc[NV];
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) bc[k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = bc[k];
  __syncthreads();
}

// sum_k val[k] x[col[k]] over row i of a SELL-32 operator.  For WMAX > 0 the
// loads are fully unrolled and predicated so a thread issues all its column
// and value loads back to back (memory-level parallelism); WMAX = 0 loops.
template <int WMAX, bool CROSS, class T = double>
__device__ __forceinline__ T sell_row(const int64_t* __restrict__ sptr, const int* __restrict__ swidth,
                                      const int* __restrict__ colv, const T* __restrict__ val, const T* x, int i) {
  const int s = i >> 5;
  const int64_t base = sptr[s] + (i & 31);
  const int w = swidth[s];
  T acc = T(0);
  if constexpr (WMAX > 0) {
    // chunks of BD_SELL_CHUNK entries: all loads of a chunk in flight at
    // once, without holding a whole 32-wide row in registers.  Measured on
    // GB300 (TP06 257^2 sheet, 101x101x26 slab, LV shell), 2 beats 3, 4, 6
    // and 8: the solver kernels are register-bound, and longer chunks spill.
    constexpr int CH = BD_SELL_CHUNK;
    for (int k0 = 0; k0 < w; k0 += CH) {
      int c[CH];
      T v[CH], g[CH];
#pragma unroll
      for (int k = 0; k < CH; ++k)
        if (k0 + k < w) {
          c[k] = colv[base + 32 * (k0 + k)];
          v[k] = val[base + 32 * (k0 + k)];
        }
#pragma unroll
      for (int k = 0; k < CH; ++k)
        if (k0 + k < w) g[k] = CROSS ? __ldcg(x + c[k]) : x[c[k]];
#pragma unroll
      for (int k = 0; k < CH; ++k)
        if (k0 + k < w) acc += v[k] * g[k];
    }
  } else {
    for (int k = 0; k < w; ++k) {
      const int c = colv[base + 32 * k];
      acc += val[base + 32 * k] * (CROSS ? __ldcg(x + c) : x[c]);
    }
  }
  return acc;
}


// Up to NV products of operators sharing one SELL pattern, out[q] = sum_k
// val[q][k] x[q][col[k]] for every q with on[q], in one pass over the row:
// the slice header and the column indices are loaded once, and every sum is
// formed in the order sell_row forms it (bit-identical).  Vectors are read
// through L2.
template <int NV, class T = double>
__device__ __forceinline__ void sell_row_multi(const int64_t* __restrict__ sptr, const int* __restrict__ swidth,
                                               const int* __restrict__ colv, const T* const (&val)[NV],
                                               const T* const (&x)[NV], const bool (&on)[NV], int i, T (&out)[NV]) {
  const int s = i >> 5;
  const int64_t base = sptr[s] + (i & 31);
  const int w = swidth[s];
  constexpr int CH = BD_SELL_CHUNK;
#pragma unroll
  for (int q = 0; q < NV; ++q) out[q] = T(0);
  for (int k0 = 0; k0 < w; k0 += CH) {
    int c[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k0 + k < w) c[k] = colv[base + 32 * (k0 + k)];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      if (!on[q]) continue;
      T v[CH], g[CH];
#pragma unroll
      for (int k = 0; k < CH; ++k)
        if (k0 + k < w) {
          v[k] = val[q][base + 32 * (k0 + k)];
          g[k] = __ldcg(x[q] + c[k]);
        }
#pragma unroll
      for (int k = 0; k < CH; ++k)
        if (k0 + k < w) out[q] += v[k] * g[k];
    }
  }
}

template <int WMAX, bool CROSS>
__device__ __forceinline__ double sell_row(const PcgLaunch& a, const double* __restrict__ val, const double* x, int i) {
  return sell_row<WMAX, CROSS>(a.sptr, a.swidth, a.col, val, x, i);
}

}  // namespace bd
