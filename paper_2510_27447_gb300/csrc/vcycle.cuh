// vcycle.cuh -- one AMG V(1,1) cycle inside a persistent cooperative kernel,
// generic in the value type (FP64 for the FP64 path, FP32 for the inner
// solves of the mixed path).  See amg.cu for the cycle's definition.
#pragma once
#include "bd_internal.h"
#include "sparse.cuh"

namespace bd {

template <class T>
__device__ __forceinline__ T sdot(const SellDevT<T>& M, const T* x, int i) {
  switch (M.wmax) {
    case 8: return sell_row<8, true, T>(M.sptr, M.sw, M.col, M.val, x, i);
    case 16: return sell_row<16, true, T>(M.sptr, M.sw, M.col, M.val, x, i);
    case 32: return sell_row<32, true, T>(M.sptr, M.sw, M.col, M.val, x, i);
    default: return sell_row<0, true, T>(M.sptr, M.sw, M.col, M.val, x, i);
  }
}

// For every row i of M: epi(i, (M x)_i).  SELL operators use one thread per
// row; CSR operators (long rows) one warp per row, the lanes reading the
// row's contiguous entries and a butterfly reduction giving every lane the
// same sum (deterministic); lane 0 runs the epilogue.  x and every vector an
// epilogue reads may have been written by other threads in earlier phases,
// so they are read through L2.
template <class T, class F>
__device__ __forceinline__ void apply_rows(const SellDevT<T>& M, const T* x, int i0, int stride, F&& epi) {
  if (M.rp) {
    const int lane = threadIdx.x & 31;
    for (int i = i0 >> 5; i < M.n; i += stride >> 5) {
      T s = T(0);
      const int64_t e = M.rp[i + 1];
      for (int64_t p = M.rp[i] + lane; p < e; p += 32) s += M.val[p] * __ldcg(x + M.col[p]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) epi(i, s);
    }
  } else {
    for (int i = i0; i < M.n; i += stride) epi(i, sdot<T>(M, x, i));
  }
}

// z = V(rin); returns false if a barrier gave up
template <class T>
__device__ bool vcycle(const AmgDevT<T>& M, const T* rin, T* zout, unsigned* bar, int nb, int* status) {
  const int stride = blockDim.x * gridDim.x;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int L = M.nlev;
  {
    const AmgLevelDevT<T>& l0 = M.L[0];
    for (int i = i0; i < l0.A.n; i += stride) l0.x[i] = l0.omega * l0.invd[i] * rin[i];
  }
  for (int l = 0; l < L; ++l) {
    const AmgLevelDevT<T>& Lv = M.L[l];
    const T* b = l == 0 ? rin : Lv.b;
    if (!grid_barrier(bar, nb, status)) return false;
    apply_rows(Lv.A, Lv.x, i0, stride, [&](int i, T d) { Lv.r[i] = __ldcg(b + i) - d; });
    if (!grid_barrier(bar, nb, status)) return false;
    const bool last = l + 1 == L;
    T* nb_rhs = last ? M.bc : M.L[l + 1].b;
    apply_rows(Lv.R, Lv.r, i0, stride, [&](int i, T v) {
      nb_rhs[i] = v;
      if (!last) M.L[l + 1].x[i] = M.L[l + 1].omega * M.L[l + 1].invd[i] * v;
    });
  }
  if (!grid_barrier(bar, nb, status)) return false;
  {
    // dense coarse solve, one warp per row (lanes split the dot product)
    const int lane = threadIdx.x & 31;
    const int warp = i0 >> 5;
    const int nwarps = stride >> 5;
    for (int i = warp; i < M.nc; i += nwarps) {
      const T* row = M.cinv + int64_t(i) * M.nc;
      T s = T(0);
      for (int j = lane; j < M.nc; j += 32) s += row[j] * __ldcg(M.bc + j);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) M.xc[i] = s;
    }
  }
  for (int l = L - 1; l >= 0; --l) {
    const AmgLevelDevT<T>& Lv = M.L[l];
    const T* coarse = l + 1 == L ? M.xc : M.L[l + 1].y;
    if (!grid_barrier(bar, nb, status)) return false;
    apply_rows(Lv.P, coarse, i0, stride, [&](int i, T d) { Lv.x[i] = __ldcg(Lv.x + i) + d; });
    if (!grid_barrier(bar, nb, status)) return false;
    const T* b = l == 0 ? rin : Lv.b;
    T* y = l == 0 ? zout : Lv.y;
    apply_rows(Lv.A, Lv.x, i0, stride, [&](int i, T d) {
      y[i] = __ldcg(Lv.x + i) + Lv.omega * Lv.invd[i] * (__ldcg(b + i) - d);
    });
  }
  return true;
}

}  // namespace bd
