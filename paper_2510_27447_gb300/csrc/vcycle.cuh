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

// sum_k val[k] g(col[k]) over row i of a SELL operator, entries in the same
// order as sell_row; loads issued eight at a time for memory-level parallelism
template <class T, class G>
__device__ __forceinline__ T sell_row_f(const SellDevT<T>& M, int i, G& g) {
  const int s = i >> 5;
  const int64_t base = M.sptr[s] + (i & 31);
  const int w = M.sw[s];
  T acc = T(0);
  for (int k0 = 0; k0 < w; k0 += 8) {
    int c[8];
    T v[8], gv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k0 + k < w) {
        c[k] = M.col[base + 32 * (k0 + k)];
        v[k] = M.val[base + 32 * (k0 + k)];
      }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k0 + k < w) gv[k] = g(c[k]);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k0 + k < w) acc += v[k] * gv[k];
  }
  return acc;
}

// For every row i of M: epi(i, sum_k val[k] g(col[k])) -- apply_rows with the
// gathered value given by a functor (values other threads wrote in earlier
// phases must be read through L2 inside g)
template <class T, class G, class F>
__device__ __forceinline__ void apply_rows_f(const SellDevT<T>& M, int i0, int stride, G&& g, F&& epi) {
  if (M.rp) {
    const int lane = threadIdx.x & 31;
    for (int i = i0 >> 5; i < M.n; i += stride >> 5) {
      T s = T(0);
      const int64_t e = M.rp[i + 1];
      for (int64_t p = M.rp[i] + lane; p < e; p += 32) s += M.val[p] * g(M.col[p]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) epi(i, s);
    }
  } else {
    for (int i = i0; i < M.n; i += stride) epi(i, sell_row_f<T>(M, i, g));
  }
}

// For every row i of U: epi(i, sum_k v2[k] x[col[k]], sum_k val[k] x[col[k]])
// (two operators on one pattern, one gather of x per entry)
template <class T, class F>
__device__ __forceinline__ void apply_rows2(const SellDevT<T>& M, const T* v2, const T* x, int i0, int stride,
                                            F&& epi) {
  if (M.rp) {
    const int lane = threadIdx.x & 31;
    for (int i = i0 >> 5; i < M.n; i += stride >> 5) {
      T a = T(0), b = T(0);
      const int64_t e = M.rp[i + 1];
      for (int64_t p = M.rp[i] + lane; p < e; p += 32) {
        const T xv = __ldcg(x + M.col[p]);
        a += v2[p] * xv;
        b += M.val[p] * xv;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
      if (lane == 0) epi(i, a, b);
    }
  } else {
    for (int i = i0; i < M.n; i += stride) {
      const int s = i >> 5;
      const int64_t base = M.sptr[s] + (i & 31);
      const int w = M.sw[s];
      T a = T(0), b = T(0);
      for (int k0 = 0; k0 < w; k0 += 8) {
        T xv[8], p2[8], pv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k0 + k < w) {
            const int64_t q = base + 32 * (k0 + k);
            xv[k] = __ldcg(x + M.col[q]);
            p2[k] = v2[q];
            pv[k] = M.val[q];
          }
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k0 + k < w) {
            a += p2[k] * xv[k];
            b += pv[k] * xv[k];
          }
      }
      epi(i, a, b);
    }
  }
}

// Fused V(1,1) cycle, the same operator as vcycle() below in exact arithmetic
// but with two device barriers per level instead of four.  With zero initial
// guesses the pre-smoothed iterate is x = w D^-1 b, so on the way down one
// phase per level computes, from b alone,
//   x = w D^-1 b,   r = b - A (w D^-1 b),   b_next = Q b,  Q = R (I - w A D^-1)
// (each thread recomputing the x_j of the neighbours it needs), and on the way
// up one phase per level computes prolongation and post-smoothing together,
//   y = x + P x_c + w D^-1 (r - (A P) x_c).
// b0(j) gives the level-0 right-hand side at any row j (the caller's CG
// update r - alpha q is folded in this way, saving its barrier); zhook(i, z_i)
// is called for every level-0 row of the result.  The caller must place a
// device barrier between the last writes of b0's inputs and the call.
template <class T, class B0, class Z0>
__device__ bool vcycle_fused(const AmgDevT<T>& M, B0& b0, T* zout, Z0& zhook, unsigned* bar, int nb, int* status) {
  const int stride = blockDim.x * gridDim.x;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int L = M.nlev;
  for (int l = 0; l < L; ++l) {
    const AmgLevelDevT<T>& Lv = M.L[l];
    if (l > 0 && !grid_barrier(bar, nb, status)) return false;
    const bool last = l + 1 == L;
    T* nrhs = last ? M.bc : M.L[l + 1].b;
    auto down = [&](auto& bf) {
      auto g = [&](int j) { return Lv.omega * Lv.invd[j] * bf(j); };
      apply_rows_f(Lv.A, i0, stride, g, [&](int i, T s) {
        const T bi = bf(i);
        Lv.x[i] = Lv.omega * Lv.invd[i] * bi;
        Lv.r[i] = bi - s;
      });
      apply_rows_f(Lv.Q, i0, stride, bf, [&](int k, T s) { nrhs[k] = s; });
    };
    if (l == 0) {
      down(b0);
    } else {
      auto bl = [&](int j) { return __ldcg(Lv.b + j); };
      down(bl);
    }
  }
  if (!grid_barrier(bar, nb, status)) return false;
  {
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
    const T* xc = l + 1 == L ? M.xc : M.L[l + 1].y;
    if (!grid_barrier(bar, nb, status)) return false;
    if (l == 0) {
      apply_rows2(Lv.U, Lv.uP, xc, i0, stride, [&](int i, T sp, T sap) {
        const T z = __ldcg(Lv.x + i) + sp + Lv.omega * Lv.invd[i] * (__ldcg(Lv.r + i) - sap);
        zout[i] = z;
        zhook(i, z);
      });
    } else {
      apply_rows2(Lv.U, Lv.uP, xc, i0, stride, [&](int i, T sp, T sap) {
        Lv.y[i] = __ldcg(Lv.x + i) + sp + Lv.omega * Lv.invd[i] * (__ldcg(Lv.r + i) - sap);
      });
    }
  }
  return true;
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
