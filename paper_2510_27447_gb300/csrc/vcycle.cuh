// vcycle.cuh -- one AMG V(1,1) cycle inside a persistent cooperative kernel,
// generic in the value type (FP64 for the FP64 path, FP32 for the inner
// solves of the mixed path).  See amg.cu for the cycle's definition.
#pragma once
#include "bd_internal.h"
#include "sparse.cuh"

namespace bd {

// row i of a SELL operator against x read through L2 (sell_row processes any
// width in chunks of eight, so one instantiation serves every level)
template <class T>
__device__ __forceinline__ T sdot(const SellDevT<T>& M, const T* x, int i) {
  return sell_row<8, true, T>(M.sptr, M.sw, M.col, M.val, x, i);
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

// For every row i of M: epi(i, (M x0)_i, (M x1)_i) -- two vectors through one
// pass over the operator (values and indices loaded once), each sum in the
// same order as sell_row's
template <class T, class F>
__device__ __forceinline__ void apply_rows_2v(const SellDevT<T>& M, const T* x0, const T* x1, int i0, int stride,
                                              F&& epi) {
  if (M.rp) {
    const int lane = threadIdx.x & 31;
    for (int i = i0 >> 5; i < M.n; i += stride >> 5) {
      T a = T(0), b = T(0);
      const int64_t e = M.rp[i + 1];
      for (int64_t p = M.rp[i] + lane; p < e; p += 32) {
        const int c = M.col[p];
        const T v = M.val[p];
        a += v * __ldcg(x0 + c);
        b += v * __ldcg(x1 + c);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
      if (lane == 0) epi(i, a, b);
    }
  } else {
    constexpr int CH = BD_SELL_CHUNK;
    for (int i = i0; i < M.n; i += stride) {
      const int s = i >> 5;
      const int64_t base = M.sptr[s] + (i & 31);
      const int w = M.sw[s];
      T a = T(0), b = T(0);
      for (int k0 = 0; k0 < w; k0 += CH) {
        int c[CH];
        T v[CH], g0[CH], g1[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k)
          if (k0 + k < w) {
            c[k] = M.col[base + 32 * (k0 + k)];
            v[k] = M.val[base + 32 * (k0 + k)];
          }
#pragma unroll
        for (int k = 0; k < CH; ++k)
          if (k0 + k < w) {
            g0[k] = __ldcg(x0 + c[k]);
            g1[k] = __ldcg(x1 + c[k]);
          }
#pragma unroll
        for (int k = 0; k < CH; ++k)
          if (k0 + k < w) {
            a += v[k] * g0[k];
            b += v[k] * g1[k];
          }
      }
      epi(i, a, b);
    }
  }
}

// Two V(1,1) cycles at once (z_k = V(r_k), k = 0, 1) sharing every device
// barrier and every pass over the operators.  H0 carries the operators and the
// level vectors of the first right-hand side, H1 the level vectors of the
// second (its operators are not read).  Each z_k is the cycle vcycle() below
// computes for r_k, with the same order of every sum.
template <class T>
__device__ bool vcycle2(const AmgDevT<T>& H0, const AmgDevT<T>& H1, const T* r0, const T* r1, T* z0, T* z1,
                        unsigned* bar, int nb, int* status) {
  const int stride = blockDim.x * gridDim.x;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int L = H0.nlev;
  {
    const AmgLevelDevT<T>& l0 = H0.L[0];
    T* xa = l0.x;
    T* xb = H1.L[0].x;
    for (int i = i0; i < l0.A.n; i += stride) {
      xa[i] = l0.omega * l0.invd[i] * r0[i];
      xb[i] = l0.omega * l0.invd[i] * r1[i];
    }
  }
  for (int l = 0; l < L; ++l) {
    const AmgLevelDevT<T>& Lv = H0.L[l];
    const AmgLevelDevT<T>& Lw = H1.L[l];
    const T* ba = l == 0 ? r0 : Lv.b;
    const T* bb = l == 0 ? r1 : Lw.b;
    if (!grid_barrier(bar, nb, status)) return false;
    apply_rows_2v(Lv.A, Lv.x, Lw.x, i0, stride, [&](int i, T da, T db) {
      Lv.r[i] = __ldcg(ba + i) - da;
      Lw.r[i] = __ldcg(bb + i) - db;
    });
    if (!grid_barrier(bar, nb, status)) return false;
    const bool last = l + 1 == L;
    T* na = last ? H0.bc : H0.L[l + 1].b;
    T* nbv = last ? H1.bc : H1.L[l + 1].b;
    apply_rows_2v(Lv.R, Lv.r, Lw.r, i0, stride, [&](int i, T va, T vb) {
      na[i] = va;
      nbv[i] = vb;
      if (!last) {
        const AmgLevelDevT<T>& Nx = H0.L[l + 1];
        Nx.x[i] = Nx.omega * Nx.invd[i] * va;
        H1.L[l + 1].x[i] = Nx.omega * Nx.invd[i] * vb;
      }
    });
  }
  if (!grid_barrier(bar, nb, status)) return false;
  {
    const int lane = threadIdx.x & 31;
    const int warp = i0 >> 5;
    const int nwarps = stride >> 5;
    for (int i = warp; i < H0.nc; i += nwarps) {
      const T* row = H0.cinv + int64_t(i) * H0.nc;
      T a = T(0), b = T(0);
      for (int j = lane; j < H0.nc; j += 32) {
        const T c = row[j];
        a += c * __ldcg(H0.bc + j);
        b += c * __ldcg(H1.bc + j);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
      if (lane == 0) {
        H0.xc[i] = a;
        H1.xc[i] = b;
      }
    }
  }
  for (int l = L - 1; l >= 0; --l) {
    const AmgLevelDevT<T>& Lv = H0.L[l];
    const AmgLevelDevT<T>& Lw = H1.L[l];
    const T* ca = l + 1 == L ? H0.xc : H0.L[l + 1].y;
    const T* cb = l + 1 == L ? H1.xc : H1.L[l + 1].y;
    if (!grid_barrier(bar, nb, status)) return false;
    apply_rows_2v(Lv.P, ca, cb, i0, stride, [&](int i, T da, T db) {
      Lv.x[i] = __ldcg(Lv.x + i) + da;
      Lw.x[i] = __ldcg(Lw.x + i) + db;
    });
    if (!grid_barrier(bar, nb, status)) return false;
    const T* ba = l == 0 ? r0 : Lv.b;
    const T* bb = l == 0 ? r1 : Lw.b;
    T* ya = l == 0 ? z0 : Lv.y;
    T* yb = l == 0 ? z1 : Lw.y;
    apply_rows_2v(Lv.A, Lv.x, Lw.x, i0, stride, [&](int i, T da, T db) {
      ya[i] = __ldcg(Lv.x + i) + Lv.omega * Lv.invd[i] * (__ldcg(ba + i) - da);
      yb[i] = __ldcg(Lw.x + i) + Lv.omega * Lv.invd[i] * (__ldcg(bb + i) - db);
    });
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
