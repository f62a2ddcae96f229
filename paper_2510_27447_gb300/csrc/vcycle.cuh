// vcycle.cuh -- one AMG V(1,1) cycle inside a persistent cooperative kernel,
// generic in the value type (FP64 for the FP64 path, FP32 for the inner
// solves of the mixed path).  See amg.cu for the cycle's definition.
#pragma once
#include <type_traits>

#include "bd_internal.h"
#include "sparse.cuh"

namespace bd {

// row i of a SELL operator against x read through L2 (sell_row processes any
// width in chunks, so one instantiation serves every level)
template <class T>
__device__ __forceinline__ T sdot(const SellDevT<T>& M, const T* x, int i) {
  return sell_row<8, true, T>(M.sptr, M.sw, M.col, M.val, x, i);
}

// Lanes that share one row of a SELL operator: operators with few rows
// (coarse levels) spread each row over g lanes (a power of two, at most half
// the row-width bound) while the grid has threads for g lanes a row, so that
// fewer dependent load rounds sit in each lane's part of the row.
template <class T>
__device__ __forceinline__ int lanes_per_row(const SellDevT<T>& M, int stride) {
  int g = 1;
  while (g < 32 && int64_t(M.n) * (2 * g) <= int64_t(stride) && 2 * g <= M.wmax) g *= 2;
  return g;
}

// lane sub's part of row i (entries k = sub, sub + g, ...; in k order)
template <class T, int NV>
__device__ __forceinline__ void sell_row_part(const SellDevT<T>& M, const T* const (&x)[NV], int i, int sub, int g,
                                              T (&acc)[NV]) {
  const int s = i >> 5;
  const int64_t base = M.sptr[s] + (i & 31);
  const int w = M.sw[s];
  constexpr int CH = BD_SELL_CHUNK;
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = T(0);
  for (int k0 = sub; k0 < w; k0 += g * CH) {
    int c[CH];
    T v[CH], gx[NV][CH];
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k0 + g * k < w) {
        c[k] = M.col[base + 32 * (k0 + g * k)];
        v[k] = M.val[base + 32 * (k0 + g * k)];
      }
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k0 + g * k < w)
#pragma unroll
        for (int q = 0; q < NV; ++q) gx[q][k] = __ldcg(x[q] + c[k]);
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k0 + g * k < w)
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += v[k] * gx[q][k];
  }
}

// Rows of a SELL operator with g > 1 lanes a row: warp w takes rows
// [w 32/g, (w+1) 32/g) of every round (the loop is warp-uniform, so every
// lane reaches the shuffles), a butterfly over the row's lanes gives the sum
// and the row's first lane runs epi(i, sums).
template <class T, int NV, class F>
__device__ __forceinline__ void apply_rows_spread(const SellDevT<T>& M, const T* const (&x)[NV], int g, int i0,
                                                  int stride, F&& epi) {
  const int lane = threadIdx.x & 31;
  const int rpw = 32 / g;
  const int sub = lane & (g - 1);
  for (int r0 = (i0 >> 5) * rpw; r0 < M.n; r0 += (stride >> 5) * rpw) {
    const int i = r0 + lane / g;
    T acc[NV];
    if (i < M.n) {
      sell_row_part<T, NV>(M, x, i, sub, g, acc);
    } else {
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q] = T(0);
    }
    for (int o = g >> 1; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (sub == 0 && i < M.n) epi(i, acc);
  }
}

// For every row i of M: epi(i, (M x)_i).  SELL operators use one thread per
// row, or g lanes per row (lanes_per_row) where `spread` allows it; CSR
// operators (long rows) one warp per row, the lanes reading the row's
// contiguous entries and a butterfly reduction giving every lane the same sum
// (deterministic); lane 0 runs the epilogue.  x and every vector an epilogue
// reads may have been written by other threads in earlier phases, so they are
// read through L2.  `spread` is false for operators whose output the Krylov
// loop reads back row by row without a barrier (the finest level's A).
template <class T, class F>
__device__ __forceinline__ void apply_rows(const SellDevT<T>& M, const T* x, int i0, int stride, F&& epi,
                                           bool spread = true) {
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
    const int g = spread ? lanes_per_row(M, stride) : 1;
    if (g == 1) {
      for (int i = i0; i < M.n; i += stride) epi(i, sdot<T>(M, x, i));
    } else {
      const T* xs[1] = {x};
      apply_rows_spread<T, 1>(M, xs, g, i0, stride, [&](int i, const T (&a)[1]) { epi(i, a[0]); });
    }
  }
}

// For every row i of M: epi(i, (M x0)_i, (M x1)_i) -- two vectors through one
// pass over the operator (values and indices loaded once), each sum in the
// same order as sell_row's
template <class T, class F>
__device__ __forceinline__ void apply_rows_2v(const SellDevT<T>& M, const T* x0, const T* x1, int i0, int stride,
                                              F&& epi, bool spread = true) {
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
  } else if (const int g = spread ? lanes_per_row(M, stride) : 1; g > 1) {
    const T* xs[2] = {x0, x1};
    apply_rows_spread<T, 2>(M, xs, g, i0, stride, [&](int i, const T (&a)[2]) { epi(i, a[0], a[1]); });
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

// capacity (elements) of the shared-memory copy of the coarse right-hand sides
constexpr int kCoarseStage = 1536;

__device__ __forceinline__ float dot_vec(const float4& c, const float* b) {
  return c.x * b[0] + c.y * b[1] + c.z * b[2] + c.w * b[3];
}
__device__ __forceinline__ double dot_vec(const double2& c, const double* b) { return c.x * b[0] + c.y * b[1]; }

// Dense coarsest solve xc_k = Cinv bc_k (k < NV), one warp per row, the lanes
// splitting the dot product and a butterfly sum giving the row's value.  When
// a padded row fits kCoarseStage, every block that owns rows first copies the
// right-hand sides into shared memory (one round trip for all of them) and the
// warps read their rows as 16-byte vectors, up to B vectors a lane in flight
// at once; the rows are zero padded to ldc (a multiple of 4 entries, so every
// row starts 16-byte aligned).  Wider coarse operators take a lane-strided
// loop over global memory.  bc is read through L2 (written by other blocks).
template <class T, int NV>
__device__ __forceinline__ void coarse_solve(const T* cinv, int nc, int ldc, const T* const (&bc)[NV],
                                             T* const (&xc)[NV]) {
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int E = 16 / int(sizeof(T));           // entries per vector
  constexpr int B = sizeof(T) == 4 ? 4 : 2;        // vectors per lane per batch (4 measured best)
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int warp = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * wpb;
  __shared__ __align__(16) T sbc[NV][kCoarseStage];
  if (ldc <= kCoarseStage) {
    if (blockIdx.x * wpb >= nc) return;             // block-uniform: no rows here
    for (int j = threadIdx.x; j < ldc; j += blockDim.x)
#pragma unroll
      for (int k = 0; k < NV; ++k) sbc[k][j] = j < nc ? __ldcg(bc[k] + j) : T(0);
    __syncthreads();
    const int nvec = ldc / E;
    for (int i = warp; i < nc; i += nwarps) {
      const V* row = reinterpret_cast<const V*>(cinv + int64_t(i) * ldc);
      T s[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) s[k] = T(0);
      for (int q0 = lane; q0 < nvec; q0 += 32 * B) {
        V c[B];
#pragma unroll
        for (int u = 0; u < B; ++u)
          if (q0 + 32 * u < nvec) c[u] = __ldg(row + q0 + 32 * u);
#pragma unroll
        for (int u = 0; u < B; ++u)
          if (q0 + 32 * u < nvec)
#pragma unroll
            for (int k = 0; k < NV; ++k) s[k] += dot_vec(c[u], &sbc[k][(q0 + 32 * u) * E]);
      }
#pragma unroll
      for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
        if (lane == 0) xc[k][i] = s[k];
      }
    }
  } else {
    for (int i = warp; i < nc; i += nwarps) {
      const T* row = cinv + int64_t(i) * ldc;
      T s[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) s[k] = T(0);
      for (int j = lane; j < nc; j += 32) {
        const T c = row[j];
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] += c * __ldcg(bc[k] + j);
      }
#pragma unroll
      for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
        if (lane == 0) xc[k][i] = s[k];
      }
    }
  }
}

// Two V(1,1) cycles at once (z_k = V(r_k), k = 0, 1) sharing every device
// barrier and every pass over the operators.  H0 carries the operators and the
// level vectors of the first right-hand side, H1 the level vectors of the
// second (its operators are not read).  Each z_k is the cycle vcycle_body() below
// computes for r_k, with the same order of every sum.
template <class T>
__device__ __forceinline__ bool vcycle2_body(const AmgDevT<T>& H0, const AmgDevT<T>& H1, const T* r0, const T* r1,
                                             T* z0, T* z1, unsigned* bar, int nb, int* status) {
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
    }, l > 0);
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
    const T* bcs[2] = {H0.bc, H1.bc};
    T* xcs[2] = {H0.xc, H1.xc};
    coarse_solve<T, 2>(H0.cinv, H0.nc, H0.ldc, bcs, xcs);
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
    }, l > 0);
  }
  return true;
}

// z = V(rin); returns false if a barrier gave up
template <class T>
__device__ __forceinline__ bool vcycle_body(const AmgDevT<T>& M, const T* rin, T* zout, unsigned* bar, int nb,
                                            int* status) {
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
    apply_rows(Lv.A, Lv.x, i0, stride, [&](int i, T d) { Lv.r[i] = __ldcg(b + i) - d; }, l > 0);
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
    const T* bcs[1] = {M.bc};
    T* xcs[1] = {M.xc};
    coarse_solve<T, 1>(M.cinv, M.nc, M.ldc, bcs, xcs);
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
    }, l > 0);
  }
  return true;
}

// The cycles as calls: a called cycle gets the whole register budget of the
// thread for itself, where an inlined one shares it with the Krylov loop
// around it.  Measured on GB300, the call pays in the 128-register solver
// build (mixed TP06 257^2 sheet: elliptic 1.99 -> 1.88 ms per step) and
// costs a little in the 64-register build, so kernels choose with CALL.
template <class T>
__device__ __noinline__ bool vcycle_call(const AmgDevT<T>& M, const T* rin, T* zout, unsigned* bar, int nb,
                                         int* status) {
  return vcycle_body<T>(M, rin, zout, bar, nb, status);
}
template <class T>
__device__ __noinline__ bool vcycle2_call(const AmgDevT<T>& H0, const AmgDevT<T>& H1, const T* r0, const T* r1,
                                          T* z0, T* z1, unsigned* bar, int nb, int* status) {
  return vcycle2_body<T>(H0, H1, r0, r1, z0, z1, bar, nb, status);
}
template <class T, bool CALL>
__device__ __forceinline__ bool vcycle(const AmgDevT<T>& M, const T* rin, T* zout, unsigned* bar, int nb,
                                       int* status) {
  if constexpr (CALL) return vcycle_call<T>(M, rin, zout, bar, nb, status);
  else return vcycle_body<T>(M, rin, zout, bar, nb, status);
}
template <class T, bool CALL>
__device__ __forceinline__ bool vcycle2(const AmgDevT<T>& H0, const AmgDevT<T>& H1, const T* r0, const T* r1, T* z0,
                                        T* z1, unsigned* bar, int nb, int* status) {
  if constexpr (CALL) return vcycle2_call<T>(H0, H1, r0, r1, z0, z1, bar, nb, status);
  else return vcycle2_body<T>(H0, H1, r0, r1, z0, z1, bar, nb, status);
}

}  // namespace bd
