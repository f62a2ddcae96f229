// stream2.cu -- the streaming solve of two elliptic systems on one operator.
//
// From the second sweep on, Algorithm 2 solves the elliptic constraint
// A_ie u = -A_i v (Sec. 3.3.2) at two Gauss-Lobatto nodes whose transmembrane
// potentials are both known before either solve starts: two right-hand sides
// on one operator.  Two runs of the single-system chain (stream.cu) would
// stream every operator of the solve -- A_ie for the Krylov product, the
// whole AMG hierarchy for the V-cycle, A_i and A_ie in FP64 for the
// right-hand side and the refinement residual -- twice from HBM.  Here every
// kernel of the chain runs the rows of both systems: a row's column indices
// and values are loaded once and applied to both systems' vectors.
//
// Each system keeps its own vectors (the second half of the two-system
// workspaces, the second set of AMG level vectors), scalars and decisions,
// and each computes what the single-system chain computes for it, with the
// same per-row sums.  A system stops on its own; while both iterate the
// kernels take the shared-load form (mask 3), once one has stopped they run
// the other alone (mask 1 or 2).  A loop goes on while either system still
// iterates.  A kernel reads the systems' stop flags at entry; they are
// written by earlier kernels, so every block takes the same form.
//
// The reductions of both systems share one block-partial area and one atomic
// ticket (system 0's); the last block to arrive forms both systems' totals.
// Only the AMG-preconditioned, warm-started, projected or pinned elliptic
// form is built here (no extra diagonal, no rl or second operator term).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "bd_internal.h"
#include "segment.cuh"
#include "sparse.cuh"
#include "stream_rows.cuh"
#include "vcycle.cuh"

namespace bd {

namespace {

// system 1's AMG level vectors (the operators are system 0's)
template <class T>
struct LevVec {
  T *x, *b, *r, *y;
};

template <class T>
struct Pair {
  StreamLaunch a[2];              // per-system parameters; the operator fields are read from a[0]
  AmgDevT<T> H;                   // the hierarchy with system 0's level vectors
  LevVec<T> v1[kMaxAmgLevels];    // system 1's level vectors
  T *bc1, *xc1;                   // system 1's coarse right-hand side and solution
  long long* pair_acc;            // inner iterations in which both systems advanced
  long long* pair64_acc;          // FP64 operator passes shared by both systems
  long long* pairc_acc;           // first V-cycles of an inner solve shared by both systems
};

template <class T>
__device__ __forceinline__ LevVec<T> lev(const Pair<T>& P, int k, int l) {
  if (k == 0) {
    const AmgLevelDevT<T>& L = P.H.L[l];
    return LevVec<T>{L.x, L.b, L.r, L.y};
  }
  return P.v1[l];
}

// The systems a kernel runs: mask 1 (system 0), 2 (system 1) or 3 (both);
// f is called with the mask as a compile-time constant, or not at all.
template <int M>
using Mask = std::integral_constant<int, M>;
template <class F>
__device__ __forceinline__ void by_mask(bool on0, bool on1, F&& f) {
  if (on0 && on1) f(Mask<3>{});
  else if (on0) f(Mask<1>{});
  else if (on1) f(Mask<2>{});
}
#define MASK_OF(m) constexpr int M = decltype(m)::value
#define ON(k) (((M) >> (k)) & 1)

// loop conditions of the pair: the inner loop ends when neither system
// iterates; the outer decision sets both loops
__device__ __forceinline__ void pair_vote_inner(const StreamLaunch& a, bool any) {
  if (!a.host_loop && !any) set_cond(a.h_inner, 0u);
}
__device__ __forceinline__ void pair_vote_outer(const StreamLaunch& a, bool inner_on, bool outer_on) {
  if (a.host_loop) return;
  set_cond(a.h_inner, inner_on ? 1u : 0u);
  set_cond(a.h_outer, outer_on ? 1u : 0u);
}

// ---- row products for the systems of mask M ---------------------------------
//
// acc[k] = sum_j val[j] x_k[col[j]] over a row, for k in M: the entries are
// loaded once, and each system's sum is formed in the order the single-system
// product (srow / srow4 / level_rows) forms it.

// PIPE: the next chunk's indices and values are requested before this
// chunk's gathers (two chunks of the operator stream in flight) -- faster for
// the FP64 products of the right-hand side and the refinement residual,
// slower for the FP32 level products, whose extra registers cost occupancy
template <int M, bool STREAMOP, class V, class X, bool PIPE = false>
__device__ __forceinline__ void srow_m(const int64_t* __restrict__ sptr, const int* __restrict__ sw,
                                       const int* __restrict__ col, const V* __restrict__ val,
                                       const X* __restrict__ x0, const X* __restrict__ x1, int i, X (&acc)[2]) {
  const int s = i >> 5;
  const int64_t base = sptr[s] + (i & 31);
  const int w = sw[s];
  acc[0] = X(0);
  acc[1] = X(0);
  constexpr int CH = 4;
  int c[CH];
  V v[CH];
  auto load = [&](int k0, int (&cc)[CH], V (&vv)[CH]) {
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k0 + k < w) {
        const int64_t e = base + 32 * (k0 + k);
        cc[k] = STREAMOP ? ld_stream(col + e) : __ldg(col + e);
        vv[k] = STREAMOP ? ld_stream(val + e) : __ldg(val + e);
      }
  };
  if (PIPE) load(0, c, v);
  for (int k0 = 0; k0 < w; k0 += CH) {
    int cn[CH];
    V vn[CH];
    if (!PIPE) load(k0, c, v);
    else if (k0 + CH < w) load(k0 + CH, cn, vn);
    X g0[CH], g1[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k0 + k < w) {
        if (ON(0)) g0[k] = __ldg(x0 + c[k]);
        if (ON(1)) g1[k] = __ldg(x1 + c[k]);
      }
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k0 + k < w) {
        if (ON(0)) acc[0] += X(v[k]) * g0[k];
        if (ON(1)) acc[1] += X(v[k]) * g1[k];
      }
    if (PIPE)
#pragma unroll
      for (int k = 0; k < CH; ++k) {
        c[k] = cn[k];
        v[k] = vn[k];
      }
  }
}

// the same over the SELL-32/4 copy of an FP32 operator (see srow4): one
// 4-entry group in flight per system while both run, two while one runs
template <int M, bool STREAMOP, class X>
__device__ __forceinline__ void srow4_m(const int64_t* __restrict__ sptr4, const int* __restrict__ sw,
                                        const int* __restrict__ col4, const float* __restrict__ val4,
                                        const X* __restrict__ x0, const X* __restrict__ x1, int i, X (&acc)[2]) {
  if constexpr (M != 3) {
    const X* x = ON(0) ? x0 : x1;
    acc[ON(0) ? 0 : 1] = srow4<X, STREAMOP>(sptr4, sw, col4, val4, x, i);
    acc[ON(0) ? 1 : 0] = X(0);
    return;
  } else {
    const int s = i >> 5;
    const int64_t base = sptr4[s] + 4 * (i & 31);
    const int w = sw[s];
    acc[0] = X(0);
    acc[1] = X(0);
    for (int k0 = 0; k0 < w; k0 += 4) {
      const int4 c = ld4i<STREAMOP>(col4 + base + 32 * k0);
      const float4 v = ld4f<STREAMOP>(val4 + base + 32 * k0);
      const X g0 = __ldg(x0 + c.x), g1 = __ldg(x0 + c.y), g2 = __ldg(x0 + c.z), g3 = __ldg(x0 + c.w);
      const X h0 = __ldg(x1 + c.x), h1 = __ldg(x1 + c.y), h2 = __ldg(x1 + c.z), h3 = __ldg(x1 + c.w);
      acc[0] += X(v.x) * g0;
      acc[0] += X(v.y) * g1;
      acc[0] += X(v.z) * g2;
      acc[0] += X(v.w) * g3;
      acc[1] += X(v.x) * h0;
      acc[1] += X(v.y) * h1;
      acc[1] += X(v.z) * h2;
      acc[1] += X(v.w) * h3;
    }
  }
}

// every row i of an AMG-level operator for the systems of mask M (the forms
// and their choice as in level_rows): epi(i, ax), ax[k] = (Mx x_k)_i
template <class T, int K, int M, class F>
__device__ __forceinline__ void level_rows_m(const SellDevT<T>& A, const T* x0, const T* x1, bool streamop, SegInfo sg,
                                             F&& epi) {
  const int gt = sg.lb * blockDim.x + threadIdx.x;
  const int gs = sg.nb * blockDim.x;
  T ax[2];
  if constexpr (K == kRowsSellStream) {
    if constexpr (sizeof(T) == 4) {
      if (A.col4) {
        for (int i = gt; i < A.n; i += gs) {
          srow4_m<M, true, T>(A.sptr4, A.sw, A.col4, A.val4, x0, x1, i, ax);
          epi(i, ax);
        }
        return;
      }
    }
    for (int i = gt; i < A.n; i += gs) {
      srow_m<M, true, T, T>(A.sptr, A.sw, A.col, A.val, x0, x1, i, ax);
      epi(i, ax);
    }
    return;
  }
  if ((K & kRowsCsrBlock) && A.rp && A.lpr > 32) {
    // a block per row: both systems' sums in one block reduction
    __shared__ T shb[2][32];
    for (int i = sg.lb; i < A.n; i += sg.nb) {
      const int64_t e = __ldg(A.rp + i + 1);
      T v[2] = {T(0), T(0)};
      for (int64_t p = __ldg(A.rp + i) + threadIdx.x; p < e; p += blockDim.x) {
        const T a = __ldg(A.val + p);
        const int c = __ldg(A.col + p);
        if (ON(0)) v[0] += a * __ldg(x0 + c);
        if (ON(1)) v[1] += a * __ldg(x1 + c);
      }
      block_sum<2, T>(v, shb);
      if (threadIdx.x == 0) epi(i, v);
    }
  } else if ((K & kRowsCsrLanes) && A.rp) {
    // L lanes per row, four entries L apart in flight per lane (as level_rows)
    const int L = A.lpr > 0 ? A.lpr : 32;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (L - 1);
    const int rows_per_warp = 32 / L;
    const int grp = lane / L;
    const int step = (gs >> 5) * rows_per_warp;
    int base = (gt >> 5) * rows_per_warp;
    int i = base + grp;
    int64_t pb = 0, pe = 0;
    if (i < A.n) {
      pb = __ldg(A.rp + i);
      pe = __ldg(A.rp + i + 1);
    }
    for (; base < A.n; base += step) {
      const int inext = i + step;
      int64_t nb = 0, ne = 0;
      if (inext < A.n) {
        nb = __ldg(A.rp + inext);
        ne = __ldg(A.rp + inext + 1);
      }
      T s[2][4] = {{T(0), T(0), T(0), T(0)}, {T(0), T(0), T(0), T(0)}};
      for (int64_t p = pb + sub; p < pe; p += 4 * L) {
        int c[4];
        T v[4];
        c[0] = __ldg(A.col + p);
        v[0] = __ldg(A.val + p);
#pragma unroll
        for (int u = 1; u < 4; ++u) {
          const bool in = p + u * L < pe;   // past the row: its first column, value 0
          c[u] = in ? __ldg(A.col + p + u * L) : c[0];
          v[u] = in ? __ldg(A.val + p + u * L) : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (ON(0)) s[0][u] += v[u] * __ldg(x0 + c[u]);
          if (ON(1)) s[1][u] += v[u] * __ldg(x1 + c[u]);
        }
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        T t = (s[k][0] + s[k][1]) + (s[k][2] + s[k][3]);
        for (int o = L >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        ax[k] = t;
      }
      if (sub == 0 && i < A.n) epi(i, ax);
      i = inext;
      pb = nb;
      pe = ne;
    }
  } else if ((K & kRowsSellStream) && streamop) {
    if constexpr (sizeof(T) == 4) {
      if (A.col4) {
        for (int i = gt; i < A.n; i += gs) {
          srow4_m<M, true, T>(A.sptr4, A.sw, A.col4, A.val4, x0, x1, i, ax);
          epi(i, ax);
        }
        return;
      }
    }
    for (int i = gt; i < A.n; i += gs) {
      srow_m<M, true, T, T>(A.sptr, A.sw, A.col, A.val, x0, x1, i, ax);
      epi(i, ax);
    }
  } else {
    if constexpr (sizeof(T) == 4) {
      if (A.col4) {
        for (int i = gt; i < A.n; i += gs) {
          srow4_m<M, false, T>(A.sptr4, A.sw, A.col4, A.val4, x0, x1, i, ax);
          epi(i, ax);
        }
        return;
      }
    }
    for (int i = gt; i < A.n; i += gs) {
      srow_m<M, false, T, T>(A.sptr, A.sw, A.col, A.val, x0, x1, i, ax);
      epi(i, ax);
    }
  }
}

// ---- kernels -------------------------------------------------------------------

#define PAIR_BEGIN(P)                                    \
  count_launch(P.a[0].launch_acc);                       \
  const SegInfo sg{0, int(blockIdx.x), int(gridDim.x)};  \
  const int gt = int(blockIdx.x) * blockDim.x + threadIdx.x; \
  const int gs = int(gridDim.x) * blockDim.x;            \
  const StreamLaunch& a = P.a[0];

// b_k = c1 A_i va_k in FP64 (one pass over A_i for both), a cold start's
// x = 0; the last block sets both solves up
template <class T>
__global__ void __launch_bounds__(kSB) st2_rhs_kernel(const __grid_constant__ Pair<T> P) {
  PAIR_BEGIN(P)
  if (a.gate && *a.gate == 0) {        // the sweep test closed both solves (uniform)
    if (blockIdx.x == 0 && threadIdx.x == 0) P.a[0].sc->skip = P.a[1].sc->skip = 1;
    return;
  }
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = gt; i < a.n; i += gs) {
    double sp[2];
    srow_m<3, true, double, double, true>(a.sptr, a.swidth, a.col, a.val1, P.a[0].va, P.a[1].va, i, sp);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const StreamLaunch& ak = P.a[k];
      const double b = ak.c1 * sp[k];
      ak.b64[i] = b;
      if (!ak.warm) ak.x[i] = 0.0;
      acc[2 * k] += b;
      acc[2 * k + 1] += b * b;
    }
  }
  if (last_block_total<4, double>(acc, a.part, &a.sc->ticket, sg) && threadIdx.x == 0) {
    rhs_setup(P.a[0], acc[0], acc[1]);
    rhs_setup(P.a[1], acc[2], acc[3]);
    if (P.pair64_acc) atomicAdd(reinterpret_cast<unsigned long long*>(P.pair64_acc), 1ull);
  }
}

// FP64 outer residuals r_k = b_k - mean_k - A x_k and the outer decisions.  A
// system runs a pass while it has not failed and still wants one (its first
// pass, or more = 1 from its last decision).
template <class T>
__global__ void __launch_bounds__(kSB) st2_outer_kernel(const __grid_constant__ Pair<T> P) {
  PAIR_BEGIN(P)
  bool on[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const StreamScal& c = *P.a[k].sc;
    on[k] = !c.skip && !c.fail && (c.outer == 0 || c.more);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int k = 0; k < 2; ++k)
      if (!on[k]) {
        StreamScal& c = *P.a[k].sc;
        c.inner_ran = 0;
        c.stop = 1;
        c.more = 0;
      }
  if (!on[0] && !on[1]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) pair_vote_outer(a, false, false);
    return;
  }
  double acc[2] = {0.0, 0.0};
  by_mask(on[0], on[1], [&](auto m) {
    MASK_OF(m);
    const double mean[2] = {P.a[0].sc->mean_b, P.a[1].sc->mean_b};
    for (int i = gt; i < a.n; i += gs) {
      double ax[2];
      srow_m<M, true, double, double, true>(a.sptr, a.swidth, a.col, a.valA, P.a[0].x, P.a[1].x, i, ax);
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (ON(k)) {
          double r = P.a[k].b64[i] - mean[k];
          r -= ax[k];
          P.a[k].r64[i] = r;
          acc[k] += r * r;
        }
    }
  });
  if (last_block_total<2, double>(acc, a.part, &a.sc->ticket, sg) && threadIdx.x == 0) {
    bool inner = false, outer = false;
    for (int k = 0; k < 2; ++k)
      if (on[k] && outer_decide<T>(P.a[k], acc[k])) {
        inner = true;
        outer = outer || P.a[k].max_outer > 1;
      }
    if (on[0] && on[1] && P.pair64_acc) atomicAdd(reinterpret_cast<unsigned long long*>(P.pair64_acc), 1ull);
    pair_vote_outer(a, inner, outer);
  }
}

// inner start: r_k = r64_k / |r_k|, d_k = 0, the level-0 pre-smoothing
template <class T>
__global__ void __launch_bounds__(kSB) st2_inner_init_kernel(const __grid_constant__ Pair<T> P) {
  PAIR_BEGIN(P)
  const bool on0 = !P.a[0].sc->stop, on1 = !P.a[1].sc->stop;
  if (!on0 && !on1) return;
  const T* invd0 = static_cast<const T*>(a.h0_invd);
  const T omega0 = T(a.h0_omega);
  T acc[2] = {T(0), T(0)};
  by_mask(on0, on1, [&](auto m) {
    MASK_OF(m);
    const double inv_scale[2] = {1.0 / P.a[0].sc->scale, 1.0 / P.a[1].sc->scale};
    for (int i = gt; i < a.n; i += gs) {
      const T w = omega0 * invd0[i];
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (ON(k)) {
          const StreamLaunch& ak = P.a[k];
          const T ri = T(ak.r64[i] * inv_scale[k]);
          static_cast<T*>(ak.r)[i] = ri;
          static_cast<T*>(ak.d)[i] = T(0);
          acc[k] += ri * ri;
          static_cast<T*>(ak.h0_x)[i] = w * ri;
        }
    }
  });
  if (last_block_total<2, T>(acc, a.part, &a.sc->ticket, sg) && threadIdx.x == 0) {
    if (on0) P.a[0].sc->rr_new = double(acc[0]);
    if (on1) P.a[1].sc->rr_new = double(acc[1]);
    if (on0 && on1 && P.pairc_acc) atomicAdd(reinterpret_cast<unsigned long long*>(P.pairc_acc), 1ull);
  }
}

// p_k = z_k + beta_k p_k, q_k = A z_k + beta_k q_k, p_k.q_k and alpha_k
template <class T>
__global__ void __launch_bounds__(kSB) st2_pq_kernel(const __grid_constant__ Pair<T> P) {
  PAIR_BEGIN(P)
  const bool on0 = !P.a[0].sc->stop, on1 = !P.a[1].sc->stop;
  if (!on0 && !on1) return;
  T acc[2] = {T(0), T(0)};
  by_mask(on0, on1, [&](auto m) {
    MASK_OF(m);
    const T* z[2] = {static_cast<const T*>(P.a[0].z), static_cast<const T*>(P.a[1].z)};
    const bool first[2] = {P.a[0].sc->it == 0, P.a[1].sc->it == 0};
    const T beta[2] = {T(P.a[0].sc->beta), T(P.a[1].sc->beta)};
    const bool v4 = sizeof(T) == 4 && a.col4 != nullptr;
    for (int i = gt; i < a.n; i += gs) {
      T zi[2], az[2], pv[2], qv[2];   // the row's vector entries, requested before its products
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (ON(k)) {
          zi[k] = z[k][i];
          pv[k] = first[k] ? T(0) : static_cast<const T*>(P.a[k].p)[i];
          qv[k] = first[k] ? T(0) : static_cast<const T*>(P.a[k].q)[i];
        }
      if (v4) {
        float azf[2];
        srow4_m<M, true, float>(a.sptr4, a.sw4, a.col4, static_cast<const float*>(a.valT4),
                                reinterpret_cast<const float*>(z[0]), reinterpret_cast<const float*>(z[1]), i, azf);
        az[0] = T(azf[0]);
        az[1] = T(azf[1]);
      } else {
        srow_m<M, true, T, T>(a.sptr, a.swidth, a.col, static_cast<const T*>(a.valT), z[0], z[1], i, az);
      }
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (ON(k)) {
          T* p = static_cast<T*>(P.a[k].p);
          T* q = static_cast<T*>(P.a[k].q);
          const T pi = first[k] ? zi[k] : zi[k] + beta[k] * pv[k];
          const T qi = first[k] ? az[k] : az[k] + beta[k] * qv[k];
          p[i] = pi;
          q[i] = qi;
          acc[k] += pi * qi;
        }
    }
  });
  if (last_block_total<2, T>(acc, a.part, &a.sc->ticket, sg) && threadIdx.x == 0) {
    const bool go0 = on0 && pq_decide<T>(P.a[0], acc[0]);
    const bool go1 = on1 && pq_decide<T>(P.a[1], acc[1]);
    if (go0 && go1 && P.pair_acc) atomicAdd(reinterpret_cast<unsigned long long*>(P.pair_acc), 1ull);
    pair_vote_inner(a, go0 || go1);
  }
}

// d_k += alpha_k p_k, r_k -= alpha_k q_k, |r_k|^2, the level-0 pre-smoothing
template <class T>
__global__ void __launch_bounds__(kSB) st2_update_kernel(const __grid_constant__ Pair<T> P) {
  PAIR_BEGIN(P)
  const bool on0 = !P.a[0].sc->stop, on1 = !P.a[1].sc->stop;
  if (!on0 && !on1) return;
  const T* invd0 = static_cast<const T*>(a.h0_invd);
  const T omega0 = T(a.h0_omega);
  T acc[2] = {T(0), T(0)};
  by_mask(on0, on1, [&](auto m) {
    MASK_OF(m);
    const T alpha[2] = {T(P.a[0].sc->alpha), T(P.a[1].sc->alpha)};
    for (int i = gt; i < a.n; i += gs) {
      const T w = omega0 * invd0[i];
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (ON(k)) {
          const StreamLaunch& ak = P.a[k];
          T* r = static_cast<T*>(ak.r);
          T* d = static_cast<T*>(ak.d);
          d[i] += alpha[k] * static_cast<const T*>(ak.p)[i];
          const T ri = r[i] - alpha[k] * static_cast<const T*>(ak.q)[i];
          r[i] = ri;
          acc[k] += ri * ri;
          static_cast<T*>(ak.h0_x)[i] = w * ri;
        }
    }
  });
  if (last_block_total<2, T>(acc, a.part, &a.sc->ticket, sg) && threadIdx.x == 0) {
    if (on0) P.a[0].sc->rr_new = double(acc[0]);
    if (on1) P.a[1].sc->rr_new = double(acc[1]);
  }
}

// ---- V(1,1) cycle for both systems, one kernel per phase and level ---------

#define PAIR_VC_BEGIN(P)                                        \
  count_launch(P.a[0].launch_acc);                              \
  const SegInfo sg{0, int(blockIdx.x), int(gridDim.x)};         \
  const bool on0 = !P.a[0].sc->stop, on1 = !P.a[1].sc->stop;    \
  const AmgDevT<T>& H = P.H;

// r_l = b_l - A_l x_l (level 0: b = the inner residual, A_0 = the operator)
template <class T, bool L0>
__global__ void __launch_bounds__(kSB) st2_vc_res_kernel(const __grid_constant__ Pair<T> P, int l) {
  PAIR_VC_BEGIN(P)
  if ((!on0 && !on1) || l >= H.nlev) return;
  const AmgLevelDevT<T>& L = H.L[l];
  const LevVec<T> v[2] = {lev(P, 0, l), lev(P, 1, l)};
  by_mask(on0, on1, [&](auto m) {
    MASK_OF(m);
    if constexpr (L0) {
      const T* b[2] = {static_cast<const T*>(P.a[0].r), static_cast<const T*>(P.a[1].r)};
      const StreamLaunch& a = P.a[0];
      auto epi = [&](int i, const T (&ax)[2]) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (ON(k)) v[k].r[i] = b[k][i] - ax[k];
      };
      if (sizeof(T) == 4 && a.col4) {
        T ax[2];
        for (int i = sg.lb * blockDim.x + threadIdx.x; i < L.A.n; i += sg.nb * blockDim.x) {
          float axf[2];
          srow4_m<M, true, float>(a.sptr4, a.sw4, a.col4, static_cast<const float*>(a.valT4),
                                  reinterpret_cast<const float*>(v[0].x), reinterpret_cast<const float*>(v[1].x), i,
                                  axf);
          ax[0] = T(axf[0]);
          ax[1] = T(axf[1]);
          epi(i, ax);
        }
        return;
      }
      level_rows_m<T, kRowsSellStream, M>(L.A, v[0].x, v[1].x, true, sg, epi);
    } else {
      level_rows_m<T, kRowsCoarse, M>(L.A, v[0].x, v[1].x, false, sg, [&](int i, const T (&ax)[2]) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (ON(k)) v[k].r[i] = v[k].b[i] - ax[k];
      });
    }
  });
}

// b_{l+1} = R_l r_l and the next level's pre-smoothing x_{l+1} = w D^-1 b_{l+1}
template <class T, int K>
__global__ void __launch_bounds__(kSB) st2_vc_restrict_kernel(const __grid_constant__ Pair<T> P, int l) {
  PAIR_VC_BEGIN(P)
  if ((!on0 && !on1) || l >= H.nlev) return;
  const AmgLevelDevT<T>& L = H.L[l];
  const bool last = l + 1 == H.nlev;
  T* bn[2];
  T* xn[2];
  for (int k = 0; k < 2; ++k) {
    if (last) {
      bn[k] = k == 0 ? H.bc : P.bc1;
      xn[k] = nullptr;
    } else {
      const LevVec<T> vn = lev(P, k, l + 1);
      bn[k] = vn.b;
      xn[k] = vn.x;
    }
  }
  const T* invdn = last ? nullptr : H.L[l + 1].invd;
  const T omegan = last ? T(0) : H.L[l + 1].omega;
  const T* r0 = lev(P, 0, l).r;
  const T* r1 = lev(P, 1, l).r;
  by_mask(on0, on1, [&](auto m) {
    MASK_OF(m);
    level_rows_m<T, K, M>(L.R, r0, r1, l == 0, sg, [&](int i, const T (&bv)[2]) {
      const T w = last ? T(0) : omegan * invdn[i];
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (ON(k)) {
          bn[k][i] = bv[k];
          if (!last) xn[k][i] = w * bv[k];
        }
    });
  });
}

// dense coarsest solves xc_k = Cinv bc_k: one warp per row of the coarse
// inverse, which is read once for both right-hand sides (staged in shared
// memory when a padded row fits)
template <class T>
__global__ void __launch_bounds__(kSB) st2_vc_coarse_kernel(const __grid_constant__ Pair<T> P) {
  PAIR_VC_BEGIN(P)
  if ((!on0 && !on1) || H.nlev == 0) return;
  using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int E = 16 / int(sizeof(T));
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int nvec = H.ldc / E;
  if (sg.lb * wpb >= H.nc) return;                 // no rows in this block (uniform)
  const T* bc[2] = {H.bc, P.bc1};
  T* xc[2] = {H.xc, P.xc1};
  __shared__ __align__(16) T sbc[2][kCoarseStage];
  const bool staged = H.ldc <= kCoarseStage;
  by_mask(on0, on1, [&](auto m) {
    MASK_OF(m);
    if (staged) {
      for (int j = threadIdx.x; j < H.ldc; j += blockDim.x)
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (ON(k)) sbc[k][j] = j < H.nc ? __ldcg(bc[k] + j) : T(0);
      __syncthreads();
    }
    for (int i = sg.lb * wpb + (threadIdx.x >> 5); i < H.nc; i += sg.nb * wpb) {
      const VT* row = reinterpret_cast<const VT*>(H.cinv + int64_t(i) * H.ldc);
      T s[2] = {T(0), T(0)};
      for (int q = lane; q < nvec; q += 32) {
        const VT cv = __ldg(row + q);
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (ON(k)) {
            if (staged) {
              s[k] += dot_vec(cv, &sbc[k][q * E]);
            } else {
              T bq[E];
#pragma unroll
              for (int u = 0; u < E; ++u) {
                const int j = q * E + u;
                bq[u] = j < H.nc ? __ldcg(bc[k] + j) : T(0);
              }
              s[k] += dot_vec(cv, bq);
            }
          }
      }
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (ON(k)) {
          T t = s[k];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          if (lane == 0) xc[k][i] = t;
        }
    }
  });
}

// x_l += P_l y_{l+1}
template <class T>
__global__ void __launch_bounds__(kSB) st2_vc_prolong_kernel(const __grid_constant__ Pair<T> P, int l) {
  PAIR_VC_BEGIN(P)
  if ((!on0 && !on1) || l >= H.nlev) return;
  const AmgLevelDevT<T>& L = H.L[l];
  const bool last = l + 1 == H.nlev;
  const T* y0 = last ? H.xc : lev(P, 0, l + 1).y;
  const T* y1 = last ? P.xc1 : lev(P, 1, l + 1).y;
  T* x[2] = {lev(P, 0, l).x, lev(P, 1, l).x};
  by_mask(on0, on1, [&](auto m) {
    MASK_OF(m);
    level_rows_m<T, kRowsAll & ~kRowsCsrBlock, M>(L.P, y0, y1, l == 0, sg, [&](int i, const T (&pv)[2]) {
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (ON(k)) x[k][i] += pv[k];
    });
  });
}

// y_l = x_l + w D^-1 (b_l - A_l x_l); on level 0 y is z_k, r_k.z_k and the
// inner decisions
template <class T, bool L0>
__global__ void __launch_bounds__(kSB) st2_vc_post_kernel(const __grid_constant__ Pair<T> P, int l) {
  PAIR_VC_BEGIN(P)
  if (!on0 && !on1) return;
  const AmgLevelDevT<T>& L = H.L[l];
  const LevVec<T> v[2] = {lev(P, 0, l), lev(P, 1, l)};
  const T* b[2];
  T* y[2];
  for (int k = 0; k < 2; ++k) {
    b[k] = L0 ? static_cast<const T*>(P.a[k].r) : v[k].b;
    y[k] = L0 ? static_cast<T*>(P.a[k].z) : v[k].y;
  }
  T acc[2] = {T(0), T(0)};
  by_mask(on0, on1, [&](auto m) {
    MASK_OF(m);
    auto post = [&](int i, const T (&ax)[2]) {
      const T w = L.omega * L.invd[i];
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (ON(k)) {
          const T bi = b[k][i];
          const T yi = v[k].x[i] + w * (bi - ax[k]);
          y[k][i] = yi;
          acc[k] += bi * yi;
        }
    };
    if constexpr (L0) {
      const StreamLaunch& a = P.a[0];
      if (sizeof(T) == 4 && a.col4) {
        T ax[2];
        for (int i = sg.lb * blockDim.x + threadIdx.x; i < L.A.n; i += sg.nb * blockDim.x) {
          float axf[2];
          srow4_m<M, true, float>(a.sptr4, a.sw4, a.col4, static_cast<const float*>(a.valT4),
                                  reinterpret_cast<const float*>(v[0].x), reinterpret_cast<const float*>(v[1].x), i,
                                  axf);
          ax[0] = T(axf[0]);
          ax[1] = T(axf[1]);
          post(i, ax);
        }
      } else {
        level_rows_m<T, kRowsSellStream, M>(L.A, v[0].x, v[1].x, true, sg, post);
      }
    } else {
      level_rows_m<T, kRowsCoarse, M>(L.A, v[0].x, v[1].x, false, sg, post);
    }
  });
  if constexpr (L0) {
    if (last_block_total<2, T>(acc, P.a[0].part, &P.a[0].sc->ticket, sg) && threadIdx.x == 0) {
      const bool go0 = on0 && inner_decide<T>(P.a[0], acc[0]);
      const bool go1 = on1 && inner_decide<T>(P.a[1], acc[1]);
      pair_vote_inner(P.a[0], go0 || go1);
    }
  }
}

// x_k += |r_k| d_k after an inner solve of system k that ran without failure
template <class T>
__global__ void __launch_bounds__(kSB) st2_xupdate_kernel(const __grid_constant__ Pair<T> P) {
  PAIR_BEGIN(P)
  const StreamScal& c0 = *P.a[0].sc;
  const StreamScal& c1 = *P.a[1].sc;
  by_mask(c0.inner_ran && !c0.fail, c1.inner_ran && !c1.fail, [&](auto m) {
    MASK_OF(m);
    const double s[2] = {c0.scale, c1.scale};
    for (int i = gt; i < a.n; i += gs)
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (ON(k)) P.a[k].x[i] += s[k] * double(static_cast<const T*>(P.a[k].d)[i]);
  });
}

// normalisation of the singular elliptic solutions: the shifts (u_k[pin], or
// the nodal means); the pin is the handle's, the same for both systems
template <class T>
__global__ void __launch_bounds__(kSB) st2_shift_kernel(const __grid_constant__ Pair<T> P) {
  PAIR_BEGIN(P)
  const bool on0 = !P.a[0].sc->skip, on1 = !P.a[1].sc->skip;
  if ((!on0 && !on1) || a.pin < -1) return;
  if (a.pin >= 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0)
      for (int k = 0; k < 2; ++k)
        if (!P.a[k].sc->skip) P.a[k].sc->shift = P.a[k].x[a.pin];
    return;
  }
  double acc[2] = {0.0, 0.0};
  by_mask(on0, on1, [&](auto m) {
    MASK_OF(m);
    for (int i = gt; i < a.n; i += gs)
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (ON(k)) acc[k] += P.a[k].x[i];
  });
  if (last_block_total<2, double>(acc, a.part, &a.sc->ticket, sg) && threadIdx.x == 0) {
    if (on0) P.a[0].sc->shift = acc[0] / double(a.n);
    if (on1) P.a[1].sc->shift = acc[1] / double(a.n);
  }
}

// x_k -= shift_k; each solve's status and counters
template <class T>
__global__ void __launch_bounds__(kSB) st2_finish_kernel(const __grid_constant__ Pair<T> P) {
  PAIR_BEGIN(P)
  const StreamScal& c0 = *P.a[0].sc;
  const StreamScal& c1 = *P.a[1].sc;
  if (a.pin >= -1)
    by_mask(!c0.skip, !c1.skip, [&](auto m) {
      MASK_OF(m);
      const double sh[2] = {c0.shift, c1.shift};
      for (int i = gt; i < a.n; i += gs)
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (ON(k)) P.a[k].x[i] -= sh[k];
    });
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int k = 0; k < 2; ++k) {
      const StreamLaunch& ak = P.a[k];
      const StreamScal& c = *ak.sc;
      if (c.skip) continue;
      if (c.fail) atomicOr(ak.status, c.fail);
      if (ak.iters_acc) atomicAdd(reinterpret_cast<unsigned long long*>(ak.iters_acc), (unsigned long long)c.inner_total);
      if (ak.outer_acc) atomicAdd(reinterpret_cast<unsigned long long*>(ak.outer_acc), (unsigned long long)c.outer_total);
      if (ak.solves_acc) atomicAdd(reinterpret_cast<unsigned long long*>(ak.solves_acc), 1ull);
    }
}

// ---- host side ------------------------------------------------------------------

// the pair's launches: its parameters and the grid-stride threads of each
// kernel family (grids from stream_fit)
template <class T>
struct PairPlan {
  Pair<T> P{};
  int nlev = 0;
  int64_t rows = 1, tcoarse = 1;
  int64_t tA[kMaxAmgLevels] = {}, tR[kMaxAmgLevels] = {}, tP[kMaxAmgLevels] = {};
};

#define PAIR_LAUNCH(KNAME, threads, stream, ...) \
  KNAME<<<stream_fit((const void*)KNAME, threads), kSB, 0, stream>>>(__VA_ARGS__)

template <class T>
void enqueue_vcycle2(const PairPlan<T>& Q, cudaStream_t s) {
  const Pair<T>& P = Q.P;
  for (int l = 0; l < Q.nlev; ++l) {
    if (l == 0) PAIR_LAUNCH((st2_vc_res_kernel<T, true>), Q.tA[l], s, P, l);
    else PAIR_LAUNCH((st2_vc_res_kernel<T, false>), Q.tA[l], s, P, l);
    if (P.H.L[l].R.lpr > 32) PAIR_LAUNCH((st2_vc_restrict_kernel<T, kRowsAll>), Q.tR[l], s, P, l);
    else PAIR_LAUNCH((st2_vc_restrict_kernel<T, kRowsAll & ~kRowsCsrBlock>), Q.tR[l], s, P, l);
  }
  PAIR_LAUNCH(st2_vc_coarse_kernel<T>, Q.tcoarse, s, P);
  for (int l = Q.nlev - 1; l >= 0; --l) {
    PAIR_LAUNCH(st2_vc_prolong_kernel<T>, Q.tP[l], s, P, l);
    if (l == 0) PAIR_LAUNCH((st2_vc_post_kernel<T, true>), Q.rows, s, P, l);
    else PAIR_LAUNCH((st2_vc_post_kernel<T, false>), Q.tA[l], s, P, l);
  }
}

// the pair's kernels and loops, appended to the capture of `st` (the loop
// structure of the single-system solve)
template <class T>
cudaError_t enqueue_pair(PairPlan<T>& Q, cudaStream_t st, const cudaStream_t* side) {
  cudaGraph_t g = stream_capture_graph(st);
  if (!g) return cudaErrorStreamCaptureUnsupported;
  cudaGraphConditionalHandle ho, hi;
  cudaError_t e = cudaGraphConditionalHandleCreate(&ho, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hi, g, 0, 0);
  if (e != cudaSuccess) return e;
  for (StreamLaunch& a : Q.P.a) {
    a.h_outer = static_cast<unsigned long long>(ho);
    a.h_inner = static_cast<unsigned long long>(hi);
  }
  const Pair<T>& P = Q.P;
  PAIR_LAUNCH(st2_rhs_kernel<T>, Q.rows, st, P);
  cudaGraph_t ob = nullptr;
  if ((e = stream_add_while(st, ho, &ob)) != cudaSuccess) return e;
  if ((e = cudaStreamBeginCaptureToGraph(side[0], ob, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return e;
  PAIR_LAUNCH(st2_outer_kernel<T>, Q.rows, side[0], P);
  PAIR_LAUNCH(st2_inner_init_kernel<T>, Q.rows, side[0], P);
  enqueue_vcycle2<T>(Q, side[0]);
  cudaGraph_t ib = nullptr;
  e = stream_add_while(side[0], hi, &ib);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(side[1], ib, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    PAIR_LAUNCH(st2_pq_kernel<T>, Q.rows, side[1], P);
    PAIR_LAUNCH(st2_update_kernel<T>, Q.rows, side[1], P);
    enqueue_vcycle2<T>(Q, side[1]);
    cudaGraph_t tmp = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(side[1], &tmp);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) PAIR_LAUNCH(st2_xupdate_kernel<T>, Q.rows, side[0], P);
  {
    cudaGraph_t tmp = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(side[0], &tmp);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return e;
  PAIR_LAUNCH(st2_shift_kernel<T>, Q.rows, st, P);
  PAIR_LAUNCH(st2_finish_kernel<T>, Q.rows, st, P);
  return cudaGetLastError();
}

// the same with the loops on the host (eager launches that tools can
// capture; the host reads both systems' decisions back after each deciding
// launch)
template <class T>
cudaError_t host_loop_pair(PairPlan<T>& Q, cudaStream_t st) {
  for (StreamLaunch& a : Q.P.a) a.host_loop = 1;
  const Pair<T>& P = Q.P;
  StreamScal c[2]{};
  auto flags = [&]() {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
      e = cudaMemcpyAsync(&c[k], P.a[k].sc, sizeof(StreamScal), cudaMemcpyDeviceToHost, st);
    return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
  };
  const int max_outer = std::max(P.a[0].max_outer, P.a[1].max_outer);
  const int inner_cap = std::max(P.a[0].inner_cap, P.a[1].inner_cap);
  cudaError_t e;
  PAIR_LAUNCH(st2_rhs_kernel<T>, Q.rows, st, P);
  for (int pass = 0; pass <= max_outer; ++pass) {
    PAIR_LAUNCH(st2_outer_kernel<T>, Q.rows, st, P);
    if ((e = flags()) != cudaSuccess) return e;
    if (!c[0].inner_ran && !c[1].inner_ran) break;
    PAIR_LAUNCH(st2_inner_init_kernel<T>, Q.rows, st, P);
    enqueue_vcycle2<T>(Q, st);
    if ((e = flags()) != cudaSuccess) return e;
    for (int it = 0; (!c[0].stop || !c[1].stop) && it <= inner_cap; ++it) {
      PAIR_LAUNCH(st2_pq_kernel<T>, Q.rows, st, P);
      PAIR_LAUNCH(st2_update_kernel<T>, Q.rows, st, P);
      enqueue_vcycle2<T>(Q, st);
      if ((e = flags()) != cudaSuccess) return e;
    }
    PAIR_LAUNCH(st2_xupdate_kernel<T>, Q.rows, st, P);
    if ((e = flags()) != cudaSuccess) return e;
    if (!(c[0].more && !c[0].fail) && !(c[1].more && !c[1].fail)) break;
  }
  PAIR_LAUNCH(st2_shift_kernel<T>, Q.rows, st, P);
  PAIR_LAUNCH(st2_finish_kernel<T>, Q.rows, st, P);
  return cudaGetLastError();
}

template <class T>
void prepare_pair_family() {
  for (const void* k : {(const void*)st2_rhs_kernel<T>, (const void*)st2_outer_kernel<T>,
                        (const void*)st2_inner_init_kernel<T>, (const void*)st2_pq_kernel<T>,
                        (const void*)st2_update_kernel<T>, (const void*)st2_xupdate_kernel<T>,
                        (const void*)st2_shift_kernel<T>, (const void*)st2_finish_kernel<T>,
                        (const void*)st2_vc_res_kernel<T, true>, (const void*)st2_vc_res_kernel<T, false>,
                        (const void*)st2_vc_restrict_kernel<T, kRowsAll>,
                        (const void*)st2_vc_restrict_kernel<T, kRowsAll & ~kRowsCsrBlock>,
                        (const void*)st2_vc_coarse_kernel<T>, (const void*)st2_vc_prolong_kernel<T>,
                        (const void*)st2_vc_post_kernel<T, true>, (const void*)st2_vc_post_kernel<T, false>})
    stream_resident_blocks(k);
}

template <class T>
cudaError_t solve_pair(const StreamLaunch (&a)[2], const AmgDevT<T>& H0, const AmgDevT<T>& H1, long long* pair_acc,
                       long long* pair64_acc, long long* pairc_acc, cudaStream_t st, const cudaStream_t* side) {
  // the form built here: the AMG-preconditioned, warm-started elliptic solve
  for (int k = 0; k < 2; ++k)
    if (!a[k].use_amg || !a[k].warm || a[k].rl || a[k].val2 || a[k].dextra || !a[k].val1 || a[k].n != a[0].n ||
        a[k].pin != a[0].pin || a[k].sc == a[1 - k].sc)
      return cudaErrorInvalidValue;
  if (H0.nlev <= 0 || H1.nlev != H0.nlev) return cudaErrorInvalidValue;
  PairPlan<T> Q;
  Pair<T>& P = Q.P;
  P.a[0] = a[0];
  P.a[1] = a[1];
  P.H = H0;
  for (int l = 0; l < H0.nlev; ++l) P.v1[l] = LevVec<T>{H1.L[l].x, H1.L[l].b, H1.L[l].r, H1.L[l].y};
  P.bc1 = H1.bc;
  P.xc1 = H1.xc;
  P.pair_acc = pair_acc;
  P.pair64_acc = pair64_acc;
  P.pairc_acc = pairc_acc;
  for (int k = 0; k < 2; ++k) {
    P.a[k].h0_invd = H0.L[0].invd;
    P.a[k].h0_omega = double(H0.L[0].omega);
  }
  P.a[0].h0_x = H0.L[0].x;
  P.a[1].h0_x = H1.L[0].x;
  Q.nlev = H0.nlev;
  Q.rows = a[0].n;
  for (int l = 0; l < Q.nlev; ++l) {
    Q.tA[l] = level_threads(H0.L[l].A);
    Q.tR[l] = level_threads(H0.L[l].R);
    Q.tP[l] = level_threads(H0.L[l].P);
  }
  Q.tcoarse = int64_t(std::max(1, H0.nc)) * 32;
  if (a[0].host_loop) return host_loop_pair<T>(Q, st);
  return stream_run_captured(st, [&]() { return enqueue_pair<T>(Q, st, side); });
}

}  // namespace

void stream_prepare_pair() {
  prepare_pair_family<float>();
  prepare_pair_family<double>();
}

cudaError_t stream_solve_pair(const StreamLaunch (&a)[2], const AmgDevF& H0, const AmgDevF& H1, long long* pair_acc,
                              long long* pair64_acc, long long* pairc_acc, cudaStream_t st, const cudaStream_t* side) {
  return solve_pair<float>(a, H0, H1, pair_acc, pair64_acc, pairc_acc, st, side);
}

cudaError_t stream_solve_pair(const StreamLaunch (&a)[2], const AmgDev& H0, const AmgDev& H1, long long* pair_acc,
                              long long* pair64_acc, long long* pairc_acc, cudaStream_t st, const cudaStream_t* side) {
  return solve_pair<double>(a, H0, H1, pair_acc, pair64_acc, pairc_acc, st, side);
}

}  // namespace bd
