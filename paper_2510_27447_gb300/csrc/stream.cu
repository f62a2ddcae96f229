// stream.cu -- streaming preconditioned conjugate gradients, for one system
// whose operators do not fit in L2 and for batches of many small systems.
// (The row products, reductions and decisions these kernels share with the
// two-system elliptic chain of stream2.cu live in stream_rows.cuh.)
//
// The persistent solvers (pcg.cu, amg.cu, mixed.cu) keep one grid resident
// for a whole solve and separate its phases with device-wide barriers; that
// caps the threads an SM keeps in flight, which is what a solve that streams
// its operators from HBM needs most.  Here every phase of an iteration is an
// ordinary kernel at full occupancy (one thread per row, grid-stride loops),
// reading the operators with evict-first loads so that the vectors stay in
// L2, and the iteration runs on the device: the loops are CUDA-graph
// conditional WHILE nodes and the kernel that finishes a reduction sets their
// conditions (cudaGraphSetConditional), so a solve has no host round trip.
//
// The algorithm is the one of the persistent mixed kernel (mixed.cu):
//   FP64  b = rl + c1 A1 va + c2 A2 vb, mean-projected for the singular
//         elliptic operator; per outer pass r = b - A x
//   inner CG on A d = r / |r| from d = 0 in the inner precision (FP32 for the
//         mixed path, FP64 otherwise), preconditioned by one AMG V(1,1) cycle
//         (the hierarchy of amg.cpp) or by Jacobi, to |r_inner| <= tol_inner
//         (or what the outer tolerance still needs)
//   FP64  x += |r| d; repeat (iterative refinement) up to max_outer passes,
//         or stop after one pass (max_outer = 1: the single inner solve is the
//         answer)
// then the pin / zero-mean shift of the elliptic solution.
//
// Every kernel takes its parameters through a policy: One (a single system,
// the parameters by value, the whole grid its own) or Many (a batch: a table
// of per-system parameters and a block -> system map; see BatchSolve).  A
// system's arithmetic does not depend on the policy or on the other systems
// of a batch (its reductions run over its own blocks in the same order), so a
// system gives the same bits alone in a batch of one and in any batch.
//
// Reductions: every block writes its partial sums, the last block of the
// system to arrive (an atomic ticket) adds them in block order and takes the
// system's scalar decisions.  A kernel whose work is skipped (a finished
// loop, a closed sweep gate) reads the flag that says so at entry; the flag
// is written by an earlier kernel, so every block of a system takes the same
// branch.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "bd_internal.h"
#include "sparse.cuh"
#include "segment.cuh"
#include "stream_rows.cuh"
#include "vcycle.cuh"

namespace bd {

namespace {


// ---- policies -------------------------------------------------------------------

struct One {
  StreamLaunch a;
};
struct Many {
  const StreamLaunch* tab;
  const int* blk;              // block prefix of this launch
  int nseg;
  BatchCtl* ctl;
  long long* launch_acc;
  unsigned long long h_outer, h_inner;
};
template <class T>
struct VcOne {
  AmgDevT<T> H;
};
template <class T>
struct VcMany {
  const AmgDevT<T>* tab;
  const int* blk;
  int nseg;
};

template <class S>
constexpr bool kMany = std::is_same_v<S, Many>;

__device__ __forceinline__ SegInfo seg_of(const One&) { return {0, int(blockIdx.x), int(gridDim.x)}; }
__device__ __forceinline__ SegInfo seg_of(const Many& m) { return seg_locate(m.blk, m.nseg); }
template <class T>
__device__ __forceinline__ SegInfo seg_of(const VcOne<T>&) { return {0, int(blockIdx.x), int(gridDim.x)}; }
template <class T>
__device__ __forceinline__ SegInfo seg_of(const VcMany<T>& m) { return seg_locate(m.blk, m.nseg); }

__device__ __forceinline__ const StreamLaunch& params(const One& o, int) { return o.a; }
__device__ __forceinline__ const StreamLaunch& params(const Many& m, int r) { return stage(m.tab, r); }
template <class T>
__device__ __forceinline__ const AmgDevT<T>& hier(const VcOne<T>& o, int) { return o.H; }
template <class T>
__device__ __forceinline__ const AmgDevT<T>& hier(const VcMany<T>& m, int r) { return stage(m.tab, r); }

// every kernel counts its launch (see stream_rows.cuh); a batched launch counts once
__device__ __forceinline__ void count_launch(const One& o) { count_launch(o.a.launch_acc); }
__device__ __forceinline__ void count_launch(const Many& m) { count_launch(m.launch_acc); }


// Loop conditions.  A single system sets them directly when it decides.  A
// batch's conditions are set by st_batch_cond_kernel at the end of each loop
// body from every system's flags (the loop continues while any system still
// iterates), with a hard cap on the passes.
__device__ __forceinline__ void vote_inner(const One&, const StreamLaunch& a, bool active) {
  if (a.host_loop) return;
  if (!active) {
    set_cond(a.h_inner, 0u);
    if (a.sc->fail) set_cond(a.h_outer, 0u);
  }
}
__device__ __forceinline__ void vote_inner(const Many&, const StreamLaunch&, bool) {}
__device__ __forceinline__ void vote_outer(const One&, const StreamLaunch& a, bool inner_on, bool outer_on) {
  if (a.host_loop) return;
  set_cond(a.h_inner, inner_on ? 1u : 0u);
  set_cond(a.h_outer, outer_on ? 1u : 0u);
}
__device__ __forceinline__ void vote_outer(const Many&, const StreamLaunch&, bool, bool) {}



#define SEG_BEGIN(src)                             \
  count_launch(src);                               \
  const SegInfo sg = seg_of(src);                  \
  const StreamLaunch& a = params(src, sg.r);       \
  const int gt = sg.lb * blockDim.x + threadIdx.x; \
  const int gs = sg.nb * blockDim.x;

// ---- kernels -------------------------------------------------------------------

// right-hand side in FP64 (two operator products sharing the pattern), the
// Jacobi scaling, a cold start's x = 0; the last block sets the solve up
template <class T, class S>
__global__ void __launch_bounds__(kSB) st_rhs_kernel(const __grid_constant__ S src) {
  SEG_BEGIN(src)
  if (a.gate && *a.gate == 0) {        // the sweep test closed this solve (uniform)
    if (sg.lb == 0 && threadIdx.x == 0) a.sc->skip = 1;
    return;
  }
  T* invd = static_cast<T*>(a.invd);
  double acc[2] = {0.0, 0.0};
  const double* const pv[2] = {a.val1, a.val2};
  const double* const px[2] = {a.va, a.vb};
  const bool pon[2] = {a.val1 != nullptr, a.val2 != nullptr};
  for (int i = gt; i < a.n; i += gs) {
    double sp[2];
    sell_row_multi<2>(a.sptr, a.swidth, a.col, pv, px, pon, i, sp);
    double b = a.rl ? a.rl[i] : 0.0;
    if (a.val1) b += a.c1 * sp[0];
    if (a.val2) b += a.c2 * sp[1];
    a.b64[i] = b;
    if (!a.use_amg) {
      double d = a.valA[a.diagpos[i]];
      if (a.dextra) d += a.dextra[i];
      invd[i] = T(1.0 / d);
    }
    if (!a.warm) a.x[i] = 0.0;
    acc[0] += b;
    acc[1] += b * b;
  }
  if (last_block_total<2, double>(acc, a.part, &a.sc->ticket, sg) && threadIdx.x == 0) rhs_setup(a, acc[0], acc[1]);
}

// FP64 outer residual r = b - A x (b projected) and the outer decision
template <class T, class S>
__global__ void __launch_bounds__(kSB) st_outer_kernel(const __grid_constant__ S src) {
  SEG_BEGIN(src)
  StreamScal& c = *a.sc;
  if (c.skip || c.fail) {
    if (sg.lb == 0 && threadIdx.x == 0) {
      c.inner_ran = 0;
      c.stop = 1;
      c.more = 0;
      vote_outer(src, a, false, false);
    }
    return;
  }
  const double mean = c.mean_b;
  const bool product = c.outer > 0 || a.warm;
  double acc[1] = {0.0};
  for (int i = gt; i < a.n; i += gs) {
    double r = a.b64[i] - mean;
    if (product) {
      double ax = srow<true, double, double>(a.sptr, a.swidth, a.col, a.valA, a.x, i);
      if (a.dextra) ax += a.dextra[i] * a.x[i];
      r -= ax;
    }
    a.r64[i] = r;
    acc[0] += r * r;
  }
  if (last_block_total<1, double>(acc, a.part, &c.ticket, sg) && threadIdx.x == 0) {
    const bool on = outer_decide<T>(a, acc[0]);
    vote_outer(src, a, on, on && a.max_outer > 1);
  }
}

// inner start: r = r64 / |r|, d = 0, the first preconditioning step
// (Jacobi z = D^-1 r and the first decision; AMG: the level-0 pre-smoothing)
template <class T, class S>
__global__ void __launch_bounds__(kSB) st_inner_init_kernel(const __grid_constant__ S src) {
  SEG_BEGIN(src)
  StreamScal& c = *a.sc;
  if (c.stop) {
    if constexpr (kMany<S>)
      if (sg.lb == 0 && threadIdx.x == 0) vote_inner(src, a, false);
    return;
  }
  T* r = static_cast<T*>(a.r);
  T* z = static_cast<T*>(a.z);
  T* d = static_cast<T*>(a.d);
  const T* invd = static_cast<const T*>(a.invd);
  const T* invd0 = static_cast<const T*>(a.h0_invd);
  T* x0 = static_cast<T*>(a.h0_x);
  const T omega0 = T(a.h0_omega);
  const double inv_scale = 1.0 / c.scale;
  T acc[2] = {T(0), T(0)};
  for (int i = gt; i < a.n; i += gs) {
    const T ri = T(a.r64[i] * inv_scale);
    r[i] = ri;
    d[i] = T(0);
    acc[0] += ri * ri;
    if (a.use_amg) {
      x0[i] = omega0 * invd0[i] * ri;
    } else {
      const T zi = invd[i] * ri;
      z[i] = zi;
      acc[1] += ri * zi;
    }
  }
  if (last_block_total<2, T>(acc, a.part, &c.ticket, sg) && threadIdx.x == 0) {
    c.rr_new = double(acc[0]);
    if (!a.use_amg) vote_inner(src, a, inner_decide<T>(a, acc[1]));
    else if constexpr (kMany<S>) vote_inner(src, a, true);
  }
}

// p = z + beta p, q = A z + beta q (q = A p by recurrence), p.q and alpha
template <class T, class S>
__global__ void __launch_bounds__(kSB) st_pq_kernel(const __grid_constant__ S src) {
  SEG_BEGIN(src)
  StreamScal& c = *a.sc;
  if (c.stop) {
    if constexpr (kMany<S>)
      if (sg.lb == 0 && threadIdx.x == 0) vote_inner(src, a, false);
    return;
  }
  const T* z = static_cast<const T*>(a.z);
  T* p = static_cast<T*>(a.p);
  T* q = static_cast<T*>(a.q);
  const T* val = static_cast<const T*>(a.valT);
  const bool first = c.it == 0;
  const T beta = T(c.beta);
  T acc[1] = {T(0)};
  const bool v4 = sizeof(T) == 4 && a.col4 != nullptr;
  for (int i = gt; i < a.n; i += gs) {
    // the row's vector entries are requested before its product
    const T zi = z[i];
    const T pv = first ? T(0) : p[i];
    const T qv = first ? T(0) : q[i];
    T az = v4 ? T(srow4<T>(a.sptr4, a.sw4, a.col4, static_cast<const float*>(a.valT4), z, i))
              : srow<true, T, T>(a.sptr, a.swidth, a.col, val, z, i);
    if (a.dextra) az += T(a.dextra[i]) * zi;
    const T pi = first ? zi : zi + beta * pv;
    const T qi = first ? az : az + beta * qv;
    p[i] = pi;
    q[i] = qi;
    acc[0] += pi * qi;
  }
  if (last_block_total<1, T>(acc, a.part, &c.ticket, sg) && threadIdx.x == 0) {
    const bool active = pq_decide<T>(a, acc[0]);   // a breakdown keeps d; the outer pass decides
    if (!active || kMany<S>) vote_inner(src, a, active);
  }
}

// d += alpha p, r -= alpha q, |r|^2; Jacobi: z = D^-1 r, r.z and the decision;
// AMG: the level-0 pre-smoothing of the next cycle
template <class T, class S>
__global__ void __launch_bounds__(kSB) st_update_kernel(const __grid_constant__ S src) {
  SEG_BEGIN(src)
  StreamScal& c = *a.sc;
  if (c.stop) {
    if constexpr (kMany<S>)
      if (sg.lb == 0 && threadIdx.x == 0) vote_inner(src, a, false);
    return;
  }
  T* r = static_cast<T*>(a.r);
  T* z = static_cast<T*>(a.z);
  T* d = static_cast<T*>(a.d);
  const T* p = static_cast<const T*>(a.p);
  const T* q = static_cast<const T*>(a.q);
  const T* invd = static_cast<const T*>(a.invd);
  const T* invd0 = static_cast<const T*>(a.h0_invd);
  T* x0 = static_cast<T*>(a.h0_x);
  const T omega0 = T(a.h0_omega);
  const T alpha = T(c.alpha);
  T acc[2] = {T(0), T(0)};
  for (int i = gt; i < a.n; i += gs) {
    d[i] += alpha * p[i];
    const T ri = r[i] - alpha * q[i];
    r[i] = ri;
    acc[0] += ri * ri;
    if (a.use_amg) {
      x0[i] = omega0 * invd0[i] * ri;
    } else {
      const T zi = invd[i] * ri;
      z[i] = zi;
      acc[1] += ri * zi;
    }
  }
  if (last_block_total<2, T>(acc, a.part, &c.ticket, sg) && threadIdx.x == 0) {
    c.rr_new = double(acc[0]);
    if (!a.use_amg) vote_inner(src, a, inner_decide<T>(a, acc[1]));
    else if constexpr (kMany<S>) vote_inner(src, a, true);
  }
}

// The batch's loop conditions (one block): phase 0 starts a solve (outer pass
// counter), 1 starts an inner loop (inner = any system iterating), 2 closes an
// inner pass, 3 closes an outer pass (outer = any system wanting another).
// The pass caps are a backstop: every system stops itself at its own caps.
__global__ void __launch_bounds__(kSB) st_batch_cond_kernel(const __grid_constant__ Many m, int phase,
                                                            unsigned cap) {
  count_launch(m);
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  if (phase != 0) {
    int mine = 0;
    for (int r = threadIdx.x; r < m.nseg; r += blockDim.x) {
      const StreamScal& c = *m.tab[r].sc;
      mine |= phase == 3 ? (c.more && !c.fail) : !c.stop;
    }
    if (mine) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  BatchCtl& b = *m.ctl;
  if (phase == 0) {
    b.outer_iters = 0u;
  } else if (phase == 1) {
    b.inner_iters = 0u;
    set_cond(m.h_inner, any ? 1u : 0u);
  } else if (phase == 2) {
    b.inner_iters += 1u;
    set_cond(m.h_inner, (any && b.inner_iters < cap) ? 1u : 0u);
  } else {
    b.outer_iters += 1u;
    set_cond(m.h_outer, (any && b.outer_iters < cap) ? 1u : 0u);
  }
}

// ---- V(1,1) cycle, one kernel per phase and level (the cycle of amg.cu) -----
//
// V (VcOne / VcMany) gives a block its system's hierarchy, S its solve (stop
// flag, level-0 vectors); both resolve the same system for a block.

// r_l = b_l - A_l x_l
// (L0: compiled for level 0 only, else for the coarser levels only)
template <class T, class V, class S, bool L0>
__global__ void __launch_bounds__(kSB) st_vc_res_kernel(const __grid_constant__ V hv, const __grid_constant__ S src,
                                                        int l) {
  count_launch(src);
  const SegInfo sg = seg_of(hv);
  const AmgDevT<T>& H = hier(hv, sg.r);
  const StreamLaunch& a = params(src, sg.r);
  if (a.sc->stop || l >= H.nlev) return;
  const AmgLevelDevT<T>& L = H.L[l];
  if constexpr (L0) {
    const T* b = static_cast<const T*>(a.r);
    if (sizeof(T) == 4 && a.col4) {
      for (int i = sg.lb * blockDim.x + threadIdx.x; i < L.A.n; i += sg.nb * blockDim.x)
        L.r[i] = b[i] - T(srow4<T>(a.sptr4, a.sw4, a.col4, static_cast<const float*>(a.valT4), L.x, i));
      return;
    }
    level_rows<T, kRowsSellStream>(L.A, L.x, true, sg, [&](int i, T ax) { L.r[i] = b[i] - ax; });
  } else {
    const T* b = L.b;
    level_rows<T, kRowsCoarse>(L.A, L.x, false, sg, [&](int i, T ax) { L.r[i] = b[i] - ax; });
  }
}

// b_{l+1} = R_l r_l and the next level's pre-smoothing x_{l+1} = w D^-1 b_{l+1}
// (K: the row forms compiled; the block-per-row form only where R_l has it)
template <class T, class V, class S, int K>
__global__ void __launch_bounds__(kSB) st_vc_restrict_kernel(const __grid_constant__ V hv,
                                                             const __grid_constant__ S src, int l) {
  count_launch(src);
  const SegInfo sg = seg_of(hv);
  const AmgDevT<T>& H = hier(hv, sg.r);
  const StreamLaunch& a = params(src, sg.r);
  if (a.sc->stop || l >= H.nlev) return;
  const AmgLevelDevT<T>& L = H.L[l];
  const bool last = l + 1 == H.nlev;
  T* bn = last ? H.bc : H.L[l + 1].b;
  T* xn = last ? nullptr : H.L[l + 1].x;
  const T* invdn = last ? nullptr : H.L[l + 1].invd;
  const T omegan = last ? T(0) : H.L[l + 1].omega;
  level_rows<T, K>(L.R, L.r, l == 0, sg, [&](int i, T v) {
    bn[i] = v;
    if (xn) xn[i] = omegan * invdn[i] * v;
  });
}

// dense coarsest solve xc = Cinv bc: one warp per row of the system's coarse
// inverse (rows padded to 16-byte multiples), 16-byte loads, butterfly sum
template <class T, class V, class S>
__global__ void __launch_bounds__(kSB) st_vc_coarse_kernel(const __grid_constant__ V hv,
                                                           const __grid_constant__ S src) {
  count_launch(src);
  const SegInfo sg = seg_of(hv);
  const AmgDevT<T>& H = hier(hv, sg.r);
  const StreamLaunch& a = params(src, sg.r);
  if (a.sc->stop || H.nlev == 0) return;
  using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int E = 16 / int(sizeof(T));
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int nvec = H.ldc / E;
  if (sg.lb * wpb >= H.nc) return;                 // no rows in this block (uniform)
  __shared__ __align__(16) T sbc[kCoarseStage];
  const bool staged = H.ldc <= kCoarseStage;       // the right-hand side in shared memory
  if (staged) {
    for (int j = threadIdx.x; j < H.ldc; j += blockDim.x) sbc[j] = j < H.nc ? __ldcg(H.bc + j) : T(0);
    __syncthreads();
  }
  for (int i = sg.lb * wpb + (threadIdx.x >> 5); i < H.nc; i += sg.nb * wpb) {
    const VT* row = reinterpret_cast<const VT*>(H.cinv + int64_t(i) * H.ldc);
    T s = T(0);
    for (int q = lane; q < nvec; q += 32) {
      const VT cv = __ldg(row + q);
      if (staged) {
        s += dot_vec(cv, &sbc[q * E]);
      } else {
        T bq[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const int j = q * E + k;
          bq[k] = j < H.nc ? __ldcg(H.bc + j) : T(0);
        }
        s += dot_vec(cv, bq);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) H.xc[i] = s;
  }
}

// x_l += P_l y_{l+1}
template <class T, class V, class S>
__global__ void __launch_bounds__(kSB) st_vc_prolong_kernel(const __grid_constant__ V hv,
                                                            const __grid_constant__ S src, int l) {
  count_launch(src);
  const SegInfo sg = seg_of(hv);
  const AmgDevT<T>& H = hier(hv, sg.r);
  const StreamLaunch& a = params(src, sg.r);
  if (a.sc->stop || l >= H.nlev) return;
  const AmgLevelDevT<T>& L = H.L[l];
  const T* yc = l + 1 == H.nlev ? H.xc : H.L[l + 1].y;
  // rows of P are short: never a block per row
  level_rows<T, kRowsAll & ~kRowsCsrBlock>(L.P, yc, l == 0, sg, [&](int i, T v) { L.x[i] += v; });
}

// y_l = x_l + w D^-1 (b_l - A_l x_l); on level 0 y is z, r.z and the decision
// (every system of a batch has at least one block here and votes)
template <class T, class V, class S, bool L0>
__global__ void __launch_bounds__(kSB) st_vc_post_kernel(const __grid_constant__ V hv, const __grid_constant__ S src,
                                                         int l) {
  count_launch(src);
  const SegInfo sg = seg_of(hv);
  const AmgDevT<T>& H = hier(hv, sg.r);
  const StreamLaunch& a = params(src, sg.r);
  StreamScal& c = *a.sc;
  if (c.stop) {
    if constexpr (kMany<S>)
      if (l == 0 && sg.lb == 0 && threadIdx.x == 0) vote_inner(src, a, false);
    return;
  }
  if (l >= H.nlev) {            // a Jacobi system of a batch: nothing to do at level 0
    if constexpr (kMany<S>)
      if (l == 0 && sg.lb == 0 && threadIdx.x == 0) vote_inner(src, a, true);
    return;
  }
  const AmgLevelDevT<T>& L = H.L[l];
  const T* b = l == 0 ? static_cast<const T*>(a.r) : L.b;
  T* y = l == 0 ? static_cast<T*>(a.z) : L.y;
  T acc[1] = {T(0)};
  auto post = [&](int i, T ax) {
    const T bi = b[i];
    const T yi = L.x[i] + L.omega * L.invd[i] * (bi - ax);
    y[i] = yi;
    acc[0] += bi * yi;
  };
  if constexpr (L0) {
    if (sizeof(T) == 4 && a.col4) {
      for (int i = sg.lb * blockDim.x + threadIdx.x; i < L.A.n; i += sg.nb * blockDim.x)
        post(i, T(srow4<T>(a.sptr4, a.sw4, a.col4, static_cast<const float*>(a.valT4), L.x, i)));
    } else {
      level_rows<T, kRowsSellStream>(L.A, L.x, true, sg, post);
    }
    if (last_block_total<1, T>(acc, a.part, &c.ticket, sg) && threadIdx.x == 0)
      vote_inner(src, a, inner_decide<T>(a, acc[0]));
  } else {
    level_rows<T, kRowsCoarse>(L.A, L.x, false, sg, post);
  }
}

// x += |r| d after an inner solve that ran without failure
template <class T, class S>
__global__ void __launch_bounds__(kSB) st_xupdate_kernel(const __grid_constant__ S src) {
  SEG_BEGIN(src)
  const StreamScal& c = *a.sc;
  if (!c.inner_ran || c.fail) return;
  const double s = c.scale;
  const T* d = static_cast<const T*>(a.d);
  for (int i = gt; i < a.n; i += gs) a.x[i] += s * double(d[i]);
}

// normalisation of the singular elliptic solution: the shift (u[pin], or the
// nodal mean)
template <class S>
__global__ void __launch_bounds__(kSB) st_shift_kernel(const __grid_constant__ S src) {
  SEG_BEGIN(src)
  StreamScal& c = *a.sc;
  if (c.skip || a.pin < -1) return;
  if (a.pin >= 0) {
    if (sg.lb == 0 && threadIdx.x == 0) c.shift = a.x[a.pin];
    return;
  }
  double acc[1] = {0.0};
  for (int i = gt; i < a.n; i += gs) acc[0] += a.x[i];
  if (last_block_total<1, double>(acc, a.part, &c.ticket, sg) && threadIdx.x == 0) c.shift = acc[0] / double(a.n);
}

// x -= shift (pin >= -1); the solve's status and counters
template <class S>
__global__ void __launch_bounds__(kSB) st_finish_kernel(const __grid_constant__ S src) {
  SEG_BEGIN(src)
  const StreamScal& c = *a.sc;
  if (c.skip) return;
  if (a.pin >= -1) {
    const double sh = c.shift;
    for (int i = gt; i < a.n; i += gs) a.x[i] -= sh;
  }
  if (sg.lb == 0 && threadIdx.x == 0) {
    if (c.fail) atomicOr(a.status, c.fail);
    if (a.iters_acc) atomicAdd(reinterpret_cast<unsigned long long*>(a.iters_acc), (unsigned long long)c.inner_total);
    if (a.outer_acc) atomicAdd(reinterpret_cast<unsigned long long*>(a.outer_acc), (unsigned long long)c.outer_total);
    if (a.solves_acc) atomicAdd(reinterpret_cast<unsigned long long*>(a.solves_acc), 1ull);
  }
}

// ---- host side ------------------------------------------------------------------

int grid_for(int64_t threads) {
  const int64_t b = (threads + kSB - 1) / kSB;
  return int(std::max<int64_t>(1, std::min<int64_t>(b, stream_grid_cap())));
}

}  // namespace

// ---- host helpers (declared in stream_rows.cuh; stream2.cu uses them too) -----

namespace {
std::mutex g_occ_mu;
std::unordered_map<const void*, int> g_occ;
}  // namespace

// resident blocks per SM of kernel k at kSB threads, queried once and cached
// (stream_prepare fills the cache before any capture)
int stream_resident_blocks(const void* k) {
  std::lock_guard<std::mutex> g(g_occ_mu);
  auto it = g_occ.find(k);
  if (it != g_occ.end()) return it->second;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kSB, 0) != cudaSuccess || nb <= 0) {
    cudaGetLastError();
    nb = 1;
  }
  nb = std::min(nb, kBlocksPerSM);
  g_occ.emplace(k, nb);
  return nb;
}

// grid of kernel k over `threads` grid-stride threads: at most one full wave
// of resident blocks (a second partial wave would run its blocks' equal
// shares of rows at a fraction of the occupancy)
int stream_fit(const void* k, int64_t threads) {
  const int64_t b = (threads + kSB - 1) / kSB;
  const int64_t wave = int64_t(stream_grid_cap() / kBlocksPerSM) * stream_resident_blocks(k);
  return int(std::max<int64_t>(1, std::min(b, wave)));
}

// add a WHILE node after the current capture frontier of `cap` and return its
// body graph; the capture continues after the node
cudaError_t stream_add_while(cudaStream_t cap, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cap, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np);
  if (e != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

cudaGraph_t stream_capture_graph(cudaStream_t s) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess) return nullptr;
  return cs == cudaStreamCaptureStatusActive ? g : nullptr;
}

namespace {

// The launches of one solve (One) or of one batch of solves (Many): the
// policies and grids of every kernel family.
template <class T>
struct Plan {
  bool many = false;
  One one{};
  Many many_base{};
  VcOne<T> vone{};
  VcMany<T> vmany{};
  const BatchSolve* bs = nullptr;
  int nlev = 0;
  // grid-stride threads of each kernel family (single system)
  int64_t rows = 1, tcoarse = 1;
  int64_t tA[kMaxAmgLevels] = {}, tR[kMaxAmgLevels] = {}, tP[kMaxAmgLevels] = {};
  bool amg = false;
  Many mk(const int* blk) const {
    Many m = many_base;
    m.blk = blk;
    return m;
  }
  VcMany<T> vmk(const int* blk) const {
    VcMany<T> v = vmany;
    v.blk = blk;
    return v;
  }
};

// a kernel of the row family under either policy (KNAME<T, policy> or,
// without the value type, KNAME<policy>)
#define ROWS_LAUNCH_T(KNAME, stream)                                                                   \
  do {                                                                                                 \
    if (P.many) KNAME<T, Many><<<P.bs->total_rows_blocks, kSB, 0, stream>>>(P.mk(P.bs->blk_rows));      \
    else KNAME<T, One><<<stream_fit((const void*)KNAME<T, One>, P.rows), kSB, 0, stream>>>(P.one);            \
  } while (0)
#define ROWS_LAUNCH_S(KNAME, stream)                                                                   \
  do {                                                                                                 \
    if (P.many) KNAME<Many><<<P.bs->total_rows_blocks, kSB, 0, stream>>>(P.mk(P.bs->blk_rows));         \
    else KNAME<One><<<stream_fit((const void*)KNAME<One>, P.rows), kSB, 0, stream>>>(P.one);                  \
  } while (0)

template <class T>
void enqueue_vcycle(const Plan<T>& P, cudaStream_t s) {
  for (int l = 0; l < P.nlev; ++l) {
    if (P.many) {
      const Many m = P.mk(P.bs->blk_rows);
      if (l == 0)
        st_vc_res_kernel<T, VcMany<T>, Many, true><<<P.bs->total_A[l], kSB, 0, s>>>(P.vmk(P.bs->blk_A[l]), m, l);
      else
        st_vc_res_kernel<T, VcMany<T>, Many, false><<<P.bs->total_A[l], kSB, 0, s>>>(P.vmk(P.bs->blk_A[l]), m, l);
      st_vc_restrict_kernel<T, VcMany<T>, Many, kRowsAll><<<P.bs->total_R[l], kSB, 0, s>>>(P.vmk(P.bs->blk_R[l]), m,
                                                                                         l);
    } else {
      if (l == 0)
        st_vc_res_kernel<T, VcOne<T>, One, true>
            <<<stream_fit((const void*)st_vc_res_kernel<T, VcOne<T>, One, true>, P.tA[l]), kSB, 0, s>>>(P.vone, P.one, l);
      else
        st_vc_res_kernel<T, VcOne<T>, One, false>
            <<<stream_fit((const void*)st_vc_res_kernel<T, VcOne<T>, One, false>, P.tA[l]), kSB, 0, s>>>(P.vone, P.one, l);
      if (P.vone.H.L[l].R.lpr > 32)
        st_vc_restrict_kernel<T, VcOne<T>, One, kRowsAll>
            <<<stream_fit((const void*)st_vc_restrict_kernel<T, VcOne<T>, One, kRowsAll>, P.tR[l]), kSB, 0, s>>>(P.vone,
                                                                                                   P.one, l);
      else
        st_vc_restrict_kernel<T, VcOne<T>, One, kRowsAll & ~kRowsCsrBlock>
            <<<stream_fit((const void*)st_vc_restrict_kernel<T, VcOne<T>, One, kRowsAll & ~kRowsCsrBlock>, P.tR[l]), kSB, 0,
               s>>>(P.vone, P.one, l);
    }
  }
  if (P.many)
    st_vc_coarse_kernel<T, VcMany<T>, Many><<<P.bs->total_coarse, kSB, 0, s>>>(P.vmk(P.bs->blk_coarse),
                                                                                P.mk(P.bs->blk_rows));
  else
    st_vc_coarse_kernel<T, VcOne<T>, One><<<stream_fit((const void*)st_vc_coarse_kernel<T, VcOne<T>, One>, P.tcoarse), kSB,
                                            0, s>>>(P.vone, P.one);
  for (int l = P.nlev - 1; l >= 0; --l) {
    if (P.many) {
      const Many m = P.mk(P.bs->blk_rows);
      st_vc_prolong_kernel<T, VcMany<T>, Many><<<P.bs->total_P[l], kSB, 0, s>>>(P.vmk(P.bs->blk_P[l]), m, l);
      if (l == 0)
        st_vc_post_kernel<T, VcMany<T>, Many, true><<<P.bs->total_post0_blocks, kSB, 0, s>>>(
            P.vmk(P.bs->blk_post0), P.mk(P.bs->blk_post0), 0);
      else
        st_vc_post_kernel<T, VcMany<T>, Many, false><<<P.bs->total_A[l], kSB, 0, s>>>(P.vmk(P.bs->blk_A[l]), m, l);
    } else {
      st_vc_prolong_kernel<T, VcOne<T>, One><<<stream_fit((const void*)st_vc_prolong_kernel<T, VcOne<T>, One>, P.tP[l]),
                                               kSB, 0, s>>>(P.vone, P.one, l);
      if (l == 0)
        st_vc_post_kernel<T, VcOne<T>, One, true>
            <<<stream_fit((const void*)st_vc_post_kernel<T, VcOne<T>, One, true>, P.rows), kSB, 0, s>>>(P.vone, P.one, l);
      else
        st_vc_post_kernel<T, VcOne<T>, One, false>
            <<<stream_fit((const void*)st_vc_post_kernel<T, VcOne<T>, One, false>, P.tA[l]), kSB, 0, s>>>(P.vone, P.one, l);
    }
  }
}

// the solve's kernels and loops, appended to the capture of `st`
template <class T>
cudaError_t enqueue_solve(Plan<T>& P, cudaStream_t st, const cudaStream_t* side) {
  cudaGraph_t g = stream_capture_graph(st);
  if (!g) return cudaErrorStreamCaptureUnsupported;
  cudaGraphConditionalHandle ho, hi;
  cudaError_t e = cudaGraphConditionalHandleCreate(&ho, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hi, g, 0, 0);
  if (e != cudaSuccess) return e;
  P.one.a.h_outer = P.many_base.h_outer = static_cast<unsigned long long>(ho);
  P.one.a.h_inner = P.many_base.h_inner = static_cast<unsigned long long>(hi);
  ROWS_LAUNCH_T(st_rhs_kernel, st);
  if (P.many) st_batch_cond_kernel<<<1, kSB, 0, st>>>(P.mk(P.bs->blk_rows), 0, 0u);
  cudaGraph_t ob = nullptr;
  if ((e = stream_add_while(st, ho, &ob)) != cudaSuccess) return e;
  // outer body: residual and decision, inner start, inner loop, x update
  if ((e = cudaStreamBeginCaptureToGraph(side[0], ob, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return e;
  ROWS_LAUNCH_T(st_outer_kernel, side[0]);
  ROWS_LAUNCH_T(st_inner_init_kernel, side[0]);
  if (P.amg) enqueue_vcycle<T>(P, side[0]);
  if (P.many) st_batch_cond_kernel<<<1, kSB, 0, side[0]>>>(P.mk(P.bs->blk_rows), 1, 0u);
  cudaGraph_t ib = nullptr;
  e = stream_add_while(side[0], hi, &ib);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(side[1], ib, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    ROWS_LAUNCH_T(st_pq_kernel, side[1]);
    ROWS_LAUNCH_T(st_update_kernel, side[1]);
    if (P.amg) enqueue_vcycle<T>(P, side[1]);
    if (P.many) st_batch_cond_kernel<<<1, kSB, 0, side[1]>>>(P.mk(P.bs->blk_rows), 2, P.bs->inner_cap + 1u);
    cudaGraph_t tmp = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(side[1], &tmp);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) ROWS_LAUNCH_T(st_xupdate_kernel, side[0]);
  if (e == cudaSuccess && P.many)
    st_batch_cond_kernel<<<1, kSB, 0, side[0]>>>(P.mk(P.bs->blk_rows), 3, P.bs->max_outer + 1u);
  {
    cudaGraph_t tmp = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(side[0], &tmp);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return e;
  ROWS_LAUNCH_S(st_shift_kernel, st);
  ROWS_LAUNCH_S(st_finish_kernel, st);
  return cudaGetLastError();
}

// The same solve with its loops on the host (a profiling form: every kernel
// is an eager launch that tools can capture; the host reads the decisions
// back after each deciding launch)
template <class T>
cudaError_t host_loop_solve(Plan<T>& P, cudaStream_t st) {
  P.one.a.host_loop = 1;
  StreamScal c{};
  auto flags = [&]() {
    const cudaError_t e = cudaMemcpyAsync(&c, P.one.a.sc, sizeof(StreamScal), cudaMemcpyDeviceToHost, st);
    return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
  };
  cudaError_t e;
  ROWS_LAUNCH_T(st_rhs_kernel, st);
  for (int pass = 0; pass <= P.one.a.max_outer; ++pass) {
    ROWS_LAUNCH_T(st_outer_kernel, st);
    if ((e = flags()) != cudaSuccess) return e;
    if (!c.inner_ran) break;
    ROWS_LAUNCH_T(st_inner_init_kernel, st);
    if (P.amg) enqueue_vcycle<T>(P, st);
    if ((e = flags()) != cudaSuccess) return e;
    for (int it = 0; !c.stop && it <= P.one.a.inner_cap; ++it) {
      ROWS_LAUNCH_T(st_pq_kernel, st);
      ROWS_LAUNCH_T(st_update_kernel, st);
      if (P.amg) enqueue_vcycle<T>(P, st);
      if ((e = flags()) != cudaSuccess) return e;
    }
    ROWS_LAUNCH_T(st_xupdate_kernel, st);
    if ((e = flags()) != cudaSuccess) return e;
    if (!c.more || c.fail) break;
  }
  ROWS_LAUNCH_S(st_shift_kernel, st);
  ROWS_LAUNCH_S(st_finish_kernel, st);
  return cudaGetLastError();
}

template <class T>
Plan<T> one_plan(const StreamLaunch& a, const AmgDevT<T>* M) {
  Plan<T> P;
  P.one.a = a;
  P.amg = a.use_amg && M && M->nlev > 0;
  if (P.amg) {
    P.vone.H = *M;
    P.nlev = M->nlev;
    for (int l = 0; l < P.nlev; ++l) {
      P.tA[l] = level_threads(M->L[l].A);
      P.tR[l] = level_threads(M->L[l].R);
      P.tP[l] = level_threads(M->L[l].P);
    }
    P.tcoarse = int64_t(std::max(1, M->nc)) * 32;
    P.one.a.h0_invd = M->L[0].invd;
    P.one.a.h0_x = M->L[0].x;
    P.one.a.h0_omega = double(M->L[0].omega);
  } else {
    P.one.a.use_amg = 0;
  }
  P.rows = a.n;
  return P;
}

}  // namespace

int stream_grid_cap() {
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess) {
      cudaGetLastError();
      return 152 * kBlocksPerSM;
    }
    cap = sms * kBlocksPerSM;
  }
  return cap;
}

int stream_grid(int64_t rows) { return grid_for(rows); }

namespace {
template <class T>
void prepare_family() {
  for (const void* k : {(const void*)st_rhs_kernel<T, One>, (const void*)st_outer_kernel<T, One>,
                        (const void*)st_inner_init_kernel<T, One>, (const void*)st_pq_kernel<T, One>,
                        (const void*)st_update_kernel<T, One>, (const void*)st_xupdate_kernel<T, One>,
                        (const void*)st_vc_res_kernel<T, VcOne<T>, One, true>,
                        (const void*)st_vc_res_kernel<T, VcOne<T>, One, false>,
                        (const void*)st_vc_restrict_kernel<T, VcOne<T>, One, kRowsAll>,
                        (const void*)st_vc_restrict_kernel<T, VcOne<T>, One, kRowsAll & ~kRowsCsrBlock>,
                        (const void*)st_vc_coarse_kernel<T, VcOne<T>, One>,
                        (const void*)st_vc_prolong_kernel<T, VcOne<T>, One>,
                        (const void*)st_vc_post_kernel<T, VcOne<T>, One, true>,
                        (const void*)st_vc_post_kernel<T, VcOne<T>, One, false>})
    stream_resident_blocks(k);
}
}  // namespace

void stream_prepare() {
  stream_grid_cap();
  prepare_family<float>();
  prepare_family<double>();
  stream_resident_blocks((const void*)st_shift_kernel<One>);
  stream_resident_blocks((const void*)st_finish_kernel<One>);
  stream_prepare_pair();
}

cudaError_t stream_solve(const StreamLaunch& a, int f32, const AmgDevF* M32, const AmgDev* M64, cudaStream_t st,
                         const cudaStream_t* side) {
  if (f32) {
    Plan<float> P = one_plan<float>(a, M32);
    if (a.host_loop) return host_loop_solve<float>(P, st);
    return stream_run_captured(st, [&]() { return enqueue_solve<float>(P, st, side); });
  }
  Plan<double> P = one_plan<double>(a, M64);
  if (a.host_loop) return host_loop_solve<double>(P, st);
  return stream_run_captured(st, [&]() { return enqueue_solve<double>(P, st, side); });
}

cudaError_t stream_solve_batch(const BatchSolve& b, cudaStream_t st, const cudaStream_t* side) {
  auto run = [&](auto tag) {
    using T = decltype(tag);
    Plan<T> P;
    P.many = true;
    P.bs = &b;
    P.many_base.tab = b.tab;
    P.many_base.nseg = b.nseg;
    P.many_base.ctl = b.ctl;
    P.many_base.launch_acc = b.launch_acc;
    P.vmany.tab = static_cast<const AmgDevT<T>*>(b.hier);
    P.vmany.nseg = b.nseg;
    P.nlev = b.nlev_max;
    P.amg = b.nlev_max > 0;
    return stream_run_captured(st, [&]() { return enqueue_solve<T>(P, st, side); });
  };
  return b.f32 ? run(float{}) : run(double{});
}

}  // namespace bd
