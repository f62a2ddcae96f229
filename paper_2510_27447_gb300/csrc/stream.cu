// stream.cu -- streaming preconditioned conjugate gradients for operators
// that do not fit in L2.
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
//         answer, to tol relative to |b|)
// then the pin / zero-mean shift of the elliptic solution.
//
// Reductions: every block writes its partial sums, the last block to arrive
// (an atomic ticket) adds them in block order -- deterministic for a fixed
// grid -- and takes the solve's scalar decisions.  A kernel whose work is
// skipped (a finished loop, a closed sweep gate) reads the flag that says so
// at entry; the flag is written by an earlier kernel, so every block of a
// launch takes the same branch.
#include <cuda_runtime.h>

#include <algorithm>

#include "bd_internal.h"
#include "sparse.cuh"
#include "vcycle.cuh"

namespace bd {

namespace {

constexpr int kSB = 256;       // threads per block of every streaming kernel
constexpr int kBlocksPerSM = 8;

// ---- row products ------------------------------------------------------------

// evict-first load (operator streams: read once per use, larger than L2)
template <class V>
__device__ __forceinline__ V ld_stream(const V* p) {
  return __ldcs(p);
}

// sum_k val[k] x[col[k]] over row i of a SELL-32 operator, entries in order,
// four loads of each stream in flight per thread
template <bool STREAMOP, class V, class X>
__device__ __forceinline__ X srow(const int64_t* __restrict__ sptr, const int* __restrict__ sw,
                                  const int* __restrict__ col, const V* __restrict__ val, const X* __restrict__ x,
                                  int i) {
  const int s = i >> 5;
  const int64_t base = sptr[s] + (i & 31);
  const int w = sw[s];
  X acc = X(0);
  constexpr int CH = 4;
  for (int k0 = 0; k0 < w; k0 += CH) {
    int c[CH];
    V v[CH];
    X g[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k0 + k < w) {
        const int64_t e = base + 32 * (k0 + k);
        c[k] = STREAMOP ? ld_stream(col + e) : __ldg(col + e);
        v[k] = STREAMOP ? ld_stream(val + e) : __ldg(val + e);
      }
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k0 + k < w) g[k] = __ldg(x + c[k]);
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (k0 + k < w) acc += X(v[k]) * g[k];
  }
  return acc;
}

// every row i of an AMG-level operator (SELL: thread per row; CSR: warp per
// row, butterfly sum): epi(i, (M x)_i), run by one lane per row
// (level 0's operators are streamed with evict-first loads, the coarser
// levels' stay cacheable: they are read twice a cycle and fit in L2)
template <class T, class F>
__device__ __forceinline__ void level_rows(const SellDevT<T>& M, const T* x, bool streamop, F&& epi) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int gs = gridDim.x * blockDim.x;
  if (M.rp) {
    const int lane = threadIdx.x & 31;
    for (int i = gt >> 5; i < M.n; i += gs >> 5) {
      T s = T(0);
      const int64_t e = M.rp[i + 1];
      for (int64_t p = M.rp[i] + lane; p < e; p += 32) s += __ldg(M.val + p) * __ldg(x + __ldg(M.col + p));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) epi(i, s);
    }
  } else if (streamop) {
    for (int i = gt; i < M.n; i += gs) epi(i, srow<true, T, T>(M.sptr, M.sw, M.col, M.val, x, i));
  } else {
    for (int i = gt; i < M.n; i += gs) epi(i, srow<false, T, T>(M.sptr, M.sw, M.col, M.val, x, i));
  }
}

// every kernel of a streaming solve counts its launch (the loops run on the
// device, so the host cannot)
__device__ __forceinline__ void count_launch(long long* acc) {
  if (acc && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(acc), 1ull);
}

// ---- reductions ----------------------------------------------------------------

// Block sums of v[0..NV) into part, an atomic ticket, and in the last block to
// arrive the grid totals (block order, fixed tree): returns true there, with
// v holding the totals in every thread of that block; false elsewhere.
template <int NV, class T>
__device__ __forceinline__ bool last_block_total(T (&v)[NV], void* partv, unsigned* ticket) {
  __shared__ T sh[NV][32];
  __shared__ T tot[NV];
  __shared__ int amlast;
  T* part = static_cast<T*>(partv);
  block_sum<NV, T>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[blockIdx.x * NV + k] = v[k];
    __threadfence();
    amlast = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!amlast) return false;
  __threadfence();
  T acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = T(0);
  for (int b = threadIdx.x; b < int(gridDim.x); b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(part + b * NV + k);
  block_sum<NV, T>(acc, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = acc[k];
    *ticket = 0u;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = tot[k];
  return true;
}

__device__ __forceinline__ void set_cond(unsigned long long h, unsigned v) {
  cudaGraphSetConditional(static_cast<cudaGraphConditionalHandle>(h), v);
}

// Decision after the inner residual r and the preconditioned z are complete
// (thread 0 of the last block): the first one of an inner solve sets rho,
// later ones close an iteration as the persistent kernel's loop does.
template <class T>
__device__ __forceinline__ void inner_decide(const StreamLaunch& a, T rz) {
  StreamScal& c = *a.sc;
  bool done = false;
  const T rr = T(c.rr_new);
  if (c.first) {
    c.first = 0;
    c.rho = double(rz);
    done = !(rr > T(c.tgt));
  } else {
    c.it += 1;
    if (!isfinite(rr) || !isfinite(rz)) {
      c.fail |= ST_NONFINITE;
      done = true;
    } else if (rr <= T(c.tgt)) {
      done = true;
    } else if (c.it >= a.inner_cap) {
      if (a.max_outer == 1) c.fail |= ST_NOT_CONVERGED;
      done = true;
    } else {
      c.beta = double(rz / T(c.rho));
      c.rho = double(rz);
    }
  }
  if (done) {
    c.stop = 1;
    c.inner_total += c.it;
    set_cond(a.h_inner, 0u);
    if (c.fail) set_cond(a.h_outer, 0u);
  }
}

// ---- kernels -------------------------------------------------------------------

// right-hand side in FP64 (two operator products sharing the pattern), the
// Jacobi scaling, a cold start's x = 0; the last block sets the solve up
template <class T>
__global__ void __launch_bounds__(kSB) st_rhs_kernel(const __grid_constant__ StreamLaunch a) {
  count_launch(a.launch_acc);
  if (a.gate && *a.gate == 0) {        // the sweep test closed this solve (uniform)
    if (blockIdx.x == 0 && threadIdx.x == 0) a.sc->skip = 1;
    return;
  }
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int gs = gridDim.x * blockDim.x;
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
  if (last_block_total<2, double>(acc, a.part, &a.sc->ticket) && threadIdx.x == 0) {
    StreamScal& c = *a.sc;
    const double mean = a.project ? acc[0] / double(a.n) : 0.0;
    double bb = a.project ? acc[1] - double(a.n) * mean * mean : acc[1];
    if (bb < 0.0) bb = 0.0;
    c.mean_b = mean;
    c.bb = bb;
    c.tol2 = a.tol * a.tol * bb;
    c.outer = 0;
    c.fail = 0;
    c.skip = 0;
    c.stop = 1;
    c.inner_ran = 0;
    c.inner_total = 0;
    c.outer_total = 0;
  }
}

// FP64 outer residual r = b - A x (b projected) and the outer decision
template <class T>
__global__ void __launch_bounds__(kSB) st_outer_kernel(const __grid_constant__ StreamLaunch a) {
  count_launch(a.launch_acc);
  StreamScal& c = *a.sc;
  if (c.skip || c.fail) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      c.inner_ran = 0;
      c.stop = 1;
      set_cond(a.h_inner, 0u);
      set_cond(a.h_outer, 0u);
    }
    return;
  }
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int gs = gridDim.x * blockDim.x;
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
  if (last_block_total<1, double>(acc, a.part, &c.ticket) && threadIdx.x == 0) {
    const double rr = acc[0];
    c.rr64 = rr;
    c.outer_total += 1;
    bool done = false;
    if (!isfinite(rr)) {
      c.fail |= ST_NONFINITE;
      done = true;
    } else if (a.max_outer > 1 && rr <= c.tol2) {
      done = true;
    } else if (c.outer >= a.max_outer) {
      if (a.max_outer > 1) c.fail |= ST_NOT_CONVERGED;
      done = true;
    } else if (!(rr > 0.0)) {
      done = true;
    }
    if (done) {
      c.inner_ran = 0;
      c.stop = 1;
      set_cond(a.h_inner, 0u);
      set_cond(a.h_outer, 0u);
    } else {
      c.scale = sqrt(rr);
      // inner target relative to |r|^2: the FP32 solves follow the persistent
      // mixed kernel; a single FP64 solve stops at |r| <= tol |b|, as the
      // persistent FP64 kernel does
      double tgt = a.tol_inner * a.tol_inner;
      if (a.max_outer > 1) tgt = fmax(tgt, 0.25 * c.tol2 / rr);
      else if (sizeof(T) == 8) tgt = c.tol2 / rr;
      else if (a.warm) tgt = fmax(tgt, tgt * c.bb / rr);
      c.tgt = tgt;
      c.it = 0;
      c.first = 1;
      c.stop = 0;
      c.inner_ran = 1;
      c.beta = 0.0;
      c.outer += 1;
      set_cond(a.h_inner, 1u);
      set_cond(a.h_outer, a.max_outer > 1 ? 1u : 0u);
    }
  }
}

// inner start: r = r64 / |r|, d = 0, the first preconditioning step
// (Jacobi z = D^-1 r and the first decision; AMG: the level-0 pre-smoothing)
template <class T>
__global__ void __launch_bounds__(kSB) st_inner_init_kernel(const __grid_constant__ StreamLaunch a, const T* invd0,
                                                            T omega0, T* x0) {
  count_launch(a.launch_acc);
  StreamScal& c = *a.sc;
  if (c.stop) return;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int gs = gridDim.x * blockDim.x;
  T* r = static_cast<T*>(a.r);
  T* z = static_cast<T*>(a.z);
  T* d = static_cast<T*>(a.d);
  const T* invd = static_cast<const T*>(a.invd);
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
  if (last_block_total<2, T>(acc, a.part, &c.ticket) && threadIdx.x == 0) {
    c.rr_new = double(acc[0]);
    if (!a.use_amg) inner_decide<T>(a, acc[1]);
  }
}

// p = z + beta p, q = A z + beta q (q = A p by recurrence), p.q and alpha
template <class T>
__global__ void __launch_bounds__(kSB) st_pq_kernel(const __grid_constant__ StreamLaunch a) {
  count_launch(a.launch_acc);
  StreamScal& c = *a.sc;
  if (c.stop) return;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int gs = gridDim.x * blockDim.x;
  const T* z = static_cast<const T*>(a.z);
  T* p = static_cast<T*>(a.p);
  T* q = static_cast<T*>(a.q);
  const T* val = static_cast<const T*>(a.valT);
  const bool first = c.it == 0;
  const T beta = T(c.beta);
  T acc[1] = {T(0)};
  for (int i = gt; i < a.n; i += gs) {
    const T zi = z[i];
    T az = srow<true, T, T>(a.sptr, a.swidth, a.col, val, z, i);
    if (a.dextra) az += T(a.dextra[i]) * zi;
    const T pi = first ? zi : zi + beta * p[i];
    const T qi = first ? az : az + beta * q[i];
    p[i] = pi;
    q[i] = qi;
    acc[0] += pi * qi;
  }
  if (last_block_total<1, T>(acc, a.part, &c.ticket) && threadIdx.x == 0) {
    const T pq = acc[0];
    if (!(pq > T(0))) {       // breakdown: keep d, the outer pass decides
      if (!isfinite(pq)) c.fail |= ST_NONFINITE;
      c.stop = 1;
      c.inner_total += c.it;
      set_cond(a.h_inner, 0u);
      if (c.fail) set_cond(a.h_outer, 0u);
    } else {
      c.alpha = double(T(c.rho) / pq);
    }
  }
}

// d += alpha p, r -= alpha q, |r|^2; Jacobi: z = D^-1 r, r.z and the decision;
// AMG: the level-0 pre-smoothing of the next cycle
template <class T>
__global__ void __launch_bounds__(kSB) st_update_kernel(const __grid_constant__ StreamLaunch a, const T* invd0,
                                                        T omega0, T* x0) {
  count_launch(a.launch_acc);
  StreamScal& c = *a.sc;
  if (c.stop) return;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int gs = gridDim.x * blockDim.x;
  T* r = static_cast<T*>(a.r);
  T* z = static_cast<T*>(a.z);
  T* d = static_cast<T*>(a.d);
  const T* p = static_cast<const T*>(a.p);
  const T* q = static_cast<const T*>(a.q);
  const T* invd = static_cast<const T*>(a.invd);
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
  if (last_block_total<2, T>(acc, a.part, &c.ticket) && threadIdx.x == 0) {
    c.rr_new = double(acc[0]);
    if (!a.use_amg) inner_decide<T>(a, acc[1]);
  }
}

// ---- V(1,1) cycle, one kernel per phase (the cycle of amg.cu) ----------------

// r_l = b_l - A_l x_l
template <class T>
__global__ void __launch_bounds__(kSB) st_vc_res_kernel(const StreamScal* sc, long long* lc,
                                                        const __grid_constant__ AmgLevelDevT<T> L, const T* b,
                                                        int level0) {
  count_launch(lc);
  if (sc->stop) return;
  level_rows<T>(L.A, L.x, level0 != 0, [&](int i, T ax) { L.r[i] = b[i] - ax; });
}

// b_{l+1} = R_l r_l and the next level's pre-smoothing x_{l+1} = w D^-1 b_{l+1}
template <class T>
__global__ void __launch_bounds__(kSB) st_vc_restrict_kernel(const StreamScal* sc, long long* lc,
                                                             const __grid_constant__ AmgLevelDevT<T> L, T* bn,
                                                             const T* invdn, T omegan, T* xn, int level0) {
  count_launch(lc);
  if (sc->stop) return;
  level_rows<T>(L.R, L.r, level0 != 0, [&](int i, T v) {
    bn[i] = v;
    if (xn) xn[i] = omegan * invdn[i] * v;
  });
}

template <class T>
__global__ void __launch_bounds__(kSB) st_vc_coarse_kernel(const StreamScal* sc, long long* lc, const T* cinv, int nc,
                                                           int ldc, const T* bc, T* xc) {
  count_launch(lc);
  if (sc->stop) return;
  const T* bcs[1] = {bc};
  T* xcs[1] = {xc};
  coarse_solve<T, 1>(cinv, nc, ldc, bcs, xcs);
}

// x_l += P_l y_{l+1}
template <class T>
__global__ void __launch_bounds__(kSB) st_vc_prolong_kernel(const StreamScal* sc, long long* lc,
                                                            const __grid_constant__ AmgLevelDevT<T> L, const T* yc,
                                                            int level0) {
  count_launch(lc);
  if (sc->stop) return;
  level_rows<T>(L.P, yc, level0 != 0, [&](int i, T v) { L.x[i] += v; });
}

// y_l = x_l + w D^-1 (b_l - A_l x_l); on level 0 y is z, r.z and the decision
template <class T>
__global__ void __launch_bounds__(kSB) st_vc_post_kernel(const __grid_constant__ StreamLaunch a,
                                                         const __grid_constant__ AmgLevelDevT<T> L, const T* b, T* y,
                                                         int level0) {
  count_launch(a.launch_acc);
  StreamScal& c = *a.sc;
  if (c.stop) return;
  T acc[1] = {T(0)};
  level_rows<T>(L.A, L.x, level0 != 0, [&](int i, T ax) {
    const T bi = b[i];
    const T yi = L.x[i] + L.omega * L.invd[i] * (bi - ax);
    y[i] = yi;
    acc[0] += bi * yi;
  });
  if (!level0) return;
  if (last_block_total<1, T>(acc, a.part, &c.ticket) && threadIdx.x == 0) inner_decide<T>(a, acc[0]);
}

// x += |r| d after an inner solve that ran without failure
__global__ void __launch_bounds__(kSB) st_xupdate_kernel(const __grid_constant__ StreamLaunch a, int f32) {
  count_launch(a.launch_acc);
  const StreamScal& c = *a.sc;
  if (!c.inner_ran || c.fail) return;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int gs = gridDim.x * blockDim.x;
  const double s = c.scale;
  if (f32) {
    const float* d = static_cast<const float*>(a.d);
    for (int i = gt; i < a.n; i += gs) a.x[i] += s * double(d[i]);
  } else {
    const double* d = static_cast<const double*>(a.d);
    for (int i = gt; i < a.n; i += gs) a.x[i] += s * d[i];
  }
}

// normalisation of the singular elliptic solution: the shift (u[pin], or the
// nodal mean)
__global__ void __launch_bounds__(kSB) st_shift_kernel(const __grid_constant__ StreamLaunch a) {
  count_launch(a.launch_acc);
  StreamScal& c = *a.sc;
  if (c.skip) return;
  if (a.pin >= 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) c.shift = a.x[a.pin];
    return;
  }
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int gs = gridDim.x * blockDim.x;
  double acc[1] = {0.0};
  for (int i = gt; i < a.n; i += gs) acc[0] += a.x[i];
  if (last_block_total<1, double>(acc, a.part, &c.ticket) && threadIdx.x == 0) c.shift = acc[0] / double(a.n);
}

// x -= shift (pin >= -1); the solve's status and counters
__global__ void __launch_bounds__(kSB) st_finish_kernel(const __grid_constant__ StreamLaunch a) {
  count_launch(a.launch_acc);
  const StreamScal& c = *a.sc;
  if (c.skip) return;
  if (a.pin >= -1) {
    const double sh = c.shift;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int gs = gridDim.x * blockDim.x;
    for (int i = gt; i < a.n; i += gs) a.x[i] -= sh;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
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

int level_grid(const void* rp, int n) { return grid_for(rp ? int64_t(n) * 32 : int64_t(n)); }

// the V-cycle z = V(r) of one hierarchy on stream s
template <class T>
cudaError_t enqueue_vcycle(const StreamLaunch& a, const AmgDevT<T>& M, const T* r, T* z, cudaStream_t s) {
  const int L = M.nlev;
  for (int l = 0; l < L; ++l) {
    const AmgLevelDevT<T>& Lv = M.L[l];
    const T* b = l == 0 ? r : Lv.b;
    const int l0 = l == 0 ? 1 : 0;
    st_vc_res_kernel<T><<<l0 ? a.grid : level_grid(Lv.A.rp, Lv.A.n), kSB, 0, s>>>(a.sc, a.launch_acc, Lv, b, l0);
    const bool last = l + 1 == L;
    T* bn = last ? M.bc : M.L[l + 1].b;
    const T* invdn = last ? nullptr : M.L[l + 1].invd;
    const T omegan = last ? T(0) : M.L[l + 1].omega;
    T* xn = last ? nullptr : M.L[l + 1].x;
    st_vc_restrict_kernel<T><<<level_grid(Lv.R.rp, Lv.R.n), kSB, 0, s>>>(a.sc, a.launch_acc, Lv, bn, invdn, omegan,
                                                                          xn, l0);
  }
  {
    const int warps = std::max(1, M.nc);
    st_vc_coarse_kernel<T><<<grid_for(int64_t(warps) * 32), kSB, 0, s>>>(a.sc, a.launch_acc, M.cinv, M.nc, M.ldc,
                                                                          M.bc, M.xc);
  }
  for (int l = L - 1; l >= 0; --l) {
    const AmgLevelDevT<T>& Lv = M.L[l];
    const T* yc = l + 1 == L ? M.xc : M.L[l + 1].y;
    const int l0 = l == 0 ? 1 : 0;
    st_vc_prolong_kernel<T><<<level_grid(Lv.P.rp, Lv.P.n), kSB, 0, s>>>(a.sc, a.launch_acc, Lv, yc, l0);
    const T* b = l == 0 ? r : Lv.b;
    T* y = l == 0 ? z : Lv.y;
    st_vc_post_kernel<T><<<l0 ? a.grid : level_grid(Lv.A.rp, Lv.A.n), kSB, 0, s>>>(a, Lv, b, y, l0);
  }
  return cudaGetLastError();
}

// add a WHILE node after the current capture frontier of `cap` and return its
// body graph; the capture continues after the node
cudaError_t add_while(cudaStream_t cap, cudaGraphConditionalHandle h, cudaGraph_t* body) {
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

cudaGraph_t capture_graph(cudaStream_t s) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess) return nullptr;
  return cs == cudaStreamCaptureStatusActive ? g : nullptr;
}

// the solve's kernels and loops, appended to the capture of `st`
template <class T>
cudaError_t enqueue_solve(StreamLaunch a, const AmgDevT<T>* M, cudaStream_t st, const cudaStream_t* side) {
  cudaGraph_t g = capture_graph(st);
  if (!g) return cudaErrorStreamCaptureUnsupported;
  cudaGraphConditionalHandle ho, hi;
  cudaError_t e = cudaGraphConditionalHandleCreate(&ho, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hi, g, 0, 0);
  if (e != cudaSuccess) return e;
  a.h_outer = static_cast<unsigned long long>(ho);
  a.h_inner = static_cast<unsigned long long>(hi);
  const bool amg = a.use_amg && M;
  const T* invd0 = amg ? M->L[0].invd : nullptr;
  const T omega0 = amg ? M->L[0].omega : T(0);
  T* x0 = amg ? M->L[0].x : nullptr;
  T* r = static_cast<T*>(a.r);
  T* z = static_cast<T*>(a.z);

  st_rhs_kernel<T><<<a.grid, kSB, 0, st>>>(a);
  cudaGraph_t ob = nullptr;
  if ((e = add_while(st, ho, &ob)) != cudaSuccess) return e;
  // outer body: residual and decision, inner start, inner loop, x update
  if ((e = cudaStreamBeginCaptureToGraph(side[0], ob, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return e;
  st_outer_kernel<T><<<a.grid, kSB, 0, side[0]>>>(a);
  st_inner_init_kernel<T><<<a.grid, kSB, 0, side[0]>>>(a, invd0, omega0, x0);
  if (amg) enqueue_vcycle<T>(a, *M, r, z, side[0]);
  cudaGraph_t ib = nullptr;
  e = add_while(side[0], hi, &ib);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(side[1], ib, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    st_pq_kernel<T><<<a.grid, kSB, 0, side[1]>>>(a);
    st_update_kernel<T><<<a.grid, kSB, 0, side[1]>>>(a, invd0, omega0, x0);
    if (amg) enqueue_vcycle<T>(a, *M, r, z, side[1]);
    cudaGraph_t tmp = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(side[1], &tmp);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) st_xupdate_kernel<<<a.grid, kSB, 0, side[0]>>>(a, sizeof(T) == 4 ? 1 : 0);
  {
    cudaGraph_t tmp = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(side[0], &tmp);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return e;
  if (a.pin >= -1) st_shift_kernel<<<a.grid, kSB, 0, st>>>(a);
  st_finish_kernel<<<a.grid, kSB, 0, st>>>(a);
  return cudaGetLastError();
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

// Outside a capture the solve is captured into a graph of its own, launched
// and destroyed (the eager and profiling paths); inside one it is appended.
cudaError_t stream_solve(const StreamLaunch& a, int f32, const AmgDevF* M32, const AmgDev* M64, cudaStream_t st,
                         const cudaStream_t* side) {
  cudaStreamCaptureStatus cs;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  auto body = [&]() { return f32 ? enqueue_solve<float>(a, M32, st, side) : enqueue_solve<double>(a, M64, st, side); };
  if (cs == cudaStreamCaptureStatusActive) return body();
  if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
  const cudaError_t r = body();
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(st, &g);
  if (r != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return e;
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return e;
  e = cudaGraphLaunch(ex, st);
  cudaGraphExecDestroy(ex);   // released once the launch completes
  return e;
}

}  // namespace bd
