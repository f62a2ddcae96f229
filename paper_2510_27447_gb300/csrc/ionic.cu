// ionic.cu -- node-wise kernels of the partitioned SDC step (one thread per
// mesh node, the node's state vector in registers).
//
// Every kernel evaluates the membrane model of Sec. 2 with its exact
// Jacobian (Sec. 3.3.2) through the compile-time sparse dual type and
// eliminates the node's ODE states from the linear system of the ROS2 stage
// (Eq. (3.13)) or of the SDC correction (Eq. (3.20)), leaving one condensed
// unknown per node for the parabolic CG solve.
#include <cuda_runtime.h>
#include <algorithm>
#include <utility>

#include "bd_internal.h"
#include "models.cuh"
#include "segment.cuh"

namespace bd {

namespace {

constexpr int kBlock = kNodeBlock;

__device__ __forceinline__ double stim_current(const uint32_t* bits, int64_t i, const StimTable& st,
                                               double t, double dt) {
  uint32_t b = bits ? bits[i] : 0u;
  double s = 0.0;
  const double eps = 1e-9 * dt;
  while (b) {
    const int k = __ffs(b) - 1;
    b &= b - 1u;
    if ((t - st.t_on[k]) > -eps && (t - st.t_on[k] - st.dur[k]) < -eps) s += st.amp[k];
  }
  return s;
}

template <template <class> class Model>
struct Params;
template <>
struct Params<LR91> {
  template <class T>
  static LR91<T> get(int model) { return LR91<T>::make(model == BD_LR91_PAPER_MOD); }
};
template <>
struct Params<TP06> {
  template <class T>
  static TP06<T> get(int) { return TP06<T>::make(); }
};

// ROS2 stage-2 evaluation point X* = X + k1/gamma with k1_y = z1 + w1 k1_v
// (Eq. (3.13)); z1, w1 point at the node's entry of stage 1's vectors
// (stride n).  On the FP64 path everything is FP64.  On the FP32 path z1 and
// w1 are FP32 values, so k1_y is formed in FP32 and added to the rounded
// state; the voltage xs0 stays FP64 (it also feeds the elliptic and
// parabolic right-hand sides).
template <class T, int NS>
__device__ __forceinline__ void stage_point(const double* xj, double xs0, double k1v, const T* z1, const T* w1,
                                            int64_t n, double inv_gamma, T* xst, T* k1y) {
  xst[0] = T(xs0);
  const T kv = T(k1v), ig = T(inv_gamma);
#pragma unroll
  for (int k = 1; k < NS; ++k) {
    k1y[k - 1] = z1[(k - 1) * n] + w1[(k - 1) * n] * kv;
    xst[k] = T(xj[k]) + k1y[k - 1] * ig;
  }
}

// ---------------------------------------------------------------------------
// condensation kernel: S1, S2 and correction modes
// ---------------------------------------------------------------------------
template <template <class> class Model, class T, int MODE, int NQ = 0>
__device__ __forceinline__ void ionic_body(const IonicLaunch& L, const Model<T>& P, int64_t i) {
  using Mod = Model<T>;
  constexpr int NS = Mod::NS;
  if (i >= L.n) return;
  if (L.gate && *L.gate == 0) return;
  const int64_t n = L.n;
  const double t = *L.t_now;
  const double istim = stim_current(L.stim_bits, i, L.stim, t, L.dt);

  double xj[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) xj[k] = L.XJ[k * n + i];

  if constexpr (MODE == MODE_S2P) {
    // stage 2 without a second Jacobian: field at X* = X + k1/gamma, then
    // z = A^-1 rho with stage 1's stored condensation; the condensed diagonal
    // and w are stage 1's (unchanged)
    const double k1v = L.k1v[i];
    const double xs0 = xj[0] + k1v * L.inv_gamma;
    T xst[NS];
    T k1y[NS - 1];
    stage_point<T, NS>(xj, xs0, k1v, static_cast<const T*>(L.z1) + i, static_cast<const T*>(L.w1) + i, n,
                       L.inv_gamma, xst, k1y);
    ValSink<T, Mod> fs;
    P.eval(xst, T(istim), T(L.inv_cm), fs);
    T rho[NS - 1];
    const T ck1 = T(L.ck1);
#pragma unroll
    for (int k = 1; k < NS; ++k) rho[k - 1] = fs.f[k] - ck1 * k1y[k - 1];
    T corr, z[NS - 1];
    cond_solve<T, Mod>(static_cast<const T*>(L.pack) + i, n, rho, corr, z);
    L.rl[i] = L.ML[i] * (double(fs.f[0]) + double(corr));
    T* zo = static_cast<T*>(L.z);
#pragma unroll
    for (int k = 0; k < NS - 1; ++k) zo[k * n + i] = z[k];
    L.avec[i] = xs0 + L.u[i];
    if (L.bvec) L.bvec[i] = k1v;
  } else {
    T xt[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) xt[k] = T(xj[k]);

    JacSink<T, Mod> e;
    // field and Jacobian at this state may have been stored by an earlier
    // launch (same state, time and stimulus): load them, no evaluation.  The
    // FP32 predictor has no load path: it would cost it registers and, at
    // 66k nodes, its single wave of blocks.
    constexpr bool kLoad = MODE == MODE_CORR || (MODE == MODE_S1 && sizeof(T) == 8);
    if (kLoad && L.jac_in) {
      jac_load<T, Mod>(e, static_cast<const T*>(L.jac_in) + i, n);
    } else {
      P.eval(xt, T(istim), T(L.inv_cm), e);
    }

    T rho[NS - 1];
    double fv;                        // node field f_v at the F point
    double avec = 0.0, bvec = 0.0;
    if constexpr (MODE == MODE_S1) {
#pragma unroll
      for (int k = 1; k < NS; ++k) rho[k - 1] = e.f[k];
      fv = double(e.f[0]);
      avec = xj[0] + L.u[i];
      if (L.pack) cond_store<T, Mod>(e, T(L.alpha), static_cast<T*>(L.pack) + i, n);
      // the field goes with the Jacobian only where a later predictor loads
      // both (FP64); the FP32 predictor keeps fewer values live without it
      if (L.jac_out) jac_store<T, Mod, sizeof(T) == 8>(e, static_cast<T*>(L.jac_out) + i, n);
      if (L.fq_out) {
        T* fo = static_cast<T*>(L.fq_out);
#pragma unroll
        for (int k = 0; k < NS; ++k) fo[k * n + i] = e.f[k];
      }
    } else if constexpr (MODE == MODE_S2) {
      // F point X* = X + k1/gamma, k1_y = z1 + w1 k1_v
      const double k1v = L.k1v[i];
      const double xs0 = xj[0] + k1v * L.inv_gamma;
      T xst[NS];
      T k1y[NS - 1];
      stage_point<T, NS>(xj, xs0, k1v, static_cast<const T*>(L.z1) + i, static_cast<const T*>(L.w1) + i, n,
                         L.inv_gamma, xst, k1y);
      ValSink<T, Mod> fs;
      P.eval(xst, T(istim), T(L.inv_cm), fs);
      const T ck1 = T(L.ck1);
#pragma unroll
      for (int k = 1; k < NS; ++k) rho[k - 1] = fs.f[k] - ck1 * k1y[k - 1];
      fv = double(fs.f[0]);
      avec = xs0 + L.u[i];
      bvec = k1v;
    } else {
      // correction: rho = [(X_m^new - X~_{m+1}) + sum_j S_j f_j] / dt_m on the y rows
      // (the stored fields are values of T: the quadrature sum runs in T, the
      // state difference in FP64 before it is rounded)
      T q[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) q[k] = T(0);
      double av = 0.0;
      // NQ quadrature nodes, known at compile time: the node loop unrolls and
      // every pointer of L is read at a constant offset
#pragma unroll
      for (int jn = 0; jn < NQ; ++jn) {
        const T S = T(L.S[jn]);
        const T* fj = static_cast<const T*>(L.fq[jn]);
#pragma unroll
        for (int k = 0; k < NS; ++k) q[k] += S * fj[k * n + i];
        av += L.S[jn] * (L.Xq[jn][i] + L.uq[jn][i]);
      }
      const T idt = T(L.inv_dt);
#pragma unroll
      for (int k = 1; k < NS; ++k) rho[k - 1] = (T(L.Xprev[k * n + i] - xj[k]) + q[k]) * idt;
      fv = double(q[0]) * L.inv_dt;
      avec = av;
      bvec = L.Xprev[i] - xj[0];
    }

    T s, corr;
    T z[NS - 1], w[NS - 1];
    condense<T, Mod>(e, T(L.alpha), rho, s, corr, z, w);
    double sd = double(s);
    if (sd < L.smin) {
      sd = L.smin;
      atomicAdd(L.clamp_count, 1ull);
    }
    const double ml = L.ML[i];
    L.dgs[i] = ml * sd;
    L.rl[i] = ml * (fv + double(corr));
    T* zo = static_cast<T*>(L.z);
    T* wo = static_cast<T*>(L.w);
#pragma unroll
    for (int k = 0; k < NS - 1; ++k) {
      zo[k * n + i] = z[k];
      wo[k * n + i] = w[k];
    }
    L.avec[i] = avec;
    if (L.bvec) L.bvec[i] = bvec;
  }
}

template <template <class> class Model, class T, int MODE, int NQ = 0>
__global__ void __launch_bounds__(kBlock) ionic_kernel(const IonicLaunch L, const Model<T> P) {
  ionic_body<Model, T, MODE, NQ>(L, P, int64_t(blockIdx.x) * blockDim.x + threadIdx.x);
}

// the same over the nodes of a batch of handles (parameters per handle)
template <template <class> class Model, class T, int MODE, int NQ = 0>
__global__ void __launch_bounds__(kBlock) ionic_batch_kernel(const IonicLaunch* tab, const int* blk, int nseg,
                                                             const Model<T> P) {
  const SegInfo sg = seg_locate(blk, nseg);
  const IonicLaunch& L = stage(tab, sg.r);
  ionic_body<Model, T, MODE, NQ>(L, P, int64_t(sg.lb) * blockDim.x + threadIdx.x);
}

template <template <class> class Model, class T>
__device__ __forceinline__ void field_body(int64_t n, const double* X, double inv_cm, double dt,
                                           const uint32_t* stim_bits, const double* t_now, const StimTable& stim,
                                           void* foutv, const Model<T>& P, const int* gate, int64_t i) {
  using Mod = Model<T>;
  constexpr int NS = Mod::NS;
  if (i >= n) return;
  if (gate && *gate == 0) return;
  const double t = t_now ? *t_now : 0.0;
  const double istim = stim_current(stim_bits, i, stim, t, dt);
  T x[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) x[k] = T(X[k * n + i]);
  ValSink<T, Mod> fs;
  P.eval(x, T(istim), T(inv_cm), fs);
  T* fout = static_cast<T*>(foutv);
#pragma unroll
  for (int k = 0; k < NS; ++k) fout[k * n + i] = fs.f[k];
}

template <template <class> class Model, class T>
__global__ void __launch_bounds__(kBlock) field_kernel(int64_t n, const double* X, double inv_cm, double dt,
                                                       const uint32_t* stim_bits, const double* t_now,
                                                       const StimTable stim, void* fout, const Model<T> P,
                                                       const int* gate) {
  field_body<Model, T>(n, X, inv_cm, dt, stim_bits, t_now, stim, fout, P, gate,
                       int64_t(blockIdx.x) * blockDim.x + threadIdx.x);
}

template <template <class> class Model, class T>
__global__ void __launch_bounds__(kBlock) field_batch_kernel(const FieldArgs* tab, const int* blk, int nseg,
                                                             const Model<T> P) {
  const SegInfo sg = seg_locate(blk, nseg);
  const FieldArgs& a = stage(tab, sg.r);
  field_body<Model, T>(a.n, a.X, a.inv_cm, a.dt, a.stim_bits, a.t_now, a.stim, a.fout, P, nullptr,
                       int64_t(sg.lb) * blockDim.x + threadIdx.x);
}

// X_{m+1} = X + m1 k1 + m2 k2, k_y = z + w k_v  (ROS2 combination, Eq. (3.14)).
// With err != nullptr also the embedded error estimate: X_hat = X + k1/gamma,
// |X_{m+1} - X_hat| / (etol (1 + |X_{m+1}|)), maximum over the launch
// accumulated with an order-independent atomicMax on the bit pattern.
template <int NS, class ZT>
__global__ void __launch_bounds__(kBlock) combine_kernel(int64_t n, const double* src, const double* k1v,
                                                         const ZT* z1, const ZT* w1, const double* k2v,
                                                         const ZT* z2, const ZT* w2, double m1, double m2,
                                                         double* dst, const int* gate, double mhat1, double etol,
                                                         unsigned long long* err) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (i < n && !(gate && *gate == 0)) {
    const double a = k1v[i], b = k2v[i];
    const double x0 = src[i] + m1 * a + m2 * b;
    dst[i] = x0;
    if (err) e = fabs(x0 - (src[i] + mhat1 * a)) / (etol * (1.0 + fabs(x0)));
    if constexpr (sizeof(ZT) == 4) {
      // FP32 stage vectors: the increment m1 k1 + m2 k2 is formed in FP32
      // and added to the FP64 state (one conversion and one FP64 add per
      // variable: GB300's FP64 pipe, not memory, bounds the FP64 form)
      const float af = float(a), bf = float(b), m1f = float(m1), m2f = float(m2), mhf = float(mhat1);
#pragma unroll
      for (int k = 1; k < NS; ++k) {
        const int64_t o = (k - 1) * n + i;
        const float k1 = z1[o] + w1[o] * af;
        const float k2 = z2[o] + w2[o] * bf;
        const float inc = m1f * k1 + m2f * k2;
        const double xk = src[k * n + i] + double(inc);
        dst[k * n + i] = xk;
        if (err) e = fmax(e, double(fabsf(inc - mhf * k1)) / (etol * (1.0 + fabs(xk))));
      }
    } else {
#pragma unroll
      for (int k = 1; k < NS; ++k) {
        const int64_t o = (k - 1) * n + i;
        const double k1 = z1[o] + w1[o] * a;
        const double k2 = z2[o] + w2[o] * b;
        const double xs = src[k * n + i];
        const double xk = xs + m1 * k1 + m2 * k2;
        dst[k * n + i] = xk;
        if (err) e = fmax(e, fabs(xk - (xs + mhat1 * k1)) / (etol * (1.0 + fabs(xk))));
      }
    }
  }
  if (err) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = fmax(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0 && e > 0.0) atomicMax(err, (unsigned long long)__double_as_longlong(e));
  }
}

// Reaction half step of the CN-RK2 splitting (Sec. 3.3.3): the explicit
// midpoint rule over h = dt/2 on the node ODE system with the step's stimulus,
//   X_mid = X + (h/2) f(X),   X_out = X + h f(X_mid),
// starting from X with dv added to v (the Crank-Nicolson increment, or none).
// With avec != nullptr also writes avec = v_out + u, the operand of the
// diffusion step's right-hand side.
template <template <class> class Model, class T>
__global__ void __launch_bounds__(kBlock) rk2_kernel(int64_t n, const double* X, const double* dv, double* Xout,
                                                     double h, double inv_cm, double dt, const uint32_t* stim_bits,
                                                     const double* t_now, const StimTable stim, const double* u,
                                                     double* avec, const Model<T> P) {
  using Mod = Model<T>;
  constexpr int NS = Mod::NS;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double istim = stim_current(stim_bits, i, stim, *t_now, dt);
  double x[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) x[k] = X[k * n + i];
  if (dv) x[0] += dv[i];
  T xt[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) xt[k] = T(x[k]);
  ValSink<T, Mod> f1;
  P.eval(xt, T(istim), T(inv_cm), f1);
#pragma unroll
  for (int k = 0; k < NS; ++k) xt[k] = T(x[k] + 0.5 * h * double(f1.f[k]));
  ValSink<T, Mod> f2;
  P.eval(xt, T(istim), T(inv_cm), f2);
#pragma unroll
  for (int k = 0; k < NS; ++k) Xout[k * n + i] = x[k] + h * double(f2.f[k]);
  if (avec) avec[i] = x[0] + h * double(f2.f[0]) + u[i];
}

// X^new_{m+1} = X~_{m+1} + eps, eps_y = z + w eps_v
template <int NS, class ZT>
__global__ void __launch_bounds__(kBlock) update_kernel(int64_t n, const double* Xt, const double* ev,
                                                        const ZT* z, const ZT* w, double* dst,
                                                        const int* gate) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (gate && *gate == 0) return;
  const double e = ev[i];
  dst[i] = Xt[i] + e;
  if constexpr (sizeof(ZT) == 4) {   // FP32 increment added to the FP64 state
    const float ef = float(e);
#pragma unroll
    for (int k = 1; k < NS; ++k) {
      const int64_t o = (k - 1) * n + i;
      dst[k * n + i] = Xt[k * n + i] + double(z[o] + w[o] * ef);
    }
  } else {
#pragma unroll
    for (int k = 1; k < NS; ++k) {
      const int64_t o = (k - 1) * n + i;
      dst[k * n + i] = Xt[k * n + i] + z[o] + w[o] * e;
    }
  }
}

// end of step: activation times, X^n <- X^{n+1}, u^n <- u^{n+1}
__global__ void __launch_bounds__(256) finish_kernel(int ns, int64_t n, int64_t nu, double* Xn, const double* Xlast,
                                                     double* u0, const double* ulast, double* t_act, double v_act,
                                                     double dt, const double* t_now, int* status) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const double t = *t_now;
  if (i < n) {
    const double vo = Xn[i], vn = Xlast[i];
    if (!isfinite(vn)) atomicOr(status, ST_NONFINITE);
    if (isnan(t_act[i]) && vo < v_act && vn >= v_act) t_act[i] = t + (v_act - vo) / (vn - vo) * dt;
    for (int k = 0; k < ns; ++k) Xn[k * n + i] = Xlast[k * n + i];
  }
  if (i < nu) u0[i] = ulast[i];
  // every block reads the clock above; it advances in a separate one-thread
  // launch so no block can see the new value early
}

// simulated time t^{n+1} = t^n + dt (t_now[1] keeps t^n) and the step counter
__global__ void bump_kernel(long long* step_n, double* t_now, double dt) {
  *step_n += 1;
  t_now[1] = t_now[0];
  t_now[0] += dt;
}

// Initial guesses of the elliptic solves of sweep 2 (a warm start only: the
// solves converge to their tolerance from any guess).  e = u2 holds the
// sweep-1 solution E(v^n) at every node; with ep = the same quantity of the
// previous step, u at t^n + c dt is extrapolated linearly in time:
// u1 = e + c1 r (e - ep), u2 = e + r (e - ep), r = dt / (t^n - t^{n-1}).
// clk = (t^n, t^{n-1}, valid); ep becomes e.
__global__ void extrap_kernel(int64_t n, double* u1, double* u2, double* ep, double c1, double dt,
                              const double* clk, const int* gate) {
  if (gate && *gate == 0) return;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double h = clk[0] - clk[1];
  const double r = (clk[2] != 0.0 && h > 0.0) ? fmin(dt / h, 4.0) : 0.0;
  const double e = u2[i];
  const double d = e - ep[i];
  if (u1) u1[i] = e + c1 * r * d;
  u2[i] = e + r * d;
  ep[i] = e;
}

__global__ void set_valid_kernel(double* clk, const int* gate) {
  if (gate && *gate == 0) return;
  clk[2] = 1.0;
}

__global__ void sweep_delta_kernel(int64_t n, const double* a, const double* b, unsigned long long* dmax,
                                   const int* gate) {
  if (gate && *gate == 0) return;
  double m = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    m = fmax(m, fabs(a[i] - b[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  // non-negative doubles order like their bit patterns: the maximum is exact
  // and independent of the order of the updates
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(dmax, (unsigned long long)__double_as_longlong(m));
}

__global__ void sweep_gate_kernel(const unsigned long long* dmax, double tol, int* gate, long long* sweeps) {
  if (*gate == 0) return;
  const double d = __longlong_as_double((long long)*dmax);
  if (d < tol) *gate = 0;
  else *sweeps += 1;
}

__global__ void set_int_kernel(int* p, int v, unsigned long long* clear) {
  *p = v;
  if (clear) *clear = 0ull;
}

__global__ void clear_gated_kernel(unsigned long long* p, const int* gate) {
  if (gate && *gate == 0) return;
  *p = 0ull;
}

// ---- batched forms of the node-wise kernels (one launch over many handles)
// Each block works on one handle's nodes with that handle's arguments; the
// arithmetic per node is the one of the single-handle kernels above.

template <int NS, class ZT>
__global__ void __launch_bounds__(kBlock) combine_batch_kernel(const CombineArgs* tab, const int* blk, int nseg) {
  const SegInfo sg = seg_locate(blk, nseg);
  const CombineArgs& a = stage(tab, sg.r);
  const int64_t i = int64_t(sg.lb) * blockDim.x + threadIdx.x;
  const int64_t n = a.n;
  if (i >= n) return;
  const double k1 = a.k1v[i], k2 = a.k2v[i];
  a.dst[i] = a.src[i] + a.m1 * k1 + a.m2 * k2;
  const ZT *z1 = static_cast<const ZT*>(a.z1), *w1 = static_cast<const ZT*>(a.w1);
  const ZT *z2 = static_cast<const ZT*>(a.z2), *w2 = static_cast<const ZT*>(a.w2);
  if constexpr (sizeof(ZT) == 4) {   // as combine_kernel: FP32 increment, FP64 state
    const float af = float(k1), bf = float(k2), m1f = float(a.m1), m2f = float(a.m2);
#pragma unroll
    for (int k = 1; k < NS; ++k) {
      const int64_t o = (k - 1) * n + i;
      const float y1 = z1[o] + w1[o] * af;
      const float y2 = z2[o] + w2[o] * bf;
      a.dst[k * n + i] = a.src[k * n + i] + double(m1f * y1 + m2f * y2);
    }
  } else {
#pragma unroll
    for (int k = 1; k < NS; ++k) {
      const int64_t o = (k - 1) * n + i;
      const double y1 = z1[o] + w1[o] * k1;
      const double y2 = z2[o] + w2[o] * k2;
      a.dst[k * n + i] = a.src[k * n + i] + a.m1 * y1 + a.m2 * y2;
    }
  }
}

template <int NS, class ZT>
__global__ void __launch_bounds__(kBlock) update_batch_kernel(const UpdateArgs* tab, const int* blk, int nseg) {
  const SegInfo sg = seg_locate(blk, nseg);
  const UpdateArgs& a = stage(tab, sg.r);
  const int64_t i = int64_t(sg.lb) * blockDim.x + threadIdx.x;
  const int64_t n = a.n;
  if (i >= n) return;
  const double e = a.ev[i];
  a.dst[i] = a.Xt[i] + e;
  const ZT *z = static_cast<const ZT*>(a.z), *w = static_cast<const ZT*>(a.w);
  if constexpr (sizeof(ZT) == 4) {   // as update_kernel: FP32 increment, FP64 state
    const float ef = float(e);
#pragma unroll
    for (int k = 1; k < NS; ++k) {
      const int64_t o = (k - 1) * n + i;
      a.dst[k * n + i] = a.Xt[k * n + i] + double(z[o] + w[o] * ef);
    }
  } else {
#pragma unroll
    for (int k = 1; k < NS; ++k) {
      const int64_t o = (k - 1) * n + i;
      a.dst[k * n + i] = a.Xt[k * n + i] + z[o] + w[o] * e;
    }
  }
}

__global__ void __launch_bounds__(kVecBlock) copy_batch_kernel(const CopyArgs* tab, const int* blk, int nseg) {
  const SegInfo sg = seg_locate(blk, nseg);
  const CopyArgs& a = stage(tab, sg.r);
  const int64_t i = int64_t(sg.lb) * blockDim.x + threadIdx.x;
  if (i < a.n) a.dst[i] = a.src[i];
}

// extrap_kernel per handle; the clock's valid flag is set by the per-handle
// kernel below, after every block of the handle has read the clock
__global__ void __launch_bounds__(kVecBlock) extrap_batch_kernel(const ExtrapArgs* tab, const int* blk, int nseg) {
  const SegInfo sg = seg_locate(blk, nseg);
  const ExtrapArgs& a = stage(tab, sg.r);
  const int64_t i = int64_t(sg.lb) * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const double h = a.clk[0] - a.clk[1];
  const double r = (a.clk[2] != 0.0 && h > 0.0) ? fmin(a.dt / h, 4.0) : 0.0;
  const double e = a.u2[i];
  const double d = e - a.ep[i];
  if (a.u1) a.u1[i] = e + a.c1 * r * d;
  a.u2[i] = e + r * d;
  a.ep[i] = e;
}
__global__ void set_valid_batch_kernel(const ExtrapArgs* tab, int nseg) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nseg) tab[r].clk[2] = 1.0;
}

__global__ void __launch_bounds__(kVecBlock) finish_batch_kernel(const FinishArgs* tab, const int* blk, int nseg) {
  const SegInfo sg = seg_locate(blk, nseg);
  const FinishArgs& a = stage(tab, sg.r);
  const int64_t i = int64_t(sg.lb) * blockDim.x + threadIdx.x;
  const double t = *a.t_now;
  if (i < a.n) {
    const double vo = a.Xn[i], vn = a.Xlast[i];
    if (!isfinite(vn)) atomicOr(a.status, ST_NONFINITE);
    if (isnan(a.t_act[i]) && vo < a.v_act && vn >= a.v_act) a.t_act[i] = t + (a.v_act - vo) / (vn - vo) * a.dt;
    for (int k = 0; k < a.ns; ++k) a.Xn[k * a.n + i] = a.Xlast[k * a.n + i];
  }
  if (i < a.nu) a.u0[i] = a.ulast[i];
}
__global__ void bump_batch_kernel(const FinishArgs* tab, int nseg) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nseg) return;
  const FinishArgs& a = tab[r];
  *a.step_n += 1;
  a.t_now[1] = a.t_now[0];
  a.t_now[0] += a.dt;
}

template <template <class> class Model, class T>
cudaError_t launch_ionic_batch_t(const IonicLaunch& L, const IonicLaunch* tab, const int* blk, int nseg, int nb,
                                 cudaStream_t st) {
  const auto P = Params<Model>::template get<T>(L.model);
  switch (L.mode) {
    case MODE_S1: ionic_batch_kernel<Model, T, MODE_S1><<<nb, kBlock, 0, st>>>(tab, blk, nseg, P); break;
    case MODE_S2: ionic_batch_kernel<Model, T, MODE_S2><<<nb, kBlock, 0, st>>>(tab, blk, nseg, P); break;
    case MODE_S2P: ionic_batch_kernel<Model, T, MODE_S2P><<<nb, kBlock, 0, st>>>(tab, blk, nseg, P); break;
    default:
      if (L.n_nodes == 3) ionic_batch_kernel<Model, T, MODE_CORR, 3><<<nb, kBlock, 0, st>>>(tab, blk, nseg, P);
      else ionic_batch_kernel<Model, T, MODE_CORR, 2><<<nb, kBlock, 0, st>>>(tab, blk, nseg, P);
      break;
  }
  return cudaGetLastError();
}

template <template <class> class Model, class T>
cudaError_t launch_ionic_t(const IonicLaunch& L, cudaStream_t st) {
  const auto P = Params<Model>::template get<T>(L.model);
  const unsigned grid = unsigned((L.n + kBlock - 1) / kBlock);
  switch (L.mode) {
    case MODE_S1: ionic_kernel<Model, T, MODE_S1><<<grid, kBlock, 0, st>>>(L, P); break;
    case MODE_S2: ionic_kernel<Model, T, MODE_S2><<<grid, kBlock, 0, st>>>(L, P); break;
    case MODE_S2P: ionic_kernel<Model, T, MODE_S2P><<<grid, kBlock, 0, st>>>(L, P); break;
    default:
      if (L.n_nodes == 3) ionic_kernel<Model, T, MODE_CORR, 3><<<grid, kBlock, 0, st>>>(L, P);
      else ionic_kernel<Model, T, MODE_CORR, 2><<<grid, kBlock, 0, st>>>(L, P);
      break;
  }
  return cudaGetLastError();
}

}  // namespace

int cond_pack_values(int model) {
  return model == BD_TP06_EPI ? cond_pack_size<TP06<double>>() : cond_pack_size<LR91<double>>();
}

int jac_pack_values(int model) {
  return model == BD_TP06_EPI ? jac_pack_size<TP06<double>>() : jac_pack_size<LR91<double>>();
}

int model_ns(int model) {
  switch (model) {
    case BD_LR91:
    case BD_LR91_PAPER_MOD: return 8;
    case BD_TP06_EPI: return 19;
    default: return 0;
  }
}

cudaError_t launch_ionic(const IonicLaunch& L, cudaStream_t st) {
  if (L.n == 0) return cudaSuccess;
  const bool f32 = L.precision == BD_MIXED;
  if (L.model == BD_TP06_EPI) return f32 ? launch_ionic_t<TP06, float>(L, st) : launch_ionic_t<TP06, double>(L, st);
  return f32 ? launch_ionic_t<LR91, float>(L, st) : launch_ionic_t<LR91, double>(L, st);
}

cudaError_t launch_ionic_batch(const IonicLaunch& L, const IonicLaunch* tab, const int* blk, int nseg, int nb,
                               cudaStream_t st) {
  if (nb == 0) return cudaSuccess;
  const bool f32 = L.precision == BD_MIXED;
  if (L.model == BD_TP06_EPI)
    return f32 ? launch_ionic_batch_t<TP06, float>(L, tab, blk, nseg, nb, st)
               : launch_ionic_batch_t<TP06, double>(L, tab, blk, nseg, nb, st);
  return f32 ? launch_ionic_batch_t<LR91, float>(L, tab, blk, nseg, nb, st)
             : launch_ionic_batch_t<LR91, double>(L, tab, blk, nseg, nb, st);
}

cudaError_t launch_field_batch(int model, int precision, const FieldArgs* tab, const int* blk, int nseg, int nb,
                               cudaStream_t st) {
  if (nb == 0) return cudaSuccess;
  const bool f32 = precision == BD_MIXED;
  if (model == BD_TP06_EPI) {
    if (f32) field_batch_kernel<TP06, float><<<nb, kBlock, 0, st>>>(tab, blk, nseg, TP06<float>::make());
    else field_batch_kernel<TP06, double><<<nb, kBlock, 0, st>>>(tab, blk, nseg, TP06<double>::make());
  } else {
    const bool pm = model == BD_LR91_PAPER_MOD;
    if (f32) field_batch_kernel<LR91, float><<<nb, kBlock, 0, st>>>(tab, blk, nseg, LR91<float>::make(pm));
    else field_batch_kernel<LR91, double><<<nb, kBlock, 0, st>>>(tab, blk, nseg, LR91<double>::make(pm));
  }
  return cudaGetLastError();
}

cudaError_t launch_combine_batch(int model, int zw32, const CombineArgs* tab, const int* blk, int nseg, int nb,
                                 cudaStream_t st) {
  if (nb == 0) return cudaSuccess;
  const bool tp = model == BD_TP06_EPI;
  if (zw32) {
    if (tp) combine_batch_kernel<19, float><<<nb, kBlock, 0, st>>>(tab, blk, nseg);
    else combine_batch_kernel<8, float><<<nb, kBlock, 0, st>>>(tab, blk, nseg);
  } else {
    if (tp) combine_batch_kernel<19, double><<<nb, kBlock, 0, st>>>(tab, blk, nseg);
    else combine_batch_kernel<8, double><<<nb, kBlock, 0, st>>>(tab, blk, nseg);
  }
  return cudaGetLastError();
}

cudaError_t launch_update_batch(int model, int zw32, const UpdateArgs* tab, const int* blk, int nseg, int nb,
                                cudaStream_t st) {
  if (nb == 0) return cudaSuccess;
  const bool tp = model == BD_TP06_EPI;
  if (zw32) {
    if (tp) update_batch_kernel<19, float><<<nb, kBlock, 0, st>>>(tab, blk, nseg);
    else update_batch_kernel<8, float><<<nb, kBlock, 0, st>>>(tab, blk, nseg);
  } else {
    if (tp) update_batch_kernel<19, double><<<nb, kBlock, 0, st>>>(tab, blk, nseg);
    else update_batch_kernel<8, double><<<nb, kBlock, 0, st>>>(tab, blk, nseg);
  }
  return cudaGetLastError();
}

cudaError_t launch_copy_batch(const CopyArgs* tab, const int* blk, int nseg, int nb, cudaStream_t st) {
  if (nb == 0) return cudaSuccess;
  copy_batch_kernel<<<nb, kVecBlock, 0, st>>>(tab, blk, nseg);
  return cudaGetLastError();
}

cudaError_t launch_extrap_batch(const ExtrapArgs* tab, const int* blk, int nseg, int nb, cudaStream_t st) {
  if (nb > 0) extrap_batch_kernel<<<nb, kVecBlock, 0, st>>>(tab, blk, nseg);
  set_valid_batch_kernel<<<(nseg + 127) / 128, 128, 0, st>>>(tab, nseg);
  return cudaGetLastError();
}

cudaError_t launch_finish_batch(const FinishArgs* tab, const int* blk, int nseg, int nb, cudaStream_t st) {
  if (nb > 0) finish_batch_kernel<<<nb, kVecBlock, 0, st>>>(tab, blk, nseg);
  bump_batch_kernel<<<(nseg + 127) / 128, 128, 0, st>>>(tab, nseg);
  return cudaGetLastError();
}

cudaError_t launch_field(int model, int precision, int64_t n, const double* X, double inv_cm, double dt,
                         const uint32_t* stim_bits, const double* step_n, const StimTable& stim, void* fout,
                         cudaStream_t st, const int* gate) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = unsigned((n + kBlock - 1) / kBlock);
  const bool f32 = precision == BD_MIXED;
  if (model == BD_TP06_EPI) {
    if (f32) field_kernel<TP06, float><<<grid, kBlock, 0, st>>>(n, X, inv_cm, dt, stim_bits, step_n, stim, fout, TP06<float>::make(), gate);
    else field_kernel<TP06, double><<<grid, kBlock, 0, st>>>(n, X, inv_cm, dt, stim_bits, step_n, stim, fout, TP06<double>::make(), gate);
  } else {
    const bool pm = model == BD_LR91_PAPER_MOD;
    if (f32) field_kernel<LR91, float><<<grid, kBlock, 0, st>>>(n, X, inv_cm, dt, stim_bits, step_n, stim, fout, LR91<float>::make(pm), gate);
    else field_kernel<LR91, double><<<grid, kBlock, 0, st>>>(n, X, inv_cm, dt, stim_bits, step_n, stim, fout, LR91<double>::make(pm), gate);
  }
  return cudaGetLastError();
}

cudaError_t launch_rk2(int model, int precision, int64_t n, const double* X, const double* dv, double* Xout,
                       double h, double inv_cm, double dt, const uint32_t* stim_bits, const double* t_now,
                       const StimTable& stim, const double* u, double* avec, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = unsigned((n + kBlock - 1) / kBlock);
  const bool f32 = precision == BD_MIXED;
  if (model == BD_TP06_EPI) {
    if (f32) rk2_kernel<TP06, float><<<grid, kBlock, 0, st>>>(n, X, dv, Xout, h, inv_cm, dt, stim_bits, t_now, stim, u, avec, TP06<float>::make());
    else rk2_kernel<TP06, double><<<grid, kBlock, 0, st>>>(n, X, dv, Xout, h, inv_cm, dt, stim_bits, t_now, stim, u, avec, TP06<double>::make());
  } else {
    const bool pm = model == BD_LR91_PAPER_MOD;
    if (f32) rk2_kernel<LR91, float><<<grid, kBlock, 0, st>>>(n, X, dv, Xout, h, inv_cm, dt, stim_bits, t_now, stim, u, avec, LR91<float>::make(pm));
    else rk2_kernel<LR91, double><<<grid, kBlock, 0, st>>>(n, X, dv, Xout, h, inv_cm, dt, stim_bits, t_now, stim, u, avec, LR91<double>::make(pm));
  }
  return cudaGetLastError();
}

namespace {
template <class ZT>
void combine_typed(int model, unsigned grid, cudaStream_t st, int64_t n, const double* src, const double* k1v,
                   const void* z1, const void* w1, const double* k2v, const void* z2, const void* w2, double m1,
                   double m2, double* dst, const int* gate, double mhat1, double etol, unsigned long long* err) {
  const ZT *a = static_cast<const ZT*>(z1), *b = static_cast<const ZT*>(w1);
  const ZT *c = static_cast<const ZT*>(z2), *d = static_cast<const ZT*>(w2);
  if (model == BD_TP06_EPI)
    combine_kernel<19, ZT><<<grid, kBlock, 0, st>>>(n, src, k1v, a, b, k2v, c, d, m1, m2, dst, gate, mhat1, etol, err);
  else
    combine_kernel<8, ZT><<<grid, kBlock, 0, st>>>(n, src, k1v, a, b, k2v, c, d, m1, m2, dst, gate, mhat1, etol, err);
}
}  // namespace

cudaError_t launch_combine(int model, int zw32, int64_t n, const double* src, const double* k1v, const void* z1,
                           const void* w1, const double* k2v, const void* z2, const void* w2, double m1,
                           double m2, double* dst, cudaStream_t st, const int* gate, double mhat1, double etol,
                           unsigned long long* err) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = unsigned((n + kBlock - 1) / kBlock);
  if (zw32) combine_typed<float>(model, grid, st, n, src, k1v, z1, w1, k2v, z2, w2, m1, m2, dst, gate, mhat1, etol, err);
  else combine_typed<double>(model, grid, st, n, src, k1v, z1, w1, k2v, z2, w2, m1, m2, dst, gate, mhat1, etol, err);
  return cudaGetLastError();
}

cudaError_t launch_update(int model, int zw32, int64_t n, const double* Xt, const double* ev, const void* z,
                          const void* w, double* dst, cudaStream_t st, const int* gate) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = unsigned((n + kBlock - 1) / kBlock);
  const bool tp = model == BD_TP06_EPI;
  if (zw32) {
    const float *a = static_cast<const float*>(z), *b = static_cast<const float*>(w);
    if (tp) update_kernel<19, float><<<grid, kBlock, 0, st>>>(n, Xt, ev, a, b, dst, gate);
    else update_kernel<8, float><<<grid, kBlock, 0, st>>>(n, Xt, ev, a, b, dst, gate);
  } else {
    const double *a = static_cast<const double*>(z), *b = static_cast<const double*>(w);
    if (tp) update_kernel<19, double><<<grid, kBlock, 0, st>>>(n, Xt, ev, a, b, dst, gate);
    else update_kernel<8, double><<<grid, kBlock, 0, st>>>(n, Xt, ev, a, b, dst, gate);
  }
  return cudaGetLastError();
}

cudaError_t launch_extrap(int64_t n, double* u1, double* u2, double* ep, double c1, double dt, double* clk,
                          const int* gate, cudaStream_t st) {
  if (n > 0) extrap_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(n, u1, u2, ep, c1, dt, clk, gate);
  set_valid_kernel<<<1, 1, 0, st>>>(clk, gate);
  return cudaGetLastError();
}

cudaError_t launch_finish(int ns, int64_t n, int64_t nu, double* Xn, const double* Xlast, double* u0,
                          const double* ulast, double* t_act, double v_act, double dt, long long* step_n,
                          double* t_now, int* status, cudaStream_t st) {
  const int64_t m = std::max(n, nu);
  if (m > 0) {
    const unsigned grid = unsigned((m + 255) / 256);
    finish_kernel<<<grid, 256, 0, st>>>(ns, n, nu, Xn, Xlast, u0, ulast, t_act, v_act, dt, t_now, status);
  }
  bump_kernel<<<1, 1, 0, st>>>(step_n, t_now, dt);
  return cudaGetLastError();
}

cudaError_t launch_sweep_delta(int64_t n, const double* a, const double* b, unsigned long long* dmax,
                               const int* gate, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = unsigned(std::min<int64_t>((n + 255) / 256, 4096));
  sweep_delta_kernel<<<grid, 256, 0, st>>>(n, a, b, dmax, gate);
  return cudaGetLastError();
}

cudaError_t launch_sweep_gate(const unsigned long long* dmax, double tol, int* gate, long long* sweeps,
                              cudaStream_t st) {
  sweep_gate_kernel<<<1, 1, 0, st>>>(dmax, tol, gate, sweeps);
  return cudaGetLastError();
}

cudaError_t launch_set_int(int* p, int v, unsigned long long* clear, cudaStream_t st) {
  set_int_kernel<<<1, 1, 0, st>>>(p, v, clear);
  return cudaGetLastError();
}

cudaError_t launch_clear_gated(unsigned long long* p, const int* gate, cudaStream_t st) {
  clear_gated_kernel<<<1, 1, 0, st>>>(p, gate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host-side helpers: rest state and the standalone evaluation entry point
// ---------------------------------------------------------------------------

namespace {

template <class Mod>
void field_host(const Mod& P, const double* x, double* f, double J[kMaxNS][kMaxNS]) {
  DenseSink<double, Mod> s;
  P.eval(x, 0.0, 1.0, s);
  for (int r = 0; r < Mod::NS; ++r) {
    f[r] = s.f[r];
    for (int c = 0; c < Mod::NS; ++c) J[r][c] = s.J[r][c];
  }
}

// Newton on the single-cell field f(x) = 0 with dense partial pivoting.
template <class Mod>
void newton_rest(const Mod& P, double* x) {
  constexpr int n = Mod::NS;
  for (int it = 0; it < 60; ++it) {
    double f[kMaxNS], J[kMaxNS][kMaxNS];
    field_host(P, x, f, J);
    double A[kMaxNS][kMaxNS + 1];
    for (int r = 0; r < n; ++r) {
      for (int c = 0; c < n; ++c) A[r][c] = J[r][c];
      A[r][n] = -f[r];
    }
    for (int k = 0; k < n; ++k) {
      int piv = k;
      for (int r = k + 1; r < n; ++r)
        if (std::fabs(A[r][k]) > std::fabs(A[piv][k])) piv = r;
      if (piv != k)
        for (int c = 0; c <= n; ++c) std::swap(A[k][c], A[piv][c]);
      for (int r = k + 1; r < n; ++r) {
        const double l = A[r][k] / A[k][k];
        for (int c = k; c <= n; ++c) A[r][c] -= l * A[k][c];
      }
    }
    double dx[kMaxNS];
    double rel = 0.0;
    for (int r = n - 1; r >= 0; --r) {
      double s = A[r][n];
      for (int c = r + 1; c < n; ++c) s -= A[r][c] * dx[c];
      dx[r] = s / A[r][r];
    }
    for (int r = 0; r < n; ++r) {
      x[r] += dx[r];
      rel = std::fmax(rel, std::fabs(dx[r]) / std::fmax(std::fabs(x[r]), 1e-12));
    }
    if (rel < 1e-13) break;
  }
}

template <template <class> class Model, class T>
__global__ void eval_kernel(int64_t n, const double* X, const double* istim, double inv_cm, double* f, double* jac,
                            const Model<T> P) {
  using Mod = Model<T>;
  constexpr int NS = Mod::NS;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T x[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) x[k] = T(X[k * n + i]);
  const T is = istim ? T(istim[i]) : T(0);
  DenseSink<T, Mod> s;
  P.eval(x, is, T(inv_cm), s);
  for (int r = 0; r < NS; ++r) {
    f[r * n + i] = double(s.f[r]);
    if (jac)
      for (int c = 0; c < NS; ++c) jac[(i * NS + r) * NS + c] = double(s.J[r][c]);
  }
}

}  // namespace

void rest_state_host(int model, double* x) {
  if (model == BD_TP06_EPI) {
    // TP06 conserves charge (the stimulus is carried by K+), so its Jacobian
    // is singular at rest; the published initial values are used instead.
    TP06<double>::initial(x);
    return;
  }
  LR91<double>::initial(x);
  newton_rest(LR91<double>::make(model == BD_LR91_PAPER_MOD), x);
}

cudaError_t launch_eval(int model, int precision, int64_t n, const double* X, const double* istim, double inv_cm,
                        double* f, double* jac, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = unsigned((n + 63) / 64);
  const bool f32 = precision == BD_MIXED;
  if (model == BD_TP06_EPI) {
    if (f32) eval_kernel<TP06, float><<<grid, 64, 0, st>>>(n, X, istim, inv_cm, f, jac, TP06<float>::make());
    else eval_kernel<TP06, double><<<grid, 64, 0, st>>>(n, X, istim, inv_cm, f, jac, TP06<double>::make());
  } else {
    const bool pm = model == BD_LR91_PAPER_MOD;
    if (f32) eval_kernel<LR91, float><<<grid, 64, 0, st>>>(n, X, istim, inv_cm, f, jac, LR91<float>::make(pm));
    else eval_kernel<LR91, double><<<grid, 64, 0, st>>>(n, X, istim, inv_cm, f, jac, LR91<double>::make(pm));
  }
  return cudaGetLastError();
}

void pattern_host(int model, uint32_t* masks) {
  if (model == BD_TP06_EPI) {
    for (int r = 0; r < 19; ++r) masks[r] = TP06<double>::ROWMASK[r];
  } else {
    for (int r = 0; r < 8; ++r) masks[r] = LR91<double>::ROWMASK[r];
  }
}

}  // namespace bd
