// mixed.cu -- mixed-precision conjugate gradients for the mixed path.
//
// One persistent cooperative kernel:
//   FP64   b (right-hand side; mean-projected for the singular elliptic
//          operator) and, per outer step, the residual r = b - A x of the
//          FP64 solution x
//   FP32   an inner CG on A d = r from d = 0 with FP32 operator values,
//          vectors and accumulation, preconditioned by Jacobi or by one
//          FP32 AMG V(1,1) cycle, until |r_inner| <= tol_inner |r|
//   FP64   x += d
// With max_outer > 1 the outer step repeats until |b - A x| <= tol |b| in
// FP64 (iterative refinement: the elliptic solve keeps FP64 accuracy while
// every Krylov iteration runs in FP32); with max_outer = 1 the single FP32
// solve is the answer (the well-conditioned condensed parabolic systems).
// FP64 partial sums use their own slots (part), FP32 ones another buffer
// (partf); each slot is rewritten only after a barrier that follows its
// last read, as in pcg.cu.
#include <cuda_runtime.h>

#include "bd_internal.h"
#include "sparse.cuh"
#include "vcycle.cuh"

namespace bd {

namespace {

template <int WMAX, bool AMG, int TPB, int MINB = BD_SOLVER_MIN_BLOCKS>
__global__ void __launch_bounds__(TPB, MINB) pcg_mixed_kernel(const __grid_constant__ PcgLaunch a,
                                                             const __grid_constant__ MixedLaunch m,
                                                             const AmgDevF* __restrict__ Mp, float* partf) {
  __shared__ AmgDevF sM;    // descriptor staged in shared memory (see pcg_amg_kernel)
  if constexpr (AMG) load_descriptor(sM, Mp);
  const AmgDevF& M = sM;
  __shared__ double shd[4][32];
  __shared__ float shf[4][32];
  if (a.gate && *a.gate == 0) return;
  const int n = a.n;
  const int nb = gridDim.x;
  const int stride = blockDim.x * gridDim.x;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;

  // ---- FP64 right-hand side, FP32 Jacobi scaling ---------------------------
  // Without mean projection the first outer residual is final here and is
  // formed in the same pass (one device barrier fewer).
  const bool fused = !a.project;
  double acc0[3] = {0.0, 0.0, 0.0};
  // the right-hand side products and the warm residual's A x share the
  // operator pattern: one pass over each row
  const double* const pv[3] = {a.val1, a.val2, a.valA};
  const double* const px[3] = {a.va, a.vb, a.x};
  const bool pon[3] = {a.val1 != nullptr, a.val2 != nullptr, fused && a.warm != 0};
  for (int i = i0; i < n; i += stride) {
    double sp[3];
    sell_row_multi<3>(a.sptr, a.swidth, a.col, pv, px, pon, i, sp);
    double b = a.rl ? a.rl[i] : 0.0;
    if (a.val1) b += a.c1 * sp[0];
    if (a.val2) b += a.c2 * sp[1];
    m.b64[i] = b;
    double d = a.valA[a.diagpos[i]];
    if (a.dextra) d += a.dextra[i];
    m.invd32[i] = float(1.0 / d);
    acc0[0] += b;
    acc0[1] += b * b;
    if (fused) {
      double r = b;
      if (a.warm) r = b - ((a.dextra ? a.dextra[i] * a.x[i] : 0.0) + sp[2]);
      m.r64[i] = r;
      acc0[2] += r * r;
    }
  }
  if (!a.warm)
    for (int i = i0; i < n; i += stride) a.x[i] = 0.0;
  block_sum<3, double>(acc0, shd);
  if (threadIdx.x == 0) {
    a.part[blockIdx.x * 4 + 0] = acc0[0];
    a.part[blockIdx.x * 4 + 1] = acc0[1];
    a.part[blockIdx.x * 4 + 2] = acc0[2];
  }
  if (!grid_barrier(a.bar, nb, a.status)) return;
  double tot[3] = {0.0, 0.0, 0.0};
  if (fused) {
    grid_total<3, double>(a.part, {0, 1, 2}, nb, tot, shd);
  } else {
    double t01[2];
    grid_total<2, double>(a.part, {0, 1}, nb, t01, shd);
    tot[0] = t01[0];
    tot[1] = t01[1];
  }
  const double mean_b = a.project ? tot[0] / double(n) : 0.0;
  double bb = a.project ? tot[1] - double(n) * mean_b * mean_b : tot[1];
  if (bb < 0.0) bb = 0.0;
  const double tol2 = a.tol * a.tol * bb;
  if (a.project)
    for (int i = i0; i < n; i += stride) m.b64[i] -= mean_b;

  int fail = 0;
  long long inner_total = 0;
  long long outer_total = 0;
  for (int outer = 0;; ++outer) {
    ++outer_total;
    // ---- FP64 outer residual ---------------------------------------------
    double rr64 = tot[2];   // the first pass of a fused start has it already
    if (!(outer == 0 && fused)) {
      double accr[1] = {0.0};
      if (outer == 0 && !a.warm) {
        for (int i = i0; i < n; i += stride) {
          const double r = m.b64[i];
          m.r64[i] = r;
          accr[0] += r * r;
        }
      } else {
        for (int i = i0; i < n; i += stride) {
          const double ax = (a.dextra ? a.dextra[i] * a.x[i] : 0.0) + sell_row<WMAX, true>(a, a.valA, a.x, i);
          const double r = m.b64[i] - ax;
          m.r64[i] = r;
          accr[0] += r * r;
        }
      }
      block_sum<1, double>(accr, shd);
      if (threadIdx.x == 0) a.part[blockIdx.x * 4 + 2] = accr[0];
      if (!grid_barrier(a.bar, nb, a.status)) return;
      double t1[1];
      grid_total<1, double>(a.part, {2}, nb, t1, shd);
      rr64 = t1[0];
    }
    if (!isfinite(rr64)) {
      fail = ST_NONFINITE;
      break;
    }
    if (m.max_outer > 1 && rr64 <= tol2) break;
    if (outer >= m.max_outer) {
      if (m.max_outer > 1) fail = ST_NOT_CONVERGED;
      break;
    }
    if (!(rr64 > 0.0)) break;   // b = 0 with x = 0
    // the inner system is scaled to a unit residual (FP32 range is then never
    // an issue, whatever the magnitude of b) and solved until its residual is
    // tol_inner, or just what the outer tolerance still needs
    const double scale = sqrt(rr64);
    const double inv_scale = 1.0 / scale;
    double tgt = double(m.tol_inner) * double(m.tol_inner);
    if (m.max_outer > 1) tgt = fmax(tgt, 0.25 * tol2 / rr64);
    // single solve: the target is tol_inner |b|, so a warm start that already
    // reduced the residual needs fewer iterations (cold: rr64 = |b|^2)
    else if (a.warm) tgt = fmax(tgt, tgt * bb / rr64);
    const float target2 = float(tgt);

    // ---- FP32 inner CG on A d = r / |r| ----------------------------------
    for (int i = i0; i < n; i += stride) {
      m.r32[i] = float(m.r64[i] * inv_scale);
      m.d32[i] = 0.0f;
    }
    int it = 0;
    if (!AMG && m.pipelined) {
      // Pipelined Jacobi-PCG (Ghysels & Vanroose, Parallel Computing 40, 2014):
      // the recurrences w = A u, s = A p, q = M s and z = A q let ONE device
      // barrier per iteration carry both the dot products (r, u), (w, u),
      // (r, r) and the input m = M w of the next product A m.  m is double
      // buffered (neighbours read it while its successor is written); the
      // per-block partial sums alternate between two slot groups.  Its
      // recursively updated residual drifts from b - A d faster than the
      // classic one's, so the host asks for it only for the well-conditioned
      // parabolic systems in the latency-bound 128-register build.
      float* const r = m.r32;
      float* const u = m.r32 + n;
      float* const w = m.z32;
      float* const z = m.z32 + n;
      float* const p = m.p32;
      float* const s = m.p32 + n;
      float* const q = m.q32;
      float* const d = m.d32;
      float* const mb[2] = {m.q32 + n, m.d32 + n};
      for (int i = i0; i < n; i += stride) u[i] = m.invd32[i] * r[i];
      if (!grid_barrier(a.bar, nb, a.status)) return;
      {
        float acc[3] = {0.0f, 0.0f, 0.0f};
        for (int i = i0; i < n; i += stride) {
          const float ui = u[i], ri = r[i];
          float au = a.dextra ? float(a.dextra[i]) * ui : 0.0f;
          au += sell_row<WMAX, true, float>(a.sptr, a.swidth, a.col, m.valA32, u, i);
          w[i] = au;
          mb[0][i] = m.invd32[i] * au;
          acc[0] += ri * ui;
          acc[1] += au * ui;
          acc[2] += ri * ri;
        }
        block_sum<3, float>(acc, shf);
        if (threadIdx.x == 0)
#pragma unroll
          for (int k = 0; k < 3; ++k) partf[blockIdx.x * 8 + k] = acc[k];
        if (!grid_barrier(a.bar, nb, a.status)) return;
      }
      float gam_prev = 1.0f, alpha_prev = 1.0f;
      for (;;) {
        const int par = it & 1;
        const int sl[3] = {4 * par, 4 * par + 1, 4 * par + 2};
        float t[3];
        grid_total<3, float, 8>(partf, sl, nb, t, shf);
        const float gam = t[0], del = t[1], rr = t[2];
        if (!isfinite(rr) || !isfinite(gam) || !isfinite(del)) {
          fail = ST_NONFINITE;
          break;
        }
        if (!(rr > target2)) break;
        if (it >= m.inner_cap) {
          if (m.max_outer == 1) fail = ST_NOT_CONVERGED;
          break;
        }
        const float beta = it == 0 ? 0.0f : gam / gam_prev;
        const float den = it == 0 ? del : del - beta * gam / alpha_prev;
        if (!(den > 0.0f)) {
          if (!isfinite(den)) fail = ST_NONFINITE;
          break;     // FP32 breakdown: keep d, the outer step decides
        }
        const float alpha = gam / den;
        const float* const mc = mb[par];
        float* const mn = mb[par ^ 1];
        float acc[3] = {0.0f, 0.0f, 0.0f};
        for (int i = i0; i < n; i += stride) {
          const float mi = mc[i];
          float ni = a.dextra ? float(a.dextra[i]) * mi : 0.0f;
          ni += sell_row<WMAX, true, float>(a.sptr, a.swidth, a.col, m.valA32, mc, i);
          const float zi = it == 0 ? ni : ni + beta * z[i];
          const float qi = it == 0 ? mi : mi + beta * q[i];
          const float si = it == 0 ? w[i] : w[i] + beta * s[i];
          const float pi = it == 0 ? u[i] : u[i] + beta * p[i];
          z[i] = zi;
          q[i] = qi;
          s[i] = si;
          p[i] = pi;
          d[i] += alpha * pi;
          const float ri = r[i] - alpha * si;
          const float ui = u[i] - alpha * qi;
          const float wi = w[i] - alpha * zi;
          r[i] = ri;
          u[i] = ui;
          w[i] = wi;
          mn[i] = m.invd32[i] * wi;
          acc[0] += ri * ui;
          acc[1] += wi * ui;
          acc[2] += ri * ri;
        }
        block_sum<3, float>(acc, shf);
        if (threadIdx.x == 0)
#pragma unroll
          for (int k = 0; k < 3; ++k) partf[blockIdx.x * 8 + 4 * (par ^ 1) + k] = acc[k];
        if (!grid_barrier(a.bar, nb, a.status)) return;
        gam_prev = gam;
        alpha_prev = alpha;
        ++it;
      }
    } else {
      if constexpr (AMG) {
        if (!vcycle<float, TPB == 512>(M, m.r32, m.z32, a.bar, nb, a.status)) return;
      } else {
        for (int i = i0; i < n; i += stride) m.z32[i] = m.invd32[i] * m.r32[i];
      }
      float accf[2] = {0.0f, 0.0f};
      for (int i = i0; i < n; i += stride) {
        accf[0] += m.r32[i] * m.z32[i];
        accf[1] += m.r32[i] * m.r32[i];
      }
      block_sum<2, float>(accf, shf);
      if (threadIdx.x == 0) {
        partf[blockIdx.x * 4 + 2] = accf[0];
        partf[blockIdx.x * 4 + 3] = accf[1];
      }
      if (!grid_barrier(a.bar, nb, a.status)) return;
      float tf[2];
      grid_total<2, float>(partf, {2, 3}, nb, tf, shf);
      float rho = tf[0];
      float rr = tf[1];
      float beta = 0.0f;
      bool done = !(rr > target2);
      while (!done) {
        float pq[1] = {0.0f};
        for (int i = i0; i < n; i += stride) {
          const float z = m.z32[i];
          float az = a.dextra ? float(a.dextra[i]) * z : 0.0f;
          az += sell_row<WMAX, true, float>(a.sptr, a.swidth, a.col, m.valA32, m.z32, i);
          const float p = it == 0 ? z : z + beta * m.p32[i];
          const float q = it == 0 ? az : az + beta * m.q32[i];
          m.p32[i] = p;
          m.q32[i] = q;
          pq[0] += p * q;
        }
        block_sum<1, float>(pq, shf);
        if (threadIdx.x == 0) partf[blockIdx.x * 4 + 0] = pq[0];
        if (!grid_barrier(a.bar, nb, a.status)) return;
        float tq[1];
        grid_total<1, float>(partf, {0}, nb, tq, shf);
        if (!(tq[0] > 0.0f)) {
          if (!isfinite(tq[0])) fail = ST_NONFINITE;
          break;     // FP32 breakdown: keep d, the outer step decides
        }
        const float alpha = rho / tq[0];
        float rrl = 0.0f;
        for (int i = i0; i < n; i += stride) {
          m.d32[i] += alpha * m.p32[i];
          const float r = m.r32[i] - alpha * m.q32[i];
          m.r32[i] = r;
          rrl += r * r;
        }
        if constexpr (AMG) {
          if (!vcycle<float, TPB == 512>(M, m.r32, m.z32, a.bar, nb, a.status)) return;
        } else {
          for (int i = i0; i < n; i += stride) m.z32[i] = m.invd32[i] * m.r32[i];
        }
        float acc[2] = {0.0f, rrl};
        for (int i = i0; i < n; i += stride) acc[0] += m.r32[i] * m.z32[i];
        block_sum<2, float>(acc, shf);
        if (threadIdx.x == 0) {
          partf[blockIdx.x * 4 + 2] = acc[0];
          partf[blockIdx.x * 4 + 3] = acc[1];
        }
        if (!grid_barrier(a.bar, nb, a.status)) return;
        grid_total<2, float>(partf, {2, 3}, nb, tf, shf);
        ++it;
        rr = tf[1];
        if (!isfinite(rr) || !isfinite(tf[0])) {
          fail = ST_NONFINITE;
          break;
        }
        if (rr <= target2) break;
        if (it >= m.inner_cap) {
          if (m.max_outer == 1) fail = ST_NOT_CONVERGED;
          break;
        }
        beta = tf[0] / rho;
        rho = tf[0];
      }
    }
    inner_total += it;
    if (fail) break;
    for (int i = i0; i < n; i += stride) a.x[i] += scale * double(m.d32[i]);
    if (m.max_outer == 1) break;
    if (!grid_barrier(a.bar, nb, a.status)) return;   // x complete before the next residual
  }

  if (a.pin >= 0) {
    if (!grid_barrier(a.bar, nb, a.status)) return;
    const double shift = __ldcg(a.x + a.pin);
    if (!grid_barrier(a.bar, nb, a.status)) return;
    for (int i = i0; i < n; i += stride) a.x[i] -= shift;
  } else if (a.pin == -1) {
    double sx[1] = {0.0};
    for (int i = i0; i < n; i += stride) sx[0] += a.x[i];
    block_sum<1, double>(sx, shd);
    if (threadIdx.x == 0) a.part[blockIdx.x * 4 + 0] = sx[0];
    if (!grid_barrier(a.bar, nb, a.status)) return;
    double tm[1];
    grid_total<1, double>(a.part, {0}, nb, tm, shd);
    const double mean = tm[0] / double(n);
    for (int i = i0; i < n; i += stride) a.x[i] -= mean;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (fail) atomicOr(a.status, fail);
    if (a.iters_acc) atomicAdd((unsigned long long*)a.iters_acc, (unsigned long long)inner_total);
    if (a.outer_acc) atomicAdd((unsigned long long*)a.outer_acc, (unsigned long long)outer_total);
    if (a.solves_acc) atomicAdd((unsigned long long*)a.solves_acc, 1ull);
  }
}

// Two elliptic solves A_ie u_k = c1 A_i v_k (k = 0, 1; the rhs mean-projected)
// in one launch: the mixed-precision AMG-CG above, run for both right-hand
// sides in lock-step so that they share every device barrier and every pass
// over the operators.  Each right-hand side keeps its own Krylov scalars,
// refinement passes and convergence test; a converged one stops changing.
// Workspace vectors of the second system sit n entries after the first's;
// partd / partf hold 8 values per block.
template <int WMAX, int TPB, int MINB = BD_SOLVER_MIN_BLOCKS>
__global__ void __launch_bounds__(TPB, MINB) pcg_mixed2_kernel(const __grid_constant__ PcgLaunch a,
                                                              const double* va1, double* x1,
                                                              const __grid_constant__ MixedLaunch m,
                                                              const AmgDevF* __restrict__ H0p,
                                                              const AmgDevF* __restrict__ H1p, float* partf,
                                                              double* partd) {
  __shared__ AmgDevF sH0, sH1;   // descriptors staged in shared memory
  load_descriptor(sH0, H0p);
  load_descriptor(sH1, H1p);
  const AmgDevF& H0 = sH0;
  const AmgDevF& H1 = sH1;
  __shared__ double shd[4][32];
  __shared__ float shf[4][32];
  if (a.gate && *a.gate == 0) return;
  const int n = a.n;
  const int nb = gridDim.x;
  const int stride = blockDim.x * gridDim.x;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  double* X[2] = {a.x, x1};
  const double* V[2] = {a.va, va1};
  double* b64[2] = {m.b64, m.b64 + n};
  double* r64[2] = {m.r64, m.r64 + n};
  float* r32[2] = {m.r32, m.r32 + n};
  float* z32[2] = {m.z32, m.z32 + n};
  float* p32[2] = {m.p32, m.p32 + n};
  float* q32[2] = {m.q32, m.q32 + n};
  float* d32[2] = {m.d32, m.d32 + n};

  // ---- FP64 right-hand sides ----------------------------------------------
  double acc0[4] = {0.0, 0.0, 0.0, 0.0};
  const double* const v1v[2] = {a.val1, a.val1};
  const bool both[2] = {true, true};
  for (int i = i0; i < n; i += stride) {
    double sp[2];
    sell_row_multi<2>(a.sptr, a.swidth, a.col, v1v, V, both, i, sp);   // both products in one pass
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double b = a.c1 * sp[k];
      b64[k][i] = b;
      acc0[2 * k] += b;
      acc0[2 * k + 1] += b * b;
    }
  }
  if (!a.warm)
    for (int i = i0; i < n; i += stride) {
      X[0][i] = 0.0;
      X[1][i] = 0.0;
    }
  block_sum<4, double>(acc0, shd);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) partd[blockIdx.x * 8 + k] = acc0[k];
  if (!grid_barrier(a.bar, nb, a.status)) return;
  {
    double t[4];
    grid_total<4, double, 8>(partd, {0, 1, 2, 3}, nb, t, shd);
    for (int k = 0; k < 4; ++k) acc0[k] = t[k];
  }
  double tol2[2];
  for (int k = 0; k < 2; ++k) {
    const double mean_b = a.project ? acc0[2 * k] / double(n) : 0.0;
    double bb = a.project ? acc0[2 * k + 1] - double(n) * mean_b * mean_b : acc0[2 * k + 1];
    if (bb < 0.0) bb = 0.0;
    tol2[k] = a.tol * a.tol * bb;
    if (a.project)
      for (int i = i0; i < n; i += stride) b64[k][i] -= mean_b;
  }

  int fail = 0;
  long long inner_total[2] = {0, 0};
  long long outer_total = 0, shared = 0;
  for (int outer = 0;; ++outer) {
    ++outer_total;
    // ---- FP64 outer residuals -----------------------------------------------
    double accr[2] = {0.0, 0.0};
    const double* const vAv[2] = {a.valA, a.valA};
    const double* const Xc[2] = {X[0], X[1]};
    const bool prod = !(outer == 0 && !a.warm);
    const bool on2[2] = {prod, prod};
    for (int i = i0; i < n; i += stride) {
      double ax[2];
      sell_row_multi<2>(a.sptr, a.swidth, a.col, vAv, Xc, on2, i, ax);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const double r = prod ? b64[k][i] - ax[k] : b64[k][i];
        r64[k][i] = r;
        accr[k] += r * r;
      }
    }
    block_sum<2, double>(accr, shd);
    if (threadIdx.x == 0) {
      partd[blockIdx.x * 8 + 4] = accr[0];
      partd[blockIdx.x * 8 + 5] = accr[1];
    }
    if (!grid_barrier(a.bar, nb, a.status)) return;
    double rr64[2];
    grid_total<2, double, 8>(partd, {4, 5}, nb, rr64, shd);
    if (!isfinite(rr64[0]) || !isfinite(rr64[1])) {
      fail = ST_NONFINITE;
      break;
    }
    bool active[2];
    for (int k = 0; k < 2; ++k) active[k] = rr64[k] > tol2[k] && rr64[k] > 0.0;
    if (!active[0] && !active[1]) break;
    if (outer >= m.max_outer) {
      fail = ST_NOT_CONVERGED;
      break;
    }
    double scale[2] = {1.0, 1.0};
    float target2[2] = {0.0f, 0.0f};
    for (int k = 0; k < 2; ++k)
      if (active[k]) {
        scale[k] = sqrt(rr64[k]);
        double tgt = double(m.tol_inner) * double(m.tol_inner);
        tgt = fmax(tgt, 0.25 * tol2[k] / rr64[k]);
        target2[k] = float(tgt);
      }

    // ---- FP32 inner CG on both unit-scaled systems ---------------------------
    for (int i = i0; i < n; i += stride) {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        r32[k][i] = active[k] ? float(r64[k][i] / scale[k]) : 0.0f;
        d32[k][i] = 0.0f;
      }
    }
    if (!vcycle2<float, TPB == 512>(H0, H1, r32[0], r32[1], z32[0], z32[1], a.bar, nb, a.status)) return;
    float accf[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int i = i0; i < n; i += stride) {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        accf[2 * k] += r32[k][i] * z32[k][i];
        accf[2 * k + 1] += r32[k][i] * r32[k][i];
      }
    }
    block_sum<4, float>(accf, shf);
    if (threadIdx.x == 0)
      for (int k = 0; k < 4; ++k) partf[blockIdx.x * 8 + 2 + k] = accf[k];
    if (!grid_barrier(a.bar, nb, a.status)) return;
    float tf[4];
    grid_total<4, float, 8>(partf, {2, 3, 4, 5}, nb, tf, shf);
    float rho[2] = {tf[0], tf[2]};
    bool done[2];
    for (int k = 0; k < 2; ++k) done[k] = !active[k] || !(tf[2 * k + 1] > target2[k]);
    int it[2] = {0, 0};
    float beta[2] = {0.0f, 0.0f};
    while (!(done[0] && done[1])) {
      float pq[2] = {0.0f, 0.0f};
      for (int i = i0; i < n; i += stride) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (done[k]) continue;
          const float z = z32[k][i];
          const float az = sell_row<WMAX, true, float>(a.sptr, a.swidth, a.col, m.valA32, z32[k], i);
          const float p = it[k] == 0 ? z : z + beta[k] * p32[k][i];
          const float q = it[k] == 0 ? az : az + beta[k] * q32[k][i];
          p32[k][i] = p;
          q32[k][i] = q;
          pq[k] += p * q;
        }
      }
      block_sum<2, float>(pq, shf);
      if (threadIdx.x == 0) {
        partf[blockIdx.x * 8 + 0] = pq[0];
        partf[blockIdx.x * 8 + 1] = pq[1];
      }
      if (!grid_barrier(a.bar, nb, a.status)) return;
      float tq[2];
      grid_total<2, float, 8>(partf, {0, 1}, nb, tq, shf);
      float alpha[2] = {0.0f, 0.0f};
      bool upd[2] = {false, false};
      for (int k = 0; k < 2; ++k) {
        if (done[k]) continue;
        if (!(tq[k] > 0.0f)) {
          if (!isfinite(tq[k])) fail = ST_NONFINITE;
          done[k] = true;          // FP32 breakdown: keep d, the outer step decides
          continue;
        }
        alpha[k] = rho[k] / tq[k];
        upd[k] = true;
      }
      if (upd[0] && upd[1]) ++shared;
      float rrl[2] = {0.0f, 0.0f};
      for (int i = i0; i < n; i += stride) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (!upd[k]) continue;
          d32[k][i] += alpha[k] * p32[k][i];
          const float r = r32[k][i] - alpha[k] * q32[k][i];
          r32[k][i] = r;
          rrl[k] += r * r;
        }
      }
      if (!vcycle2<float, TPB == 512>(H0, H1, r32[0], r32[1], z32[0], z32[1], a.bar, nb, a.status)) return;
      float acc[4] = {0.0f, rrl[0], 0.0f, rrl[1]};
      for (int i = i0; i < n; i += stride) {
        acc[0] += r32[0][i] * z32[0][i];
        acc[2] += r32[1][i] * z32[1][i];
      }
      block_sum<4, float>(acc, shf);
      if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) partf[blockIdx.x * 8 + 2 + k] = acc[k];
      if (!grid_barrier(a.bar, nb, a.status)) return;
      grid_total<4, float, 8>(partf, {2, 3, 4, 5}, nb, tf, shf);
      for (int k = 0; k < 2; ++k) {
        if (!upd[k]) continue;
        ++it[k];
        const float rzk = tf[2 * k], rrk = tf[2 * k + 1];
        if (!isfinite(rrk) || !isfinite(rzk)) {
          fail = ST_NONFINITE;
          done[k] = true;
          continue;
        }
        if (rrk <= target2[k] || it[k] >= m.inner_cap) {
          done[k] = true;
          continue;
        }
        beta[k] = rzk / rho[k];
        rho[k] = rzk;
      }
      if (fail) break;
    }
    inner_total[0] += it[0];
    inner_total[1] += it[1];
    if (fail) break;
    for (int i = i0; i < n; i += stride) {
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (active[k]) X[k][i] += scale[k] * double(d32[k][i]);
    }
    if (!grid_barrier(a.bar, nb, a.status)) return;   // x complete before the next residual
  }

  // ---- normalisation of both singular solutions --------------------------------
  if (a.pin >= 0) {
    const double s0 = __ldcg(X[0] + a.pin), s1 = __ldcg(X[1] + a.pin);
    if (!grid_barrier(a.bar, nb, a.status)) return;
    for (int i = i0; i < n; i += stride) {
      X[0][i] -= s0;
      X[1][i] -= s1;
    }
  } else if (a.pin == -1) {
    double sx[2] = {0.0, 0.0};
    for (int i = i0; i < n; i += stride) {
      sx[0] += X[0][i];
      sx[1] += X[1][i];
    }
    block_sum<2, double>(sx, shd);
    if (threadIdx.x == 0) {
      partd[blockIdx.x * 8 + 0] = sx[0];
      partd[blockIdx.x * 8 + 1] = sx[1];
    }
    if (!grid_barrier(a.bar, nb, a.status)) return;
    double tm[2];
    grid_total<2, double, 8>(partd, {0, 1}, nb, tm, shd);
    for (int i = i0; i < n; i += stride) {
      X[0][i] -= tm[0] / double(n);
      X[1][i] -= tm[1] / double(n);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (fail) atomicOr(a.status, fail);
    if (a.iters_acc) atomicAdd((unsigned long long*)a.iters_acc, (unsigned long long)(inner_total[0] + inner_total[1]));
    if (a.outer_acc) atomicAdd((unsigned long long*)a.outer_acc, (unsigned long long)(2 * outer_total));
    if (a.solves_acc) atomicAdd((unsigned long long*)a.solves_acc, 2ull);
    if (a.pair_acc) atomicAdd((unsigned long long*)a.pair_acc, (unsigned long long)shared);
  }
}

template <int W, int TPB, int MINB = BD_SOLVER_MIN_BLOCKS>
int max_blocks2_t(int block) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pcg_mixed2_kernel<W, TPB, MINB>, block, 0) != cudaSuccess)
    return 0;
  return sms * per;
}

template <int W, bool AMG, int TPB, int MINB = BD_SOLVER_MIN_BLOCKS>
int max_blocks_t(int block) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pcg_mixed_kernel<W, AMG, TPB, MINB>, block, 0) !=
      cudaSuccess)
    return 0;
  return sms * per;
}

// the smallest co-resident count over a build's instantiations keeps every
// launch legal; AMG_MINB is the occupancy bound of its AMG kernels
template <int TPB, int AMG_MINB>
int tier_max_blocks(int block) {
  int m = max_blocks_t<8, false, TPB>(block);
  m = std::min(m, max_blocks_t<0, false, TPB>(block));
  m = std::min(m, max_blocks_t<8, true, TPB, AMG_MINB>(block));
  m = std::min(m, max_blocks_t<0, true, TPB, AMG_MINB>(block));
  m = std::min(m, max_blocks2_t<8, TPB, AMG_MINB>(block));
  m = std::min(m, max_blocks2_t<0, TPB, AMG_MINB>(block));
  return m;
}

// the AMG kernels alone (tier 2 sizes their grid separately)
template <int TPB, int AMG_MINB>
int tier_amg_max_blocks(int block) {
  int m = max_blocks_t<8, true, TPB, AMG_MINB>(block);
  m = std::min(m, max_blocks_t<0, true, TPB, AMG_MINB>(block));
  m = std::min(m, max_blocks2_t<8, TPB, AMG_MINB>(block));
  m = std::min(m, max_blocks2_t<0, TPB, AMG_MINB>(block));
  return m;
}

template <int TPB, int AMG_MINB>
cudaError_t launch_mixed_tier(const cudaLaunchConfig_t& cfg, const PcgLaunch& K, const MixedLaunch& X,
                              const AmgDevF* M, int wmax, float* partf) {
  if (X.use_amg)
    return wmax > 0 ? cudaLaunchKernelEx(&cfg, pcg_mixed_kernel<8, true, TPB, AMG_MINB>, K, X, M, partf)
                    : cudaLaunchKernelEx(&cfg, pcg_mixed_kernel<0, true, TPB, AMG_MINB>, K, X, M, partf);
  return wmax > 0 ? cudaLaunchKernelEx(&cfg, pcg_mixed_kernel<8, false, TPB>, K, X, M, partf)
                  : cudaLaunchKernelEx(&cfg, pcg_mixed_kernel<0, false, TPB>, K, X, M, partf);
}

template <int TPB, int AMG_MINB>
cudaError_t launch_mixed2_tier(const cudaLaunchConfig_t& cfg, const PcgLaunch& K, const double* va1, double* x1,
                               const MixedLaunch& X, const AmgDevF* H0, const AmgDevF* H1, int wmax,
                               float* partf8, double* partd8) {
  return wmax > 0
             ? cudaLaunchKernelEx(&cfg, pcg_mixed2_kernel<8, TPB, AMG_MINB>, K, va1, x1, X, H0, H1, partf8, partd8)
             : cudaLaunchKernelEx(&cfg, pcg_mixed2_kernel<0, TPB, AMG_MINB>, K, va1, x1, X, H0, H1, partf8, partd8);
}

__global__ void to_float_kernel(int64_t n, const double* src, float* dst) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = float(src[i]);
}

}  // namespace

// sell_row's chunked loop serves every width bound (8, 16, 32) with the same
// code, so one instantiation covers them; 0 (rows wider than 32) loops
int pcg_mixed_max_blocks(int block, int tier) {
  if (tier == 1) return tier_max_blocks<512, 1>(block);
  return tier_max_blocks<1024, 1>(block);
}

int pcg_mixed_amg_max_blocks(int block, int tier) {
  if (tier == 1) return tier_amg_max_blocks<512, 1>(block);
  if (tier == 2) return tier_amg_max_blocks<1024, 2>(block);
  return tier_amg_max_blocks<1024, 1>(block);
}

cudaError_t launch_pcg_mixed(const PcgLaunch& P, const MixedLaunch& X, const AmgDevF* M, int wmax, cudaStream_t st,
                             float* partf) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  PcgLaunch K;
  solver_launch_config(P, st, &cfg, attr, &K);
  if (K.tier == 1) return launch_mixed_tier<512, 1>(cfg, K, X, M, wmax, partf);
  if (K.tier == 2) return launch_mixed_tier<1024, 2>(cfg, K, X, M, wmax, partf);
  return launch_mixed_tier<1024, 1>(cfg, K, X, M, wmax, partf);
}

cudaError_t launch_pcg_mixed2(const PcgLaunch& P, const double* va1, double* x1, const MixedLaunch& X,
                              const AmgDevF* H0, const AmgDevF* H1, int wmax, cudaStream_t st, float* partf8,
                              double* partd8) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  PcgLaunch K;
  solver_launch_config(P, st, &cfg, attr, &K);
  if (K.tier == 1) return launch_mixed2_tier<512, 1>(cfg, K, va1, x1, X, H0, H1, wmax, partf8, partd8);
  if (K.tier == 2) return launch_mixed2_tier<1024, 2>(cfg, K, va1, x1, X, H0, H1, wmax, partf8, partd8);
  return launch_mixed2_tier<1024, 1>(cfg, K, va1, x1, X, H0, H1, wmax, partf8, partd8);
}

// cluster launches use tier 0 (full-size blocks)
bool mixed_cluster_ok(int block, int size) {
  return solver_cluster_ok(pcg_mixed_kernel<8, true, 1024>, block, size) &&
         solver_cluster_ok(pcg_mixed_kernel<0, true, 1024>, block, size) &&
         solver_cluster_ok(pcg_mixed_kernel<8, false, 1024>, block, size) &&
         solver_cluster_ok(pcg_mixed_kernel<0, false, 1024>, block, size) &&
         solver_cluster_ok(pcg_mixed2_kernel<8, 1024>, block, size) &&
         solver_cluster_ok(pcg_mixed2_kernel<0, 1024>, block, size);
}

// values of a SELL-32 operator into the SELL-32/4 layout (one thread per row
// of a slice; the slice's SELL-32 width w, its SELL-32/4 width w4 = the next
// multiple of 4)
__global__ void sell_v4_kernel(int64_t n_slices, const int64_t* sptr, const int* sw, const int64_t* sptr4,
                               const float* src, float* dst) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t s = t >> 5;
  const int l = int(t & 31);
  if (s >= n_slices) return;
  const int w = sw[s], w4 = (w + 3) & ~3;
  for (int k = 0; k < w4; ++k)
    dst[sptr4[s] + 128 * (k >> 2) + 4 * l + (k & 3)] = k < w ? src[sptr[s] + 32 * k + l] : 0.0f;
}

cudaError_t launch_sell_v4(int64_t n_slices, const int64_t* sptr, const int* sw, const int64_t* sptr4,
                           const float* src, float* dst, cudaStream_t st) {
  if (n_slices == 0) return cudaSuccess;
  sell_v4_kernel<<<unsigned((n_slices * 32 + 255) / 256), 256, 0, st>>>(n_slices, sptr, sw, sptr4, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_to_float(int64_t n, const double* src, float* dst, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  to_float_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(n, src, dst);
  return cudaGetLastError();
}

}  // namespace bd
