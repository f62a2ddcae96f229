// pcg.cu -- Jacobi-preconditioned conjugate gradients as one persistent,
// cooperatively launched kernel.
//
// Used for the elliptic constraint A_ie u = -A_i v (Eq. (3.15)) and for the
// condensed parabolic systems (alpha M + A_i + M_L diag(s)) k_v = r of the
// ROS2 stages (Eq. (3.13)) and of the SDC correction (Eq. (3.20)).  The
// paper solves these with BiCGSTAB + block Jacobi / AMG (Sec. 3.3.2); the
// node-wise elimination done in the ionic kernels makes the systems
// symmetric positive (semi-)definite, so plain PCG applies.
//
// One launch runs the whole solve: rows are distributed over all threads of
// a grid that is resident on the device at once (cooperative launch), and
// the iteration synchronises with a device-wide barrier.  Per iteration:
//   phase A  beta, p = z + beta p, q = A z + beta q   (q = A p by recurrence;
//            reads z of other rows, written before the previous barrier)
//            partial p.q                                          -> barrier
//   phase B  alpha = rho / p.q, x += alpha p, r -= alpha q, z = D^-1 r,
//            partial r.z and r.r                                  -> barrier
// Reductions are deterministic: per-block partials, then every block sums
// the partials in the same fixed order.  Every barrier wait is bounded; on
// timeout the kernel records ST_TIMEOUT and returns.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "bd_internal.h"
#include "sparse.cuh"

namespace bd {

namespace {

template <int WMAX, int TPB>
__global__ void __launch_bounds__(TPB, BD_SOLVER_MIN_BLOCKS) pcg_kernel(const __grid_constant__ PcgLaunch a) {
  __shared__ double sh[4][32];
  if (a.gate && *a.gate == 0) return;   // same value for every block: all skip together
  const int n = a.n;
  const int nb = gridDim.x;
  const int stride = blockDim.x * gridDim.x;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;

  // ---- phase 0: right-hand side, initial residual --------------------------
  // Without mean projection the residual is final here, so phase 1 (z = D^-1 r
  // and its dot products) runs in the same pass: one device barrier fewer.
  const bool fused = !a.project;
  double acc0[4] = {0.0, 0.0, 0.0, 0.0};
  // the right-hand side products and the warm residual's A x share the
  // operator pattern: one pass over each row
  const double* const pv[3] = {a.val1, a.val2, a.valA};
  const double* const px[3] = {a.va, a.vb, a.x};
  const bool pon[3] = {a.val1 != nullptr, a.val2 != nullptr, a.warm != 0};
  for (int i = i0; i < n; i += stride) {
    double sp[3];
    sell_row_multi<3>(a.sptr, a.swidth, a.col, pv, px, pon, i, sp);
    double b = a.rl ? a.rl[i] : 0.0;
    if (a.val1) b += a.c1 * sp[0];
    if (a.val2) b += a.c2 * sp[1];
    double d = a.valA[a.diagpos[i]];
    if (a.dextra) d += a.dextra[i];
    a.invd[i] = 1.0 / d;
    double r = b;
    if (a.warm) {
      const double ax = (a.dextra ? a.dextra[i] * a.x[i] : 0.0) + sp[2];
      r -= ax;
    }
    a.r[i] = r;
    acc0[0] += b;
    acc0[1] += b * b;
    if (fused) {
      const double z = r * a.invd[i];
      a.z[i] = z;
      acc0[2] += r * z;
      acc0[3] += r * r;
    }
  }
  if (!a.warm)
    for (int i = i0; i < n; i += stride) a.x[i] = 0.0;
  block_sum<4>(acc0, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) a.part[blockIdx.x * 4 + k] = acc0[k];
  if (!grid_barrier(a.bar, nb, a.status)) return;
  double tot[4] = {0.0, 0.0, 0.0, 0.0};
  if (fused) {
    grid_total<4>(a.part, {0, 1, 2, 3}, nb, tot, sh);
  } else {
    double t01[2];
    grid_total<2>(a.part, {0, 1}, nb, t01, sh);
    tot[0] = t01[0];
    tot[1] = t01[1];
  }
  const double mean_b = a.project ? tot[0] / double(n) : 0.0;
  double bb = a.project ? tot[1] - double(n) * mean_b * mean_b : tot[1];
  if (bb < 0.0) bb = 0.0;
  const double tol2 = a.tol * a.tol * bb;

  // ---- phase 1: z = D^-1 r, p = z (projected systems) ---------------------
  if (!fused) {
    double acc1[2] = {0.0, 0.0};
    for (int i = i0; i < n; i += stride) {
      const double r = a.r[i] - mean_b;
      a.r[i] = r;
      const double z = r * a.invd[i];
      a.z[i] = z;
      acc1[0] += r * z;
      acc1[1] += r * r;
    }
    block_sum<2>(acc1, sh);
    if (threadIdx.x == 0) {
      a.part[blockIdx.x * 4 + 2] = acc1[0];
      a.part[blockIdx.x * 4 + 3] = acc1[1];
    }
    if (!grid_barrier(a.bar, nb, a.status)) return;
    double t23[2];
    grid_total<2>(a.part, {2, 3}, nb, t23, sh);
    tot[2] = t23[0];
    tot[3] = t23[1];
  }
  double rho = tot[2];
  double rr = tot[3];

  int it = 0;
  int fail = 0;
  bool done = !(rr > tol2);      // includes b = 0
  double beta = 0.0;
  while (!done) {
    // phase A
    double pq[1] = {0.0};
    for (int i = i0; i < n; i += stride) {
      const double z = a.z[i];
      double az = a.dextra ? a.dextra[i] * z : 0.0;
      az += sell_row<WMAX, true>(a, a.valA, a.z, i);   // reads other blocks' z through L2
      const double p = it == 0 ? z : z + beta * a.p[i];
      const double q = it == 0 ? az : az + beta * a.q[i];
      a.p[i] = p;
      a.q[i] = q;
      pq[0] += p * q;
    }
    block_sum<1>(pq, sh);
    if (threadIdx.x == 0) a.part[blockIdx.x * 4 + 0] = pq[0];
    if (!grid_barrier(a.bar, nb, a.status)) return;
    double t1[1];
    grid_total<1>(a.part, {0}, nb, t1, sh);
    if (!(t1[0] > 0.0)) {
      fail = isfinite(t1[0]) ? ST_INDEFINITE : ST_NONFINITE;
      break;
    }
    const double alpha = rho / t1[0];
    // phase B
    double acc[2] = {0.0, 0.0};
    for (int i = i0; i < n; i += stride) {
      a.x[i] += alpha * a.p[i];
      const double r = a.r[i] - alpha * a.q[i];
      a.r[i] = r;
      const double z = r * a.invd[i];
      a.z[i] = z;
      acc[0] += r * z;
      acc[1] += r * r;
    }
    block_sum<2>(acc, sh);
    if (threadIdx.x == 0) {
      a.part[blockIdx.x * 4 + 2] = acc[0];
      a.part[blockIdx.x * 4 + 3] = acc[1];
    }
    if (!grid_barrier(a.bar, nb, a.status)) return;
    double tk[2];
    grid_total<2>(a.part, {2, 3}, nb, tk, sh);
    ++it;
    rr = tk[1];
    if (!isfinite(rr)) {
      fail = ST_NONFINITE;
      break;
    }
    if (rr <= tol2) break;
    if (it >= a.maxit) {
      fail = ST_NOT_CONVERGED;
      break;
    }
    beta = tk[0] / rho;
    rho = tk[0];
  }

  // ---- normalisation of the singular elliptic solution ----------------------
  if (a.pin >= 0) {
    const double shift = __ldcg(a.x + a.pin);
    if (!grid_barrier(a.bar, nb, a.status)) return;
    for (int i = i0; i < n; i += stride) a.x[i] -= shift;
  } else if (a.pin == -1) {
    double sx[1] = {0.0};
    for (int i = i0; i < n; i += stride) sx[0] += a.x[i];
    block_sum<1>(sx, sh);
    if (threadIdx.x == 0) a.part[blockIdx.x * 4 + 0] = sx[0];
    if (!grid_barrier(a.bar, nb, a.status)) return;
    double t1[1];
    grid_total<1>(a.part, {0}, nb, t1, sh);
    const double mean = t1[0] / double(n);
    for (int i = i0; i < n; i += stride) a.x[i] -= mean;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (fail) atomicOr(a.status, fail);
    if (a.iters_acc) atomicAdd((unsigned long long*)a.iters_acc, (unsigned long long)it);
    if (a.solves_acc) atomicAdd((unsigned long long*)a.solves_acc, 1ull);
  }
}

__global__ void axpby_kernel(int64_t n, double a, const double* X, double b, const double* Y, double* out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * X[i] + b * Y[i];
}

__global__ void copy_kernel(int64_t n, const double* src, double* dst, const int* gate) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gate && *gate == 0) return;
  if (i < n) dst[i] = src[i];
}

}  // namespace

namespace {
template <int W, int TPB>
int max_blocks_t(int block) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pcg_kernel<W, TPB>, block, 0) != cudaSuccess) return 0;
  return sms * per;
}
}  // namespace

// one block waits at a device-wide barrier sized for two blocks: the second
// never exists, so the wait runs out and records ST_TIMEOUT
__global__ void wait_selftest_kernel(unsigned* bar, int* status) { grid_barrier(bar, 2u, status); }

cudaError_t launch_wait_selftest(unsigned* bar, int* status, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(bar, status);
  return cudaGetLastError();
}

// cluster launches use tier 0 (full-size blocks)
bool pcg_cluster_ok(int block, int size) {
  return solver_cluster_ok(pcg_kernel<8, 1024>, block, size) && solver_cluster_ok(pcg_kernel<0, 1024>, block, size);
}

// sell_row's chunked loop serves every width bound (8, 16, 32) with the same
// code, so one instantiation covers them; 0 (rows wider than 32) loops
int pcg_max_blocks(int block, int wmax, int tier) {
  if (tier == 1) return wmax > 0 ? max_blocks_t<8, 512>(block) : max_blocks_t<0, 512>(block);
  return wmax > 0 ? max_blocks_t<8, 1024>(block) : max_blocks_t<0, 1024>(block);
}

void solver_launch_config(const PcgLaunch& P, cudaStream_t st, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr,
                          PcgLaunch* Pk) {
  *cfg = cudaLaunchConfig_t{};
  *Pk = P;
  cfg->blockDim = dim3(unsigned(P.block));
  cfg->dynamicSmemBytes = 0;
  cfg->stream = st;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
  if (P.cluster > 0) {
    cfg->gridDim = dim3(unsigned(P.cluster));
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(P.cluster);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    Pk->bar = nullptr;
    Pk->grid = P.cluster;
    Pk->tier = 0;
  } else {
    cfg->gridDim = dim3(unsigned(P.grid));
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
  }
}

cudaError_t launch_pcg(const PcgLaunch& P, int wmax, cudaStream_t st) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  PcgLaunch K;
  solver_launch_config(P, st, &cfg, attr, &K);
  if (K.tier == 1)
    return wmax > 0 ? cudaLaunchKernelEx(&cfg, pcg_kernel<8, 512>, K) : cudaLaunchKernelEx(&cfg, pcg_kernel<0, 512>, K);
  return wmax > 0 ? cudaLaunchKernelEx(&cfg, pcg_kernel<8, 1024>, K)
                  : cudaLaunchKernelEx(&cfg, pcg_kernel<0, 1024>, K);
}

cudaError_t launch_axpby_vals(int64_t n, double a, const double* X, double b, const double* Y, double* out,
                              cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  axpby_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(n, a, X, b, Y, out);
  return cudaGetLastError();
}

cudaError_t launch_copy(int64_t n, const double* src, double* dst, cudaStream_t st, const int* gate) {
  if (n == 0) return cudaSuccess;
  copy_kernel<<<unsigned((n + 255) / 256), 256, 0, st>>>(n, src, dst, gate);
  return cudaGetLastError();
}

}  // namespace bd
