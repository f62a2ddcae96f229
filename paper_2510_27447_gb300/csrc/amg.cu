// amg.cu -- conjugate gradients preconditioned by one algebraic-multigrid
// V(1,1) cycle per iteration, as one persistent cooperative kernel.
//
// The paper solves the elliptic equation (Eq. (3.15)) with an AMG-
// preconditioned Krylov method (Sec. 3.3.2); the hierarchy is built on the
// host (amg.cpp).  Cycle, for levels l = 0..L-1 and the coarsest operator:
//   down:   x_l = w_l D_l^-1 b_l ; r_l = b_l - A_l x_l ; b_{l+1} = R_l r_l
//   coarse: x_L = C b_L   (C: dense inverse of A_L + c 1 1^T)
//   up:     x_l += P_l y_{l+1} ; y_l = x_l + w_l D_l^-1 (b_l - A_l x_l)
// with b_0 the CG residual and y_0 the preconditioned residual z.  Damped
// Jacobi before and after, R = P^T and an exact coarse solve make the cycle a
// symmetric positive definite preconditioner on the range of A.  Every step
// that reads another row's value waits at a bounded device-wide barrier (4
// per level + 1); the CG part is the same two-barrier iteration as the
// Jacobi kernel in pcg.cu.
#include <cuda_runtime.h>

#include "bd_internal.h"
#include "sparse.cuh"
#include "vcycle.cuh"

namespace bd {

namespace {

template <int WMAX, int TPB>
__global__ void __launch_bounds__(TPB, BD_SOLVER_MIN_BLOCKS) pcg_amg_kernel(const __grid_constant__ PcgLaunch a,
                                                           const AmgDev* __restrict__ Mp) {
  // level loops index the descriptor at run time: a by-value kernel parameter
  // would be copied to local memory, so it is staged in shared memory
  __shared__ AmgDev sM;
  load_descriptor(sM, Mp);
  const AmgDev& M = sM;
  __shared__ double sh[4][32];
  if (a.gate && *a.gate == 0) return;
  const int n = a.n;
  const int nb = gridDim.x;
  const int stride = blockDim.x * gridDim.x;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;

  // ---- right-hand side and initial residual (as in pcg.cu) -------------------
  double acc0[2] = {0.0, 0.0};
  for (int i = i0; i < n; i += stride) {
    double b = a.rl ? a.rl[i] : 0.0;
    if (a.val1) b += a.c1 * sell_row<WMAX, false>(a, a.val1, a.va, i);
    if (a.val2) b += a.c2 * sell_row<WMAX, false>(a, a.val2, a.vb, i);
    double r = b;
    if (a.warm) r -= (a.dextra ? a.dextra[i] * a.x[i] : 0.0) + sell_row<WMAX, false>(a, a.valA, a.x, i);
    a.r[i] = r;
    acc0[0] += b;
    acc0[1] += b * b;
  }
  if (!a.warm)
    for (int i = i0; i < n; i += stride) a.x[i] = 0.0;
  block_sum<2>(acc0, sh);
  if (threadIdx.x == 0) {
    a.part[blockIdx.x * 4 + 0] = acc0[0];
    a.part[blockIdx.x * 4 + 1] = acc0[1];
  }
  if (!grid_barrier(a.bar, nb, a.status)) return;
  double tot[2];
  grid_total<2>(a.part, {0, 1}, nb, tot, sh);
  const double mean_b = a.project ? tot[0] / double(n) : 0.0;
  double bb = a.project ? tot[1] - double(n) * mean_b * mean_b : tot[1];
  if (bb < 0.0) bb = 0.0;
  const double tol2 = a.tol * a.tol * bb;
  double rr_loc = 0.0;
  for (int i = i0; i < n; i += stride) {
    const double r = a.r[i] - mean_b;
    a.r[i] = r;
    rr_loc += r * r;
  }
  if (!vcycle<double, TPB == 512>(M, a.r, a.z, a.bar, nb, a.status)) return;
  double acc1[2] = {0.0, rr_loc};
  for (int i = i0; i < n; i += stride) acc1[0] += a.r[i] * a.z[i];
  block_sum<2>(acc1, sh);
  if (threadIdx.x == 0) {
    a.part[blockIdx.x * 4 + 2] = acc1[0];
    a.part[blockIdx.x * 4 + 3] = acc1[1];
  }
  if (!grid_barrier(a.bar, nb, a.status)) return;
  grid_total<2>(a.part, {2, 3}, nb, tot, sh);
  double rho = tot[0];
  double rr = tot[1];

  int it = 0, fail = 0;
  bool done = !(rr > tol2);
  double beta = 0.0;
  while (!done) {
    double pq[1] = {0.0};
    for (int i = i0; i < n; i += stride) {
      const double z = a.z[i];
      const double az = (a.dextra ? a.dextra[i] * z : 0.0) + sell_row<WMAX, true>(a, a.valA, a.z, i);
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
    double rrl = 0.0;
    for (int i = i0; i < n; i += stride) {
      a.x[i] += alpha * a.p[i];
      const double r = a.r[i] - alpha * a.q[i];
      a.r[i] = r;
      rrl += r * r;
    }
    if (!vcycle<double, TPB == 512>(M, a.r, a.z, a.bar, nb, a.status)) return;
    double acc[2] = {0.0, rrl};
    for (int i = i0; i < n; i += stride) acc[0] += a.r[i] * a.z[i];
    block_sum<2>(acc, sh);
    if (threadIdx.x == 0) {
      a.part[blockIdx.x * 4 + 2] = acc[0];
      a.part[blockIdx.x * 4 + 3] = acc[1];
    }
    if (!grid_barrier(a.bar, nb, a.status)) return;
    grid_total<2>(a.part, {2, 3}, nb, tot, sh);
    ++it;
    rr = tot[1];
    if (!isfinite(rr) || !isfinite(tot[0])) {
      fail = ST_NONFINITE;
      break;
    }
    if (rr <= tol2) break;
    if (it >= a.maxit) {
      fail = ST_NOT_CONVERGED;
      break;
    }
    beta = tot[0] / rho;
    rho = tot[0];
  }

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

template <int W, int TPB>
int max_blocks_t(int block) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pcg_amg_kernel<W, TPB>, block, 0) != cudaSuccess) return 0;
  return sms * per;
}

}  // namespace

int pcg_amg_max_blocks(int block, int tier) {
  // the smallest co-resident count over the tier's instantiations keeps every launch legal
  if (tier == 1) return std::min(max_blocks_t<8, 512>(block), max_blocks_t<0, 512>(block));
  return std::min(max_blocks_t<8, 1024>(block), max_blocks_t<0, 1024>(block));
}

cudaError_t launch_pcg_amg(const PcgLaunch& P, const AmgDev* M, int wmax, cudaStream_t st) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  PcgLaunch K;
  solver_launch_config(P, st, &cfg, attr, &K);
  if (K.tier == 1)
    return wmax > 0 ? cudaLaunchKernelEx(&cfg, pcg_amg_kernel<8, 512>, K, M)
                    : cudaLaunchKernelEx(&cfg, pcg_amg_kernel<0, 512>, K, M);
  return wmax > 0 ? cudaLaunchKernelEx(&cfg, pcg_amg_kernel<8, 1024>, K, M)
                  : cudaLaunchKernelEx(&cfg, pcg_amg_kernel<0, 1024>, K, M);
}

bool amg_cluster_ok(int block, int size) {
  return solver_cluster_ok(pcg_amg_kernel<8, 1024>, block, size) &&
         solver_cluster_ok(pcg_amg_kernel<0, 1024>, block, size);
}

}  // namespace bd
