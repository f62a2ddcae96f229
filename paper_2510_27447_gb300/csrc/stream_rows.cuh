// stream_rows.cuh -- device pieces shared by the streaming solve kernels:
// the row products of the shared SELL pattern and of the AMG level operators,
// the last-block reductions and the inner decision (stream.cu: one system or
// a batch of systems; stream2.cu: two systems on one operator), and the host
// helpers that size their grids and build their loops.
#pragma once

#include <cuda_runtime.h>

#include "bd_internal.h"
#include "segment.cuh"
#include "sparse.cuh"

namespace bd {

namespace {

constexpr int kSB = 256;       // threads per block of every streaming kernel
static_assert(kSB == kCsrBlockLanes, "a block-per-row CSR level needs blocks of kCsrBlockLanes threads");
constexpr int kBlocksPerSM = 8;

// every kernel counts its launch (the loops run on the device, so the host
// cannot)
__device__ __forceinline__ void count_launch(long long* acc) {
  if (acc && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(acc), 1ull);
}

__device__ __forceinline__ void set_cond(unsigned long long h, unsigned v) {
  cudaGraphSetConditional(static_cast<cudaGraphConditionalHandle>(h), v);
}

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

// the same over the SELL-32/4 copy of an FP32 operator: four column indices
// and four values per 16-byte load (evict-first when STREAMOP, else through
// the read-only cache), the entries added in the SELL-32 order
template <bool STREAMOP>
__device__ __forceinline__ int4 ld4i(const int* p) {
  if constexpr (STREAMOP) return __ldcs(reinterpret_cast<const int4*>(p));
  else return __ldg(reinterpret_cast<const int4*>(p));
}
template <bool STREAMOP>
__device__ __forceinline__ float4 ld4f(const float* p) {
  if constexpr (STREAMOP) return __ldcs(reinterpret_cast<const float4*>(p));
  else return __ldg(reinterpret_cast<const float4*>(p));
}
template <class X, bool STREAMOP = true>
__device__ __forceinline__ X srow4(const int64_t* __restrict__ sptr4, const int* __restrict__ sw,
                                   const int* __restrict__ col4, const float* __restrict__ val4,
                                   const X* __restrict__ x, int i) {
  const int s = i >> 5;
  const int64_t base = sptr4[s] + 4 * (i & 31);
  const int w = sw[s];
  X acc = X(0);
  for (int k0 = 0; k0 < w; k0 += 8) {      // two 4-entry groups in flight
    const int4 c0 = ld4i<STREAMOP>(col4 + base + 32 * k0);
    const float4 v0 = ld4f<STREAMOP>(val4 + base + 32 * k0);
    const bool two = k0 + 4 < w;
    int4 c1 = c0;
    float4 v1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (two) {
      c1 = ld4i<STREAMOP>(col4 + base + 32 * (k0 + 4));
      v1 = ld4f<STREAMOP>(val4 + base + 32 * (k0 + 4));
    }
    const X g0 = __ldg(x + c0.x), g1 = __ldg(x + c0.y), g2 = __ldg(x + c0.z), g3 = __ldg(x + c0.w);
    X h0 = X(0), h1 = X(0), h2 = X(0), h3 = X(0);
    if (two) {
      h0 = __ldg(x + c1.x);
      h1 = __ldg(x + c1.y);
      h2 = __ldg(x + c1.z);
      h3 = __ldg(x + c1.w);
    }
    acc += X(v0.x) * g0;
    acc += X(v0.y) * g1;
    acc += X(v0.z) * g2;
    acc += X(v0.w) * g3;
    if (two) {
      acc += X(v1.x) * h0;
      acc += X(v1.y) * h1;
      acc += X(v1.z) * h2;
      acc += X(v1.w) * h3;
    }
  }
  return acc;
}

// every row i of an AMG-level operator (SELL: thread per row; CSR: warp per
// row, butterfly sum): epi(i, (M x)_i), run by one lane per row.  Level 0's
// operators are streamed with evict-first loads, the coarser levels' stay
// cacheable (read twice a cycle, they fit in L2).  K is the set of forms a
// kernel compiles (kRows* flags): a kernel that never meets a form leaves
// it out, which keeps registers low and resident warps high for the
// latency-bound coarse products.
constexpr int kRowsSellStream = 1, kRowsSellCache = 2, kRowsCsrLanes = 4, kRowsCsrBlock = 8;
constexpr int kRowsAll = 15;
constexpr int kRowsCoarse = kRowsSellCache | kRowsCsrLanes | kRowsCsrBlock;   // levels >= 1

template <class T, int K, class F>
__device__ __forceinline__ void level_rows(const SellDevT<T>& M, const T* x, bool streamop, SegInfo sg, F&& epi) {
  const int gt = sg.lb * blockDim.x + threadIdx.x;
  const int gs = sg.nb * blockDim.x;
  if constexpr (K == kRowsSellStream) {
    for (int i = gt; i < M.n; i += gs) epi(i, srow<true, T, T>(M.sptr, M.sw, M.col, M.val, x, i));
    return;
  }
  if ((K & kRowsCsrBlock) && M.rp && M.lpr > 32) {
    // a block per row (blockDim.x == kCsrBlockLanes): the row's entries
    // strided over the block's threads (a few each: the rows are long, not
    // huge), then the block's fixed-order sum; the row loop is block-uniform
    // so every thread reaches the block sum's barriers
    __shared__ T shb[1][32];
    for (int i = sg.lb; i < M.n; i += sg.nb) {
      const int64_t e = __ldg(M.rp + i + 1);
      T v[1] = {T(0)};
      for (int64_t p = __ldg(M.rp + i) + threadIdx.x; p < e; p += blockDim.x)
        v[0] += __ldg(M.val + p) * __ldg(x + __ldg(M.col + p));
      block_sum<1, T>(v, shb);
      if (threadIdx.x == 0) epi(i, v[0]);
    }
  } else if ((K & kRowsCsrLanes) && M.rp) {
    // L lanes per row (a power of two), 32 / L rows per warp pass; a lane
    // keeps four entries L apart in flight, four partial sums added in a
    // fixed order, then a butterfly over the row's lanes (deterministic).
    // The pass loop is warp-uniform so every shuffle has all 32 lanes.
    const int L = M.lpr > 0 ? M.lpr : 32;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (L - 1);
    const int rows_per_warp = 32 / L;
    const int grp = lane / L;
    const int step = (gs >> 5) * rows_per_warp;
    int base = (gt >> 5) * rows_per_warp;
    int i = base + grp;
    int64_t pb = 0, pe = 0;
    if (i < M.n) {
      pb = __ldg(M.rp + i);
      pe = __ldg(M.rp + i + 1);
    }
    for (; base < M.n; base += step) {
      // the next pass's row pointers are requested before this pass's entries
      const int inext = i + step;
      int64_t nb = 0, ne = 0;
      if (inext < M.n) {
        nb = __ldg(M.rp + inext);
        ne = __ldg(M.rp + inext + 1);
      }
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      {
        const int64_t e = pe;
        for (int64_t p = pb + sub; p < e; p += 4 * L) {
          const bool b1 = p + L < e, b2 = p + 2 * L < e, b3 = p + 3 * L < e;
          const int c0 = __ldg(M.col + p);
          const int c1 = b1 ? __ldg(M.col + p + L) : c0;
          const int c2 = b2 ? __ldg(M.col + p + 2 * L) : c0;
          const int c3 = b3 ? __ldg(M.col + p + 3 * L) : c0;
          const T v0 = __ldg(M.val + p);
          const T v1 = b1 ? __ldg(M.val + p + L) : T(0);
          const T v2 = b2 ? __ldg(M.val + p + 2 * L) : T(0);
          const T v3 = b3 ? __ldg(M.val + p + 3 * L) : T(0);
          s0 += v0 * __ldg(x + c0);
          s1 += v1 * __ldg(x + c1);
          s2 += v2 * __ldg(x + c2);
          s3 += v3 * __ldg(x + c3);
        }
      }
      T s = (s0 + s1) + (s2 + s3);
      for (int o = L >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (sub == 0 && i < M.n) epi(i, s);
      i = inext;
      pb = nb;
      pe = ne;
    }
  } else if ((K & kRowsSellStream) && streamop) {
    if constexpr (sizeof(T) == 4) {
      if (M.col4) {   // SELL-32/4 copy of a large FP32 level operator
        for (int i = gt; i < M.n; i += gs) epi(i, srow4<T, true>(M.sptr4, M.sw, M.col4, M.val4, x, i));
        return;
      }
    }
    for (int i = gt; i < M.n; i += gs) epi(i, srow<true, T, T>(M.sptr, M.sw, M.col, M.val, x, i));
  } else {
    if constexpr (sizeof(T) == 4) {
      if (M.col4) {
        for (int i = gt; i < M.n; i += gs) epi(i, srow4<T, false>(M.sptr4, M.sw, M.col4, M.val4, x, i));
        return;
      }
    }
    for (int i = gt; i < M.n; i += gs) epi(i, srow<false, T, T>(M.sptr, M.sw, M.col, M.val, x, i));
  }
}

// ---- reductions ----------------------------------------------------------------

// Block sums of v[0..NV) into part, the system's atomic ticket, and in its last
// block to arrive the system's totals (block order, fixed tree): returns true
// there, with v holding the totals in every thread of that block.
template <int NV, class T>
__device__ __forceinline__ bool last_block_total(T (&v)[NV], void* partv, unsigned* ticket, SegInfo sg) {
  __shared__ T sh[NV][32];
  __shared__ T tot[NV];
  __shared__ int amlast;
  T* part = static_cast<T*>(partv);
  block_sum<NV, T>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[sg.lb * NV + k] = v[k];
    __threadfence();
    amlast = atomicAdd(ticket, 1u) == unsigned(sg.nb) - 1u;
  }
  __syncthreads();
  if (!amlast) return false;
  __threadfence();
  T acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = T(0);
  for (int b = threadIdx.x; b < sg.nb; b += blockDim.x)
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

// Decision after the inner residual r and the preconditioned z are complete
// (thread 0 of the system's last block): the first one of an inner solve sets
// rho, later ones close an iteration as the persistent kernel's loop does.
// Returns whether the inner loop continues.
template <class T>
__device__ __forceinline__ bool inner_decide(const StreamLaunch& a, T rz) {
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
  }
  return !done;
}

// Set-up of a solve once its right-hand side b is complete (thread 0 of the
// system's last block): sum = sum_i b_i, sumsq = sum_i b_i^2.  A projected
// (singular) system solves for b - mean(b), so its |b|^2 is the centred sum.
__device__ __forceinline__ void rhs_setup(const StreamLaunch& a, double sum, double sumsq) {
  StreamScal& c = *a.sc;
  const double mean = a.project ? sum / double(a.n) : 0.0;
  double bb = a.project ? sumsq - double(a.n) * mean * mean : sumsq;
  if (bb < 0.0) bb = 0.0;
  c.mean_b = mean;
  c.bb = bb;
  c.tol2 = a.tol * a.tol * bb;
  c.outer = 0;
  c.fail = 0;
  c.skip = 0;
  c.stop = 1;
  c.more = 0;
  c.inner_ran = 0;
  c.inner_total = 0;
  c.outer_total = 0;
}

// Decision after an outer pass's FP64 residual |r|^2 = rr (thread 0 of the
// system's last block): the solve ends (converged, out of passes, or a zero
// residual), or the next inner solve is set up on r / |r|.  Returns whether
// that inner solve runs.
template <class T>
__device__ __forceinline__ bool outer_decide(const StreamLaunch& a, double rr) {
  StreamScal& c = *a.sc;
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
    c.more = 0;
    return false;
  }
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
  c.more = a.max_outer > 1 ? 1 : 0;
  return true;
}

// Decision after p.q of an inner iteration (thread 0 of the system's last
// block): alpha, or a breakdown that ends the inner solve (the outer pass
// decides what follows).  Returns whether the iteration goes on.
template <class T>
__device__ __forceinline__ bool pq_decide(const StreamLaunch& a, T pq) {
  StreamScal& c = *a.sc;
  if (!(pq > T(0))) {
    if (!isfinite(pq)) c.fail |= ST_NONFINITE;
    c.stop = 1;
    c.inner_total += c.it;
    return false;
  }
  c.alpha = double(T(c.rho) / pq);
  return true;
}

}  // namespace

// ---- host side (stream.cu) ------------------------------------------------------

// grid of kernel k (kSB threads a block) over `threads` grid-stride threads:
// at most one full wave of its resident blocks (queried once and cached; the
// first query of a kernel must come before any capture)
int stream_fit(const void* k, int64_t threads);
// resident blocks per SM of kernel k at kSB threads (cached)
int stream_resident_blocks(const void* k);
// add a WHILE node after the current capture frontier of `cap` and return its
// body graph; the capture continues after the node
cudaError_t stream_add_while(cudaStream_t cap, cudaGraphConditionalHandle h, cudaGraph_t* body);
// the graph `s` is capturing into, or NULL when it is not capturing
cudaGraph_t stream_capture_graph(cudaStream_t s);

// Outside a capture `body` (which enqueues a solve on st) is captured into a
// graph of its own, launched and destroyed; inside one it is appended.
template <class F>
cudaError_t stream_run_captured(cudaStream_t st, F&& body) {
  cudaStreamCaptureStatus cs;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
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
  e = cudaGraphUpload(ex, st);
  if (e == cudaSuccess) e = cudaGraphLaunch(ex, st);
  cudaGraphExecDestroy(ex);   // released once the launch completes
  return e;
}

}  // namespace bd
