// bd.cu -- handle, C ABI and the step driver of the partitioned SDC method.
//
// One step (Sec. 3.3.2, Algorithm 2, on M Gauss-Lobatto nodes; M = 2 is the
// paper's two-node trapezoidal correction, Eq. (3.20)):
//
//   f_0 = f(X^n)                                          node field, stored
//   for sweep k = 1..K:
//     elliptic   u_m = E(v_m) for m >= 1  (k = 1: once, from v^n)   Eq. (3.15)
//     predictor  X~_0 = X^n; for m: ROS2 over [t_m, t_m+1] with u_{m+1}
//                stage 1: ionic(S1) -> PCG -> k1 ; stage 2: ionic(S2) -> PCG -> k2
//                X~_{m+1} = X~_m + 3/(2g) k1 + 1/(2g) k2            Eq. (3.13)-(3.14)
//     correction f(X~_{M-1}); for m: ionic(C) -> PCG -> eps,
//                X_{m+1} = X~_{m+1} + eps                           Eq. (3.20)
//   activation times, X^{n+1} = X_{M-1}, u^{n+1} = u_{M-1}
//
// All of it runs on the handle's stream; after the first step of a given
// (dt, M, K) the launch sequence is captured once into a CUDA graph and
// replayed.  The device is touched by the host only at create/set/get calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "bd_internal.h"

namespace bd {
cudaError_t launch_eval(int model, int precision, int64_t n, const double* X, const double* istim, double inv_cm,
                        double* f, double* jac, cudaStream_t st);
void pattern_host(int model, uint32_t* masks);
}  // namespace bd

using namespace bd;

// relative residual reduction of each FP32 inner solve of the mixed elliptic
// refinement
#ifndef BD_MIXED_TOL_INNER
#define BD_MIXED_TOL_INNER 1e-4f
#endif

// ---------------------------------------------------------------------------
// fixed scratch of bd_solve_elliptic_noalloc (see include/bd.h)
// layout in doubles: r, z, p, q, 1/D (5 x max nodes), partial sums (4 x max
// blocks), then 4 control words: barrier (2 x uint32), status (int32),
// iteration counter (int64)
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t kNoAllocRows = BD_NOALLOC_MAX_NODES;
constexpr int64_t kNoAllocBlocks = 4096;
constexpr int64_t kNoAllocWords = 5 * kNoAllocRows + 4 * kNoAllocBlocks + 4;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocWords];
}  // namespace

struct bd_state {
  int model = 0, ns = 0, dim = 0, precision = 0;
  int device = 0;                 // CUDA device current at bd_create (the handle's device)
  int64_t N = 0, nnz = 0;
  int64_t NT = 0;                 // tissue nodes (v, membrane state); N - NT bath nodes follow them
  int64_t nnz_t = 0;              // nonzeros of the tissue block (rows and columns < NT)
  double* vfull = nullptr;        // bath: v on all N nodes, zero on the bath nodes
  bd_opts_t opts{};
  double inv_cm = 1.0, lambda_M = 0.25;
  int64_t* sptr = nullptr;      // SELL-32 layout of the shared operator pattern
  int* swidth = nullptr;
  int* col = nullptr;
  int* diagpos = nullptr;
  int64_t ell_n = 0;
  int wmax = 0;
  HostOps host;                   // CSR copies (bd_operator_csr)
  bool use_amg = false;
  AmgDev amg{};
  AmgDevF amgf{};                 // FP32 copy of the hierarchy (mixed path)
  AmgDevF amgf2{};                // its operators with a second set of level vectors (two-RHS solves)
  AmgDev amg2{};                  // FP64 streaming: the hierarchy with a second set of level vectors (two-system solves)
  bool pair64 = false;            // amg2 and two-system FP64 streaming workspaces are set up
  AmgDevF* d_amgf2 = nullptr;
  bool two_rhs = false;           // sweeps >= 2 solve their elliptic pair in one launch (mixed AMG path)
  float* partf8 = nullptr;
  double* partd8 = nullptr;
  double* vfull2 = nullptr;
  AmgDev* d_amg = nullptr;        // device copies of the two descriptors (kernel arguments)
  AmgDevF* d_amgf = nullptr;
  // mixed path: FP32 operator values and CG workspaces
  float* fAie = nullptr;
  bool vec4 = false;            // FP32 operators also in SELL-32/4 (streaming, mixed)
  int64_t n_slices = 0;         // SELL-32 slices of the shared pattern
  int64_t ell_n4 = 0;           // stored entries of the SELL-32/4 layout
  int64_t* sptr4 = nullptr;
  int* col4 = nullptr;
  float* fAie4 = nullptr;
  struct PCF { double alpha; float* val; float* val4; };   // val4: SELL-32/4 copy (vec4)
  std::vector<PCF> fpcache;
  float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *invd32 = nullptr, *d32 = nullptr;
  float* partf = nullptr;
  double *b64 = nullptr, *r64 = nullptr;
  int mixed_grid = 1;
  int mixed_amg_grid = 1;                  // grid of the mixed AMG kernels (differs in tier 2)
  int amg_grid = 1;
  int amg_levels = 0;
  std::vector<int64_t> amg_shape;   // per level: rows, entries, form of A, R, P (bd_amg_level)
  double amg_cycle_bytes[2] = {0.0, 0.0};   // algorithmic bytes of one V-cycle's smoothed levels (FP64, FP32)
  double amg_cycle_opbytes[2] = {0.0, 0.0}; // ... of which operator values and indices
  double amg_coarse_bytes[2] = {0.0, 0.0};  // dense coarsest-level solve of one cycle
  double *Ai = nullptr, *Aie = nullptr, *Mv = nullptr, *Mc = nullptr, *ML = nullptr;
  struct PC { double alpha; double* val; };
  std::vector<PC> pcache;
  double *Xn = nullptr, *Xt[kMaxNodes] = {}, *Xc[kMaxNodes] = {}, *u[kMaxNodes] = {};
  void* fq[kMaxNodes] = {};     // node fields f(X~_m), ns x NT values of the model's type
  double *dgs = nullptr, *rl = nullptr;
  // condensation vectors z, w of ROS2 stage 1 / the correction (z1, w1) and
  // z of stage 2, (ns-1) x NT values of the membrane model's type (float on
  // the mixed path: the condensation computes them in FP32)
  void *z1 = nullptr, *w1 = nullptr, *z2 = nullptr;
  double *k1v = nullptr, *k2v = nullptr, *avec = nullptr, *bvec = nullptr;
  // increments of each (sub-interval, ROS2 stage 1 / 2, correction): every
  // solve warm-starts from the previous sweep's (sweep 1: the previous step's)
  double* kinc[kMaxNodes - 1][3] = {};
  double *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_q = nullptr, *cg_invd = nullptr, *cg_part = nullptr;
  unsigned* bar = nullptr;
  double* t_act = nullptr;
  uint32_t* stim_bits = nullptr;
  StimTable stim{};
  long long* step_n = nullptr;
  int* d_status = nullptr;
  long long* d_stats = nullptr;            // [iters_e, solves_e, iters_p, solves_p, outer_e, outer_p, extra sweeps,
                                           //  paired elliptic iterations, launches, paired FP64 operator
                                           //  passes, paired first V-cycles]
  int* gate = nullptr;                     // sweep test of Algorithm 2 (sweep_tol > 0)
  unsigned long long* dmax = nullptr;
  double* Xsave = nullptr;
  unsigned long long* d_clamps = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // one captured graph per step shape (dt, M, K, embedded-error estimate on/off)
  struct GraphEntry { double dt; int M, K, adapt; cudaGraphExec_t exec; int64_t launches; };
  std::vector<GraphEntry> graphs;
  double* t_now = nullptr;                 // clock: t^n, t^{n-1}, previous-step data valid (0/1)
  double* uprev = nullptr;                 // sweep-1 elliptic solution of the previous step
  void* pack = nullptr;                    // stage-1 condensation of the current ROS2 step (stage 2 reuses it)
  void* jpack = nullptr;                   // node Jacobian at X~_1 (the correction at that state reuses it)
  void* jpack0 = nullptr;                  // node field and Jacobian at X^n (later sweeps' first predictor)
  // adaptive stepping (bd_step_adaptive)
  bool adapt_on = false;                   // the step being enqueued estimates its error
  double adapt_tol = 1.0;
  double dt_adapt = 0.0;                   // next step size (0: start at dt_max)
  unsigned long long* d_err = nullptr;
  double *Xbak = nullptr, *ubak = nullptr, *tbak = nullptr, *upbak = nullptr;
  // streaming solver (operators that do not fit in L2): device scalars, block
  // partials, FP64-path workspaces and two streams that capture loop bodies
  bool streaming = false;
  StreamScal* d_sc = nullptr;     // two: a solve's (or a pair's first system's) and a pair's second system's
  double* spart = nullptr;
  double *sb64 = nullptr, *sr64 = nullptr;
  double *sr = nullptr, *sz = nullptr, *sp = nullptr, *sq = nullptr, *sd = nullptr, *sinvd = nullptr;
  int s64_sys = 1;                // systems the FP64 workspaces above (but sinvd) hold
  cudaStream_t side[2] = {nullptr, nullptr};
  int pcg_grid = 1, pcg_block = 512, pcg_max = 1;
  int tier = 0;                            // solver register tier (kSolverTierBlock)
  int cluster = 0;                         // > 0: solvers run as one cluster of this many 1024-thread blocks
  std::vector<void*> allocs;
  std::string err;
  int64_t steps = 0, sweeps = 0, ionic_evals = 0, launches = 0;
  int64_t launches_per_step = 0;
  // profiling: an event pair per launch while prof is set
  struct Ev { int kind; cudaEvent_t a, b; };
  bool prof = false;
  std::vector<Ev> evpool;
  size_t evused = 0;
  int64_t enq_launches = 0;
};

namespace {

thread_local std::string g_err;

int fail(bd_state* s, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (s) s->err = buf;
  g_err = buf;
  return code;
}

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(s, BD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

void* dalloc(bd_state* s, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (s->opts.alloc) {
    p = s->opts.alloc(bytes, s->opts.alloc_ctx);
    if (p && (reinterpret_cast<uintptr_t>(p) & 15u) != 0) {   // vector loads need 16-byte alignment
      if (s->opts.free) s->opts.free(p, s->opts.alloc_ctx);
      p = nullptr;
    }
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) s->allocs.push_back(p);
  return p;
}

template <class T>
bool alloc_n(bd_state* s, T** out, int64_t count) {
  *out = static_cast<T*>(dalloc(s, size_t(count) * sizeof(T)));
  return *out != nullptr;
}

// count values of the membrane model's type (float on the mixed path)
bool alloc_zw(bd_state* s, void** out, int64_t count) {
  *out = dalloc(s, size_t(count) * (s->precision == BD_MIXED ? sizeof(float) : sizeof(double)));
  return *out != nullptr;
}

void release(bd_state* s) {
  for (auto& e : s->evpool) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  s->evpool.clear();
  for (auto& g : s->graphs) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
  for (void* p : s->allocs) {
    if (s->opts.free) s->opts.free(p, s->opts.alloc_ctx);
    else cudaFree(p);
  }
  s->allocs.clear();
  for (cudaStream_t& x : s->side) {
    if (x) cudaStreamDestroy(x);
    x = nullptr;
  }
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  s->stream = nullptr;
}

// brackets one launch with an event pair while profiling; counts launches
struct Timed {
  bd_state* s;
  int kind;
  int nlaunch;
  size_t slot;
  Timed(bd_state* st, int k, int nl = 1) : s(st), kind(k), nlaunch(nl), slot(0) {
    s->enq_launches += nl;
    if (!s->prof) return;
    if (s->evused == s->evpool.size()) {
      bd_state::Ev e{k, nullptr, nullptr};
      cudaEventCreate(&e.a);
      cudaEventCreate(&e.b);
      s->evpool.push_back(e);
    }
    slot = s->evused++;
    s->evpool[slot].kind = k;
    // profiled steps are captured: the records become event nodes of the graph
    cudaEventRecordWithFlags(s->evpool[slot].a, s->stream, cudaEventRecordExternal);
  }
  ~Timed() {
    if (s->prof) cudaEventRecordWithFlags(s->evpool[slot].b, s->stream, cudaEventRecordExternal);
  }
};

int status_code(int st) {
  if (st & ST_TIMEOUT) return BD_ERR_TIMEOUT;
  if (st & ST_NONFINITE) return BD_ERR_NONFINITE;
  if (st & ST_INDEFINITE) return BD_ERR_INDEFINITE;
  if (st & ST_NOT_CONVERGED) return BD_ERR_NOT_CONVERGED;
  return BD_OK;
}

int read_status(bd_state* s) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  const int c = status_code(st);
  if (c != BD_OK) {
    const char* what = c == BD_ERR_TIMEOUT ? "a device barrier wait timed out"
                       : c == BD_ERR_NONFINITE ? "non-finite value in a solve or the state"
                       : c == BD_ERR_INDEFINITE ? "CG met non-positive curvature"
                                                : "a CG solve reached its iteration cap";
    fail(s, c, "%s", what);
  }
  return c;
}

// values of alpha M_v + A_i on the shared pattern, cached per alpha
double* p_values(bd_state* s, double alpha) {
  for (auto& pc : s->pcache)
    if (pc.alpha == alpha) return pc.val;
  double* v = nullptr;
  if (!alloc_n(s, &v, s->ell_n)) return nullptr;
  if (launch_axpby_vals(s->ell_n, alpha, s->Mv, 1.0, s->Ai, v, s->stream) != cudaSuccess) return nullptr;
  s->pcache.push_back({alpha, v});
  return v;
}

// FP32 copy of alpha M_v + A_i (mixed path), cached per alpha
float* p_values_f(bd_state* s, double alpha) {
  for (auto& pc : s->fpcache)
    if (pc.alpha == alpha) return pc.val;
  double* dv = p_values(s, alpha);
  float* v = nullptr;
  if (!dv || !alloc_n(s, &v, s->ell_n)) return nullptr;
  if (launch_to_float(s->ell_n, dv, v, s->stream) != cudaSuccess) return nullptr;
  float* v4 = nullptr;
  if (s->vec4 && (!alloc_n(s, &v4, s->ell_n4) ||
                  launch_sell_v4(s->n_slices, s->sptr, s->swidth, s->sptr4, v, v4, s->stream) != cudaSuccess))
    return nullptr;
  s->fpcache.push_back({alpha, v, v4});
  return v;
}

// the SELL-32/4 copy of p_values_f(s, alpha) (NULL without vec4)
float* p_values_f4(bd_state* s, double alpha) {
  if (!p_values_f(s, alpha)) return nullptr;
  for (auto& pc : s->fpcache)
    if (pc.alpha == alpha) return pc.val4;
  return nullptr;
}

MixedLaunch mixed_base(bd_state* s) {
  MixedLaunch X{};
  X.r32 = s->r32;
  X.z32 = s->z32;
  X.p32 = s->p32;
  X.q32 = s->q32;
  X.invd32 = s->invd32;
  X.d32 = s->d32;
  X.b64 = s->b64;
  X.r64 = s->r64;
  return X;
}

PcgLaunch pcg_base(bd_state* s) {
  PcgLaunch P{};
  P.n = int(s->N);
  P.sptr = s->sptr;
  P.swidth = s->swidth;
  P.col = s->col;
  P.diagpos = s->diagpos;
  P.r = s->cg_r;
  P.z = s->cg_z;
  P.p = s->cg_p;
  P.q = s->cg_q;
  P.invd = s->cg_invd;
  P.part = s->cg_part;
  P.bar = s->bar;
  P.status = s->d_status;
  P.grid = s->pcg_grid;
  P.block = s->pcg_block;
  P.cluster = s->cluster;
  P.tier = s->tier;
  if (s->cluster > 0) P.block = kSolverTierBlock[0];
  P.gate = s->opts.sweep_tol > 0 ? s->gate : nullptr;
  return P;
}

// the SELL-32/4 copy (values val4) of a launch's FP32 operator, when the
// handle keeps one
void set_vec4(const bd_state* s, StreamLaunch& A, const float* val4) {
  if (!s->vec4 || !val4) return;
  A.sptr4 = s->sptr4;
  A.sw4 = s->swidth;
  A.col4 = s->col4;
  A.valT4 = val4;
}

StreamLaunch stream_base(bd_state* s, int n) {
  StreamLaunch A{};
  A.n = n;
  A.sptr = s->sptr;
  A.swidth = s->swidth;
  A.col = s->col;
  A.diagpos = s->diagpos;
  A.part = s->spart;
  A.sc = s->d_sc;
  A.status = s->d_status;
  A.launch_acc = s->d_stats + 8;
  A.gate = s->opts.sweep_tol > 0 ? s->gate : nullptr;
  A.grid = int(std::max<int64_t>(1, std::min<int64_t>((int64_t(n) + 255) / 256, stream_grid_cap())));
  A.host_loop = s->opts.streaming == 2 ? 1 : 0;
  const bool mixed = s->precision == BD_MIXED;
  A.b64 = mixed ? s->b64 : s->sb64;
  A.r64 = mixed ? s->r64 : s->sr64;
  A.r = mixed ? static_cast<void*>(s->r32) : static_cast<void*>(s->sr);
  A.z = mixed ? static_cast<void*>(s->z32) : static_cast<void*>(s->sz);
  A.p = mixed ? static_cast<void*>(s->p32) : static_cast<void*>(s->sp);
  A.q = mixed ? static_cast<void*>(s->q32) : static_cast<void*>(s->sq);
  A.d = mixed ? static_cast<void*>(s->d32) : static_cast<void*>(s->sd);
  A.invd = mixed ? static_cast<void*>(s->invd32) : static_cast<void*>(s->sinvd);
  return A;
}

// the streaming elliptic solve u = E(v) over all N rows (v holds every node);
// k = 1: the second system of a pair, whose vectors are the second halves of
// the two-system workspaces and whose scalars are d_sc[1]
StreamLaunch elliptic_launch(bd_state* s, const double* v, double* u, int k = 0) {
  StreamLaunch A = stream_base(s, int(s->N));
  const bool mixed = s->precision == BD_MIXED;
  A.valA = s->Aie;
  A.valT = mixed ? static_cast<const void*>(s->fAie) : static_cast<const void*>(s->Aie);
  set_vec4(s, A, s->fAie4);
  A.val1 = s->Ai;
  A.va = v;
  A.c1 = -1.0;
  A.project = 1;
  A.warm = 1;
  A.x = u;
  A.pin = s->opts.pin_node >= 0 ? s->opts.pin_node : -1;
  A.max_outer = mixed ? 12 : 1;
  A.inner_cap = s->opts.cg_cap_e;
  A.use_amg = s->use_amg ? 1 : 0;
  A.tol = s->opts.cg_tol_e;
  A.tol_inner = mixed ? double(BD_MIXED_TOL_INNER) : s->opts.cg_tol_e;
  A.iters_acc = s->d_stats + 0;
  A.solves_acc = s->d_stats + 1;
  A.outer_acc = s->d_stats + 4;
  if (k == 1) {
    const int64_t N = s->N;
    A.sc = s->d_sc + 1;
    A.b64 += N;
    A.r64 += N;
    auto second = [&](void*& v) {
      v = mixed ? static_cast<void*>(static_cast<float*>(v) + N) : static_cast<void*>(static_cast<double*>(v) + N);
    };
    for (void** v : {&A.r, &A.z, &A.p, &A.q, &A.d}) second(*v);
  }
  return A;
}

int elliptic(bd_state* s, const double* v, double* u) {
  if (s->streaming) {
    if (s->NT < s->N) {
      Timed t(s, BD_K_COMBINE);
      CK(launch_copy(s->NT, v, s->vfull, s->stream, s->opts.sweep_tol > 0 ? s->gate : nullptr));
      v = s->vfull;
    }
    const StreamLaunch A = elliptic_launch(s, v, u);
    const bool mixed = s->precision == BD_MIXED;
    Timed t(s, BD_K_PCG_ELLIPTIC, 0);   // its kernels count themselves on the device
    CK(stream_solve(A, mixed ? 1 : 0, &s->amgf, &s->amg, s->stream, s->side));
    return BD_OK;
  }
  PcgLaunch P = pcg_base(s);
  if (s->NT < s->N) {   // the right-hand side -A_i v gathers v over all columns
    Timed t(s, BD_K_COMBINE);
    CK(launch_copy(s->NT, v, s->vfull, s->stream, P.gate));
    v = s->vfull;
  }
  P.valA = s->Aie;
  P.val1 = s->Ai;
  P.va = v;
  P.c1 = -1.0;
  P.project = 1;
  P.x = u;
  P.warm = 1;
  P.tol = s->opts.cg_tol_e;
  P.maxit = s->opts.cg_cap_e;
  P.pin = s->opts.pin_node >= 0 ? s->opts.pin_node : -1;
  P.iters_acc = s->d_stats + 0;
  P.solves_acc = s->d_stats + 1;
  P.outer_acc = s->d_stats + 4;
  Timed t(s, BD_K_PCG_ELLIPTIC);
  if (s->precision == BD_MIXED) {
    MixedLaunch X = mixed_base(s);
    X.valA32 = s->fAie;
    X.tol_inner = BD_MIXED_TOL_INNER;
    X.max_outer = 12;
    X.inner_cap = s->opts.cg_cap_e;
    X.use_amg = s->use_amg ? 1 : 0;
    P.grid = s->use_amg ? s->mixed_amg_grid : s->mixed_grid;
    CK(launch_pcg_mixed(P, X, s->d_amgf, s->wmax, s->stream, s->partf));
  } else if (s->use_amg) {
    P.grid = s->amg_grid;
    CK(launch_pcg_amg(P, s->d_amg, s->wmax, s->stream));
  } else {
    CK(launch_pcg(P, s->wmax, s->stream));
  }
  return BD_OK;
}

// u1 = E(v1) and u2 = E(v2): one two-RHS launch on the mixed AMG path, else
// two solves
int elliptic2(bd_state* s, const double* v1, double* u1, const double* v2, double* u2) {
  const bool mixed = s->precision == BD_MIXED;
  // pairs: mixed AMG solves in both forms, FP64 AMG solves in the streaming form
  const bool pair = s->use_amg && s->opts.pair_solve >= 0 && (mixed ? s->two_rhs : s->streaming && s->pair64);
  if (!pair) {
    const int r = elliptic(s, v1, u1);
    if (r != BD_OK) return r;
    return elliptic(s, v2, u2);
  }
  if (s->streaming) {   // one chain for both systems (stream2.cu)
    if (s->NT < s->N) {
      if (!s->vfull || !s->vfull2) return fail(s, BD_ERR_ARG, "two-system solve without its full-length potentials");
      Timed t(s, BD_K_COMBINE, 2);
      const int* gate = s->opts.sweep_tol > 0 ? s->gate : nullptr;
      CK(launch_copy(s->NT, v1, s->vfull, s->stream, gate));
      CK(launch_copy(s->NT, v2, s->vfull2, s->stream, gate));
      v1 = s->vfull;
      v2 = s->vfull2;
    }
    const StreamLaunch A[2] = {elliptic_launch(s, v1, u1, 0), elliptic_launch(s, v2, u2, 1)};
    Timed t(s, BD_K_PCG_ELLIPTIC, 0);   // its kernels count themselves on the device
    if (mixed)
      CK(stream_solve_pair(A, s->amgf, s->amgf2, s->d_stats + 7, s->d_stats + 9, s->d_stats + 10, s->stream,
                           s->side));
    else
      CK(stream_solve_pair(A, s->amg, s->amg2, s->d_stats + 7, s->d_stats + 9, s->d_stats + 10, s->stream,
                           s->side));
    return BD_OK;
  }
  PcgLaunch P = pcg_base(s);
  if (s->NT < s->N) {
    Timed t(s, BD_K_COMBINE, 2);
    CK(launch_copy(s->NT, v1, s->vfull, s->stream, P.gate));
    CK(launch_copy(s->NT, v2, s->vfull2, s->stream, P.gate));
    v1 = s->vfull;
    v2 = s->vfull2;
  }
  P.valA = s->Aie;
  P.val1 = s->Ai;
  P.va = v1;
  P.c1 = -1.0;
  P.project = 1;
  P.x = u1;
  P.warm = 1;
  P.tol = s->opts.cg_tol_e;
  P.maxit = s->opts.cg_cap_e;
  P.pin = s->opts.pin_node >= 0 ? s->opts.pin_node : -1;
  P.iters_acc = s->d_stats + 0;
  P.solves_acc = s->d_stats + 1;
  P.outer_acc = s->d_stats + 4;
  P.pair_acc = s->d_stats + 7;
  P.grid = s->mixed_amg_grid;
  MixedLaunch X = mixed_base(s);
  X.valA32 = s->fAie;
  X.tol_inner = BD_MIXED_TOL_INNER;
  X.max_outer = 12;
  X.inner_cap = s->opts.cg_cap_e;
  X.use_amg = 1;
  Timed t(s, BD_K_PCG_ELLIPTIC);
  CK(launch_pcg_mixed2(P, v2, u2, X, s->d_amgf, s->d_amgf2, s->wmax, s->stream, s->partf8, s->partd8));
  return BD_OK;
}

// (alpha M_v + A_i + diag(dgs)) x = rl + c1 A_i va + c2 M_v vb; node_terms =
// false drops diag(dgs) and rl (the plain Crank-Nicolson operator)
int parabolic(bd_state* s, double alpha, double c1, const double* va, double c2, const double* vb, double* x,
              bool node_terms = true, bool warm = false) {
  if (s->streaming) {
    StreamLaunch A = stream_base(s, int(s->NT));   // tissue rows; their bath columns hold zeros
    const bool mixed = s->precision == BD_MIXED;
    A.valA = p_values(s, alpha);
    A.valT = mixed ? static_cast<const void*>(p_values_f(s, alpha)) : static_cast<const void*>(A.valA);
    if (mixed) set_vec4(s, A, p_values_f4(s, alpha));
    A.dextra = node_terms ? s->dgs : nullptr;
    A.rl = node_terms ? s->rl : nullptr;
    A.val1 = s->Ai;
    A.va = va;
    A.c1 = c1;
    if (vb) {
      A.val2 = s->Mv;
      A.vb = vb;
      A.c2 = c2;
    }
    A.project = 0;
    A.warm = warm ? 1 : 0;
    A.x = x;
    A.pin = -2;
    A.max_outer = 1;
    A.inner_cap = s->opts.cg_cap_p;
    A.use_amg = 0;
    A.tol = s->opts.cg_tol_p;
    A.tol_inner = mixed ? std::max(s->opts.cg_tol_p, 1e-6) : s->opts.cg_tol_p;
    A.iters_acc = s->d_stats + 2;
    A.solves_acc = s->d_stats + 3;
    A.outer_acc = s->d_stats + 5;
    Timed t(s, BD_K_PCG_PARABOLIC, 0);
    CK(stream_solve(A, mixed ? 1 : 0, nullptr, nullptr, s->stream, s->side));
    return BD_OK;
  }
  PcgLaunch P = pcg_base(s);
  P.n = int(s->NT);   // tissue rows; their bath columns hold zeros
  P.valA = p_values(s, alpha);
  P.dextra = node_terms ? s->dgs : nullptr;
  P.rl = node_terms ? s->rl : nullptr;
  P.val1 = s->Ai;
  P.va = va;
  P.c1 = c1;
  if (vb) {
    P.val2 = s->Mv;
    P.vb = vb;
    P.c2 = c2;
  }
  P.project = 0;
  P.x = x;
  P.warm = warm ? 1 : 0;
  P.tol = s->opts.cg_tol_p;
  P.maxit = s->opts.cg_cap_p;
  P.pin = -2;
  P.iters_acc = s->d_stats + 2;
  P.solves_acc = s->d_stats + 3;
  P.outer_acc = s->d_stats + 5;
  Timed t(s, BD_K_PCG_PARABOLIC);
  if (s->precision == BD_MIXED) {
    MixedLaunch X = mixed_base(s);
    X.valA32 = p_values_f(s, alpha);
    X.tol_inner = float(std::max(s->opts.cg_tol_p, 1e-6));
    X.max_outer = 1;
    X.inner_cap = s->opts.cg_cap_p;
    X.use_amg = 0;
    X.pipelined = s->tier == 1 ? 1 : 0;   // measured: pays where the barriers dominate
    P.grid = s->mixed_grid;
    CK(launch_pcg_mixed(P, X, s->d_amgf, s->wmax, s->stream, s->partf));
  } else {
    CK(launch_pcg(P, s->wmax, s->stream));
  }
  return BD_OK;
}

IonicLaunch ionic_base(bd_state* s, int mode, double dt) {
  IonicLaunch L{};
  L.model = s->model;
  L.precision = s->precision;
  L.mode = mode;
  L.n = s->NT;
  L.inv_cm = s->inv_cm;
  L.dt = dt;
  L.ML = s->ML;
  L.stim_bits = s->stim_bits;
  L.t_now = s->t_now;
  L.stim = s->stim;
  L.dgs = s->dgs;
  L.rl = s->rl;
  L.avec = s->avec;
  L.clamp_count = s->d_clamps;
  L.gate = s->opts.sweep_tol > 0 ? s->gate : nullptr;
  return L;
}

void lobatto(int M, double* c) {
  if (M == 2) { c[0] = 0.0; c[1] = 1.0; }
  else { c[0] = 0.0; c[1] = 0.5; c[2] = 1.0; }
}

// S[m][j] = int_{c_m}^{c_{m+1}} l_j  (unit interval)
void integration_matrix(int M, double S[kMaxNodes - 1][kMaxNodes]) {
  if (M == 2) {
    S[0][0] = 0.5; S[0][1] = 0.5;
  } else {
    S[0][0] = 5.0 / 24; S[0][1] = 1.0 / 3; S[0][2] = -1.0 / 24;
    S[1][0] = -1.0 / 24; S[1][1] = 1.0 / 3; S[1][2] = 5.0 / 24;
  }
}

// prepare everything a step allocates or computes outside the launch sequence
// (M = 0: the CN-RK2 step)
int prepare_step(bd_state* s, double dt, int M) {
  if (M == 0) {
    if (!p_values(s, 2.0 / dt) || (s->precision == BD_MIXED && !p_values_f(s, 2.0 / dt)))
      return fail(s, BD_ERR_OOM, "device allocation failed");
    return BD_OK;
  }
  const double gam = 1.0 + 1.0 / std::sqrt(2.0);
  double c[kMaxNodes];
  lobatto(M, c);
  for (int m = 0; m + 1 < M; ++m) {
    const double h = dt * (c[m + 1] - c[m]);
    for (double alpha : {1.0 / (gam * h), 1.0 / h}) {
      if (!p_values(s, alpha)) return fail(s, BD_ERR_OOM, "device allocation failed");
      if (s->precision == BD_MIXED && !p_values_f(s, alpha)) return fail(s, BD_ERR_OOM, "device allocation failed");
    }
  }
  return BD_OK;
}

// build the AMG hierarchy of A_ie on the host and upload it (SELL-32 operators)
int setup_amg(bd_state* s, const HostOps& H) {
  HCsr A;
  A.n = A.m = s->N;
  A.rp.assign(H.rowptr.begin(), H.rowptr.end());
  A.ci = H.col;
  A.v = H.Aie;
  AmgHost AH;
  std::string err;
  AmgParams prm;
  if (s->opts.amg_coarse_max > 0) prm.coarse_max = s->opts.amg_coarse_max;
  const int rc = amg_build(A, prm, &AH, &err);
  if (rc != BD_OK) return fail(s, rc, "%s", err.c_str());
  if (AH.lev.empty()) return BD_OK;   // small operator: Jacobi-PCG is used
  if (int(AH.lev.size()) > kMaxAmgLevels)
    return fail(s, BD_ERR_ARG, "AMG hierarchy has %d levels", int(AH.lev.size()));
  auto upload = [&](const void* h, size_t bytes) -> void* {
    void* d = dalloc(s, bytes);
    if (d && cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) return nullptr;
    return d;
  };
  s->amg_shape.assign(AH.lev.size() * 9, 0);
  // rows, entries and storage form (0 SELL-32, -1 wide SELL-32, k > 0 CSR
  // with k lanes per row) of one operator of the hierarchy
  auto shape = [&](size_t l, int which, const HCsr& M, const SellDev& d) {
    int64_t* o = s->amg_shape.data() + l * 9 + 3 * which;
    o[0] = M.n;
    o[1] = int64_t(M.ci.size());
    o[2] = d.rp ? d.lpr : (d.wmax == 0 ? -1 : 0);
  };
  auto sell_dev = [&](const HCsr& M, SellDev* out) {
    const SellHost S = sell_from_csr(M, s->streaming ? s->opts.wide_sell + 1 : 0);
    out->n = int(S.n);
    out->wmax = S.wmax;
    const bool csr = !S.rp.empty();
    out->rp = csr ? static_cast<const int64_t*>(upload(S.rp.data(), S.rp.size() * 8)) : nullptr;
    out->lpr = csr ? (s->opts.csr_lanes > 0 ? s->opts.csr_lanes : csr_lanes(S.rp.back(), S.n)) : 0;
    out->sptr = csr ? nullptr : static_cast<const int64_t*>(upload(S.sptr.data(), S.sptr.size() * 8));
    out->sw = csr ? nullptr : static_cast<const int*>(upload(S.sw.data(), S.sw.size() * 4));
    out->col = static_cast<const int*>(upload(S.col.data(), S.col.size() * 4));
    out->val = static_cast<const double*>(upload(S.val.data(), S.val.size() * 8));
    // the host vectors die with S: wait for the copies
    return (csr ? out->rp != nullptr : (out->sptr && out->sw)) && out->col && out->val &&
           cudaStreamSynchronize(s->stream) == cudaSuccess;
  };
  AmgDev& M = s->amg;
  M.nlev = int(AH.lev.size());
  for (int l = 0; l < M.nlev; ++l) {
    const AmgHostLevel& Lh = AH.lev[l];
    AmgLevelDev& Ld = M.L[l];
    bool ok = true;
    if (l == 0) {
      Ld.A = SellDev{int(s->N), s->wmax, s->sptr, s->swidth, s->col, s->Aie, nullptr};
    } else {
      ok = sell_dev(Lh.A, &Ld.A);
    }
    ok = ok && sell_dev(Lh.P, &Ld.P) && sell_dev(Lh.R, &Ld.R);
    if (ok) {
      shape(size_t(l), 0, Lh.A, Ld.A);
      shape(size_t(l), 1, Lh.R, Ld.R);
      shape(size_t(l), 2, Lh.P, Ld.P);
    }
    Ld.invd = static_cast<const double*>(upload(Lh.invdiag.data(), Lh.invdiag.size() * 8));
    Ld.omega = Lh.omega;
    const int64_t n = Lh.A.n;
    ok = ok && Ld.invd && alloc_n(s, &Ld.x, n) && alloc_n(s, &Ld.r, n);
    if (l > 0) ok = ok && alloc_n(s, &Ld.b, n) && alloc_n(s, &Ld.y, n);
    if (!ok || cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, BD_ERR_OOM, "AMG upload failed");
  }
  // the dense coarse inverse with rows padded to a multiple of 4 entries, so
  // that every row starts on a 16-byte boundary (vector loads)
  const int64_t ncr = AH.nc, ldc = (ncr + 3) & ~int64_t(3);
  std::vector<double> cpad(size_t(ncr * ldc), 0.0);
  for (int64_t i = 0; i < ncr; ++i)
    std::copy(AH.cinv.begin() + i * ncr, AH.cinv.begin() + (i + 1) * ncr, cpad.begin() + i * ldc);
  M.nc = int(ncr);
  M.ldc = int(ldc);
  M.cinv = static_cast<const double*>(upload(cpad.data(), cpad.size() * 8));
  if (!M.cinv || !alloc_n(s, &M.bc, AH.nc) || !alloc_n(s, &M.xc, AH.nc) ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return fail(s, BD_ERR_OOM, "AMG upload failed");
  if (s->precision == BD_FP64 && s->streaming && s->opts.pair_solve >= 0) {
    // the same hierarchy with its own level vectors: the second system of the
    // streaming two-system solves (sweeps >= 2)
    AmgDev& G = s->amg2;
    G = M;
    bool ok2 = alloc_n(s, &G.bc, AH.nc) && alloc_n(s, &G.xc, AH.nc);
    for (int l = 0; ok2 && l < G.nlev; ++l) {
      const int64_t n = AH.lev[l].A.n;
      ok2 = alloc_n(s, &G.L[l].x, n) && alloc_n(s, &G.L[l].r, n);
      if (ok2 && l > 0) ok2 = alloc_n(s, &G.L[l].b, n) && alloc_n(s, &G.L[l].y, n);
    }
    if (!ok2) return fail(s, BD_ERR_OOM, "AMG upload failed");
    s->pair64 = true;
  }
  if (s->precision == BD_MIXED) {
    auto sell_devf = [&](const HCsr& Mh, SellDevT<float>* out) {
      const SellHost S = sell_from_csr(Mh, s->streaming ? s->opts.wide_sell + 1 : 0);
      std::vector<float> fv(S.val.begin(), S.val.end());
      out->n = int(S.n);
      out->wmax = S.wmax;
      const bool csr = !S.rp.empty();
      out->rp = csr ? static_cast<const int64_t*>(upload(S.rp.data(), S.rp.size() * 8)) : nullptr;
      out->lpr = csr ? (s->opts.csr_lanes > 0 ? s->opts.csr_lanes : csr_lanes(S.rp.back(), S.n)) : 0;
      out->sptr = csr ? nullptr : static_cast<const int64_t*>(upload(S.sptr.data(), S.sptr.size() * 8));
      out->sw = csr ? nullptr : static_cast<const int*>(upload(S.sw.data(), S.sw.size() * 4));
      out->col = static_cast<const int*>(upload(S.col.data(), S.col.size() * 4));
      out->val = static_cast<const float*>(upload(fv.data(), fv.size() * 4));
      // SELL-32/4 copy for the streaming kernels: operators of at least 2^17
      // rows (vec4 = 0) or every SELL operator (vec4 = 1)
      const bool v4 = !csr && s->vec4 && (s->opts.vec4 == 1 || S.n >= (int64_t(1) << 17));
      std::vector<int64_t> p4;
      std::vector<int> c4;
      std::vector<float> f4;
      if (v4) {
        const int64_t nsl = int64_t(S.sw.size());
        p4.resize(nsl);
        int64_t off = 0;
        for (int64_t sl = 0; sl < nsl; ++sl) {
          p4[sl] = off;
          off += 32 * int64_t((S.sw[sl] + 3) & ~3);
        }
        c4.assign(off, 0);
        f4.assign(off, 0.0f);
        for (int64_t sl = 0; sl < nsl; ++sl)
          for (int l = 0; l < 32; ++l)
            for (int k = 0; k < S.sw[sl]; ++k) {
              const int64_t src = S.sptr[sl] + 32 * int64_t(k) + l;
              const int64_t dst = p4[sl] + 128 * int64_t(k / 4) + 4 * l + k % 4;
              c4[dst] = S.col[src];
              f4[dst] = fv[src];
            }
        out->sptr4 = static_cast<const int64_t*>(upload(p4.data(), p4.size() * 8));
        out->col4 = static_cast<const int*>(upload(c4.data(), c4.size() * 4));
        out->val4 = static_cast<const float*>(upload(f4.data(), f4.size() * 4));
      }
      return (csr ? out->rp != nullptr : (out->sptr && out->sw)) && out->col && out->val &&
             (!v4 || (out->sptr4 && out->col4 && out->val4)) && cudaStreamSynchronize(s->stream) == cudaSuccess;
    };
    AmgDevF& F = s->amgf;
    F.nlev = M.nlev;
    for (int l = 0; l < F.nlev; ++l) {
      const AmgHostLevel& Lh = AH.lev[l];
      AmgLevelDevT<float>& Ld = F.L[l];
      bool ok = true;
      if (l == 0) Ld.A = SellDevT<float>{int(s->N), s->wmax, s->sptr, s->swidth, s->col, s->fAie, nullptr};
      else ok = sell_devf(Lh.A, &Ld.A);
      ok = ok && sell_devf(Lh.P, &Ld.P) && sell_devf(Lh.R, &Ld.R);
      std::vector<float> fid(Lh.invdiag.begin(), Lh.invdiag.end());
      Ld.invd = static_cast<const float*>(upload(fid.data(), fid.size() * 4));
      Ld.omega = float(Lh.omega);
      const int64_t n = Lh.A.n;
      ok = ok && Ld.invd && alloc_n(s, &Ld.x, n) && alloc_n(s, &Ld.r, n);
      if (l > 0) ok = ok && alloc_n(s, &Ld.b, n) && alloc_n(s, &Ld.y, n);
      if (!ok || cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(s, BD_ERR_OOM, "AMG upload failed");
    }
    std::vector<float> fci(cpad.begin(), cpad.end());
    F.nc = int(ncr);
    F.ldc = int(ldc);
    F.cinv = static_cast<const float*>(upload(fci.data(), fci.size() * 4));
    if (!F.cinv || !alloc_n(s, &F.bc, AH.nc) || !alloc_n(s, &F.xc, AH.nc) ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
      return fail(s, BD_ERR_OOM, "AMG upload failed");
    // the same hierarchy with its own level vectors: the second system of the
    // two-RHS solves (sweeps >= 2 solve the elliptic constraint at two nodes)
    AmgDevF& G = s->amgf2;
    G = F;
    bool ok2 = alloc_n(s, &G.bc, AH.nc) && alloc_n(s, &G.xc, AH.nc);
    for (int l = 0; ok2 && l < G.nlev; ++l) {
      const int64_t n = AH.lev[l].A.n;
      ok2 = alloc_n(s, &G.L[l].x, n) && alloc_n(s, &G.L[l].r, n);
      if (ok2 && l > 0) ok2 = alloc_n(s, &G.L[l].b, n) && alloc_n(s, &G.L[l].y, n);
    }
    if (!ok2) return fail(s, BD_ERR_OOM, "AMG upload failed");
    s->two_rhs = true;
  }
  const int mx = pcg_amg_max_blocks(s->pcg_block, s->tier);
  if (mx <= 0) return fail(s, BD_ERR_CUDA, "cannot size the cooperative AMG-CG grid");
  s->amg_grid = std::min(s->pcg_grid, mx);
  for (int v = 0; v < 2; ++v) {
    const double vb = v == 0 ? 8.0 : 4.0;
    double b = 0.0, ob = 0.0;
    for (size_t l = 0; l < AH.lev.size(); ++l) {
      const AmgHostLevel& Lh = AH.lev[l];
      const double n = double(Lh.A.n), nn = double(Lh.P.m);
      ob += double(2 * Lh.A.ci.size() + Lh.R.ci.size() + Lh.P.ci.size()) * (vb + 4);
      // one product y = B x: (vb + 4) per entry, gather of x + result + row pointer per row
      const double spA = double(Lh.A.ci.size()) * (vb + 4) + n * (2 * vb + 4);
      const double spR = double(Lh.R.ci.size()) * (vb + 4) + nn * (vb + 4) + n * vb;
      const double spP = double(Lh.P.ci.size()) * (vb + 4) + n * (vb + 4) + nn * vb;
      // 2 A products (residual, post-smoothing), R, P; vector streams of the
      // pre-smoothing (b, 1/D in, x out), residual (b in), prolongation (x in
      // and out) and post-smoothing (b, 1/D in, y out)
      b += 2 * spA + spR + spP + vb * (3 * n + n + 2 * n + 3 * n);
    }
    const double nc = double(AH.nc);
    s->amg_cycle_bytes[v] = b;
    s->amg_coarse_bytes[v] = vb * (nc * nc + 2 * nc);
    s->amg_cycle_opbytes[v] = ob + vb * nc * nc;
  }
  s->amg_levels = M.nlev;
  // the kernels read the descriptors from device memory
  if (cudaMemcpyAsync(s->d_amg, &s->amg, sizeof(AmgDev), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(s->d_amgf, &s->amgf, sizeof(AmgDevF), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      (s->d_amgf2 &&
       cudaMemcpyAsync(s->d_amgf2, &s->amgf2, sizeof(AmgDevF), cudaMemcpyHostToDevice, s->stream) != cudaSuccess) ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return fail(s, BD_ERR_CUDA, "AMG descriptor upload failed");
  s->use_amg = true;
  return BD_OK;
}

#define RUN(x)                     \
  do {                             \
    const int r_ = (x);            \
    if (r_ != BD_OK) return r_;    \
  } while (0)

}  // namespace

namespace bd {
int solver_cluster_size(int block, int want) {
  for (int size : {16, 8}) {
    if (size > want) continue;
    if (pcg_cluster_ok(block, size) && amg_cluster_ok(block, size) && mixed_cluster_ok(block, size)) return size;
  }
  return 0;
}
}  // namespace bd

namespace {

// adaptive stepping: ladder dt_max 2^-k, k = 0..kAdaptLadder-1, controller
// factor 0.9 err^(-1/2) clamped to [0.5, 2] (embedded solution of order 1)
constexpr int kAdaptLadder = 8;
double ladder_step(double dt_max, double want) {
  for (int k = 0; k < kAdaptLadder; ++k) {
    const double d = dt_max * std::ldexp(1.0, -k);
    if (d <= want * (1.0 + 1e-12)) return d;
  }
  return dt_max * std::ldexp(1.0, -(kAdaptLadder - 1));
}
double controller_factor(double err) {
  if (!(err > 0.0)) return 2.0;
  return std::min(2.0, std::max(0.5, 0.9 / std::sqrt(err)));
}

int enqueue_step(bd_state* s, double dt, int M, int K) {
  const double gam = 1.0 + 1.0 / std::sqrt(2.0);
  const int64_t N = s->NT, Nu = s->N;
  const int ns = s->ns;
  double c[kMaxNodes], S[kMaxNodes - 1][kMaxNodes];
  lobatto(M, c);
  integration_matrix(M, S);
  StimTable st = s->stim;
  const int* gate = s->opts.sweep_tol > 0 ? s->gate : nullptr;
  if (gate) {
    Timed t(s, BD_K_COMBINE);
    CK(launch_set_int(s->gate, 1, s->dmax, s->stream));
  }
  {
    Timed t(s, BD_K_FIELD);
    CK(launch_field(s->model, s->precision, N, s->Xn, s->inv_cm, dt, s->stim_bits, s->t_now, st, s->fq[0], s->stream));
  }
  for (int k = 1; k <= K; ++k) {
    // ---- elliptic constraint at the nodes m >= 1 ----
    if (k == 1) {
      RUN(elliptic(s, s->Xn, s->u[M - 1]));
      for (int m = 1; m + 1 < M; ++m) {
        Timed t(s, BD_K_COMBINE);
        CK(launch_copy(Nu, s->u[M - 1], s->u[m], s->stream, gate));
      }
    } else {
      if (k == 2) {
        // warm starts extrapolated in time from this and the previous step's
        // sweep-1 solutions (u_m still holds E(v^n) at every node)
        Timed t(s, BD_K_COMBINE, 2);
        CK(launch_extrap(Nu, M == 3 ? s->u[1] : nullptr, s->u[M - 1], s->uprev, 0.5, dt, s->t_now, gate,
                         s->stream));
      }
      if (M == 3) {
        RUN(elliptic2(s, s->Xc[1], s->u[1], s->Xc[2], s->u[2]));
      } else {
        for (int m = 1; m < M; ++m) RUN(elliptic(s, s->Xc[m], s->u[m]));
      }
    }
    // ---- ROS2 predictor ----
    if (s->adapt_on) {   // the estimate is the one of the last sweep that ran
      Timed t(s, BD_K_COMBINE);
      CK(launch_clear_gated(s->d_err, gate, s->stream));
    }
    for (int m = 0; m + 1 < M; ++m) {
      const double h = dt * (c[m + 1] - c[m]);
      const double alpha = 1.0 / (gam * h);
      const double* src = m == 0 ? s->Xn : s->Xt[m];
      IonicLaunch L = ionic_base(s, MODE_S1, dt);
      L.alpha = alpha;
      L.smin = s->opts.spd_margin > 0 ? -s->opts.spd_margin * alpha * s->lambda_M : -INFINITY;
      L.XJ = src;
      L.u = s->u[m + 1];
      L.z = s->z1;
      L.w = s->w1;
      L.fq_out = (m >= 1 && s->opts.sdc_correction) ? s->fq[m] : nullptr;
      L.pack = s->pack;
      // the correction of interval m - 1 takes its Jacobian at this same
      // state; at m = 0 (state X^n, the same in every sweep) the first FP64
      // sweep stores the field and Jacobian and the later sweeps load them
      // (in FP32 the store costs more than the evaluation it saves)
      const bool reuse0 = s->precision == BD_FP64 && K > 1;
      if (m >= 1) L.jac_out = s->opts.sdc_correction ? s->jpack : nullptr;
      else if (reuse0 && k == 1) L.jac_out = s->jpack0;
      else if (reuse0) L.jac_in = s->jpack0;
      {
        Timed t(s, BD_K_IONIC);
        CK(launch_ionic(L, s->stream));
      }
      double* k1 = s->kinc[m][0];
      double* k2 = s->kinc[m][1];
      RUN(parabolic(s, alpha, -1.0, s->avec, 0.0, nullptr, k1, true, true));
      IonicLaunch L2 = ionic_base(s, MODE_S2P, dt);   // reuses stage 1's condensation
      L2.pack = s->pack;
      L2.alpha = alpha;
      L2.smin = L.smin;
      L2.XJ = src;
      L2.u = s->u[m + 1];
      L2.k1v = k1;
      L2.z1 = s->z1;
      L2.w1 = s->w1;
      L2.ck1 = 2.0 / (gam * h);
      L2.inv_gamma = 1.0 / gam;
      L2.z = s->z2;
      L2.bvec = s->bvec;
      {
        Timed t(s, BD_K_IONIC);
        CK(launch_ionic(L2, s->stream));
      }
      RUN(parabolic(s, alpha, -1.0, s->avec, -L2.ck1, s->bvec, k2, true, true));
      {
        Timed t(s, BD_K_COMBINE);
        CK(launch_combine(s->model, s->precision == BD_MIXED, N, src, k1, s->z1, s->w1, k2, s->z2, s->w1, 1.5 / gam,
                          0.5 / gam,
                          s->Xt[m + 1], s->stream, gate, 1.0 / gam, s->adapt_tol,
                          s->adapt_on ? s->d_err : nullptr));
      }
      s->ionic_evals += 3;
    }
    // ---- SDC correction ----
    if (s->opts.sdc_correction) {
      {
        Timed t(s, BD_K_FIELD);
        CK(launch_field(s->model, s->precision, N, s->Xt[M - 1], s->inv_cm, dt, s->stim_bits, s->t_now, st,
                        s->fq[M - 1], s->stream, gate));
      }
      s->ionic_evals += 1;
      for (int m = 0; m + 1 < M; ++m) {
        const double h = dt * (c[m + 1] - c[m]);
        const double alpha = 1.0 / h;
        IonicLaunch L = ionic_base(s, MODE_CORR, dt);
        L.alpha = alpha;
        L.smin = s->opts.spd_margin > 0 ? -s->opts.spd_margin * alpha * s->lambda_M : -INFINITY;
        L.inv_dt = 1.0 / h;
        L.XJ = s->Xt[m + 1];
        L.Xprev = m == 0 ? s->Xn : s->Xc[m];
        L.n_nodes = M;
        // the predictor of interval m + 1 stored the Jacobian at X~_{m+1}
        L.jac_in = m + 2 < M ? s->jpack : nullptr;
        for (int j = 0; j < M; ++j) {
          L.S[j] = dt * S[m][j];
          L.Xq[j] = j == 0 ? s->Xn : s->Xt[j];
          L.uq[j] = s->u[j];
          L.fq[j] = s->fq[j];
        }
        L.z = s->z1;
        L.w = s->w1;
        L.bvec = s->bvec;
        {
          Timed t(s, BD_K_IONIC);
          CK(launch_ionic(L, s->stream));
        }
        double* ek = s->kinc[m][2];
        RUN(parabolic(s, alpha, -1.0 / h, s->avec, 1.0 / h, s->bvec, ek, true, true));
        {
          Timed t(s, BD_K_COMBINE);
          CK(launch_update(s->model, s->precision == BD_MIXED, N, s->Xt[m + 1], ek, s->z1, s->w1, s->Xc[m + 1],
                           s->stream, gate));
        }
        s->ionic_evals += 1;
      }
    } else {
      for (int m = 1; m < M; ++m) {
        Timed t(s, BD_K_COMBINE);
        CK(launch_copy(int64_t(ns) * N, s->Xt[m], s->Xc[m], s->stream, gate));
      }
    }
    // Algorithm 2's test: stop the sweeps once max |X^k - X^(k-1)| < sweep_tol
    if (gate && k < K) {
      Timed t(s, BD_K_COMBINE, 4);
      CK(cudaMemsetAsync(s->dmax, 0, 8, s->stream));
      CK(launch_sweep_delta(int64_t(ns) * N, s->Xc[M - 1], k == 1 ? s->Xn : s->Xsave, s->dmax, gate, s->stream));
      CK(launch_sweep_gate(s->dmax, s->opts.sweep_tol, s->gate, s->d_stats + 6, s->stream));
      CK(launch_copy(int64_t(ns) * N, s->Xc[M - 1], s->Xsave, s->stream, gate));
    }
  }
  {
    Timed t(s, BD_K_FINISH, 2);
    CK(launch_finish(ns, N, Nu, s->Xn, s->Xc[M - 1], s->u[0], s->u[M - 1], s->t_act, s->opts.v_act_mV, dt,
                     s->step_n, s->t_now, s->d_status, s->stream));
  }
  return BD_OK;
}

// One step of the decoupled CN-RK2 scheme (Sec. 3.3.3, the paper's reference
// decoupled strategy): Strang splitting of the node reaction and the
// diffusion, the elliptic constraint solved last.
//   X*      = reaction half step (dt/2) from X^n               rk2 kernel
//   (2/dt M_v + A_i) dv = -2 A_i (v* + u^n)                   CG, Crank-Nicolson
//   X^{n+1} = reaction half step from (v* + dv, y*)            rk2 kernel
//   A_ie u^{n+1} = -A_i v^{n+1}                                 CG (Eq. (3.15) form)
int enqueue_cnrk2(bd_state* s, double dt) {
  const int64_t N = s->NT, Nu = s->N;
  if (s->gate) {   // an earlier SDC step's sweep test may have closed the gate
    Timed t(s, BD_K_COMBINE);
    CK(launch_set_int(s->gate, 1, nullptr, s->stream));
  }
  {
    Timed t(s, BD_K_IONIC);
    CK(launch_rk2(s->model, s->precision, N, s->Xn, nullptr, s->Xt[1], 0.5 * dt, s->inv_cm, dt, s->stim_bits,
                  s->t_now, s->stim, s->u[0], s->avec, s->stream));
  }
  RUN(parabolic(s, 2.0 / dt, -2.0, s->avec, 0.0, nullptr, s->k1v, false));
  {
    Timed t(s, BD_K_IONIC);
    CK(launch_rk2(s->model, s->precision, N, s->Xt[1], s->k1v, s->Xc[1], 0.5 * dt, s->inv_cm, dt, s->stim_bits,
                  s->t_now, s->stim, nullptr, nullptr, s->stream));
  }
  RUN(elliptic(s, s->Xc[1], s->u[1]));
  {
    Timed t(s, BD_K_FINISH, 2);
    CK(launch_finish(s->ns, N, Nu, s->Xn, s->Xc[1], s->u[0], s->u[1], s->t_act, s->opts.v_act_mV, dt,
                     s->step_n, s->t_now, s->d_status, s->stream));
  }
  s->ionic_evals += 4;
  return BD_OK;
}

int enqueue_any(bd_state* s, double dt, int M, int K) {
  return M == 0 ? enqueue_cnrk2(s, dt) : enqueue_step(s, dt, M, K);
}

int do_step(bd_state* s, double dt, int M, int K) {
  RUN(prepare_step(s, dt, M));
  if (s->prof && s->opts.streaming != 2) {
    // a profiled step is captured with its event records and replayed, so
    // every event pair brackets device work only (launched eagerly, a fast
    // kernel's pair would also hold the time the GPU waits for the host)
    while (s->evpool.size() < 1024) {
      bd_state::Ev e{0, nullptr, nullptr};
      CK(cudaEventCreate(&e.a));
      CK(cudaEventCreate(&e.b));
      s->evpool.push_back(e);
    }
    cudaGraph_t g = nullptr;
    s->enq_launches = 0;
    CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    const int r = enqueue_any(s, dt, M, K);
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    if (r != BD_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (e != cudaSuccess) return fail(s, BD_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(s, BD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    e = cudaGraphUpload(ex, s->stream);   // the upload precedes the first event node
    if (e == cudaSuccess) e = cudaGraphLaunch(ex, s->stream);
    cudaGraphExecDestroy(ex);
    if (e != cudaSuccess) return fail(s, BD_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    s->launches += s->enq_launches;
  } else if (!s->opts.use_graph || s->prof) {
    s->enq_launches = 0;
    RUN(enqueue_any(s, dt, M, K));
    s->launches += s->enq_launches;
  } else {
    const int adapt = s->adapt_on ? 1 : 0;
    bd_state::GraphEntry* ge = nullptr;
    for (auto& g : s->graphs)
      if (g.dt == dt && g.M == M && g.K == K && g.adapt == adapt) ge = &g;
    if (!ge) {
      if (s->graphs.size() >= 16) {   // keep the cache bounded
        cudaGraphExecDestroy(s->graphs.front().exec);
        s->graphs.erase(s->graphs.begin());
      }
      cudaGraph_t g = nullptr;
      const int64_t ev0 = s->ionic_evals;
      s->enq_launches = 0;
      CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
      const int r = enqueue_any(s, dt, M, K);
      const int64_t nl = s->enq_launches;
      cudaError_t e = cudaStreamEndCapture(s->stream, &g);
      if (r != BD_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      if (e != cudaSuccess) return fail(s, BD_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
      cudaGraphExec_t ex = nullptr;
      e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(s, BD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
      s->graphs.push_back({dt, M, K, adapt, ex, nl});
      ge = &s->graphs.back();
      s->ionic_evals = ev0;   // counted per replay below
    }
    s->launches_per_step = ge->launches;
    CK(cudaGraphLaunch(ge->exec, s->stream));
    s->launches += s->launches_per_step;
    s->ionic_evals += M == 0 ? 4 : int64_t(K) * (3 * (M - 1) + (s->opts.sdc_correction ? M : 0)) + 1;
  }
  s->steps += 1;
  s->sweeps += K;
  return BD_OK;
}

void invalidate_graph(bd_state* s) {
  for (auto& g : s->graphs) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
}

// ---------------------------------------------------------------------------
// batched steps (bd_batch_step): one launch per phase over the concatenated
// nodes of many handles, the whole step captured as one graph per (dt, M, K)
// ---------------------------------------------------------------------------
//
// Every phase of enqueue_step becomes one batched launch (segment.cuh): the
// node-wise kernels over the handles' tissue nodes, every elliptic or
// parabolic solve one batched streaming solve (stream.cu) whose systems keep
// their own reductions, scalars, stopping tests and iteration caps.  The
// per-handle argument tables and block prefixes are written into a device
// arena when the step is captured; the graph reads them at replay.

struct BatchPlan {
  std::vector<bd_state*> m;
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  BatchCtl* ctl = nullptr;
  // arena chunks (one per captured step shape; graphs keep pointing into theirs)
  std::vector<char*> chunks;
  char* cur = nullptr;             // chunk of the capture in progress
  size_t cap = 0, used = 0;
  bool overflow = false;
  std::vector<char> host;          // host image of the current chunk
  struct G {
    double dt;
    int M, K;
    cudaGraphExec_t exec;
    int64_t launches;
  };
  std::vector<G> graphs;
  int64_t enq = 0;                 // launches enqueued by the capture in progress
  uint64_t last_use = 0;
  ~BatchPlan() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    for (char* c : chunks) cudaFree(c);
    if (ctl) cudaFree(ctl);
    for (cudaStream_t x : side)
      if (x) cudaStreamDestroy(x);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
  }
};

std::mutex g_batch_mu;
std::vector<std::unique_ptr<BatchPlan>> g_batches;
uint64_t g_batch_clock = 0;
constexpr size_t kMaxBatchPlans = 16;   // plans kept (least recently used dropped first)

// copy a table into the chunk of the capture in progress; returns its device address
template <class T>
T* put(BatchPlan& B, const T* v, size_t count) {
  const size_t bytes = sizeof(T) * count, at = (B.used + 255) & ~size_t(255);
  if (at + bytes > B.cap) {
    B.overflow = true;
    return reinterpret_cast<T*>(B.cur);
  }
  if (B.host.size() < at + bytes) B.host.resize(at + bytes);
  std::memcpy(B.host.data() + at, v, bytes);
  B.used = at + bytes;
  return reinterpret_cast<T*>(B.cur + at);
}
template <class T>
T* put(BatchPlan& B, const std::vector<T>& v) {
  return put(B, v.data(), v.size());
}

// block prefix of per-handle block counts; *total receives the sum
int* prefix(BatchPlan& B, const std::vector<int>& counts, int* total) {
  std::vector<int> p(counts.size() + 1, 0);
  for (size_t i = 0; i < counts.size(); ++i) p[i + 1] = p[i] + counts[i];
  *total = p.back();
  return put(B, p);
}
std::vector<int> blocks_of(const BatchPlan& B, const std::function<int64_t(const bd_state*)>& n, int block) {
  std::vector<int> c;
  for (const bd_state* s : B.m) c.push_back(int((n(s) + block - 1) / block));
  return c;
}

#define BCK(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(s0, BD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// the streaming workspaces a handle needs to take part in a batch (its own
// steps may use the persistent solvers and never allocate them)
int ensure_stream_ws(bd_state* s) {
  const int64_t N = s->N;
  bool ok = true;
  if (!s->d_sc)
    ok = alloc_n(s, reinterpret_cast<char**>(&s->d_sc), int64_t(2 * sizeof(StreamScal))) &&
         cudaMemsetAsync(s->d_sc, 0, 2 * sizeof(StreamScal), s->stream) == cudaSuccess;
  if (ok && !s->spart) ok = alloc_n(s, &s->spart, int64_t(stream_grid_cap()) * 4);
  if (ok && s->precision == BD_FP64 && !s->sb64) {
    ok = alloc_n(s, &s->sb64, N) && alloc_n(s, &s->sr64, N) && alloc_n(s, &s->sr, N) && alloc_n(s, &s->sz, N) &&
         alloc_n(s, &s->sp, N) && alloc_n(s, &s->sq, N) && alloc_n(s, &s->sd, N) && alloc_n(s, &s->sinvd, N);
    for (double* v : {s->sb64, s->sr64, s->sr, s->sz, s->sp, s->sq, s->sd, s->sinvd})
      if (ok && v) ok = cudaMemsetAsync(v, 0, N * 8, s->stream) == cudaSuccess;
  }
  if (!ok) return fail(s, BD_ERR_OOM, "device allocation failed (batch workspaces)");
  return BD_OK;
}

// one batched solve: elliptic (v -> u, all nodes) or parabolic (the
// condensed systems of the tissue rows)
struct BatchSolveArgs {
  bool elliptic;
  double alpha, c1, c2;            // parabolic: shift and right-hand-side factors
  bool node_terms;
  std::vector<const double*> va, vb;
  std::vector<double*> x;
};

int batch_solve(BatchPlan& B, const BatchSolveArgs& q, cudaStream_t st) {
  bd_state* s0 = B.m[0];
  const int nseg = int(B.m.size());
  const bool mixed = s0->precision == BD_MIXED;
  std::vector<StreamLaunch> tab(nseg);
  std::vector<int> rows(nseg), post0(nseg), coarse(nseg);
  int nlev_max = 0;
  std::vector<AmgDevF> hf(q.elliptic && mixed ? nseg : 0);
  std::vector<AmgDev> hd(q.elliptic && !mixed ? nseg : 0);
  std::vector<std::vector<int>> lA(kMaxAmgLevels, std::vector<int>(nseg, 0)), lR = lA, lP = lA;
  for (int r = 0; r < nseg; ++r) {
    bd_state* s = B.m[r];
    const int n = int(q.elliptic ? s->N : s->NT);
    StreamLaunch A = stream_base(s, n);
    A.launch_acc = nullptr;
    A.gate = nullptr;
    A.grid = stream_grid(n);
    if (q.elliptic) {
      A.valA = s->Aie;
      A.valT = mixed ? static_cast<const void*>(s->fAie) : static_cast<const void*>(s->Aie);
      set_vec4(s, A, s->fAie4);
      A.val1 = s->Ai;
      A.va = q.va[r];
      A.c1 = -1.0;
      A.project = 1;
      A.warm = 1;
      A.pin = s->opts.pin_node >= 0 ? s->opts.pin_node : -1;
      A.max_outer = mixed ? 12 : 1;
      A.inner_cap = s->opts.cg_cap_e;
      A.use_amg = s->use_amg ? 1 : 0;
      A.tol = s->opts.cg_tol_e;
      A.tol_inner = mixed ? double(BD_MIXED_TOL_INNER) : s->opts.cg_tol_e;
      A.iters_acc = s->d_stats + 0;
      A.solves_acc = s->d_stats + 1;
      A.outer_acc = s->d_stats + 4;
      int nlev = 0;
      if (s->use_amg) {
        nlev = mixed ? s->amgf.nlev : s->amg.nlev;
        const int nc = mixed ? s->amgf.nc : s->amg.nc;
        A.h0_invd = mixed ? static_cast<const void*>(s->amgf.L[0].invd) : static_cast<const void*>(s->amg.L[0].invd);
        A.h0_x = mixed ? static_cast<void*>(s->amgf.L[0].x) : static_cast<void*>(s->amg.L[0].x);
        A.h0_omega = mixed ? double(s->amgf.L[0].omega) : s->amg.L[0].omega;
        for (int l = 0; l < nlev; ++l) {
          auto grid_of = [&](const auto& M) { return stream_grid(level_threads(M)); };
          if (mixed) {
            lA[l][r] = grid_of(s->amgf.L[l].A);
            lR[l][r] = grid_of(s->amgf.L[l].R);
            lP[l][r] = grid_of(s->amgf.L[l].P);
          } else {
            lA[l][r] = grid_of(s->amg.L[l].A);
            lR[l][r] = grid_of(s->amg.L[l].R);
            lP[l][r] = grid_of(s->amg.L[l].P);
          }
        }
        coarse[r] = stream_grid(int64_t(std::max(1, nc)) * 32);
        if (mixed) hf[r] = s->amgf;
        else hd[r] = s->amg;
      } else {
        if (mixed) hf[r] = AmgDevF{};
        else hd[r] = AmgDev{};
      }
      nlev_max = std::max(nlev_max, nlev);
      post0[r] = s->use_amg ? lA[0][r] : 1;
    } else {
      A.valA = p_values(s, q.alpha);
      A.valT = mixed ? static_cast<const void*>(p_values_f(s, q.alpha)) : static_cast<const void*>(A.valA);
      if (!A.valA || !A.valT) return fail(s0, BD_ERR_OOM, "device allocation failed");
      if (mixed) set_vec4(s, A, p_values_f4(s, q.alpha));
      A.dextra = q.node_terms ? s->dgs : nullptr;
      A.rl = q.node_terms ? s->rl : nullptr;
      A.val1 = s->Ai;
      A.va = q.va[r];
      A.c1 = q.c1;
      if (!q.vb.empty() && q.vb[r]) {
        A.val2 = s->Mv;
        A.vb = q.vb[r];
        A.c2 = q.c2;
      }
      A.project = 0;
      A.warm = 1;
      A.pin = -2;
      A.max_outer = 1;
      A.inner_cap = s->opts.cg_cap_p;
      A.use_amg = 0;
      A.tol = s->opts.cg_tol_p;
      A.tol_inner = mixed ? std::max(s->opts.cg_tol_p, 1e-6) : s->opts.cg_tol_p;
      A.iters_acc = s->d_stats + 2;
      A.solves_acc = s->d_stats + 3;
      A.outer_acc = s->d_stats + 5;
      post0[r] = 1;
    }
    A.x = q.x[r];
    rows[r] = A.grid;
    tab[r] = A;
  }
  BatchSolve bs{};
  bs.tab = put(B, tab);
  bs.nseg = nseg;
  bs.f32 = mixed ? 1 : 0;
  bs.ctl = B.ctl;
  bs.launch_acc = s0->d_stats + 8;
  bs.blk_rows = prefix(B, rows, &bs.total_rows_blocks);
  bs.blk_post0 = prefix(B, post0, &bs.total_post0_blocks);
  bs.nlev_max = nlev_max;
  for (int l = 0; l < nlev_max; ++l) {
    bs.blk_A[l] = prefix(B, lA[l], &bs.total_A[l]);
    bs.blk_R[l] = prefix(B, lR[l], &bs.total_R[l]);
    bs.blk_P[l] = prefix(B, lP[l], &bs.total_P[l]);
  }
  bs.blk_coarse = prefix(B, coarse, &bs.total_coarse);
  for (const StreamLaunch& A : tab) {
    bs.inner_cap = std::max(bs.inner_cap, unsigned(std::max(A.inner_cap, 1)));
    bs.max_outer = std::max(bs.max_outer, unsigned(std::max(A.max_outer, 1)));
  }
  bs.hier = mixed ? static_cast<const void*>(put(B, hf)) : static_cast<const void*>(put(B, hd));
  BCK(stream_solve_batch(bs, st, B.side));   // its kernels count themselves on the device
  return BD_OK;
}

int enqueue_batch_step(BatchPlan& B, double dt, int M, int K) {
  bd_state* s0 = B.m[0];
  const cudaStream_t st = s0->stream;
  const int nseg = int(B.m.size());
  const int model = s0->model, prec = s0->precision, ns = s0->ns;
  const double gam = 1.0 + 1.0 / std::sqrt(2.0);
  double c[kMaxNodes], S[kMaxNodes - 1][kMaxNodes];
  lobatto(M, c);
  integration_matrix(M, S);
  auto NT = [](const bd_state* s) { return s->NT; };
  auto NU = [](const bd_state* s) { return s->N; };
  int tot = 0;
  int* blk_node = prefix(B, blocks_of(B, NT, kNodeBlock), &tot);
  const int nb_node = tot;
  int* blk_vec_u = prefix(B, blocks_of(B, NU, kVecBlock), &tot);
  const int nb_vec_u = tot;
  int* blk_fin = prefix(B, blocks_of(B, [](const bd_state* s) { return std::max(s->NT, s->N); }, kVecBlock), &tot);
  const int nb_fin = tot;
  auto field = [&](auto Xof, auto fof) {
    std::vector<FieldArgs> t;
    for (bd_state* s : B.m) t.push_back({s->NT, Xof(s), s->inv_cm, dt, s->stim_bits, s->t_now, s->stim, fof(s)});
    B.enq += 1;
    return launch_field_batch(model, prec, put(B, t), blk_node, nseg, nb_node, st);
  };
  auto copy_u = [&](auto src, auto dst) {
    std::vector<CopyArgs> t;
    for (bd_state* s : B.m) t.push_back({s->N, src(s), dst(s)});
    B.enq += 1;
    return launch_copy_batch(put(B, t), blk_vec_u, nseg, nb_vec_u, st);
  };
  // the elliptic constraint u_m = E(v) for every handle (bath meshes gather v
  // into the zero-padded N-vector first)
  auto elliptic_all = [&](auto vof, auto uof) -> int {
    bool bath = false;
    for (bd_state* s : B.m) bath = bath || s->NT < s->N;
    if (bath) {                     // copies for the bath members only
      std::vector<CopyArgs> t;
      std::vector<int> cnt;
      for (bd_state* s : B.m) {
        const bool b = s->NT < s->N;
        t.push_back({b ? s->NT : 0, vof(s), b ? s->vfull : nullptr});
        cnt.push_back(b ? int((s->NT + kVecBlock - 1) / kVecBlock) : 0);
      }
      int nb = 0;
      int* blk = prefix(B, cnt, &nb);
      B.enq += 1;
      BCK(launch_copy_batch(put(B, t), blk, nseg, nb, st));
    }
    BatchSolveArgs q{};
    q.elliptic = true;
    for (bd_state* s : B.m) {
      q.va.push_back(s->NT < s->N ? s->vfull : vof(s));
      q.x.push_back(uof(s));
    }
    return batch_solve(B, q, st);
  };
  auto parabolic_all = [&](double alpha, double c1, double c2, bool with_b, int m, int g) -> int {
    BatchSolveArgs q{};
    q.elliptic = false;
    q.alpha = alpha;
    q.c1 = c1;
    q.c2 = c2;
    q.node_terms = true;
    for (bd_state* s : B.m) {
      q.va.push_back(s->avec);
      q.vb.push_back(with_b ? s->bvec : nullptr);
      q.x.push_back(s->kinc[m][g]);
    }
    return batch_solve(B, q, st);
  };
  auto ionic_all = [&](auto build) {
    std::vector<IonicLaunch> t;
    for (bd_state* s : B.m) t.push_back(build(s));
    B.enq += 1;
    return launch_ionic_batch(t[0], put(B, t), blk_node, nseg, nb_node, st);
  };

  BCK(field([](bd_state* s) { return s->Xn; }, [](bd_state* s) { return s->fq[0]; }));
  for (int k = 1; k <= K; ++k) {
    if (k == 1) {
      RUN(elliptic_all([](bd_state* s) { return s->Xn; }, [M](bd_state* s) { return s->u[M - 1]; }));
      for (int m = 1; m + 1 < M; ++m)
        BCK(copy_u([M](bd_state* s) { return s->u[M - 1]; }, [m](bd_state* s) { return s->u[m]; }));
    } else {
      if (k == 2) {
        std::vector<ExtrapArgs> t;
        for (bd_state* s : B.m) t.push_back({s->N, M == 3 ? s->u[1] : nullptr, s->u[M - 1], s->uprev, 0.5, dt, s->t_now});
        B.enq += 2;
        BCK(launch_extrap_batch(put(B, t), blk_vec_u, nseg, nb_vec_u, st));
      }
      for (int m = 1; m < M; ++m)
        RUN(elliptic_all([m](bd_state* s) { return s->Xc[m]; }, [m](bd_state* s) { return s->u[m]; }));
    }
    // ROS2 predictor (the launch arguments of enqueue_step)
    for (int m = 0; m + 1 < M; ++m) {
      const double h = dt * (c[m + 1] - c[m]);
      const double alpha = 1.0 / (gam * h);
      const bool reuse0 = prec == BD_FP64 && K > 1;
      auto s1 = [&](bd_state* s) {
        IonicLaunch L = ionic_base(s, MODE_S1, dt);
        L.gate = nullptr;
        L.alpha = alpha;
        L.smin = s->opts.spd_margin > 0 ? -s->opts.spd_margin * alpha * s->lambda_M : -INFINITY;
        L.XJ = m == 0 ? s->Xn : s->Xt[m];
        L.u = s->u[m + 1];
        L.z = s->z1;
        L.w = s->w1;
        L.fq_out = (m >= 1 && s->opts.sdc_correction) ? s->fq[m] : nullptr;
        L.pack = s->pack;
        if (m >= 1) L.jac_out = s->opts.sdc_correction ? s->jpack : nullptr;
        else if (reuse0 && k == 1) L.jac_out = s->jpack0;
        else if (reuse0) L.jac_in = s->jpack0;
        return L;
      };
      BCK(ionic_all(s1));
      RUN(parabolic_all(alpha, -1.0, 0.0, false, m, 0));
      auto s2 = [&](bd_state* s) {
        IonicLaunch L2 = ionic_base(s, MODE_S2P, dt);
        L2.gate = nullptr;
        L2.pack = s->pack;
        L2.alpha = alpha;
        L2.smin = s->opts.spd_margin > 0 ? -s->opts.spd_margin * alpha * s->lambda_M : -INFINITY;
        L2.XJ = m == 0 ? s->Xn : s->Xt[m];
        L2.u = s->u[m + 1];
        L2.k1v = s->kinc[m][0];
        L2.z1 = s->z1;
        L2.w1 = s->w1;
        L2.ck1 = 2.0 / (gam * h);
        L2.inv_gamma = 1.0 / gam;
        L2.z = s->z2;
        L2.bvec = s->bvec;
        return L2;
      };
      BCK(ionic_all(s2));
      RUN(parabolic_all(alpha, -1.0, -2.0 / (gam * h), true, m, 1));
      {
        std::vector<CombineArgs> t;
        for (bd_state* s : B.m)
          t.push_back({s->NT, m == 0 ? s->Xn : s->Xt[m], s->kinc[m][0], s->z1, s->w1, s->kinc[m][1], s->z2, s->w1,
                       1.5 / gam, 0.5 / gam, s->Xt[m + 1]});
        B.enq += 1;
        BCK(launch_combine_batch(model, s0->precision == BD_MIXED, put(B, t), blk_node, nseg, nb_node, st));
      }
    }
    // SDC correction
    if (s0->opts.sdc_correction) {
      BCK(field([M](bd_state* s) { return s->Xt[M - 1]; }, [M](bd_state* s) { return s->fq[M - 1]; }));
      for (int m = 0; m + 1 < M; ++m) {
        const double h = dt * (c[m + 1] - c[m]);
        const double alpha = 1.0 / h;
        auto cr = [&](bd_state* s) {
          IonicLaunch L = ionic_base(s, MODE_CORR, dt);
          L.gate = nullptr;
          L.alpha = alpha;
          L.smin = s->opts.spd_margin > 0 ? -s->opts.spd_margin * alpha * s->lambda_M : -INFINITY;
          L.inv_dt = 1.0 / h;
          L.XJ = s->Xt[m + 1];
          L.Xprev = m == 0 ? s->Xn : s->Xc[m];
          L.n_nodes = M;
          L.jac_in = m + 2 < M ? s->jpack : nullptr;
          for (int j = 0; j < M; ++j) {
            L.S[j] = dt * S[m][j];
            L.Xq[j] = j == 0 ? s->Xn : s->Xt[j];
            L.uq[j] = s->u[j];
            L.fq[j] = s->fq[j];
          }
          L.z = s->z1;
          L.w = s->w1;
          L.bvec = s->bvec;
          return L;
        };
        BCK(ionic_all(cr));
        RUN(parabolic_all(alpha, -1.0 / h, 1.0 / h, true, m, 2));
        std::vector<UpdateArgs> t;
        for (bd_state* s : B.m) t.push_back({s->NT, s->Xt[m + 1], s->kinc[m][2], s->z1, s->w1, s->Xc[m + 1]});
        B.enq += 1;
        BCK(launch_update_batch(model, s0->precision == BD_MIXED, put(B, t), blk_node, nseg, nb_node, st));
      }
    } else {
      for (int m = 1; m < M; ++m) {
        std::vector<CopyArgs> t;
        for (bd_state* s : B.m) t.push_back({int64_t(ns) * s->NT, s->Xt[m], s->Xc[m]});
        std::vector<int> cnt;
        for (bd_state* s : B.m) cnt.push_back(int((int64_t(ns) * s->NT + kVecBlock - 1) / kVecBlock));
        int nb = 0;
        int* blk = prefix(B, cnt, &nb);
        B.enq += 1;
        BCK(launch_copy_batch(put(B, t), blk, nseg, nb, st));
      }
    }
  }
  {
    std::vector<FinishArgs> t;
    for (bd_state* s : B.m)
      t.push_back({ns, s->NT, s->N, s->Xn, s->Xc[M - 1], s->u[0], s->u[M - 1], s->t_act, s->opts.v_act_mV, dt,
                   s->t_now, s->step_n, s->d_status});
    B.enq += 2;
    BCK(launch_finish_batch(put(B, t), blk_fin, nseg, nb_fin, st));
  }
  return BD_OK;
}

// capture the batched step of shape (dt, M, K) into a graph of its own, with
// its tables in a fresh arena chunk (grown and captured again if too small)
int capture_batch_step(BatchPlan& B, double dt, int M, int K, BatchPlan::G* out) {
  bd_state* s0 = B.m[0];
  size_t want = size_t(1) << 22;
  for (int attempt = 0; attempt < 8; ++attempt) {
    char* chunk = nullptr;
    BCK(cudaMalloc(&chunk, want));
    B.cur = chunk;
    B.cap = want;
    B.used = 0;
    B.overflow = false;
    B.host.clear();
    B.enq = 0;
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(s0->stream, cudaStreamCaptureModeThreadLocal));
    const int r = enqueue_batch_step(B, dt, M, K);
    const cudaError_t e = cudaStreamEndCapture(s0->stream, &g);
    if (r != BD_OK || e != cudaSuccess || B.overflow) {
      if (g) cudaGraphDestroy(g);
      cudaFree(chunk);
      if (r != BD_OK) return r;
      if (e != cudaSuccess) return fail(s0, BD_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e));
      want *= 4;                      // the tables did not fit: larger chunk, capture again
      continue;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      cudaFree(chunk);
      return fail(s0, BD_ERR_CUDA, "batch graph instantiate: %s", cudaGetErrorString(ei));
    }
    if (cudaMemcpy(chunk, B.host.data(), B.used, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGraphExecDestroy(ex);
      cudaFree(chunk);
      return fail(s0, BD_ERR_CUDA, "batch table upload failed");
    }
    B.chunks.push_back(chunk);
    *out = {dt, M, K, ex, B.enq};
    return BD_OK;
  }
  return fail(s0, BD_ERR_OOM, "batch tables do not fit");
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void bd_default_options(bd_opts_t* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = BD_FP64;
  o->mass_lumped = 0;
  o->pin_node = 0;
  o->sdc_correction = 1;
  o->cg_tol_e = 1e-10;
  o->cg_tol_p = 1e-10;
  o->cg_cap_e = 20000;
  o->cg_cap_p = 2000;
  o->sweep_tol = 0.0;
  o->v_act_mV = -30.0;
  o->spd_margin = 0.9;
  o->use_graph = 1;
  o->elliptic_precond = 1;
  o->cg_cluster = 0;
}

int bd_num_states(bd_ionic_t model) { return model_ns(int(model)); }

int bd_create(const bd_mesh_t* mesh, const bd_cond_t* cond, bd_ionic_t model, const bd_opts_t* opts,
              bd_state_t** out) {
  bd_state* s = nullptr;
  if (!out) return fail(nullptr, BD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!mesh || !cond || !mesh->xyz || !mesh->elems) return fail(nullptr, BD_ERR_ARG, "mesh/cond missing");
  if (mesh->dim != 2 && mesh->dim != 3) return fail(nullptr, BD_ERR_ARG, "dim must be 2 or 3");
  if (mesh->n_nodes < 2 || mesh->n_elems < 1) return fail(nullptr, BD_ERR_ARG, "empty mesh");
  if (model_ns(int(model)) == 0) return fail(nullptr, BD_ERR_ARG, "unknown ionic model %d", int(model));
  if (!(cond->chi > 0) || !(cond->cm > 0) || !(cond->sil >= 0) || !(cond->sit >= 0) || !(cond->sel >= 0) ||
      !(cond->set >= 0))
    return fail(nullptr, BD_ERR_ARG, "conductivities must be >= 0 and chi, cm > 0");
  s = new bd_state();
  if (opts) s->opts = *opts;
  else bd_default_options(&s->opts);
  if (s->opts.pin_node >= mesh->n_nodes || s->opts.pin_node < -1) {
    delete s;
    return fail(nullptr, BD_ERR_ARG, "pin_node out of range");
  }
  if (!(s->opts.sweep_tol >= 0.0)) {
    delete s;
    return fail(nullptr, BD_ERR_ARG, "sweep_tol must be >= 0");
  }
  if (s->opts.precision != BD_FP64 && s->opts.precision != BD_MIXED) {
    delete s;
    return fail(nullptr, BD_ERR_ARG, "unknown precision");
  }
  s->model = int(model);
  s->ns = model_ns(int(model));
  s->dim = mesh->dim;
  s->precision = s->opts.precision;
  s->N = mesh->n_nodes;
  s->inv_cm = 1.0 / cond->cm;
  s->lambda_M = s->opts.mass_lumped ? 1.0 : (mesh->dim == 2 ? 0.25 : 0.2);

  HostOps H;
  std::string err;
  int rc = assemble_host(mesh, cond, &H, &err);
  if (rc != BD_OK) {
    delete s;
    return fail(nullptr, rc, "%s", err.c_str());
  }
  s->nnz = H.rowptr[s->N];
  s->NT = H.n_tissue;
  for (int64_t i = 0; i < s->NT; ++i)
    for (int64_t p = H.rowptr[i]; p < H.rowptr[i + 1]; ++p) s->nnz_t += H.col[p] < s->NT ? 1 : 0;
  if (s->opts.pin_node >= s->N) {
    delete s;
    return fail(nullptr, BD_ERR_ARG, "pin_node out of range");
  }
  // SELL-32 layout of the shared pattern
  const int64_t nsl = (s->N + 31) / 32;
  std::vector<int64_t> h_sptr(nsl);
  std::vector<int> h_sw(nsl);
  int maxw = 0;
  {
    int64_t off = 0;
    for (int64_t sl = 0; sl < nsl; ++sl) {
      int w = 0;
      for (int64_t i = sl * 32; i < std::min<int64_t>(s->N, sl * 32 + 32); ++i)
        w = std::max(w, H.rowptr[i + 1] - H.rowptr[i]);
      h_sw[sl] = w;
      h_sptr[sl] = off;
      off += 32 * int64_t(w);
      maxw = std::max(maxw, w);
    }
    s->ell_n = off;
  }
  s->wmax = maxw <= 8 ? 8 : maxw <= 16 ? 16 : maxw <= 32 ? 32 : 0;
  std::vector<int> e_col(s->ell_n, 0), e_diag(s->N);
  auto to_ell = [&](const std::vector<double>& v) {
    std::vector<double> e(s->ell_n, 0.0);
    for (int64_t i = 0; i < s->N; ++i) {
      const int64_t base = h_sptr[i / 32] + (i % 32);
      for (int k = 0; k < H.rowptr[i + 1] - H.rowptr[i]; ++k) e[base + 32 * k] = v[H.rowptr[i] + k];
    }
    return e;
  };
  for (int64_t i = 0; i < s->N; ++i) {
    const int64_t base = h_sptr[i / 32] + (i % 32);
    const int len = H.rowptr[i + 1] - H.rowptr[i];
    for (int k = 0; k < h_sw[i / 32]; ++k) e_col[base + 32 * k] = k < len ? H.col[H.rowptr[i] + k] : int(i);
    e_diag[i] = int(base + 32 * int64_t(H.diagpos[i] - H.rowptr[i]));
  }
  if (s->ell_n > int64_t(0x7fffffff)) {
    delete s;
    return fail(nullptr, BD_ERR_ARG, "operator too large for 32-bit SELL offsets");
  }

  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return fail(nullptr, BD_ERR_CUDA, "cudaGetDevice failed (no CUDA device?)");
  }
  if (s->opts.stream) {
    s->stream = static_cast<cudaStream_t>(s->opts.stream);
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return fail(nullptr, BD_ERR_CUDA, "cudaStreamCreate failed (no CUDA device?)");
    }
    s->own_stream = true;
  }
  // N: all nodes (u, elliptic); NT: tissue nodes (v, membrane state, parabolic)
  const int64_t N = s->N, NT = s->NT, nnz = s->nnz, ns = s->ns;
  const int64_t en = s->ell_n;
  bool ok = alloc_n(s, &s->sptr, nsl) && alloc_n(s, &s->swidth, nsl) && alloc_n(s, &s->col, en) &&
            alloc_n(s, &s->diagpos, N) && alloc_n(s, &s->Ai, en) && alloc_n(s, &s->Aie, en) &&
            alloc_n(s, &s->Mc, en) && alloc_n(s, &s->Mv, en) && alloc_n(s, &s->ML, NT) && alloc_n(s, &s->Xn, ns * NT) &&
            alloc_n(s, &s->dgs, NT) && alloc_n(s, &s->rl, NT) && alloc_zw(s, &s->z1, (ns - 1) * NT) &&
            alloc_zw(s, &s->w1, (ns - 1) * NT) && alloc_zw(s, &s->z2, (ns - 1) * NT) && alloc_n(s, &s->k1v, N) && alloc_n(s, &s->k2v, N) &&
            alloc_n(s, &s->avec, N) && alloc_n(s, &s->bvec, N) && alloc_n(s, &s->cg_r, N) &&
            alloc_n(s, &s->cg_z, N) && alloc_n(s, &s->cg_p, N) && alloc_n(s, &s->cg_q, N) &&
            alloc_n(s, &s->cg_invd, N) && alloc_n(s, &s->uprev, N) &&
            alloc_n(s, reinterpret_cast<double**>(&s->pack), int64_t(cond_pack_values(s->model)) * NT) &&
            alloc_n(s, reinterpret_cast<double**>(&s->jpack), int64_t(jac_pack_values(s->model)) * NT) &&
            alloc_n(s, reinterpret_cast<double**>(&s->jpack0), int64_t(jac_pack_values(s->model)) * NT) &&
            alloc_n(s, &s->kinc[0][0], N) &&
            alloc_n(s, &s->kinc[0][1], N) && alloc_n(s, &s->kinc[0][2], N) && alloc_n(s, &s->kinc[1][0], N) &&
            alloc_n(s, &s->kinc[1][1], N) && alloc_n(s, &s->kinc[1][2], N) && alloc_n(s, &s->t_act, NT) &&
            alloc_n(s, &s->stim_bits, NT) &&
            (NT == N || alloc_n(s, &s->vfull, N)) &&
            alloc_n(s, &s->step_n, 1) && alloc_n(s, &s->t_now, 3) && alloc_n(s, &s->d_err, 1) &&
            alloc_n(s, &s->d_status, 1) && alloc_n(s, &s->d_stats, 16) &&
            alloc_n(s, &s->d_clamps, 1) && alloc_n(s, &s->bar, 2) &&
            alloc_n(s, reinterpret_cast<char**>(&s->d_amg), int64_t(sizeof(AmgDev))) &&
            alloc_n(s, reinterpret_cast<char**>(&s->d_amgf), int64_t(sizeof(AmgDevF)));
  for (int m = 0; ok && m < kMaxNodes; ++m)
    ok = alloc_n(s, &s->Xt[m], ns * NT) && alloc_n(s, &s->Xc[m], ns * NT) && alloc_zw(s, &s->fq[m], ns * NT) &&
         alloc_n(s, &s->u[m], N);
  s->pcg_block = s->opts.cg_block > 0 ? s->opts.cg_block : 512;
  if (s->pcg_block % 32 != 0 || s->pcg_block > kSolverTierBlock[0]) {
    release(s);
    delete s;
    return fail(nullptr, BD_ERR_ARG, "cg_block must be a multiple of 32 up to 1024");
  }
  const int64_t want = s->opts.cg_grid > 0 ? s->opts.cg_grid : (N + s->pcg_block - 1) / s->pcg_block;
  // register tier (no cluster launches): the 128-register build when every
  // solver kernel of it holds the whole grid co-resident, else the 64-register
  // build, with the mixed AMG kernels at full occupancy on large operators;
  // solver_tier = 1..3 forces tier 0..2
  const int force = s->opts.solver_tier;
  if (force < 0 || force > 3 || (force == 2 && s->pcg_block > kSolverTierBlock[1])) {
    release(s);
    delete s;
    return fail(nullptr, BD_ERR_ARG, "solver_tier must be 0..3 (2 needs cg_block <= 512)");
  }
  s->tier = 0;
  if (s->opts.cg_cluster == 0) {
    if (force == 2 || (force == 0 && s->pcg_block <= kSolverTierBlock[1])) {
      int m1 = std::min(pcg_max_blocks(s->pcg_block, s->wmax, 1), pcg_amg_max_blocks(s->pcg_block, 1));
      if (s->precision == BD_MIXED) m1 = std::min(m1, pcg_mixed_max_blocks(s->pcg_block, 1));
      if (force == 2 || m1 >= want) s->tier = 1;
    }
    if (s->tier == 0 && s->precision == BD_MIXED && (force == 3 || (force == 0 && nnz >= kTier2Nnz))) s->tier = 2;
  }
  s->pcg_max = pcg_max_blocks(s->pcg_block, s->wmax, s->tier);
  if (ok && s->pcg_max <= 0) {
    release(s);
    delete s;
    return fail(nullptr, BD_ERR_CUDA, "cannot size the cooperative CG grid");
  }
  s->pcg_grid = int(std::max<int64_t>(1, std::min<int64_t>(want, s->pcg_max)));
  {
    const int cc = s->opts.cg_cluster;
    if (cc != 0 && cc != 8 && cc != 16) {
      release(s);
      delete s;
      return fail(nullptr, BD_ERR_ARG, "cg_cluster must be 0, 8 or 16");
    }
    if (cc > 0) s->cluster = solver_cluster_size(kSolverTierBlock[0], cc);
  }
  // per-block partial sums: room for the largest grid of any solver launch
  int part_blocks = s->pcg_max;
  if (s->precision == BD_MIXED) {
    const int mx = pcg_mixed_max_blocks(s->pcg_block, s->tier);
    const int ma = pcg_mixed_amg_max_blocks(s->pcg_block, s->tier);
    if (mx <= 0 || ma <= 0) ok = false;
    s->mixed_grid = std::min(s->pcg_grid, std::max(mx, 1));
    s->mixed_amg_grid = s->tier == 2 ? int(std::max<int64_t>(1, std::min<int64_t>(want, ma))) : s->mixed_grid;
    part_blocks = std::max(part_blocks, s->mixed_amg_grid);
  }
  if (ok) ok = alloc_n(s, &s->cg_part, int64_t(part_blocks) * 4);
  if (ok && s->opts.sweep_tol > 0)
    ok = alloc_n(s, &s->gate, 1) && alloc_n(s, &s->dmax, 1) && alloc_n(s, &s->Xsave, ns * NT);
  if (ok && s->precision == BD_MIXED) {
    // r, z, p, q, d, b, r64 hold two systems (two-RHS elliptic solves)
    ok = alloc_n(s, &s->fAie, s->ell_n) && alloc_n(s, &s->r32, 2 * N) && alloc_n(s, &s->z32, 2 * N) &&
         alloc_n(s, &s->p32, 2 * N) && alloc_n(s, &s->q32, 2 * N) && alloc_n(s, &s->invd32, N) &&
         alloc_n(s, &s->d32, 2 * N) && alloc_n(s, &s->b64, 2 * N) && alloc_n(s, &s->r64, 2 * N) &&
         alloc_n(s, &s->partf8, int64_t(part_blocks) * 8) && alloc_n(s, &s->partd8, int64_t(part_blocks) * 8) &&
         (NT == N || alloc_n(s, &s->vfull2, N)) &&
         alloc_n(s, reinterpret_cast<char**>(&s->d_amgf2), int64_t(sizeof(AmgDevF))) &&
         alloc_n(s, &s->partf, int64_t(part_blocks) * 8);
  }
  {
    const int so = s->opts.streaming;
    if (so < -1 || so > 2) {
      release(s);
      delete s;
      return fail(nullptr, BD_ERR_ARG, "streaming must be -1, 0, 1 or 2");
    }
    if (so == 2 && s->opts.sweep_tol > 0) {
      release(s);
      delete s;
      return fail(nullptr, BD_ERR_ARG, "streaming = 2 (host-driven loops) needs sweep_tol = 0");
    }
    s->streaming = s->opts.cg_cluster == 0 && (so >= 1 || (so == 0 && nnz >= kStreamNnz));
    if (so == 2) s->opts.use_graph = 0;   // host-driven loops cannot be captured
  }
  if (ok && s->streaming) {
    stream_prepare();   // kernel occupancies, queried outside any capture
    ok = alloc_n(s, reinterpret_cast<char**>(&s->d_sc), int64_t(2 * sizeof(StreamScal))) &&
         alloc_n(s, &s->spart, int64_t(stream_grid_cap()) * 4);
    if (ok && s->precision == BD_FP64) {
      // b, r64, r, z, p, q, d hold two systems (two-system elliptic solves)
      const int64_t N2 = s->opts.pair_solve >= 0 ? 2 * N : N;
      s->s64_sys = N2 == N ? 1 : 2;
      ok = alloc_n(s, &s->sb64, N2) && alloc_n(s, &s->sr64, N2) && alloc_n(s, &s->sr, N2) &&
           alloc_n(s, &s->sz, N2) && alloc_n(s, &s->sp, N2) && alloc_n(s, &s->sq, N2) && alloc_n(s, &s->sd, N2) &&
           alloc_n(s, &s->sinvd, N);
      // a bath mesh's second system gathers its potential over all nodes too
      if (ok && N2 > N && NT < N && !s->vfull2) ok = alloc_n(s, &s->vfull2, N);
    }
    for (cudaStream_t& x : s->side)
      if (ok && cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ok = false;
      }
  }
  // SELL-32/4 copy of the FP32 elliptic operator: four consecutive entries of
  // a row per 16-byte load in the streaming products
  if (s->opts.vec4 < -1 || s->opts.vec4 > 1) {
    release(s);
    delete s;
    return fail(nullptr, BD_ERR_ARG, "vec4 must be -1, 0 or 1");
  }
  {
    const int cl = s->opts.csr_lanes;
    if (!(cl == 0 || cl == 4 || cl == 8 || cl == 16 || cl == 32 || cl == kCsrBlockLanes) ||
        s->opts.wide_sell < -1 || s->opts.wide_sell > 1) {
      release(s);
      delete s;
      return fail(nullptr, BD_ERR_ARG, "csr_lanes must be 0, 4, 8, 16, 32 or 256 and wide_sell -1, 0 or 1");
    }
    if (s->opts.pair_solve < -1 || s->opts.pair_solve > 0) {
      release(s);
      delete s;
      return fail(nullptr, BD_ERR_ARG, "pair_solve must be -1 or 0");
    }
  }
  s->vec4 = s->streaming && s->precision == BD_MIXED && s->opts.vec4 >= 0;
  std::vector<int64_t> h_sptr4;
  std::vector<int> e_col4;
  int64_t en4 = 0;
  if (ok && s->vec4) {
    h_sptr4.resize(nsl);
    for (int64_t sl = 0; sl < nsl; ++sl) {
      h_sptr4[sl] = en4;
      en4 += 32 * int64_t((h_sw[sl] + 3) & ~3);
    }
    e_col4.assign(en4, 0);
    for (int64_t sl = 0; sl < nsl; ++sl) {
      const int w = h_sw[sl], w4 = (w + 3) & ~3;
      for (int l = 0; l < 32; ++l) {
        const int64_t i = sl * 32 + l;
        for (int k = 0; k < w4; ++k)
          e_col4[h_sptr4[sl] + 128 * (k / 4) + 4 * l + k % 4] =
              k < w ? e_col[h_sptr[sl] + 32 * k + l] : (i < N ? int(i) : 0);
      }
    }
    s->n_slices = nsl;
    s->ell_n4 = en4;
    ok = alloc_n(s, &s->sptr4, nsl) && alloc_n(s, &s->col4, en4) && alloc_n(s, &s->fAie4, en4);
  }
  if (!ok) {
    release(s);
    delete s;
    return fail(nullptr, BD_ERR_OOM, "device allocation failed");
  }
  std::vector<double> Mlump(nnz, 0.0);
  for (int64_t i = 0; i < N; ++i) Mlump[H.diagpos[i]] = H.ML[i];
  const std::vector<double> eAi = to_ell(H.Ai), eAie = to_ell(H.Aie), eM = to_ell(H.M),
                            eMv = s->opts.mass_lumped ? to_ell(Mlump) : eM;
  auto up = [&](void* d, const void* h, size_t b) { return cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, s->stream); };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = up(s->sptr, h_sptr.data(), nsl * 8);
  if (e == cudaSuccess) e = up(s->swidth, h_sw.data(), nsl * 4);
  if (e == cudaSuccess) e = up(s->col, e_col.data(), en * 4);
  if (e == cudaSuccess && s->vec4) e = up(s->sptr4, h_sptr4.data(), nsl * 8);
  if (e == cudaSuccess && s->vec4) e = up(s->col4, e_col4.data(), en4 * 4);
  if (e == cudaSuccess) e = up(s->diagpos, e_diag.data(), N * 4);
  if (e == cudaSuccess) e = up(s->Ai, eAi.data(), en * 8);
  if (e == cudaSuccess) e = up(s->Aie, eAie.data(), en * 8);
  if (e == cudaSuccess) e = up(s->Mc, eM.data(), en * 8);
  if (e == cudaSuccess) e = up(s->Mv, eMv.data(), en * 8);
  if (e == cudaSuccess) e = up(s->ML, H.ML.data(), NT * 8);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->stim_bits, 0, NT * 4, s->stream);
  // The parabolic solves run over the tissue rows only, and their bath
  // columns hold zero operator values; the vectors those rows gather from
  // must still hold finite numbers there (0 * NaN would poison a row), so
  // every node-length vector starts at zero.  Afterwards only the elliptic
  // solves write the bath entries, with finite values.
  for (double* v : {s->k1v, s->k2v, s->avec, s->bvec, s->cg_r, s->cg_z, s->cg_p, s->cg_q, s->cg_invd,
                    s->vfull, s->vfull2, s->uprev, s->kinc[0][0], s->kinc[0][1], s->kinc[0][2],
                    s->kinc[1][0], s->kinc[1][1], s->kinc[1][2]})
    if (e == cudaSuccess && v) e = cudaMemsetAsync(v, 0, N * 8, s->stream);
  for (double* v : {s->b64, s->r64})
    if (e == cudaSuccess && v) e = cudaMemsetAsync(v, 0, 2 * N * 8, s->stream);
  for (float* v : {s->r32, s->z32, s->p32, s->q32, s->d32})
    if (e == cudaSuccess && v) e = cudaMemsetAsync(v, 0, 2 * N * 4, s->stream);
  if (e == cudaSuccess && s->invd32) e = cudaMemsetAsync(s->invd32, 0, N * 4, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->bar, 0, 8, s->stream);
  for (double* v : {s->sb64, s->sr64, s->sr, s->sz, s->sp, s->sq, s->sd})
    if (e == cudaSuccess && v) e = cudaMemsetAsync(v, 0, s->s64_sys * N * 8, s->stream);
  if (e == cudaSuccess && s->sinvd) e = cudaMemsetAsync(s->sinvd, 0, N * 8, s->stream);
  if (e == cudaSuccess && s->d_sc) e = cudaMemsetAsync(s->d_sc, 0, 2 * sizeof(StreamScal), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_status, 0, 4, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_stats, 0, 128, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_clamps, 0, 8, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_amg, 0, sizeof(AmgDev), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_amgf, 0, sizeof(AmgDevF), s->stream);
  // the mass values outlive this scope only through the device copies; wait
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    release(s);
    delete s;
    return fail(nullptr, BD_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
  }
  if (s->precision == BD_MIXED &&
      (launch_to_float(s->ell_n, s->Aie, s->fAie, s->stream) != cudaSuccess ||
       (s->vec4 && launch_sell_v4(nsl, s->sptr, s->swidth, s->sptr4, s->fAie, s->fAie4, s->stream) != cudaSuccess) ||
       cudaStreamSynchronize(s->stream) != cudaSuccess)) {
    release(s);
    delete s;
    return fail(nullptr, BD_ERR_CUDA, "FP32 operator copy failed");
  }
  if (s->opts.elliptic_precond == 1) {
    rc = setup_amg(s, H);
    if (rc != BD_OK) {
      std::string m = s->err;
      release(s);
      delete s;
      return fail(nullptr, rc, "%s", m.c_str());
    }
  }
  s->host = std::move(H);
  // resting initial state
  std::vector<double> x0(ns), X(ns * NT);
  rest_state_host(s->model, x0.data());
  for (int k = 0; k < ns; ++k)
    for (int64_t i = 0; i < NT; ++i) X[k * NT + i] = x0[k];
  rc = bd_set_initial(s, X.data(), nullptr);
  if (rc != BD_OK) {
    std::string m = s->err;
    release(s);
    delete s;
    return fail(nullptr, rc, "%s", m.c_str());
  }
  *out = s;
  return BD_OK;
}

int bd_add_stimulus(bd_state_t* s, const uint8_t* mask, double t_on, double dur, double amp) {
  if (!s || !mask) return fail(s, BD_ERR_ARG, "NULL argument");
  if (s->stim.n >= kMaxStim) return fail(s, BD_ERR_ARG, "at most %d stimuli", kMaxStim);
  if (!std::isfinite(t_on) || !(dur >= 0) || !std::isfinite(amp)) return fail(s, BD_ERR_ARG, "bad stimulus timing/amplitude");
  std::vector<uint32_t> bits(s->NT);
  CK(cudaMemcpyAsync(bits.data(), s->stim_bits, s->NT * 4, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  const int k = s->stim.n;
  for (int64_t i = 0; i < s->NT; ++i)
    if (mask[i]) bits[i] |= (1u << k);
  CK(cudaMemcpyAsync(s->stim_bits, bits.data(), s->NT * 4, cudaMemcpyHostToDevice, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->stim.t_on[k] = t_on;
  s->stim.dur[k] = dur;
  s->stim.amp[k] = amp;
  s->stim.n = k + 1;
  invalidate_graph(s);
  return BD_OK;
}

int bd_set_initial(bd_state_t* s, const double* X, const double* u) {
  if (!s || !X) return fail(s, BD_ERR_ARG, "NULL argument");
  const int64_t N = s->NT, Nu = s->N, ns = s->ns;
  for (int64_t i = 0; i < ns * N; ++i)
    if (!std::isfinite(X[i])) return fail(s, BD_ERR_ARG, "non-finite initial state");
  CK(cudaMemcpyAsync(s->Xn, X, ns * N * 8, cudaMemcpyHostToDevice, s->stream));
  for (int m = 0; m < kMaxNodes; ++m) {
    if (u) CK(cudaMemcpyAsync(s->u[m], u, Nu * 8, cudaMemcpyHostToDevice, s->stream));
    else CK(cudaMemsetAsync(s->u[m], 0, Nu * 8, s->stream));
  }
  std::vector<double> nanv(N, std::nan(""));
  CK(cudaMemcpyAsync(s->t_act, nanv.data(), N * 8, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemsetAsync(s->step_n, 0, 8, s->stream));
  CK(cudaMemsetAsync(s->t_now, 0, 24, s->stream));
  CK(cudaMemsetAsync(s->uprev, 0, Nu * 8, s->stream));
  for (int m = 0; m < kMaxNodes - 1; ++m)
    for (int g = 0; g < 3; ++g) CK(cudaMemsetAsync(s->kinc[m][g], 0, Nu * 8, s->stream));
  s->dt_adapt = 0.0;
  CK(cudaStreamSynchronize(s->stream));
  return BD_OK;
}

int bd_step(bd_state_t* s, double dt, int M, int K) {
  if (!s) return fail(s, BD_ERR_ARG, "NULL handle");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(s, BD_ERR_ARG, "dt must be positive");
  if (M != 2 && M != 3) return fail(s, BD_ERR_ARG, "n_sdc_nodes must be 2 or 3");
  if (K < 1) return fail(s, BD_ERR_ARG, "n_sweeps must be >= 1");
  return do_step(s, dt, M, K);
}

int bd_selftest_wait_timeout(bd_state_t* s) {
  if (!s) return fail(s, BD_ERR_ARG, "NULL handle");
  CK(cudaStreamSynchronize(s->stream));
  CK(cudaMemsetAsync(s->bar, 0, 8, s->stream));
  CK(launch_wait_selftest(s->bar, s->d_status, s->stream));
  const int rc = read_status(s);   // synchronises; BD_ERR_TIMEOUT expected
  std::string msg = s->err;
  bd_clear_status(s);              // status word and barrier back to zero
  if (rc != BD_OK) fail(s, rc, "%s", msg.c_str());
  return rc;
}

int bd_step_decoupled(bd_state_t* s, double dt) {
  if (!s) return fail(s, BD_ERR_ARG, "NULL handle");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(s, BD_ERR_ARG, "dt must be positive");
  return do_step(s, dt, 0, 0);
}

int bd_batch_step(bd_state_t* const* states, int n, double dt, int M, int K) {
  if (!states || n < 1) return fail(nullptr, BD_ERR_ARG, "bad batch");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(nullptr, BD_ERR_ARG, "dt must be positive");
  if (M != 2 && M != 3) return fail(nullptr, BD_ERR_ARG, "n_sdc_nodes must be 2 or 3");
  if (K < 1) return fail(nullptr, BD_ERR_ARG, "n_sweeps must be >= 1");
  bd_state* const s0 = states[0];
  bd_state* s = s0;                 // error reports go to the first handle
  for (int i = 0; i < n; ++i) {
    bd_state* h = states[i];
    if (!h) return fail(nullptr, BD_ERR_ARG, "NULL handle in batch");
    for (int j = 0; j < i; ++j)
      if (states[j] == h) return fail(s0, BD_ERR_ARG, "a handle appears twice in the batch");
    if (h->model != s0->model || h->precision != s0->precision || h->device != s0->device ||
        h->opts.sdc_correction != s0->opts.sdc_correction)
      return fail(s0, BD_ERR_ARG, "batched handles must share model, precision, device and sdc_correction");
    if (h->opts.sweep_tol > 0) return fail(s0, BD_ERR_ARG, "batched handles must have sweep_tol = 0");
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchPlan* B = nullptr;
  for (auto& p : g_batches)
    if (int(p->m.size()) == n && std::equal(p->m.begin(), p->m.end(), states)) B = p.get();
  if (!B) {
    auto P = std::make_unique<BatchPlan>();
    P->m.assign(states, states + n);
    if (cudaSetDevice(s0->device) != cudaSuccess) return fail(s0, BD_ERR_CUDA, "cudaSetDevice failed");
    for (cudaStream_t& x : P->side)
      if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess)
        return fail(s0, BD_ERR_CUDA, "batch stream creation failed");
    if (cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&P->ctl, sizeof(BatchCtl)) != cudaSuccess || cudaMemset(P->ctl, 0, sizeof(BatchCtl)) != cudaSuccess)
      return fail(s0, BD_ERR_CUDA, "batch set-up failed");
    g_batches.push_back(std::move(P));
    B = g_batches.back().get();
    if (g_batches.size() > kMaxBatchPlans) {   // drop the least recently used other plan
      size_t lru = 0;
      for (size_t i = 1; i < g_batches.size(); ++i)
        if (g_batches[i]->last_use < g_batches[lru]->last_use) lru = i;
      if (g_batches[lru].get() != B) {
        for (bd_state* o : g_batches[lru]->m)
          if (o->stream) cudaStreamSynchronize(o->stream);
        g_batches.erase(g_batches.begin() + lru);
        B = nullptr;
        for (auto& p : g_batches)
          if (int(p->m.size()) == n && std::equal(p->m.begin(), p->m.end(), states)) B = p.get();
      }
    }
  }
  B->last_use = ++g_batch_clock;
  for (bd_state* h : B->m) {
    RUN(ensure_stream_ws(h));
    RUN(prepare_step(h, dt, M));
  }
  // the members' queued work precedes the batch on the first handle's stream
  for (bd_state* h : B->m) {
    if (h == s0) continue;
    CK(cudaEventRecord(B->ev_in, h->stream));
    CK(cudaStreamWaitEvent(s0->stream, B->ev_in, 0));
  }
  BatchPlan::G* ge = nullptr;
  for (auto& g : B->graphs)
    if (g.dt == dt && g.M == M && g.K == K) ge = &g;
  if (!ge) {
    BatchPlan::G g{};
    RUN(capture_batch_step(*B, dt, M, K, &g));
    B->graphs.push_back(g);
    ge = &B->graphs.back();
  }
  CK(cudaGraphLaunch(ge->exec, s0->stream));
  // the members' later work follows the batch
  CK(cudaEventRecord(B->ev_out, s0->stream));
  for (bd_state* m : B->m)
    if (m != s0) CK(cudaStreamWaitEvent(m->stream, B->ev_out, 0));
  s0->launches += ge->launches;
  const int64_t evals = int64_t(K) * (3 * (M - 1) + (s0->opts.sdc_correction ? M : 0)) + 1;
  for (bd_state* m : B->m) {
    m->steps += 1;
    m->sweeps += K;
    m->ionic_evals += evals;
  }
  return BD_OK;
}

int bd_sync(bd_state_t* s) {
  if (!s) return fail(s, BD_ERR_ARG, "NULL handle");
  return read_status(s);
}

int bd_query(bd_state_t* s) {
  if (!s) return fail(s, BD_ERR_ARG, "NULL handle");
  const cudaError_t e = cudaStreamQuery(s->stream);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  return fail(s, BD_ERR_CUDA, "cudaStreamQuery: %s", cudaGetErrorString(e));
}

void bd_clear_status(bd_state_t* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  cudaMemsetAsync(s->d_status, 0, 4, s->stream);
  cudaMemsetAsync(s->bar, 0, 8, s->stream);
  cudaStreamSynchronize(s->stream);
  s->err.clear();
}

int bd_activation_times(const bd_state_t* cs, double* out, int64_t n) {
  bd_state* s = const_cast<bd_state*>(cs);
  if (!s || !out || n != s->NT) return fail(s, BD_ERR_ARG, "bad arguments");
  CK(cudaStreamSynchronize(s->stream));
  CK(cudaMemcpy(out, s->t_act, n * 8, cudaMemcpyDeviceToHost));
  return read_status(s);
}

int bd_get_fields(const bd_state_t* cs, double* vm, double* phie, double* X) {
  bd_state* s = const_cast<bd_state*>(cs);
  if (!s) return fail(s, BD_ERR_ARG, "NULL handle");
  // copies ordered on the handle's stream after the queued steps; one
  // synchronisation (in read_status) for all of them
  if (vm) CK(cudaMemcpyAsync(vm, s->Xn, s->NT * 8, cudaMemcpyDeviceToHost, s->stream));
  if (phie) CK(cudaMemcpyAsync(phie, s->u[0], s->N * 8, cudaMemcpyDeviceToHost, s->stream));
  if (X) CK(cudaMemcpyAsync(X, s->Xn, int64_t(s->ns) * s->NT * 8, cudaMemcpyDeviceToHost, s->stream));
  return read_status(s);
}

int bd_device_fields(const bd_state_t* s, const double** X_dev, const double** u_dev) {
  if (!s) return fail(nullptr, BD_ERR_ARG, "NULL handle");
  if (X_dev) *X_dev = s->Xn;
  if (u_dev) *u_dev = s->u[0];
  return BD_OK;
}

// state blob: 64-byte header (magic, model, N, step counter, t^n, next adaptive
// step, t^{n-1}, previous-step-data flag), then X (ns*NT), u (N), activation
// times (NT), the previous step's sweep-1 elliptic solution (N) and the last
// parabolic increments (6 x NT; warm starts)
static size_t state_bytes(const bd_state* s) {
  return 64 + (size_t(s->ns + 1 + 3 * (kMaxNodes - 1)) * size_t(s->NT) + 2 * size_t(s->N)) * 8;
}

int bd_get_state(const bd_state_t* cs, void* buf, size_t* bytes) {
  bd_state* s = const_cast<bd_state*>(cs);
  if (!s || !bytes) return fail(s, BD_ERR_ARG, "NULL argument");
  const size_t need = state_bytes(s);
  if (!buf) {
    *bytes = need;
    return BD_OK;
  }
  if (*bytes < need) return fail(s, BD_ERR_ARG, "buffer too small (%zu < %zu)", *bytes, need);
  // copies ordered on the handle's stream after the queued steps, one
  // synchronisation before the header is filled in
  const cudaStream_t st = s->stream;
  char* const p0 = static_cast<char*>(buf);
  char* p = p0 + 64;
  int64_t hdr[8] = {0x62647376, s->model, s->N, 0, 0, 0, 0, 0};
  double clk[3];
  CK(cudaMemcpyAsync(&hdr[3], s->step_n, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(clk, s->t_now, 24, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(p, s->Xn, int64_t(s->ns) * s->NT * 8, cudaMemcpyDeviceToHost, st));
  p += int64_t(s->ns) * s->NT * 8;
  CK(cudaMemcpyAsync(p, s->u[0], s->N * 8, cudaMemcpyDeviceToHost, st));
  p += s->N * 8;
  CK(cudaMemcpyAsync(p, s->t_act, s->NT * 8, cudaMemcpyDeviceToHost, st));
  p += s->NT * 8;
  CK(cudaMemcpyAsync(p, s->uprev, s->N * 8, cudaMemcpyDeviceToHost, st));
  p += s->N * 8;
  for (int m = 0; m < kMaxNodes - 1; ++m)
    for (int g = 0; g < 3; ++g) {
      CK(cudaMemcpyAsync(p, s->kinc[m][g], s->NT * 8, cudaMemcpyDeviceToHost, st));
      p += s->NT * 8;
    }
  CK(cudaStreamSynchronize(st));
  std::memcpy(&hdr[4], &clk[0], 8);
  std::memcpy(&hdr[5], &s->dt_adapt, 8);
  std::memcpy(&hdr[6], &clk[1], 8);
  std::memcpy(&hdr[7], &clk[2], 8);
  std::memcpy(p0, hdr, 64);
  *bytes = need;
  return BD_OK;
}

int bd_set_state(bd_state_t* s, const void* buf, size_t bytes) {
  if (!s || !buf) return fail(s, BD_ERR_ARG, "NULL argument");
  const size_t need = state_bytes(s);
  if (bytes != need) return fail(s, BD_ERR_ARG, "state blob has %zu bytes, expected %zu", bytes, need);
  const char* p = static_cast<const char*>(buf);
  int64_t hdr[8];
  std::memcpy(hdr, p, 64);
  if (hdr[0] != 0x62647376 || hdr[1] != s->model || hdr[2] != s->N)
    return fail(s, BD_ERR_ARG, "state blob belongs to another model or mesh");
  p += 64;
  // every copy is ordered on the handle's stream after the work already
  // queued; one synchronisation at the end (the caller's buffer and the
  // header copies on this stack frame are read by then)
  const cudaStream_t st = s->stream;
  CK(cudaMemcpyAsync(s->Xn, p, int64_t(s->ns) * s->NT * 8, cudaMemcpyHostToDevice, st));
  p += int64_t(s->ns) * s->NT * 8;
  CK(cudaMemcpyAsync(s->u[0], p, s->N * 8, cudaMemcpyHostToDevice, st));
  for (int m = 1; m < kMaxNodes; ++m) CK(cudaMemcpyAsync(s->u[m], s->u[0], s->N * 8, cudaMemcpyDeviceToDevice, st));
  p += s->N * 8;
  CK(cudaMemcpyAsync(s->t_act, p, s->NT * 8, cudaMemcpyHostToDevice, st));
  p += s->NT * 8;
  CK(cudaMemcpyAsync(s->uprev, p, s->N * 8, cudaMemcpyHostToDevice, st));
  p += s->N * 8;
  for (int m = 0; m < kMaxNodes - 1; ++m)
    for (int g = 0; g < 3; ++g) {
      CK(cudaMemcpyAsync(s->kinc[m][g], p, s->NT * 8, cudaMemcpyHostToDevice, st));
      p += s->NT * 8;
    }
  double clk[3];
  std::memcpy(&clk[0], &hdr[4], 8);
  std::memcpy(&clk[1], &hdr[6], 8);
  std::memcpy(&clk[2], &hdr[7], 8);
  CK(cudaMemcpyAsync(s->step_n, &hdr[3], 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(s->t_now, clk, 24, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  std::memcpy(&s->dt_adapt, &hdr[5], 8);
  return BD_OK;
}

int bd_get_time(const bd_state_t* cs, double* t, int64_t* steps) {
  bd_state* s = const_cast<bd_state*>(cs);
  if (!s) return fail(s, BD_ERR_ARG, "NULL handle");
  CK(cudaStreamSynchronize(s->stream));
  if (t) CK(cudaMemcpy(t, s->t_now, 8, cudaMemcpyDeviceToHost));
  if (steps) CK(cudaMemcpy(steps, s->step_n, 8, cudaMemcpyDeviceToHost));
  return BD_OK;
}

int bd_step_adaptive(bd_state_t* s, double dt_max, double tol, int M, int K, double* dt_taken, double* err_out,
                     int* rejected) {
  if (!s) return fail(s, BD_ERR_ARG, "NULL handle");
  if (!(dt_max > 0) || !std::isfinite(dt_max) || !(tol > 0)) return fail(s, BD_ERR_ARG, "dt_max and tol must be positive");
  if (M != 2 && M != 3) return fail(s, BD_ERR_ARG, "n_sdc_nodes must be 2 or 3");
  if (K < 1) return fail(s, BD_ERR_ARG, "n_sweeps must be >= 1");
  const int64_t N = s->NT, Nu = s->N, ns = s->ns;
  if (!s->Xbak) {
    if (!alloc_n(s, &s->Xbak, ns * N) || !alloc_n(s, &s->ubak, Nu) || !alloc_n(s, &s->tbak, N + 4) ||
        !alloc_n(s, &s->upbak, Nu))
      return fail(s, BD_ERR_OOM, "device allocation failed");
  }
  const double dt_min = dt_max * std::ldexp(1.0, -(kAdaptLadder - 1));
  double dt = s->dt_adapt > 0 ? std::min(s->dt_adapt, dt_max) : dt_max;
  dt = ladder_step(dt_max, dt);
  int rej = 0;
  double err = 0.0;
  for (;;) {
    // keep X^n, u^n, activation times and the clock for a possible rejection
    CK(cudaMemcpyAsync(s->Xbak, s->Xn, ns * N * 8, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->ubak, s->u[0], Nu * 8, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->tbak, s->t_act, N * 8, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->tbak + N, s->t_now, 24, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->tbak + N + 3, s->step_n, 8, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->upbak, s->uprev, Nu * 8, cudaMemcpyDeviceToDevice, s->stream));
    s->adapt_on = true;
    s->adapt_tol = tol;
    const int r = do_step(s, dt, M, K);
    s->adapt_on = false;
    if (r != BD_OK) return r;
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, s->d_err, 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    std::memcpy(&err, &bits, 8);
    const int st = read_status(s);
    if (st != BD_OK) return st;
    if (err <= 1.0 || dt <= dt_min * (1.0 + 1e-12)) break;
    // reject: restore X^n and retry with a smaller step
    ++rej;
    CK(cudaMemcpyAsync(s->Xn, s->Xbak, ns * N * 8, cudaMemcpyDeviceToDevice, s->stream));
    for (int m = 0; m < kMaxNodes; ++m)
      CK(cudaMemcpyAsync(s->u[m], s->ubak, Nu * 8, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->t_act, s->tbak, N * 8, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->t_now, s->tbak + N, 24, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->step_n, s->tbak + N + 3, 8, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->uprev, s->upbak, Nu * 8, cudaMemcpyDeviceToDevice, s->stream));
    s->steps -= 1;
    s->sweeps -= K;
    dt = std::min(ladder_step(dt_max, dt * controller_factor(err)), 0.5 * dt);
  }
  if (dt_taken) *dt_taken = dt;
  if (err_out) *err_out = err;
  if (rejected) *rejected = rej;
  s->dt_adapt = ladder_step(dt_max, std::min(dt_max, dt * controller_factor(err)));
  return BD_OK;
}

size_t bd_footprint_bytes(const bd_mesh_t* mesh, bd_ionic_t model, const bd_opts_t* opts) {
  if (!mesh) return 0;
  const int ns = model_ns(int(model));
  if (ns == 0) return 0;
  const double N = double(mesh->n_nodes);
  double NT = N;
  if (mesh->elem_bath && mesh->elems) {
    const int k = mesh->dim + 1;
    std::vector<uint8_t> tis(mesh->n_nodes, 0);
    for (int64_t e = 0; e < mesh->n_elems; ++e)
      if (!mesh->elem_bath[e])
        for (int a = 0; a < k; ++a) {
          const int32_t q = mesh->elems[e * k + a];
          if (q >= 0 && q < mesh->n_nodes) tis[q] = 1;
        }
    NT = 0.0;
    for (uint8_t t : tis) NT += t;
  }
  bd_opts_t o;
  if (opts) o = *opts;
  else bd_default_options(&o);
  const bool mixed = o.precision == BD_MIXED;
  const double nnz = N * (mesh->dim == 2 ? 7.0 : 15.0);   // P1 node graph, upper estimate for structured meshes
  // pattern + A_i, A_ie, M_c, M_v and up to four cached parabolic shifts (FP64)
  const double mat = nnz * (4 + 8 * 4 + 8 * 4) + N * (4 * 3 + 8);
  const double st = NT * 8 * (ns * (1 + 3 * kMaxNodes) + 4 * (ns - 1) + 4) + N * 8 * (3 * kMaxNodes + 12);
  const double packs = NT * 8.0 * (cond_pack_values(model) + 2 * jac_pack_values(model));
  double extra = 0.0;
  // FP32 copies of A_ie and of the parabolic shifts, FP32 workspaces
  if (mixed) extra += nnz * 4 * 5 + N * 4 * 16;
  // AMG hierarchy below level 0: measured about 2.1 x (3-D) and 1.2 x (2-D)
  // the entries of A_0 over all A, R, P; SELL padding, FP64 values and
  // indices, an FP32 copy on the mixed path, the dense coarse inverse
  const bool amg = o.elliptic_precond == 1 && N > 1500;
  const double lev = amg ? nnz * (mesh->dim == 2 ? 1.2 : 2.1) * 1.3 : 0.0;
  const double nc = std::min(1500.0, N / 50.0 + 1.0);    // dense coarsest level (measured 1247 at 66k nodes)
  if (amg) extra += lev * (12 + (mixed ? 8 : 0)) + nc * nc * 12 + N * 8 * 10;
  // streaming form: its workspaces and, mixed, the SELL-32/4 copies of the
  // FP32 operators (8 bytes an entry, widths padded to 4)
  const bool streaming =
      o.cg_cluster == 0 && (o.streaming >= 1 || (o.streaming == 0 && nnz >= double(kStreamNnz)));
  if (streaming) {
    extra += N * 8 * 8;
    // FP64 two-system solves: second halves of seven workspaces and a second
    // set of AMG level vectors
    if (!mixed && amg && o.pair_solve >= 0) extra += N * 8 * 7 + N * 8 * 2.6;
    if (mixed && o.vec4 >= 0) extra += (nnz * 5 + lev) * 8 * 1.15;
  }
  return size_t(mat + st + packs + extra) + (size_t(1) << 20);
}

int bd_struct_sizes(size_t* mesh, size_t* cond, size_t* opts, size_t* stats) {
  if (mesh) *mesh = sizeof(bd_mesh_t);
  if (cond) *cond = sizeof(bd_cond_t);
  if (opts) *opts = sizeof(bd_opts_t);
  if (stats) *stats = sizeof(bd_stats_t);
  return BD_OK;
}

int bd_amg_level(const bd_state_t* s, int level, int64_t* out) {
  if (!s || !out) return fail(nullptr, BD_ERR_ARG, "NULL argument");
  if (level < 0 || size_t(level) * 9 >= s->amg_shape.size())
    return fail(const_cast<bd_state_t*>(s), BD_ERR_ARG, "no AMG level %d", level);
  std::copy(s->amg_shape.begin() + size_t(level) * 9, s->amg_shape.begin() + size_t(level) * 9 + 9, out);
  return BD_OK;
}

int bd_get_stats(const bd_state_t* cs, bd_stats_t* out) {
  bd_state* s = const_cast<bd_state*>(cs);
  if (!s || !out) return fail(s, BD_ERR_ARG, "NULL argument");
  long long st[9];
  unsigned long long cl = 0;
  CK(cudaStreamSynchronize(s->stream));
  CK(cudaMemcpy(st, s->d_stats, 72, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&cl, s->d_clamps, 8, cudaMemcpyDeviceToHost));
  out->steps = s->steps;
  out->sweeps = s->opts.sweep_tol > 0 ? s->steps + st[6] : s->sweeps;
  out->cg_iters_e = st[0];
  out->cg_solves_e = st[1];
  out->cg_iters_p = st[2];
  out->cg_solves_p = st[3];
  out->spd_clamps = int64_t(cl);
  out->ionic_evals = s->ionic_evals;
  out->kernel_launches = s->launches + st[8];   // host-enqueued + counted on the device (streaming solves)
  out->solver_block_bound = s->cluster > 0 ? kSolverTierBlock[0] : kSolverTierBlock[s->tier];
  out->solver_tier = s->cluster > 0 ? 0 : s->tier;
  out->amg_levels = s->use_amg ? s->amg.nlev : 0;
  out->amg_coarse_rows = s->use_amg ? s->amg.nc : 0;
  out->streaming = s->streaming ? 1 : 0;
  return BD_OK;
}

int bd_solve_elliptic_noalloc(bd_state_t* s, const double* v_dev, const double* u_guess_dev, double* u_dev,
                              int* iters) {
  static std::mutex mu;
  static double* addr[64] = {};
  if (!s || !v_dev || !u_dev) return fail(s, BD_ERR_ARG, "NULL argument");
  if (s->N > kNoAllocRows)
    return fail(s, BD_ERR_ARG, "bd_solve_elliptic_noalloc supports at most %lld nodes (mesh has %lld)",
                (long long)kNoAllocRows, (long long)s->N);
  if (s->pcg_grid > kNoAllocBlocks) return fail(s, BD_ERR_ARG, "CG grid larger than the fixed scratch allows");
  const int dev = s->device;
  if (dev < 0 || dev >= 64) return fail(s, BD_ERR_ARG, "device ordinal out of range");
  // the scratch array and the launch belong to the handle's device: make it
  // current for the call and restore the caller's device afterwards
  int prev = 0;
  CK(cudaGetDevice(&prev));
  if (prev != dev) CK(cudaSetDevice(dev));
  struct Restore {
    int d;
    bool on;
    ~Restore() {
      if (on) cudaSetDevice(d);
    }
  } restore{prev, prev != dev};
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
      void* p = nullptr;
      CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      addr[dev] = static_cast<double*>(p);
    }
    base = addr[dev];
  }
  double* part = base + 5 * kNoAllocRows;
  double* ctl = part + 4 * kNoAllocBlocks;
  unsigned* bar = reinterpret_cast<unsigned*>(ctl);
  int* status = reinterpret_cast<int*>(ctl + 1);
  long long* it = reinterpret_cast<long long*>(ctl + 2);
  CK(cudaMemsetAsync(ctl, 0, 4 * sizeof(double), s->stream));
  if (u_guess_dev && u_guess_dev != u_dev)
    CK(cudaMemcpyAsync(u_dev, u_guess_dev, s->N * 8, cudaMemcpyDeviceToDevice, s->stream));
  PcgLaunch P = pcg_base(s);
  // not part of an SDC step: the sweep test's gate (which a step may have
  // closed) must not turn this solve into a no-op
  P.gate = nullptr;
  P.r = base;
  P.z = base + kNoAllocRows;
  P.p = base + 2 * kNoAllocRows;
  P.q = base + 3 * kNoAllocRows;
  P.invd = base + 4 * kNoAllocRows;
  P.part = part;
  P.bar = bar;
  P.status = status;
  P.iters_acc = it;
  P.solves_acc = nullptr;
  P.valA = s->Aie;
  P.val1 = s->Ai;
  P.va = v_dev;
  P.c1 = -1.0;
  P.project = 1;
  P.x = u_dev;
  P.warm = u_guess_dev ? 1 : 0;
  P.tol = s->opts.cg_tol_e;
  P.maxit = s->opts.cg_cap_e;
  P.pin = s->opts.pin_node >= 0 ? s->opts.pin_node : -1;
  CK(launch_pcg(P, s->wmax, s->stream));
  long long h_ctl[2] = {0, 0};
  CK(cudaMemcpyAsync(h_ctl, ctl + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  const int st = int(h_ctl[0] & 0xffffffffll);
  if (iters) *iters = int(h_ctl[1]);
  const int c = status_code(st);
  if (c != BD_OK) return fail(s, c, "elliptic CG failed (device status %d)", st);
  return BD_OK;
}

int bd_profile_steps(bd_state_t* s, double dt, int M, int K, int n_steps, bd_profile_t* out) {
  if (!s || !out || n_steps < 0) return fail(s, BD_ERR_ARG, "bad arguments");
  if (!(dt > 0) || (M != 2 && M != 3) || K < 1) return fail(s, BD_ERR_ARG, "bad step shape");
  std::memset(out, 0, sizeof(*out));
  out->nnz = s->nnz;
  long long st0[11], st1[11];
  CK(cudaStreamSynchronize(s->stream));
  CK(cudaMemcpy(st0, s->d_stats, sizeof(st0), cudaMemcpyDeviceToHost));
  s->prof = true;
  int rc = BD_OK;
  for (int n = 0; n < n_steps && rc == BD_OK; ++n) {
    s->evused = 0;
    rc = do_step(s, dt, M, K);
    if (rc != BD_OK) break;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
      rc = fail(s, BD_ERR_CUDA, "profiled step failed");
      break;
    }
    for (size_t e = 0; e < s->evused; ++e) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, s->evpool[e].a, s->evpool[e].b);
      out->ms[s->evpool[e].kind] += ms;
      out->launches[s->evpool[e].kind] += 1;
    }
    out->launches[BD_K_FINISH] += 1;   // the step-counter launch shares the finish bracket
  }
  s->prof = false;
  if (rc != BD_OK) return rc;
  CK(cudaMemcpy(st1, s->d_stats, sizeof(st1), cudaMemcpyDeviceToHost));
  out->cg_iters[0] = st1[0] - st0[0];
  out->cg_solves[0] = st1[1] - st0[1];
  out->cg_iters[1] = st1[2] - st0[2];
  out->cg_solves[1] = st1[3] - st0[3];
  out->outer_iters[0] = st1[4] - st0[4];
  out->outer_iters[1] = st1[5] - st0[5];
  // algorithmic bytes (see bd_profile_t); vb = bytes per value of the Krylov iteration
  const bool mixed = s->precision == BD_MIXED;
  const double vb = mixed ? 4.0 : 8.0;
  const double pairs = double(st1[7] - st0[7]);     // two-RHS iterations in which both systems advanced
  const double pairs64 = double(st1[9] - st0[9]);   // FP64 operator passes shared by a streaming pair
  const double pairsc = double(st1[10] - st0[10]);  // first V-cycles shared by a streaming pair
  for (int k = 0; k < 2; ++k) {
    const bool ell = k == 0;
    // elliptic: all nodes and the whole pattern; parabolic: the tissue block
    const double n = double(ell ? s->N : s->NT), nnz = double(ell ? s->nnz : s->nnz_t);
    auto spmv = [&](double v) { return nnz * (v + 4) + n * (2 * v + 4); };
    const double iters = double(out->cg_iters[k]), solves = double(out->cg_solves[k]);
    const double extra = ell ? 0.0 : 8.0 * n;                        // condensed diagonal
    const double vec = (ell && s->use_amg ? 13.0 : 16.0) * vb * n;   // dots, axpys, (Jacobi)
    const double per_iter = spmv(vb) + vec + extra;
    // per solve: right-hand-side products (elliptic A_i v; parabolic A_i a, M b, rl),
    // the set-up passes (rhs, 1/D, x, r) and, elliptic, projection and pin shift
    const double per_solve = (ell ? 1.0 : 2.0) * spmv(8.0) + (ell ? 7.0 : 5.0) * 8.0 * n + extra;
    double b = solves * per_solve + iters * per_iter;
    if (mixed) {
      const double outer = double(out->outer_iters[k]);
      // FP64 residual product and streams (b, x in, r out), FP32 scaling (r in,
      // r32 and d32 out) and the update x += s d (x in and out, d in)
      b += outer * ((ell ? spmv(8.0) + 3.0 * 8.0 * n : 2.0 * 8.0 * n) + 16.0 * n + 20.0 * n);
    }
    if (ell && s->use_amg) b -= pairs * nnz * (vb + 4);            // shared operator pass
    if (ell) b -= pairs64 * nnz * (8.0 + 4.0);                     // shared FP64 products (A_i, A_ie)
    out->alg_bytes[k] = b;
  }
  if (s->use_amg) {
    const int v = mixed ? 1 : 0;
    // one cycle per iteration plus the first of each inner solve (mixed: every
    // refinement pass but the last, converged one of each solve)
    const double cycles = double(out->cg_iters[0]) +
                          double(mixed ? out->outer_iters[0] - out->cg_solves[0] : out->cg_solves[0]);
    out->vcycle_bytes = cycles * s->amg_cycle_bytes[v];
    out->coarse_bytes = cycles * s->amg_coarse_bytes[v];
    const double ncc = vb * double(s->amg.nc) * double(s->amg.nc);   // the dense coarse inverse
    out->vcycle_bytes -= (pairs + pairsc) * (s->amg_cycle_opbytes[v] - ncc);
    if (s->streaming) out->coarse_bytes -= (pairs + pairsc) * ncc;   // read once for both systems
  }
  return read_status(s);
}

int bd_reset_stats(bd_state_t* s) {
  if (!s) return fail(s, BD_ERR_ARG, "NULL handle");
  CK(cudaStreamSynchronize(s->stream));
  CK(cudaMemset(s->d_stats, 0, 128));
  CK(cudaMemset(s->d_clamps, 0, 8));
  s->steps = s->sweeps = s->ionic_evals = s->launches = 0;
  return BD_OK;
}

int64_t bd_num_nodes(const bd_state_t* s) { return s ? s->N : 0; }

int64_t bd_num_tissue_nodes(const bd_state_t* s) { return s ? s->NT : 0; }

const char* bd_last_error(const bd_state_t* s) {
  if (s) return s->err.c_str();
  return g_err.c_str();
}

void bd_destroy(bd_state_t* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_batches.size();) {
      auto& mm = g_batches[i]->m;
      if (std::find(mm.begin(), mm.end(), s) != mm.end()) {
        for (bd_state* o : mm)
          if (o->stream) cudaStreamSynchronize(o->stream);
        g_batches.erase(g_batches.begin() + i);
      } else {
        ++i;
      }
    }
  }
  release(s);
  delete s;
}

int bd_ionic_eval(bd_ionic_t model, int precision, int64_t n, const double* X, const double* istim, double cm,
                  double* f, double* jac) {
  bd_state* s = nullptr;
  const int ns = model_ns(int(model));
  if (ns == 0 || n < 0 || !X || !f || !(cm > 0)) return fail(nullptr, BD_ERR_ARG, "bad arguments");
  if (n == 0) return BD_OK;
  double *dX = nullptr, *dI = nullptr, *dF = nullptr, *dJ = nullptr;
  const size_t bx = size_t(ns) * n * 8;
  CK(cudaMalloc(&dX, bx));
  CK(cudaMalloc(&dF, bx));
  if (istim) CK(cudaMalloc(&dI, n * 8));
  if (jac) CK(cudaMalloc(&dJ, size_t(n) * ns * ns * 8));
  CK(cudaMemcpy(dX, X, bx, cudaMemcpyHostToDevice));
  if (istim) CK(cudaMemcpy(dI, istim, n * 8, cudaMemcpyHostToDevice));
  CK(launch_eval(int(model), precision, n, dX, dI, 1.0 / cm, dF, dJ, nullptr));
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(f, dF, bx, cudaMemcpyDeviceToHost));
  if (jac) CK(cudaMemcpy(jac, dJ, size_t(n) * ns * ns * 8, cudaMemcpyDeviceToHost));
  cudaFree(dX);
  cudaFree(dF);
  if (dI) cudaFree(dI);
  if (dJ) cudaFree(dJ);
  return BD_OK;
}

int bd_ionic_pattern(bd_ionic_t model, uint32_t* masks) {
  if (!masks || model_ns(int(model)) == 0) return fail(nullptr, BD_ERR_ARG, "bad arguments");
  pattern_host(int(model), masks);
  return BD_OK;
}

int bd_rest_state(bd_ionic_t model, double* X) {
  if (!X || model_ns(int(model)) == 0) return fail(nullptr, BD_ERR_ARG, "bad arguments");
  rest_state_host(int(model), X);
  return BD_OK;
}

int bd_operator_csr(const bd_state_t* cs, int which, int64_t* nnz, int32_t* rowptr, int32_t* col, double* val) {
  bd_state* s = const_cast<bd_state*>(cs);
  if (!s || !nnz || which < 0 || which > 3) return fail(s, BD_ERR_ARG, "bad arguments");
  *nnz = which == 3 ? s->N : s->nnz;
  if (!val) return BD_OK;   // size query
  const HostOps& H = s->host;
  if (which == 3) {
    std::memcpy(val, H.ML.data(), s->N * 8);
    return BD_OK;
  }
  if (!rowptr || !col) return fail(s, BD_ERR_ARG, "rowptr/col is NULL");
  const std::vector<double>& src = which == 0 ? H.Ai : which == 1 ? H.Aie : H.M;
  std::memcpy(rowptr, H.rowptr.data(), (s->N + 1) * 4);
  std::memcpy(col, H.col.data(), s->nnz * 4);
  std::memcpy(val, src.data(), s->nnz * 8);
  return BD_OK;
}

int bd_solve_elliptic(bd_state_t* s, const double* v, const double* u_guess, double* u, int* iters) {
  if (!s || !v || !u) return fail(s, BD_ERR_ARG, "NULL argument");
  const int64_t N = s->N;
  double *dv = s->avec, *du = s->bvec;
  CK(cudaStreamSynchronize(s->stream));
  CK(cudaMemcpyAsync(dv, v, s->NT * 8, cudaMemcpyHostToDevice, s->stream));
  if (u_guess) CK(cudaMemcpyAsync(du, u_guess, N * 8, cudaMemcpyHostToDevice, s->stream));
  else CK(cudaMemsetAsync(du, 0, N * 8, s->stream));
  long long before[2];
  CK(cudaMemcpyAsync(before, s->d_stats, 16, cudaMemcpyDeviceToHost, s->stream));
  if (s->gate) CK(launch_set_int(s->gate, 1, nullptr, s->stream));   // a step's sweep test may have closed it
  RUN(elliptic(s, dv, du));
  long long after[2];
  CK(cudaMemcpyAsync(after, s->d_stats, 16, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(u, du, N * 8, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemsetAsync(du, 0, N * 8, s->stream));
  CK(cudaMemsetAsync(dv, 0, N * 8, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (iters) *iters = int(after[0] - before[0]);
  return read_status(s);
}

}  // extern "C"
