// bd_internal.h -- shared declarations of the CUDA implementation.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/bd.h"

namespace bd {

constexpr int kMaxStim = 32;
constexpr int kMaxNodes = 3;          // Gauss-Lobatto nodes per step
constexpr int kMaxNS = 19;
// The persistent solver kernels are built for several __launch_bounds__
// ("tiers"): tier 0 allows 1024-thread blocks (64 registers a thread; two
// 512-thread blocks share an SM), tier 1 allows 512-thread blocks (128
// registers; one block an SM) and serves problems whose rows fit one block
// per SM; tier 2 is tier 0 except that the mixed AMG kernels are built for
// two 1024-thread blocks an SM (32 registers, full occupancy), for operators
// of at least kTier2Nnz entries, where the operator streams need the threads
// (measured on GB300: faster on 3-D meshes of 18M and 30M entries, slower or
// even on 2-D meshes of 4.5M and 7.3M and a 3-D mesh of 4M).
constexpr int kSolverTierBlock[3] = {1024, 512, 1024};
constexpr int64_t kTier2Nnz = 12000000;
// operators of at least kStreamNnz entries take the streaming solver form by
// default (measured on GB300, mixed, ms per step persistent / streaming:
// 513^2 sheet, 1.8M entries, 6.75 / 8.28; 3-D slab of 3.9M entries 11.7 /
// 12.0; 1025^2 sheet, 7.3M, 19.3 / 17.9; 3-D slab of 10.6M 27.3 / 22.5)
constexpr int64_t kStreamNnz = 5000000;

// device status word bits (one per bd_status_t failure kind)
enum : int {
  ST_NOT_CONVERGED = 1,
  ST_NONFINITE = 2,
  ST_INDEFINITE = 4,
  ST_TIMEOUT = 8,
};

struct StimTable {
  int n;
  double t_on[kMaxStim];
  double dur[kMaxStim];
  double amp[kMaxStim];
};

// one node-local right-hand side recipe per ionic kernel launch
// MODE_S2P: stage 2 from the condensation stage 1 stored in `pack`
enum IonicMode : int { MODE_S1 = 0, MODE_S2 = 1, MODE_CORR = 2, MODE_S2P = 3 };

struct IonicLaunch {
  int model;                 // bd_ionic_t
  int precision;             // bd_precision_t (compute type of the membrane model)
  int mode;
  int64_t n;
  double alpha;              // shift of (alpha Mt - W)
  double smin;               // safeguard floor of the condensed diagonal
  double ck1;                // stage 2: 2/(gamma h)
  double inv_gamma;          // stage 2: 1/gamma
  double inv_dt;             // correction: 1/dt_m
  double inv_cm;
  double dt;                 // step size (for the stimulus clock)
  double S[kMaxNodes];       // correction: quadrature row S_{m,j} (already times tau)
  int n_nodes;               // correction: number of quadrature nodes
  const double* XJ;          // state at which W is taken (ns x n)
  const double* u;           // S1/S2: u_{m+1}
  const double* k1v;         // S2
  const void* z1;            // S2: stage 1's z, w ((ns-1) x n, the model's type T)
  const void* w1;
  const double* Xprev;       // correction: X_m^new
  const double* Xq[kMaxNodes];   // correction: predictor nodes X~_j
  const double* uq[kMaxNodes];   // correction: u_j
  const void* fq[kMaxNodes];     // correction: stored node fields f(X~_j) (ns x n, the model's type T)
  const double* ML;
  const uint32_t* stim_bits;
  const double* t_now;       // simulated time t^n of the step
  StimTable stim;
  double* dgs;               // out: M_L * s
  double* rl;                // out: node-local part of the condensed rhs
  void* z;                   // out: (ns-1) x n values of the model's type T (exact: the
  void* w;                   //      condensation computes them in T)
  double* avec;              // out: vector multiplied by A_i in the rhs
  double* bvec;              // out: vector multiplied by M in the rhs
  void* fq_out;              // out (optional): node field at the F point (type T)
  unsigned long long* clamp_count;
  const int* gate;           // optional: kernel does nothing when *gate == 0 (sweep test)
  void* pack;                // S1: store the condensation here (optional); S2P: read it
  void* jac_out;             // S1 (optional): store the node field and Jacobian here
  const void* jac_in;        // S1, correction (optional): field and Jacobian at XJ stored by an S1 launch
};
// values per node of the stage-1 condensation pack (model, compute type)
int cond_pack_values(int model);
// values per node of a stored node Jacobian (model)
int jac_pack_values(int model);

// launchers (ionic.cu)
cudaError_t launch_ionic(const IonicLaunch& L, cudaStream_t st);
cudaError_t launch_field(int model, int precision, int64_t n, const double* X, double inv_cm, double dt,
                         const uint32_t* stim_bits, const double* t_now, const StimTable& stim,
                         void* fout, cudaStream_t st, const int* gate = nullptr);   // fout: ns x n of the model's type
// z/w arrays hold float when zw32 != 0 (the mixed path), double otherwise
cudaError_t launch_combine(int model, int zw32, int64_t n, const double* src, const double* k1v, const void* z1,
                           const void* w1, const double* k2v, const void* z2, const void* w2, double m1,
                           double m2, double* dst, cudaStream_t st, const int* gate = nullptr, double mhat1 = 0.0,
                           double etol = 1.0, unsigned long long* err = nullptr);
// CN-RK2 reaction half step: Xout = X' + h f(X' + (h/2) f(X')), X' = X with
// v += dv (dv may be NULL); avec = v_out + u when avec != NULL
cudaError_t launch_rk2(int model, int precision, int64_t n, const double* X, const double* dv, double* Xout,
                       double h, double inv_cm, double dt, const uint32_t* stim_bits, const double* t_now,
                       const StimTable& stim, const double* u, double* avec, cudaStream_t st);
cudaError_t launch_update(int model, int zw32, int64_t n, const double* Xt, const double* ev, const void* z,
                          const void* w, double* dst, cudaStream_t st, const int* gate = nullptr);
// sweep test of Algorithm 2: dmax = max |a - b| (dmax reset by the caller),
// then gate = (dmax >= tol) and, while open, sweeps += 1
cudaError_t launch_sweep_delta(int64_t n, const double* a, const double* b, unsigned long long* dmax,
                               const int* gate, cudaStream_t st);
cudaError_t launch_sweep_gate(const unsigned long long* dmax, double tol, int* gate, long long* sweeps,
                              cudaStream_t st);
cudaError_t launch_set_int(int* p, int v, unsigned long long* clear, cudaStream_t st);
// sweep-2 elliptic initial guesses extrapolated in time (u1 may be NULL); clk =
// (t^n, t^{n-1}, valid) is the handle's clock, marked valid afterwards
cudaError_t launch_extrap(int64_t n, double* u1, double* u2, double* ep, double c1, double dt, double* clk,
                          const int* gate, cudaStream_t st);
// *p = 0 unless *gate == 0 (gate may be NULL)
cudaError_t launch_clear_gated(unsigned long long* p, const int* gate, cudaStream_t st);
// X^n <- X_last and activation times on the n tissue nodes, u^n <- u_last on
// all nu nodes, then t^n += dt, n += 1
cudaError_t launch_finish(int ns, int64_t n, int64_t nu, double* Xn, const double* Xlast, double* u0,
                          const double* ulast, double* t_act, double v_act, double dt, long long* step_n,
                          double* t_now, int* status, cudaStream_t st);
int model_ns(int model);
void rest_state_host(int model, double* x);

// ---- batched node-wise launches (ionic.cu; see segment.cuh) ------------------
// One launch over the nodes of many handles: tab holds one argument block per
// handle (device memory), blk the block prefix (nseg + 1 ints, device), the
// launch has blk[nseg] blocks.  The model, precision and mode are the batch's.
struct FieldArgs {
  int64_t n;
  const double* X;
  double inv_cm, dt;
  const uint32_t* stim_bits;
  const double* t_now;
  StimTable stim;
  void* fout;                     // ns x n values of the model's type
};
struct CombineArgs {
  int64_t n;
  const double *src, *k1v;
  const void *z1, *w1;            // float or double (launch_combine_batch's zw32)
  const double* k2v;
  const void *z2, *w2;
  double m1, m2;
  double* dst;
};
struct UpdateArgs {
  int64_t n;
  const double *Xt, *ev;
  const void *z, *w;              // float or double (launch_update_batch's zw32)
  double* dst;
};
struct CopyArgs {
  int64_t n;
  const double* src;
  double* dst;
};
struct ExtrapArgs {
  int64_t n;
  double *u1, *u2, *ep;
  double c1, dt;
  double* clk;
};
struct FinishArgs {
  int ns;
  int64_t n, nu;
  double* Xn;
  const double* Xlast;
  double* u0;
  const double* ulast;
  double* t_act;
  double v_act, dt;
  double* t_now;
  long long* step_n;
  int* status;
};
constexpr int kNodeBlock = 128;   // block of the node-wise kernels (ionic, field, combine, update)
constexpr int kVecBlock = 256;    // block of the copy, extrapolation and finish kernels
cudaError_t launch_ionic_batch(const IonicLaunch& proto, const IonicLaunch* tab, const int* blk, int nseg,
                               int nblocks, cudaStream_t st);
cudaError_t launch_field_batch(int model, int precision, const FieldArgs* tab, const int* blk, int nseg, int nblocks,
                               cudaStream_t st);
cudaError_t launch_combine_batch(int model, int zw32, const CombineArgs* tab, const int* blk, int nseg,
                                 int nblocks, cudaStream_t st);
cudaError_t launch_update_batch(int model, int zw32, const UpdateArgs* tab, const int* blk, int nseg, int nblocks,
                                cudaStream_t st);
cudaError_t launch_copy_batch(const CopyArgs* tab, const int* blk, int nseg, int nblocks, cudaStream_t st);
cudaError_t launch_extrap_batch(const ExtrapArgs* tab, const int* blk, int nseg, int nblocks, cudaStream_t st);
cudaError_t launch_finish_batch(const FinishArgs* tab, const int* blk, int nseg, int nblocks, cudaStream_t st);

// sparse (pcg.cu)
//
// Operators are stored in sliced ELL ("SELL-32"): rows are grouped in slices
// of 32 consecutive rows; slice s has width w_s = its longest row, and entry k
// of row i = 32 s + l sits at sptr[s] + 32 k + l (column-major inside the
// slice), so one warp reads 32 consecutive values per load.  Padding entries
// carry value 0 and point at their own row.  All operators share one layout.
struct PcgLaunch {
  int n;
  const int64_t* sptr;      // slice offsets (n_slices)
  const int* swidth;        // slice widths (n_slices)
  const int* col;           // SELL column indices
  const int* diagpos;       // SELL position of each row's diagonal
  const double* valA;
  const double* dextra;     // optional extra diagonal
  const double* rl;         // rhs = rl + c1 V1 a + c2 V2 b
  const double* val1;
  const double* va;
  double c1;
  const double* val2;
  const double* vb;
  double c2;
  int project;              // subtract the mean of the rhs (singular Neumann system)
  double* x;
  int warm;
  double tol;
  int maxit;
  int pin;                  // >= 0 pin node, -1 zero mean, -2 none
  // workspaces
  double* r;
  double* z;
  double* p;
  double* q;
  double* invd;
  double* part;
  unsigned* bar;
  int* status;
  long long* iters_acc;
  long long* solves_acc;
  long long* outer_acc;     // FP64 residual passes (mixed kernel)
  long long* pair_acc;      // two-RHS kernel: inner iterations in which both systems advanced
  const int* gate;          // optional: the solve is skipped when *gate == 0
  int grid;                 // co-resident blocks
  int block;
  int cluster;              // > 0: one thread-block cluster of this many blocks (grid = cluster),
                            // hardware cluster barriers; 0: cooperative grid, device-wide barriers
  int tier;                 // register tier of the solver build launched (kSolverTierBlock)
};
// launch configuration of a persistent solver kernel: cooperative grid, or a
// single cluster (then the kernel gets bar = nullptr)
void solver_launch_config(const PcgLaunch& P, cudaStream_t st, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr,
                          PcgLaunch* Pk);
// largest usable single-cluster size (16, 8 or 0) for the solver kernels at
// this block size; enables non-portable cluster sizes where needed
int solver_cluster_size(int block, int want);
bool pcg_cluster_ok(int block, int size);     // pcg.cu
bool amg_cluster_ok(int block, int size);     // amg.cu
bool mixed_cluster_ok(int block, int size);   // mixed.cu
cudaError_t launch_pcg(const PcgLaunch& P, int wmax, cudaStream_t st);
// a device-barrier wait that must run out (bd_selftest_wait_timeout)
cudaError_t launch_wait_selftest(unsigned* bar, int* status, cudaStream_t st);
int pcg_max_blocks(int block, int wmax, int tier);
cudaError_t launch_axpby_vals(int64_t nnz, double a, const double* X, double b, const double* Y, double* out,
                              cudaStream_t st);
cudaError_t launch_copy(int64_t n, const double* src, double* dst, cudaStream_t st, const int* gate = nullptr);

// ---- algebraic multigrid (amg.cpp host setup, amg.cu device V-cycle) -------
struct HCsr {                      // host CSR, n x m
  int64_t n = 0, m = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> v;
};
struct AmgParams {
  double theta = 0.08;             // strength-of-connection threshold
  int64_t coarse_max = 1500;       // rows of the dense coarsest solve
  int max_levels = 9;
};
struct AmgHostLevel {
  HCsr A, P, R;                    // A: n x n, P: n x n_next, R = P^T
  std::vector<double> invdiag;
  double omega = 0.0;              // damped-Jacobi weight 4 / (3 rho(D^-1 A))
};
struct AmgHost {
  std::vector<AmgHostLevel> lev;   // smoothed levels (fine to coarse)
  int64_t nc = 0;                  // rows of the coarsest operator
  std::vector<double> cinv;        // dense inverse of A_c + c 1 1^T (nc x nc, row-major)
};
int amg_build(const HCsr& A, const AmgParams& prm, AmgHost* out, std::string* err);

struct SellHost {
  int64_t n = 0;
  std::vector<int64_t> sptr;
  std::vector<int> sw;
  std::vector<int> col;
  std::vector<double> val;
  int wmax = 0;                    // 8, 16 or 32 (SELL, thread per row); 0 with rp empty: wide SELL
  std::vector<int64_t> rp;         // non-empty: CSR layout, one warp per row (rows longer than 32)
};
// SELL-32 for rows of at most 32 entries, else CSR.  For operators only the
// streaming kernels read, wide > 0 also allows SELL-32 for longer rows when
// padding stores at most 1.5x the entries (SellHost.wmax = 0 then): wide = 1
// only for operators of at least 2^17 rows averaging at most 96 entries,
// wide = 2 whenever the padding allows
SellHost sell_from_csr(const HCsr& A, int wide = 0);

constexpr int kMaxAmgLevels = 10;
template <class T>
struct SellDevT {
  int n;
  int wmax;
  const int64_t* sptr;
  const int* sw;
  const int* col;
  const T* val;
  const int64_t* rp;               // non-null: CSR (col/val row-major), one warp per row
  int lpr;                         // CSR in the streaming kernels: lanes per row (power of 2; 0: 32)
  // optional SELL-32/4 copy (FP32 operators of streaming handles, see
  // launch_sell_v4 for the layout; the slice widths are sw): NULL = none
  const int64_t* sptr4;
  const int* col4;
  const T* val4;
};

// lanes per CSR row in the streaming level kernels: the smallest power of two
// at least a quarter of the mean row length, within [4, 32] (a lane keeps
// four entries in flight, so most rows take one pass); rows of 256 entries
// and more on average (restrictions onto the coarsest level: few rows, long)
// get a whole block of kCsrBlockLanes threads each
constexpr int kCsrBlockLanes = 256;
inline int csr_lanes(int64_t nnz, int64_t n) {
  if (n > 0 && nnz >= 256 * n) return kCsrBlockLanes;
  const int64_t q = n > 0 ? (nnz + 4 * n - 1) / (4 * n) : 1;
  int l = 4;
  while (l < 32 && l < q) l *= 2;
  return l;
}

// threads a streaming level kernel runs over M: one per row (SELL), lpr per row (CSR)
template <class T>
inline int64_t level_threads(const SellDevT<T>& M) {
  return M.rp ? int64_t(M.n) * (M.lpr > 0 ? M.lpr : 32) : int64_t(M.n);
}
template <class T>
struct AmgLevelDevT {
  SellDevT<T> A, P, R;
  const T* invd;
  T omega;
  T* x;                            // pre-smoothed / prolongation-corrected iterate
  T* b;                            // right-hand side (level >= 1)
  T* r;                            // residual
  T* y;                            // post-smoothed result (level >= 1)
};
template <class T>
struct AmgDevT {
  int nlev;                        // smoothed levels
  AmgLevelDevT<T> L[kMaxAmgLevels];
  int nc;
  int ldc;                         // row stride of cinv: nc rounded up to 4 (zero padded)
  const T* cinv;
  T* bc;
  T* xc;
};
using SellDev = SellDevT<double>;
using AmgLevelDev = AmgLevelDevT<double>;
using AmgDev = AmgDevT<double>;
using AmgDevF = AmgDevT<float>;
// M: device copy of the hierarchy descriptor (read through L1 by the level loops)
cudaError_t launch_pcg_amg(const PcgLaunch& P, const AmgDev* M, int wmax, cudaStream_t st);
int pcg_amg_max_blocks(int block, int tier);

// mixed precision (mixed.cu): FP64 right-hand side and outer residual, FP32
// inner CG (Jacobi or the FP32 copy of the AMG hierarchy), x += d in FP64
struct MixedLaunch {
  const float* valA32;      // FP32 copy of the operator values (SELL)
  float* r32;
  float* z32;
  float* p32;
  float* q32;
  float* invd32;
  float* d32;               // inner solution
  double* b64;              // right-hand side
  double* r64;              // outer residual
  float tol_inner;          // relative residual reduction of each inner solve
  int max_outer;            // 1: single FP32 solve (x = d); > 1: iterative refinement
  int inner_cap;
  int use_amg;
  int pipelined;            // Jacobi inner CG in its pipelined form (one barrier an iteration)
};
cudaError_t launch_pcg_mixed(const PcgLaunch& P, const MixedLaunch& X, const AmgDevF* M, int wmax, cudaStream_t st,
                             float* partf);
int pcg_mixed_max_blocks(int block, int tier);
int pcg_mixed_amg_max_blocks(int block, int tier);   // the mixed AMG kernels of a tier
// two elliptic solves (right-hand sides c1 A_i va and c1 A_i va1) in one launch;
// the MixedLaunch workspaces hold 2 n entries, H1 the second system's AMG
// level vectors, partf8 / partd8 8 values per block
cudaError_t launch_pcg_mixed2(const PcgLaunch& P, const double* va1, double* x1, const MixedLaunch& X,
                              const AmgDevF* H0, const AmgDevF* H1, int wmax, cudaStream_t st, float* partf8,
                              double* partd8);
cudaError_t launch_to_float(int64_t n, const double* src, float* dst, cudaStream_t st);

// SELL-32/4: the SELL-32 layout with four consecutive entries of a row side by
// side, so a thread reads four column indices and four values with one 16-byte
// load each.  Slice s keeps its rows 32 s .. 32 s + 31, its width is rounded
// up to a multiple of 4 (w4), and entry k of row 32 s + l sits at
// sptr4[s] + 128 (k / 4) + 4 l + k % 4; padding entries hold value 0 and the
// row's own column.  Sums over a row keep the SELL-32 order (k ascending).
cudaError_t launch_sell_v4(int64_t n_slices, const int64_t* sptr, const int* sw, const int64_t* sptr4,
                           const float* src, float* dst, cudaStream_t st);

// ---- streaming solver (stream.cu) -------------------------------------------
// For operators that do not fit in L2 the solves run as chains of ordinary
// full-occupancy kernels instead of one persistent kernel; the Krylov loops
// run on the device as CUDA-graph conditional WHILE nodes whose condition the
// kernels set, so a solve needs no host round trip.
struct StreamScal {               // device scalars of one streaming solve
  double mean_b, bb, tol2;        // right-hand side mean (projected systems), |b|^2, tol^2 |b|^2
  double rr64, scale, tgt;        // outer residual, its norm, inner target (relative, squared)
  double rr_new, rho, alpha, beta, shift;
  int outer, it, fail, stop, inner_ran, skip, first, more;   // more: wants another outer pass
  long long inner_total, outer_total;
  unsigned ticket, pad2;
};
struct StreamLaunch {
  int n;                          // rows
  const int64_t* sptr;            // shared SELL-32 pattern (see PcgLaunch)
  const int* swidth;
  const int* col;
  const int* diagpos;
  const double* valA;             // FP64 operator values (outer residual, diagonal)
  const void* valT;               // operator values in the inner precision
  const double* dextra;           // optional extra diagonal
  const double* rl;               // rhs = rl + c1 V1 va + c2 V2 vb
  const double* val1;
  const double* va;
  double c1;
  const double* val2;
  const double* vb;
  double c2;
  int project, warm, pin, max_outer, inner_cap, use_amg;
  double tol, tol_inner;
  double* x;
  double* b64;                    // FP64 right-hand side
  double* r64;                    // FP64 outer residual
  void *r, *z, *p, *q, *d, *invd; // inner-precision vectors
  const void* h0_invd;            // AMG level 0 (inner precision): 1/D, pre-smoothed x, damping weight
  void* h0_x;
  double h0_omega;
  void* part;                     // block partial sums (grid x 4 doubles)
  StreamScal* sc;
  int* status;
  long long* iters_acc;
  long long* solves_acc;
  long long* outer_acc;
  long long* launch_acc;          // kernels launched (counted on the device)
  const int* gate;                // optional: the solve is skipped when *gate == 0
  int grid;                       // blocks of the row kernels (capped at a multiple of the SMs)
  int host_loop;                  // 1: the loops run on the host (eager launches, no graph conditions)
  // optional SELL-32/4 copy of the inner operator (FP32 only; see launch_sell_v4):
  // used by the Krylov product and by the AMG level-0 products, whose operator
  // is the same (elliptic) -- NULL: the SELL-32 arrays above
  const int64_t* sptr4;
  const int* sw4;
  const int* col4;
  const void* valT4;
  unsigned long long h_outer, h_inner;   // conditional handles of the two loops
};
// Enqueue one streaming solve on `st` (captured or not).  side[0..1] are two
// idle streams of the same device used to capture the loop bodies; inner type
// float or double (f32 = 1: FP32 inner iterations on valT/M32), AMG hierarchy
// M32/M64 or Jacobi when use_amg = 0.
cudaError_t stream_solve(const StreamLaunch& a, int f32, const AmgDevF* M32, const AmgDev* M64, cudaStream_t st,
                         const cudaStream_t* side);
int stream_grid_cap();
// query (once, outside any capture) the resident blocks per SM of every
// single-system streaming kernel; later plans read the cached values
void stream_prepare();
int stream_grid(int64_t rows);
// Two elliptic systems on one operator (stream2.cu): the AMG-preconditioned,
// warm-started form of the elliptic solve for the two right-hand sides of a
// later sweep, in one chain whose kernels load each operator entry once for
// both.  a[k]: system k's parameters (its own vectors, scalars sc, counters;
// the operator fields and the pin of a[0] serve both); H0 / H1: the FP32
// hierarchy with system 0's / system 1's level vectors (the same operators).
// pair_acc counts the inner iterations in which both systems advanced,
// pair64_acc the FP64 operator passes (right-hand side, refinement residual)
// and pairc_acc the first V-cycles of an inner solve shared by both.  Inner
// iterations in FP32 (AmgDevF: the mixed path) or FP64 (AmgDev);
// cudaErrorInvalidValue for any other form.
cudaError_t stream_solve_pair(const StreamLaunch (&a)[2], const AmgDevF& H0, const AmgDevF& H1, long long* pair_acc,
                              long long* pair64_acc, long long* pairc_acc, cudaStream_t st, const cudaStream_t* side);
cudaError_t stream_solve_pair(const StreamLaunch (&a)[2], const AmgDev& H0, const AmgDev& H1, long long* pair_acc,
                              long long* pair64_acc, long long* pairc_acc, cudaStream_t st, const cudaStream_t* side);
// query (outside any capture) the resident blocks of the pair kernels
void stream_prepare_pair();

// ---- batched solves (one launch per phase for many independent systems) -----
// A batch of nseg systems runs every phase of its solves as one launch over
// the concatenation of their rows: block b of a launch belongs to the system r
// with blk[r] <= b < blk[r+1] (a prefix of per-system block counts) and runs
// that system's rows with that system's parameters, reductions, scalars,
// stopping test and iteration cap.  The loops of the batch continue while any
// system still iterates: each system votes once per deciding launch and the
// last vote sets the loop conditions.
struct BatchCtl {
  unsigned inner_iters;           // passes of the batch's inner loop in this outer pass
  unsigned outer_iters;           // passes of its outer loop in this solve
};
struct BatchSolve {
  const StreamLaunch* tab;        // device: one StreamLaunch per system
  int nseg;
  int f32;
  BatchCtl* ctl;                  // device
  long long* launch_acc;          // device counter of the batch's launches
  // device block prefixes (nseg + 1 entries each): row kernels, and per
  // hierarchy level the kernels over A_l (post: at least one block a system),
  // R_l and P_l, and the coarse solve
  const int* blk_rows;
  const int* blk_post0;
  const int* blk_A[kMaxAmgLevels];
  const int* blk_R[kMaxAmgLevels];
  const int* blk_P[kMaxAmgLevels];
  const int* blk_coarse;
  int total_rows_blocks, total_post0_blocks;
  int total_A[kMaxAmgLevels], total_R[kMaxAmgLevels], total_P[kMaxAmgLevels], total_coarse;
  int nlev_max;                   // deepest hierarchy of the batch
  unsigned inner_cap, max_outer;  // largest per-system caps (the batch loops' backstop)
  const void* hier;               // device: one AmgDevT<float or double> per system (nlev = 0: Jacobi)
};
// Enqueue a batched solve (captured or not) on st; side as for stream_solve.
cudaError_t stream_solve_batch(const BatchSolve& b, cudaStream_t st, const cudaStream_t* side);

// host assembly (assemble.cpp)
struct HostOps {
  int64_t n = 0;
  int64_t n_tissue = 0;            // nodes [0, n_tissue) carry v and the membrane state
  std::vector<int32_t> rowptr, col, diagpos;
  std::vector<double> Ai, Aie, M, ML;
};
int assemble_host(const bd_mesh_t* mesh, const bd_cond_t* cond, HostOps* out, std::string* err);

}  // namespace bd
