/*
 * bd.h -- C ABI of the GB300 (sm_103a) library for the partitioned bidomain
 * time step with spectral deferred correction.
 *
 * The method (Sec. 3.3.2 of the paper, Algorithm 2): at every time step the
 * elliptic constraint A_ie u = -A_i v (Eq. (3.15)) is solved with the latest
 * transmembrane voltage, the coupled parabolic PDE + ionic ODE system
 * Mt dX/dt = F(X, u) (Eq. (3.16)) is advanced with the two-stage ROS2
 * Rosenbrock method (Eq. (3.13)-(3.14)), and the result is corrected by the
 * linearised deferred-correction system (Eq. (3.20)); the three steps are
 * repeated as inner iterations ("sweeps").
 *
 * Units: cm, ms, mV, mS/cm, uA/cm^2, uF/cm^2, 1/cm.
 *
 * Conventions for every entry point
 *   - Return value: BD_OK (0) or a negative bd_status_t.  The library never
 *     aborts, traps or prints; bd_last_error() gives a one-line reason.
 *   - Host pointers are read during the call only and stay owned by the
 *     caller; nothing is retained.  "Device" pointers are CUDA global memory
 *     of the handle's device.
 *   - A handle is used by one host thread and one stream at a time.
 *   - Device-side failures (iteration cap reached, non-finite values,
 *     indefinite curvature, a grid barrier that timed out) set a status word
 *     on the device; it is returned by the next bd_sync / bd_get_* call and
 *     cleared by bd_clear_status.
 *
 * Node-major state layout ("SoA"): a state array X of a model with ns
 * variables and N nodes holds variable k of node i at X[k*N + i].  Variable
 * order per model:
 *   BD_LR91, BD_LR91_PAPER_MOD (ns = 8):  V, m, h, j, d, f, X, Cai
 *   BD_TP06_EPI (ns = 19): V, m, h, j, d, f, f2, s, r, Xr1, Xr2, Xs, fCass,
 *                          Rbar, Ki, Nai, Cai, CaSR, CaSS
 */
#ifndef BD_H_
#define BD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BD_OK = 0,
  BD_ERR_ARG = -1,            /* invalid argument (sizes, indices, NaN input, degenerate element) */
  BD_ERR_OOM = -2,            /* device allocation failed (or allocator callback returned NULL) */
  BD_ERR_CUDA = -3,           /* a CUDA runtime call failed */
  BD_ERR_NOT_CONVERGED = -4,  /* a CG solve reached its iteration cap */
  BD_ERR_NONFINITE = -5,      /* a non-finite residual or state was produced */
  BD_ERR_INDEFINITE = -6,     /* CG met p^T A p <= 0 */
  BD_ERR_TIMEOUT = -7         /* a device-wide barrier wait exceeded its bound */
} bd_status_t;

/* Membrane models of Sec. 2.  BD_LR91: Luo-Rudy 1991 with the 1991 parameter
 * set; BD_LR91_PAPER_MOD: the same with G_si = 0.02, G_Na = 4.0, G_K = 0.423
 * (Sec. 4); BD_TP06_EPI: ten Tusscher-Panfilov 2006, epicardial cell. */
typedef enum { BD_LR91 = 0, BD_LR91_PAPER_MOD = 1, BD_TP06_EPI = 2 } bd_ionic_t;

typedef enum { BD_FP64 = 0, BD_MIXED = 1 } bd_precision_t;

/* P1 mesh (Sec. 3.2): dim = 2 (triangles, 3 nodes per element) or 3
 * (tetrahedra, 4 nodes).  xyz: n_nodes*dim doubles, node-major (x0 y0 [z0] x1 ...).
 * elems: n_elems*(dim+1) zero-based node indices.  fiber: n_elems*dim unit
 * vectors or NULL (x axis).  All copied at bd_create.
 *
 * Bidomain-bath coupling (Sec. 4, "Results for Bidomain-Bath"): elem_bath
 * (n_elems bytes, or NULL = all tissue) marks the elements of a conductive
 * bath.  The tissue nodes are the nodes of the tissue elements; they must be
 * numbered first, 0 .. n_tissue-1 (BD_ERR_ARG otherwise).  Only the tissue
 * nodes carry v and the membrane state; u lives on every node and is the
 * extracellular potential in the tissue and the bath potential in the bath
 * (continuous across the interface, no intracellular current through it). */
typedef struct {
  int dim;
  int64_t n_nodes;
  int64_t n_elems;
  const double* xyz;
  const int32_t* elems;
  const double* fiber;
  const uint8_t* elem_bath;
} bd_mesh_t;

/* Conductivities (Sec. 2, transversely isotropic along the fibre):
 * sigma = s_t I + (s_l - s_t) f f^T for the intra- (i) and extracellular (e)
 * domains, mS/cm; chi = surface-to-volume ratio (1/cm); cm = membrane
 * capacitance (uF/cm^2); sbath = isotropic bath conductivity (mS/cm, > 0 when
 * the mesh has bath elements, else ignored). */
typedef struct {
  double sil, sit, sel, set;
  double chi, cm;
  double sbath;
} bd_cond_t;

/* Options; bd_default_options() fills every field. */
typedef struct {
  int precision;         /* bd_precision_t */
  int mass_lumped;       /* 1: lumped mass also on dv/dt (default 0: consistent) */
  int pin_node;          /* >= 0: u[pin] = 0; -1: zero nodal mean (default 0) */
  int sdc_correction;    /* 1: Algorithm 2 (default); 0: Algorithm 1, no correction */
  double cg_tol_e;       /* elliptic CG: ||r|| <= tol ||b|| (default 1e-10) */
  double cg_tol_p;       /* condensed parabolic CG (default 1e-10) */
  int cg_cap_e;          /* iteration caps (default 20000 / 2000) */
  int cg_cap_p;
  double sweep_tol;      /* > 0: Algorithm 2's test -- after sweep k < n_sweeps, stop when
                            max over all nodes and states |X^k - X^(k-1)| (X^0 = X^n, last
                            Lobatto node) < sweep_tol; decided on the device, so graph
                            replay is kept (default 0: always n_sweeps sweeps) */
  double v_act_mV;       /* activation threshold (default -30) */
  double spd_margin;     /* condensed-diagonal safeguard factor (default 0.9, 0 disables) */
  int use_graph;         /* 1: capture each step shape into a CUDA graph and replay it (default 1) */
  int elliptic_precond;  /* 1: aggregation AMG V(1,1) cycle (default; meshes small enough
                            for the dense coarse level use Jacobi), 0: Jacobi */
  int amg_coarse_max;    /* rows of the dense coarsest AMG level (0 = default 1500) */
  int cg_block;          /* CG threads per block (0 = auto: 512) */
  int cg_grid;           /* CG blocks (0 = auto: one per cg_block rows, at most the co-resident maximum) */
  /* device memory hooks (NULL => cudaMalloc/cudaFree); ctx is passed back.  Blocks
     must be 16-byte aligned (kernels use vector loads); a misaligned block is
     handed back to free() and counts as a failed allocation (BD_ERR_OOM). */
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* alloc_ctx;
  void* stream;          /* cudaStream_t or NULL (the library creates one) */
  int cg_cluster;        /* 0 (default): persistent CG kernels on a cooperative grid with
                            device-wide barriers; 8 or 16: as ONE thread-block cluster of that
                            many 1024-thread blocks with hardware cluster barriers (BD_ERR_ARG
                            for other values; falls back to the grid when the device cannot
                            schedule the cluster).  Measured slower on GB300 for 4k-263k-node
                            meshes (16 SMs stream less than the grid); kept for experiments. */
  int solver_tier;       /* 0 (default): choose the register tier of the solver kernels
                            (bd_stats_t.solver_tier); 1, 2, 3: force tier 0, 1 or 2 (2 needs
                            cg_block <= 512; 3 affects only the mixed AMG kernels);
                            BD_ERR_ARG otherwise; ignored with cg_cluster */
  int streaming;         /* solver form: 0 (default) streaming for operators of at least
                            5M entries (measured crossover on GB300), persistent otherwise;
                            1: always streaming; -1: never; 2: streaming with the loops on
                            the host (a profiling form: eager launches that tools can capture,
                            one synchronisation per iteration; no graphs; sweep_tol must be 0).
                            Streaming solves chain full-occupancy kernels whose CG loops run on
                            the device as CUDA graph conditional nodes; persistent solves are
                            one cooperative kernel each (bd_stats_t.streaming reports the form
                            in use) */
  int vec4;              /* 0 (default): mixed-precision streaming solves also keep the FP32
                            elliptic and parabolic operators, and every FP32 AMG level operator
                            stored as SELL-32 with at least 2^17 rows, in the SELL-32/4 layout
                            (four consecutive entries of a row per 16-byte load; 8 more bytes
                            per stored entry) and use it in their products; 1: the same for
                            every SELL-32 level operator whatever its size (testing); -1: none
                            (the plain SELL-32 layout only); BD_ERR_ARG otherwise.  Both layouts
                            give the same sums in the same order */
  int csr_lanes;         /* streaming solves, AMG levels stored as CSR: threads per row.  0
                            (default): a quarter of the level's mean row length rounded up to a
                            power of two in [4, 32], or 256 (a block per row) for rows of 256
                            entries and more on average; 4, 8, 16, 32 or 256 force that width on
                            every CSR level (tuning and testing); BD_ERR_ARG otherwise */
  int wide_sell;         /* streaming handles, AMG levels with rows longer than 32 entries: 0
                            (default) SELL-32 (thread per row) when padding stores at most 1.5x
                            the entries and the level has at least 2^17 rows averaging at most 96
                            entries, else CSR; 1: SELL-32 whenever the padding allows; -1:
                            always CSR; BD_ERR_ARG otherwise */
  int pair_solve;        /* AMG-preconditioned elliptic solves: the two elliptic solves of
                            every sweep after the first (the constraint at two Gauss-Lobatto
                            nodes, Sec. 3.3.2) run as one two-system solve whose operator
                            passes serve both right-hand sides -- in mixed precision one
                            cooperative kernel (persistent form) or one kernel chain
                            (streaming form), in FP64 one kernel chain (streaming form; the
                            persistent FP64 form solves one after the other).  0 (default):
                            on; -1: one solve after the other (each
                            system's arithmetic is the same either way; the reductions are
                            formed over different block partitions); BD_ERR_ARG otherwise */
} bd_opts_t;

typedef struct bd_state bd_state_t;

/* Per-handle counters since creation (or the last bd_reset_stats). */
typedef struct {
  int64_t steps;
  int64_t sweeps;
  int64_t cg_iters_e;      /* summed elliptic CG iterations */
  int64_t cg_solves_e;
  int64_t cg_iters_p;      /* summed parabolic CG iterations */
  int64_t cg_solves_p;
  int64_t spd_clamps;      /* nodes whose condensed diagonal was raised */
  int64_t ionic_evals;     /* node-block evaluations (kernel launches x nodes / nodes) */
  int64_t kernel_launches; /* device kernels launched by the steps */
  int64_t solver_block_bound; /* launch bound of the solver build in use: 512 (128 registers a
                                 thread, chosen when the rows fit one block per SM) or 1024 */
  int64_t solver_tier;     /* 0: 1024-thread build (64 registers); 1: 512-thread build (128
                              registers); 2: as 0, with the mixed AMG kernels built for two
                              1024-thread blocks per SM (32 registers; operators of >= 12M
                              entries) */
  int64_t amg_levels;      /* smoothed AMG levels of the elliptic preconditioner (0: Jacobi) */
  int64_t amg_coarse_rows; /* rows of the dense coarsest AMG level (0: Jacobi) */
  int64_t streaming;       /* 1: the solves run as streaming kernel chains (bd_opts_t.streaming) */
} bd_stats_t;

/* Per-kind device time of profiled steps (bd_profile_steps). */
enum {
  BD_K_PCG_ELLIPTIC = 0,   /* persistent PCG, elliptic constraint (A2) */
  BD_K_PCG_PARABOLIC = 1,  /* persistent PCG, condensed parabolic systems (A5, A9) */
  BD_K_IONIC = 2,          /* node-wise model + Jacobian + condensation (A4, A6, A8) */
  BD_K_FIELD = 3,          /* node field only (quadrature values, A8) */
  BD_K_COMBINE = 4,        /* ROS2 combination / correction update / copies (A7, A9) */
  BD_K_FINISH = 5,         /* activation times and state rotation (A10) */
  BD_K_COUNT = 6
};
typedef struct {
  double ms[BD_K_COUNT];        /* summed kernel durations (CUDA events on the handle's stream) */
  int64_t launches[BD_K_COUNT];
  int64_t cg_iters[2];          /* elliptic, parabolic CG iterations in the profiled steps */
  int64_t cg_solves[2];
  int64_t outer_iters[2];       /* FP64 residual passes (mixed path: refinement steps) */
  int64_t nnz;                  /* nonzeros of the shared operator pattern */
  double alg_bytes[2];          /* algorithmic DRAM bytes of all elliptic / parabolic solves,
                                   Krylov level only: every SpMV moves (vb + 4) bytes per
                                   nonzero and 2 vb + 4 per row (value and column index per
                                   entry; one gather of x, the result and a row pointer per
                                   row), every CG iteration 16 vb bytes per row of vector
                                   streams (13 vb with the AMG preconditioner, whose work is
                                   counted below), every solve its FP64 right-hand-side
                                   products and set-up passes, every mixed refinement pass an
                                   FP64 residual product; vb = 4 (mixed) or 8 (FP64).  A
                                   two-system elliptic solve (bd_opts_t.pair_solve) counts an
                                   operator once where both systems use the same pass of it:
                                   the Krylov product of an iteration in which both advance
                                   and, streaming, the FP64 right-hand-side and residual
                                   products of a pass both run */
  double vcycle_bytes;          /* elliptic AMG V-cycles of the profiled steps, counted the same
                                   way: per smoothed level two products with A_l and one each
                                   with R_l and P_l plus the level's vector streams (operators
                                   read once for both systems of a cycle that serves both) */
  double coarse_bytes;          /* ... their dense coarsest-level solves (nc^2 + 2 nc values
                                   per cycle; the streaming two-system solve reads the inverse
                                   once for both): a dense equivalent, reported apart */
} bd_profile_t;

void bd_default_options(bd_opts_t* opts);

/* Assemble the P1 operators on the host (Sec. 3.2, Eqs. (3.6)-(3.9)), upload
 * them, set the resting state of the model (LR91: Newton zero of the cell
 * field; TP06: the published initial values) and return a handle.
 * BD_ERR_ARG for out-of-range indices, non-positive element measures,
 * non-finite coordinates or an unknown model. */
int bd_create(const bd_mesh_t* mesh, const bd_cond_t* cond, bd_ionic_t model,
              const bd_opts_t* opts, bd_state_t** out);

/* Add a stimulus (at most 32): membrane current density amp (uA/cm^2,
 * depolarising) on the tissue nodes with node_mask[i] != 0 (n_tissue bytes), active
 * for the steps with t_on <= t^n < t_on + dur, t^n = n*dt (Sec. 4 protocols). */
int bd_add_stimulus(bd_state_t* s, const uint8_t* node_mask, double t_on_ms, double dur_ms,
                    double amp);

/* Set X (ns*n_tissue doubles, state-major: X[k*n_tissue + i]) and u
 * (n_nodes doubles or NULL => zeros) from host memory; resets the step
 * counter, the clock and the activation times. */
int bd_set_initial(bd_state_t* s, const double* X, const double* u);

/* Advance one time step of size dt_ms with Algorithm 2 on n_sdc_nodes (2 or
 * 3) Gauss-Lobatto nodes and n_sweeps (>= 1) inner iterations.  Enqueued on
 * the handle's stream; returns the status word of the last completed step
 * that was read back (bd_sync waits and reads it). */
int bd_step(bd_state_t* s, double dt_ms, int n_sdc_nodes, int n_sweeps);

/* One step of the decoupled CN-RK2 scheme, the paper's reference decoupled
 * strategy (Sec. 3.3.3): Strang splitting of the node reaction (explicit
 * midpoint rule over two half steps dt/2, the step's stimulus included) and
 * the diffusion (one Crank-Nicolson step of M dv/dt = -A_i (v + u^n),
 * solved by CG for the increment), then the elliptic constraint
 * A_ie u^{n+1} = -A_i v^{n+1}.  Explicit in the membrane model, so dt must
 * resolve its fastest gate (the paper uses dt = 0.001 ms).  Shares the
 * handle, its operators, precision, statistics, activation times and clock
 * with bd_step; one CUDA graph per dt. */
int bd_step_decoupled(bd_state_t* s, double dt_ms);

/* Adaptive step (the paper's production mode, Sec. 3.3.2 and Sec. 4.3: the
 * embedded ROS2 solution X_hat = X + k1/gamma of Eq. (3.14) determines the
 * future step, at most dt_max).  Error estimate: the maximum, over the last
 * sweep's ROS2 sub-steps, nodes and state variables, of
 * |X_new - X_hat| / (tol (1 + |X_new|)).  err <= 1 accepts the step (also at
 * the smallest step dt_max 2^-7); otherwise X^n is restored and the step is
 * repeated with a smaller step.  The next step is dt * min(2, max(0.5,
 * 0.9 err^-1/2)) rounded down to the ladder dt_max 2^-k, k = 0..7 (one CUDA
 * graph per rung).  Synchronises once per attempt.  Outputs (each may be
 * NULL): the step taken, its error estimate, the number of rejections. */
int bd_step_adaptive(bd_state_t* s, double dt_max, double tol, int n_sdc_nodes, int n_sweeps,
                     double* dt_taken, double* err, int* rejected);

/* Failure-path check (the paper has no counterpart): one block waits at a
 * device-wide barrier sized for two blocks, so the wait runs out after its
 * bound of about two seconds of device time, as a solver's wait would if a
 * block never arrived.  Returns BD_ERR_TIMEOUT when the bound works (any
 * other value is a fault of the build); the handle's status word and barrier
 * are reset afterwards, so the handle stays usable. */
int bd_selftest_wait_timeout(bd_state_t* s);

/* Simulated time t^n (ms) and number of completed steps (each may be NULL). */
int bd_get_time(const bd_state_t* s, double* t_ms, int64_t* steps);

/* Advance several handles by one step each (one launch sequence per handle
 * on the first handle's stream; the handles must share one device). */
int bd_batch_step(bd_state_t* const* states, int n, double dt_ms, int n_sdc_nodes, int n_sweeps);

/* Wait for the handle's stream and return its device status word. */
int bd_sync(bd_state_t* s);

/* Non-blocking: 1 if every step enqueued on the handle has completed, 0 if
 * work is still in flight, negative on a CUDA error.  Lets one host thread
 * keep many handles (each on its own stream) busy at once. */
int bd_query(bd_state_t* s);
void bd_clear_status(bd_state_t* s);

/* Activation times of the tissue nodes (first upward crossing of v_act,
 * linearly interpolated inside the step; NaN if not activated),
 * n = n_tissue doubles to host. */
int bd_activation_times(const bd_state_t* s, double* out, int64_t n);

/* Copy v (n_tissue), u (n_nodes) and, if X != NULL, the full state
 * (ns*n_tissue) to host memory; any pointer may be NULL. */
int bd_get_fields(const bd_state_t* s, double* vm, double* phie, double* X);

/* Device pointers of the resident v-row / u so callers can read them without
 * a host copy (valid until bd_destroy). */
int bd_device_fields(const bd_state_t* s, const double** X_dev, const double** u_dev);

/* Serialise (X, u, step counter, simulated time and the previous step's,
 * adaptive step, activation times, and the solver warm starts: the previous
 * step's sweep-1 elliptic solution and the last parabolic increments) to
 * host memory, so a restored handle continues bit for bit.  With
 * buf == NULL only *bytes is set. */
int bd_get_state(const bd_state_t* s, void* buf, size_t* bytes);
int bd_set_state(bd_state_t* s, const void* buf, size_t bytes);

/* Estimate of the device bytes bd_create allocates for this mesh, model and
 * options (opts NULL: defaults): operators, state and workspaces, the FP32
 * copies of the mixed path, the AMG hierarchy (from the entry ratios of
 * structured 2-D and 3-D meshes) and the streaming form's SELL-32/4 copies.
 * Host only.  Meant for admission control; not a bound for arbitrary
 * meshes. */
size_t bd_footprint_bytes(const bd_mesh_t* mesh, bd_ionic_t model, const bd_opts_t* opts);

int bd_get_stats(const bd_state_t* s, bd_stats_t* out);

/* Sizes in bytes of the public structs as this library was compiled (a
 * binding compares them with its own layouts); NULL arguments are skipped.
 * Host only; returns BD_OK. */
int bd_struct_sizes(size_t* mesh, size_t* cond, size_t* opts, size_t* stats);

/* Allocation-free variant of bd_solve_elliptic for callers that must not
 * allocate GPU memory during the call -- for example code running under an
 * external memory budget or allocator, or a latency-critical loop that cannot
 * afford cudaMalloc/cudaFree, which may synchronise the whole device.  The
 * paper has no counterpart; this is a service of the library.
 *
 * Solves A_ie u = -A_i v by Jacobi-preconditioned CG (whatever the handle's
 * elliptic_precond and precision: the solve is FP64) with the handle's
 * resident operators, tolerance and pin.  It is not part of a time step: a
 * device-side sweep test (sweep_tol > 0) that closed the sweeps of the last
 * bd_step does not affect it.  Every call runs on the handle's device (the
 * one current at bd_create), which it makes current for the call and then
 * restores, so the caller may have another device current; the pointers
 * below are memory of the handle's device:
 * v_dev (n_nodes doubles, device; with a bath the entries of bath nodes are
 * multiplied by zero and must be finite) is read, u_dev (n_nodes doubles,
 * device) is written, u_guess_dev (device, n_nodes) warm-starts the iteration
 * or is NULL for a zero start.  The call allocates nothing: the CG work vectors, partial sums,
 * barrier words and status live in one file-scope __device__ array of the
 * library sized for at most BD_NOALLOC_MAX_NODES nodes (about 5.4 MB, held
 * by every GPU that loads the library until the process exits).  Larger
 * meshes return BD_ERR_ARG.
 *
 * The first call on a device looks up that array's device address (with the
 * handle's device current) and caches it per device, so the first call on
 * each device should come before any stream capture.  Every call shares the array: the words that must
 * start at zero are cleared at the start of each call, and calls that overlap
 * on the GPU (on different streams or handles) race with each other.  The call
 * runs on the handle's stream and waits for it; *iters (if not NULL) receives
 * the iteration count. */
#define BD_NOALLOC_MAX_NODES 131072
int bd_solve_elliptic_noalloc(bd_state_t* s, const double* v_dev, const double* u_guess_dev, double* u_dev,
                              int* iters);

/* Run n_steps steps without graph replay, with a CUDA event pair recorded on
 * the handle's stream around every kernel launch, and return the per-kind
 * device times.  The steps advance the simulation like bd_step. */
int bd_profile_steps(bd_state_t* s, double dt_ms, int n_sdc_nodes, int n_sweeps, int n_steps,
                     bd_profile_t* out);
int bd_reset_stats(bd_state_t* s);
int64_t bd_num_nodes(const bd_state_t* s);
/* Nodes that carry v and the membrane state (= bd_num_nodes without a bath). */
int64_t bd_num_tissue_nodes(const bd_state_t* s);
int bd_num_states(bd_ionic_t model);
const char* bd_last_error(const bd_state_t* s);
void bd_destroy(bd_state_t* s);

/* ---- kernel-level entry points (parity tests and tools) ---------------- */

/* Evaluate the membrane model on the device for n node states X (host,
 * ns*n node-major) with per-node stimulus current istim (host, n, may be
 * NULL): writes the node field f = (-(I_ion - I_stim)/C_m, g) (ns*n) and,
 * if jac != NULL, the dense node Jacobian df/dX (n*ns*ns, node-major
 * blocks, row = component of f) -- Sec. 2 models, Sec. 3.3.2 "exact
 * derivatives".  cm is the membrane capacitance. */
int bd_ionic_eval(bd_ionic_t model, int precision, int64_t n, const double* X,
                  const double* istim, double cm, double* f, double* jac);

/* Compile-time sparsity pattern of the node Jacobian (the paper's CTSM
 * blocks, Sec. 3.3.2): masks[r] has bit c set iff df_r/dX_c may be nonzero.
 * masks holds ns uint32 values. */
int bd_ionic_pattern(bd_ionic_t model, uint32_t* masks);

/* Resting state used by bd_create (ns doubles). */
int bd_rest_state(bd_ionic_t model, double* X);

/* Assembled operator of a handle in CSR form (A0 of the method, Sec. 3.2):
 * which = 0: A_i, 1: A_ie (both already divided by chi*C_m), 2: consistent
 * mass M, 3: lumped mass M_L (diagonal; only val is written, N doubles).
 * With val == NULL only *nnz is set; otherwise rowptr (N+1), col (nnz)
 * and val (nnz) are written to host memory.  Columns are sorted per row. */
int bd_operator_csr(const bd_state_t* s, int which, int64_t* nnz, int32_t* rowptr,
                    int32_t* col, double* val);

/* Solve the elliptic constraint A_ie u = -A_i v (Eq. (3.15)) with the
 * handle's operators, precision and pin, from a host v (n_tissue) into a host
 * u (n_nodes), warm-started from u_guess (host, n_nodes) or from zero if NULL.
 * Returns the iteration count in *iters when not NULL. */
int bd_solve_elliptic(bd_state_t* s, const double* v, const double* u_guess, double* u,
                      int* iters);

/* Shape of level `level` of the elliptic AMG hierarchy (smoothed
 * aggregation, the preconditioner class of Sec. 3.3.2; level 0's A is A_ie
 * itself).  out[9] (host) receives rows, stored entries and storage form of
 * A_l, R_l and P_l in that order; form 0: SELL-32 with rows of at most 32
 * entries, -1: SELL-32 with longer rows (streaming handles), k > 0: CSR read
 * by k threads per row in the streaming kernels.  BD_ERR_ARG when the
 * handle has no such level (Jacobi handles have none).  No device work. */
int bd_amg_level(const bd_state_t* s, int level, int64_t* out);

#ifdef __cplusplus
}
#endif
#endif /* BD_H_ */
