/* Batched ROS4 chemistry integrator for GB300 (sm_103a), FP64: the C ABI.
 *
 * The library integrates the stiff constant-pressure chemical-kinetic ODE of every cell of a
 * CFD domain independently over one operator-split step, as in Curtis, Niemeyer & Sung,
 * "Accelerating reactive-flow simulations using vectorized chemistry integration":
 *   - state of a cell: y = [T, n_1, ..., n_{Ns-1}], the last species (bath gas) closed
 *     implicitly (Sec. 2.1, Eq. e:state_vec and Eq. e:n_nsp); here on a unit-mass basis, n_k in
 *     kmol per kg of mixture, n_Ns = (1 - sum_k W_k n_k) / W_Ns, V = n_tot R T / P;
 *   - source terms dy/dt = f(y) (Sec. 2.1, Eq. e:dphidt) and the analytical Jacobian
 *     J = df/dy (Eq. e:jac), from Arrhenius, third-body, Lindemann and Troe rate constants
 *     with reverse rates from NASA-7 equilibrium constants;
 *   - a four-stage linearly implicit Rosenbrock method (ROS4, Hairer-Wanner coefficients) in
 *     the transformed form of Sec. 2.3 (Eq. e:ros and below), with an embedded error estimate
 *     and adaptive step size; the whole domain goes in one batched call that returns the
 *     updated states and the last internal step size of each cell for reuse on the next
 *     split step (Sec. 2.4.1, BatchedChemistryModel).
 *
 * Conventions for every entry point:
 *   - SI units: T [K], P [Pa], dt and h [s], n [kmol/kg], f [K/s and kmol/kg/s].
 *   - Per-cell arrays are FP64, cell-fastest ("structure of arrays"): component i of cell c
 *     is at ptr[i * ld + c], with ld >= n_cells the leading dimension.  T, P, h, status are
 *     plain [n_cells] vectors.
 *   - Array pointers are DEVICE pointers owned by the caller (e.g. torch tensors), except in
 *     chem_integrate_host.  The library owns mechanism handles and compiled modules.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream) and
 *     return once the work is enqueued.  chem_integrate in CHEM_MODE_PERSISTENT does no host
 *     synchronisation and no allocation, so it can be captured in a CUDA graph.
 *   - Return value: 0 on success, negative on an argument, CUDA or NVRTC error; the message is
 *     in chem_last_error() (thread-local).  Integration failures of single cells are never
 *     errors: they are reported per cell in `status`.
 */
#ifndef CHEM_H
#define CHEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chem_mech* chem_mech_t;

/* error codes */
#define CHEM_OK 0
#define CHEM_EARG (-1)   /* invalid argument */
#define CHEM_ECUDA (-2)  /* CUDA driver/runtime error */
#define CHEM_ENVRTC (-3) /* run-time compilation failed */
#define CHEM_EIO (-4)    /* spec file unreadable or malformed */
#define CHEM_EWS (-5)    /* workspace too small */

/* per-cell integration status (same codes as the CPU oracle) */
#define CHEM_STATUS_OK 0
#define CHEM_STATUS_MAX_STEPS 1   /* max_steps attempts used before reaching dt */
#define CHEM_STATUS_H_UNDERFLOW 2 /* step size fell below h_min */
#define CHEM_STATUS_NONFINITE 3   /* non-finite input state; cell left unchanged */
#define CHEM_STATUS_SKIPPED 4     /* T < T_min: cell left unchanged (paper's reacting cut-off) */

/* integration drivers */
#define CHEM_MODE_PERSISTENT 0 /* one persistent launch, device work queue, per-team refill */
#define CHEM_MODE_PLAIN 1      /* one launch per ROS4 step attempt over all cells, host polling */

/* Options for chem_mech_load (NULL = defaults). */
typedef struct {
  int32_t team;        /* lanes per cell for the default kernel config: 1 (block 32..128), 4, 8
                          or 16 (several cells per warp; block 32..128), 32 (block 32..256), 64,
                          128, 256 (block = team); 0 = chosen from the mechanism size */
  int32_t block;       /* threads per block; 0 = chosen with team */
  int32_t verbose;     /* print compile logs (register use) to stderr */
  const char* cache_dir; /* directory for compiled cubins; NULL = no disk cache */
  int32_t adjoint;     /* chem_mech_compile_only: compile the adjoint module instead */
  int32_t tableau;     /* chem_mech_compile_only: integration method (CHEM_ROS4 ...) */
} chem_build_opts;

/* Rosenbrock methods (the solver table of the paper, Table T:solvers) */
#define CHEM_ROS4 0   /* Hairer-Wanner L-stable, 4 stages, order 4(3): the default */
#define CHEM_ROS3 1   /* Sandu et al. (1997), 3 stages, order 3(2), L-stable */
#define CHEM_RODAS3 2 /* Sandu et al. (1997), 4 stages, order 3(2), stiffly accurate */
#define CHEM_RODAS4 3 /* Hairer-Wanner, 6 stages, order 4(3), stiffly accurate */
/* The explicit solver of the same table: Runge-Kutta-Fehlberg 4(5), 6 evaluations of f per step,
 * no Jacobian or factorisation; the fifth-order solution is propagated (error estimate = its
 * difference to the fourth-order one, controller exponent 1/5).  For non-stiff cells only: on
 * stiff chemistry its stable step sizes are tiny and cells end with CHEM_STATUS_MAX_STEPS. */
#define CHEM_RKF45 4
/* A W-method (the class the paper names, Sec. 2.3 and Conclusions, for reusing Jacobians and
 * their factorisations): ROS2 of Verwer, Spee, Blom & Hundsdorfer (1999), 2 stages, second order
 * for any matrix W in place of the Jacobian, L-stable (gamma = 1 + 1/sqrt(2)), error estimate
 * against the first-order solution (controller exponent 1/2).  With chem_int_opts.jac_cache the
 * factorisation of I/(gamma h) - W is reused across attempts and calls while the step size is
 * unchanged; without it every attempt evaluates and factorises the Jacobian. */
#define CHEM_ROS2W 5

/* Options for chem_integrate (NULL = defaults shown). */
typedef struct {
  int32_t max_steps;   /* attempts (accepted + rejected) per cell and call; default 100000 */
  double h_min;        /* smallest step size [s] before CHEM_STATUS_H_UNDERFLOW; 1e-20 */
  double T_min;        /* cells with T < T_min are skipped; 0 = none */
  int32_t mode;        /* CHEM_MODE_PERSISTENT (default) or CHEM_MODE_PLAIN */
  int32_t team;        /* kernel config override (0 = mechanism default) */
  int32_t block;
  const double* lnA;   /* device [Nr]: ln of the pre-exponential factors (SI units; for falloff
                          reactions the high-pressure limit); NULL = the mechanism's values */
  int32_t* attempts;   /* device [n_cells] out: step attempts per cell; NULL = not written */
  int32_t tableau;     /* method, CHEM_ROS4 (0, default) .. CHEM_RODAS4, CHEM_RKF45 or CHEM_ROS2W; the step-size
                          controller uses err^(-1/order); the adjoint entry points need CHEM_ROS4 */
  const int32_t* order; /* device [n_cells] (nullable): the persistent driver's work queue hands out
                          the cells in this order -- a permutation of 0..n_cells-1, e.g. the
                          cost order of chem_cost_order; entries outside [0, n_cells) are skipped.
                          The results of a cell do not depend on the order. */
  int32_t* cell_method; /* device [n_cells] in/out (nullable): per-cell switching between an
                          alternative method (alt_tableau: RKF45 by default) and the Rosenbrock
                          method `tableau` (0..3; persistent mode; workspace per
                          chem_integrate_workspace).  In: > 0 = integrate the cell with the
                          alternative method under at most that many attempts, falling back to
                          the Rosenbrock method from the cell's initial state and step size if it
                          does not reach dt within them; <= 0 = the Rosenbrock method.  Out: the
                          choice for the next call -- after the alternative succeeded with a
                          attempts, 4a + 8; after a Rosenbrock integration with a attempts (RKF45
                          alternative), 4a + 8 if dt * rho <= 3a (rho = max_i sum_j |J_ij| w_j / w_i
                          at the first attempt, w = atol + rtol |y|: the explicit method's
                          stability-limited steps would not outnumber the Rosenbrock attempts),
                          else 0.  Start from zeros.  attempts/status report the run that finished
                          the cell.  Launches, on `stream`: a routing kernel, the alternative
                          method's integrator, a fall-back kernel, the Rosenbrock integrator. */
  double* jac_cache;    /* device, chem_jac_cache_bytes(n_cells) bytes, 8-byte aligned (nullable;
                          only with CHEM_ROS2W, persistent mode): per cell the factorised matrix
                          I/(gamma h) - W of the W-method, the step size it was built for and its
                          age, kept between attempts and between calls.  An attempt of size h reuses
                          it (no Jacobian, no factorisation) when it was built for exactly h and has
                          aged fewer than 32 accepted steps; otherwise it evaluates the Jacobian at
                          the attempt's state, factorises and stores.  Zero it before the first call
                          (an all-zero cache is empty); keep it with the cells between calls. */
  int32_t alt_tableau;  /* the alternative method of cell_method switching: 0 or CHEM_RKF45 (the
                          stiffness rule above), or CHEM_ROS2W (needs jac_cache): a cell whose
                          Rosenbrock integration took a single attempt and left a next-step
                          proposal h of at least 2 dt (quiescent, e.g. near equilibrium) runs
                          the W-method on the next call with budget 12, reusing
                          its cached factorisation across calls; the Rosenbrock launch empties the
                          cache of the cells it integrates. */
} chem_int_opts;

/* Parse a mechanism spec file (format: paper_2205_05681_gb300/synth.py docstring), build its
 * tables, generate its specialised CUDA source and compile it for sm_103a with NVRTC (or load
 * the cubin from cache_dir).  Host-side; needs a current CUDA device to load the module.
 * out receives the handle.  Errors: CHEM_EIO, CHEM_ENVRTC, CHEM_ECUDA.
 * Reaction order: every per-reaction array of this interface (lnA inputs, g_lnA and the VJP's
 * gp outputs, chem_mech_lnA) is in the file's reaction order; the kernels run the reactions in
 * their own branch-grouped order internally and map back. */
int chem_mech_load(const char* spec_path, const chem_build_opts* opts, chem_mech_t* out);

/* As chem_mech_load but only generates and compiles the source (no CUDA device needed); used
 * by the build step to check that every mechanism compiles.  Writes ptxas' register report
 * into log (capacity log_cap bytes, NUL-terminated) when log != NULL. */
int chem_mech_compile_only(const char* spec_path, const chem_build_opts* opts, char* log,
                           size_t log_cap);

/* Release a mechanism and its modules. */
int chem_mech_free(chem_mech_t mech);

/* Sizes of a mechanism: species (= state length N), reactions, elements. */
int chem_mech_info(chem_mech_t mech, int32_t* n_species, int32_t* n_reactions,
                   int32_t* n_elements);

/* Built-in ln A of every reaction (SI) copied to host array lnA[Nr]. */
int chem_mech_lnA(chem_mech_t mech, double* lnA);

/* Source terms f(y) (Eq. e:dphidt) for n_cells cells.
 *   T [n_cells], P [n_cells], n [(Ns-1) x ld] species moles (state entries 1..Ns-1),
 *   f [Ns x ld] out: f[0] = dT/dt, f[1+k] = dn_k/dt.  lnA: device [Nr] or NULL. */
int chem_eval_source(chem_mech_t mech, int64_t n_cells, const double* T, const double* P,
                     const double* n, double* f, int64_t ld, const double* lnA, void* stream);

/* Analytical Jacobian J = df/dy (Eq. e:jac) on y = [T, n_1..n_{Ns-1}].
 *   J [(Ns*Ns) x ld] out: entry (i, j) of cell c at J[(i*Ns + j) * ld + c] (row-major within
 *   a cell).  Other arguments as chem_eval_source. */
int chem_eval_jacobian(chem_mech_t mech, int64_t n_cells, const double* T, const double* P,
                       const double* n, double* J, int64_t ld, const double* lnA,
                       void* stream);

/* Bytes of device workspace chem_integrate needs for n_cells cells with these options. */
size_t chem_integrate_workspace(chem_mech_t mech, int64_t n_cells, const chem_int_opts* opts);

/* Integrate every cell from t = 0 to t = dt in place (Sec. 2.3 ROS4, Sec. 2.4.1 batching).
 *   T [n_cells] in/out, P [n_cells] in (constant during the step), Y [Ns x ld] mass fractions
 *   in/out (all Ns species; the bath gas is written from the closure).
 *   h [n_cells] in/out (nullable): in, the first step size to try (<= 0 means dt); out, the
 *   step size proposed for the next call.  status [n_cells] out (nullable).
 *   rtol, atol: the error tolerances of the weighted RMS error norm.
 *   workspace: device memory of chem_integrate_workspace() bytes, caller-owned, 256-byte
 *   aligned; its content need not be preserved between calls. */
int chem_integrate(chem_mech_t mech, int64_t n_cells, double* T, const double* P, double* Y,
                   int64_t ld, double dt, double rtol, double atol, double* h, int32_t* status,
                   const chem_int_opts* opts, void* workspace, size_t ws_bytes, void* stream);

/* chem_integrate on HOST arrays (ld = n_cells): copies T, P, Y, h to the device, integrates
 * with the persistent driver and copies T, Y, h, status back, all on `stream`, and waits for
 * completion.  Device buffers are allocated by the library on first use and reused.  h and
 * status may be NULL.  This is the end-to-end entry point for callers whose data lives on the
 * host. */
int chem_integrate_host(chem_mech_t mech, int64_t n_cells, double* T, const double* P,
                        double* Y, double dt, double rtol, double atol, double* h,
                        int32_t* status, const chem_int_opts* opts, void* stream);

/* ---- discrete adjoint (gradients of a loss on the final state) -------------------------
 * The forward is differentiated as the discrete map it is: the ROS4 steps of Sec. 2.3 with the
 * accepted step sizes frozen.  chem_integrate_ckpt records, per cell, every accepted step size
 * and the state after every `interval` accepted steps ("checkpoints"); chem_adjoint walks the
 * checkpoints backwards, recomputes the states between them, and pulls the loss gradient back
 * through each step's stages, LU and Jacobian (second derivatives of f by dual numbers).
 * (The paper has no adjoint; this extends its integrator.) */

/* Caller-owned device memory for one checkpointed forward. */
typedef struct {
  void* mem;          /* device, 256-byte aligned, >= chem_tape_bytes(...) */
  size_t bytes;
  int64_t n_cells;
  int32_t capacity;   /* accepted steps per cell the tape can hold */
  int32_t interval;   /* checkpoint every `interval` accepted steps (>= 1) */
} chem_tape;

/* Bytes of a tape: per cell an int (accepted count), capacity step sizes and
 * ((capacity-1)/interval + 1) checkpoint states of Ns doubles. */
size_t chem_tape_bytes(chem_mech_t mech, int64_t n_cells, int32_t capacity, int32_t interval);

/* chem_integrate (persistent driver) that also records the tape.  A cell whose tape is full
 * (`capacity` accepted steps recorded) before it reaches dt stops there with status
 * CHEM_STATUS_TAPE_FULL: its returned T, Y are the state after exactly the recorded steps, so a
 * reverse sweep over that tape differentiates the returned state, but it has not reached dt.
 * workspace: >= 256 bytes. */
#define CHEM_STATUS_TAPE_FULL 5
int chem_integrate_ckpt(chem_mech_t mech, int64_t n_cells, double* T, const double* P, double* Y,
                        int64_t ld, double dt, double rtol, double atol, double* h,
                        int32_t* status, const chem_int_opts* opts, const chem_tape* tape,
                        void* workspace, size_t ws_bytes, void* stream);

/* Device workspace of chem_adjoint (the recomputed segment states of every team in flight and
 * per-team partial gradients). */
size_t chem_adjoint_workspace(chem_mech_t mech, int64_t n_cells, const chem_int_opts* opts,
                              int32_t interval);

/* Reverse sweep.  Inputs: P [n_cells]; gT [n_cells] = dL/dT_final; gY [Ns x ld] = dL/dY_final
 * (mass fractions, all Ns species); the tape of the matching chem_integrate_ckpt call; opts->lnA
 * the same parameters as the forward (NULL = built-in).  Outputs: g_lnA [Nr] = dL/d lnA summed
 * over cells (a fixed-order reduction, deterministic); gT0 [n_cells] = dL/dT_0; gY0 [Ns x ld] =
 * dL/dY_0 (the state carries n_k = Y_k/W_k for k < Ns, so the bath-gas entry is 0).  Needs a
 * multi-lane kernel configuration (team >= 32). */
int chem_adjoint(chem_mech_t mech, int64_t n_cells, const double* P, const double* gT,
                 const double* gY, int64_t ld, const chem_tape* tape, const chem_int_opts* opts,
                 double* g_lnA, double* gT0, double* gY0, void* workspace, size_t ws_bytes,
                 void* stream);

/* chem_adjoint for callers that cannot allocate device memory.
 * Some callers cannot call cudaMalloc: code that runs inside a CUDA stream capture (allocation
 * there is not recorded into the graph), host applications whose device memory is owned by a
 * fixed pool or by another framework, or embedded solvers that may only touch memory handed to
 * them.  This entry point needs no workspace and allocates nothing: its scratch (a queue
 * counter, the recomputed segment states and the per-team partial gradients) lives in a static
 * device array of CHEM_ADJ_SCRATCH_BYTES (8 MiB) inside the adjoint module; every GPU that loads
 * that module holds the array until the process exits.  The caller still passes every input and
 * output, as for chem_adjoint.
 *   - The first call for a mechanism and kernel configuration compiles and loads the adjoint
 *     module (as chem_adjoint does) and resolves the array's device address; make that first call
 *     before any stream capture.
 *   - The array is shared by all calls on the same module and keeps the last call's contents:
 *     the entry point zeroes what must start at zero (the queue counter).  Calls whose work
 *     overlaps on the GPU (other streams, or chem_adjoint_noalloc enqueued twice without an
 *     ordering between them) race on the array: order them.
 *   - Fewer teams are launched when the full grid's scratch would not fit; if even one block's
 *     scratch (interval x Ns + Nr doubles per cell of a block) exceeds the array, it returns
 *     CHEM_EWS with a message naming the sizes.
 * (No counterpart in the paper: an addition for callers without an allocator.) */
#define CHEM_ADJ_SCRATCH_BYTES (8 * 1024 * 1024)
int chem_adjoint_noalloc(chem_mech_t mech, int64_t n_cells, const double* P, const double* gT,
                         const double* gY, int64_t ld, const chem_tape* tape,
                         const chem_int_opts* opts, double* g_lnA, double* gT0, double* gY0,
                         void* stream);

/* Vector-Jacobian products of f (Eq. e:jac transposed), the adjoint's building block, per cell:
 * gy [Ns x ld] = J(y)^T v and gp [Nr x ld] = (d f / d lnA)^T v, for v [Ns x ld] on the state
 * rows.  T, P, n as in chem_eval_source. */
int chem_eval_vjp(chem_mech_t mech, int64_t n_cells, const double* T, const double* P,
                  const double* n, const double* v, double* gy, double* gp, int64_t ld,
                  const double* lnA, void* stream);

/* Bytes of the W-method factorisation cache of n_cells cells (chem_int_opts.jac_cache):
 * n_cells x (Ns^2 + 2 ceil(Ns/2) + 2) doubles. */
size_t chem_jac_cache_bytes(chem_mech_t mech, int64_t n_cells);

/* Cost-ordered work queue (load balancing of cells of uneven stiffness, after the paper's call
 * for stiffness-based load balancing in its Conclusions, Sec. 6): writes to order [n_cells] (device) a permutation
 * of the cells by decreasing cost [n_cells] (device int32, e.g. the attempts of the previous split
 * step from chem_int_opts.attempts), so that the most expensive cells start first and the tail of
 * the persistent launch is short.  A counting sort over 1024 cost buckets (costs above 1023 share
 * the top bucket); cells of equal cost come in no particular order.  workspace: device memory of
 * chem_cost_order_workspace() bytes, 256-byte aligned.  Asynchronous on `stream`, no allocation,
 * no host synchronisation (capturable in a CUDA graph). */
size_t chem_cost_order_workspace(void);
int chem_cost_order(chem_mech_t mech, int64_t n_cells, const int32_t* cost, int32_t* order,
                    void* workspace, size_t ws_bytes, void* stream);

/* Autotuner: picks the fastest kernel configuration (lanes per cell "team" -- from several
 * cells per warp (4, 8, 16 lanes) for small mechanisms up to a block of 256 lanes per cell -- and
 * threads per block) for this mechanism by integrating a sample of the caller's cells once per
 * candidate configuration that fits in shared memory, and makes it the mechanism's default.  The
 * sample is the first min(n_cells, max(4096, 4 x the most resident cells of any candidate)) cells
 * of T, P, Y [Ns x ld], so that every candidate runs at full occupancy.  The caller's arrays are
 * not modified (the sample is copied).  Candidate modules are compiled on first use, in parallel
 * host threads (NVRTC; cached in cache_dir).  Set-up time only: allocates temporary device memory
 * and synchronises `stream`.  Outputs (nullable): the chosen team and block and the sample's
 * integration time in ms.
 * (Not from the paper, which tunes nothing at run time: its vector width is fixed at 8.) */
int chem_autotune(chem_mech_t mech, int64_t n_cells, const double* T, const double* P,
                  const double* Y, int64_t ld, double dt, double rtol, double atol, void* stream,
                  int32_t* team, int32_t* block, float* ms);

/* Kernel configuration actually used by chem_integrate for these options (team, block,
 * dynamic shared memory bytes, registers per thread); for reports. */
int chem_kernel_config(chem_mech_t mech, const chem_int_opts* opts, int32_t* team,
                       int32_t* block, int32_t* smem_bytes, int32_t* regs);

/* Measurement aid: throughput of this GPU's FP64 pipe, measured on `stream` (current context, or
 * device 0's primary context) with kernels compiled on the spot: dfma_tflops = FLOP/s of
 * independent FMA chains (2 flops per FMA) in TFLOP/s; exp_cost and log_cost = pipe time of one
 * double-precision exp and one log, in FMAs (log's includes one add of its argument).  Host-side,
 * synchronises `stream`, allocates and frees a small device buffer.  Outputs are nullable.
 * (No counterpart in the paper: it gives the integrator's FP64 roofline its denominator.) */
int chem_fp64_probe(void* stream, double* dfma_tflops, double* exp_cost, double* log_cost);

/* Message of the last failed call on this thread. */
const char* chem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CHEM_H */
