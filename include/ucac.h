/*
 * ucac.h -- C ABI of the B300 (sm_103a) library for the inner sweep of the
 * two-level component ADMM for unit commitment with AC optimal power flow
 * (Zhang, Kim, Kim, "On Solving Unit Commitment with AC Optimal Power Flow on
 * GPU").
 *
 * One handle holds one or more independent UC-ACOPF instances on one GPU.
 * Every step of a sweep runs in the library's CUDA kernels:
 *   x-step      UC dynamic program per generator (Algorithm 2), generator and
 *               line subproblems per (period, component) (Eq. step:uc,
 *               step:opf);
 *   x-bar-step  duplicate-UC box QPs and bus power-balance projections
 *               (Eq. step:uc_bar, step:opf_bar), fused with the z and y
 *               updates (Eq. step:z, step:y) and the residual partial sums;
 *   finish      per-instance deterministic residual reduction, inner stop
 *               test and outer lambda/beta update (Eq. step:outer,
 *               Algorithm 1).
 *
 * Conventions for every entry point:
 *   - Arrays are plain C arrays, 0-based, row-major, FP64 unless noted.
 *   - Host pointers are read during the call and not retained; device memory
 *     is owned by the handle and released by ucac_destroy.
 *   - Return value 0 = success, 1 = success and every instance converged,
 *     negative = error (UCAC_E_*); no exception crosses the ABI.  After an
 *     error ucac_last_error() gives a one-line reason.
 *   - A handle is not thread-safe; all device work is issued on the CUDA
 *     stream given at creation (NULL = the legacy default stream).
 */
#ifndef UCAC_H
#define UCAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define UCAC_OK 0
#define UCAC_CONVERGED 1
#define UCAC_E_ARG (-1)          /* bad argument (NULL pointer, size, index) */
#define UCAC_E_GRID (-2)         /* invalid grid data (disconnected, r=x=0, bounds out of order, ...) */
#define UCAC_E_CUDA (-3)         /* a CUDA runtime call failed */
#define UCAC_E_NEWTON_MAXIT (-4) /* a line subproblem stopped on an iteration cap (params.stop_on_cap = 1) */
#define UCAC_E_NAN (-5)          /* a residual became NaN or Inf */
#define UCAC_E_DIVERGED (-6)     /* r_p or r_d grew past params.div_bound */

/*
 * Instance data (Sec. II: variables, Eq. acopf, Eq. set:UC, Eq. coupling).
 * Per-unit quantities on base_mva; costs in $ with c2 in $/MW^2h, c1 in $/MWh,
 * c0 in $/h while on, c_su / c_sd in $ per start-up / shut-down.
 * Layouts: Pd, Qd are [T][n_bus]; bus arrays [n_bus]; branch arrays
 * [n_branch]; generator arrays [n_gen].  br_b is the total line charging.
 * TU/TD are the minimum up/down times in periods, u0 the status in period 0,
 * L0/F0 the number of initial periods forced on/off (Eq. uc_initial_on/off),
 * p0 the output in period 0.  Branches have no taps or phase shifters.
 */
typedef struct ucac_grid {
  int32_t n_bus, n_branch, n_gen, T, ref_bus;
  const double *Pd, *Qd;
  const double *Gs, *Bs, *Vmin, *Vmax;
  const int32_t *br_from, *br_to;
  const double *br_r, *br_x, *br_b, *br_rate;
  const int32_t *gen_bus;
  const double *Pmin, *Pmax, *Qmin, *Qmax, *c2, *c1, *c0, *c_su, *c_sd, *RU, *RD, *SU, *SD;
  const int32_t *TU, *TD, *u0, *L0, *F0;
  const double *p0;
  double base_mva;
} ucac_grid;

/* Penalties for the power rows, the voltage/angle rows and the UC rows (Sec. IV-A). */
typedef struct ucac_rho {
  double pq, va, uc;
} ucac_rho;

/*
 * Algorithm parameters.  eps_in: inner stop on the RMS primal and dual
 * residuals; eps_out: outer stop on the RMS of z; tau, theta: outer beta rule
 * (Eq. step:outer, tau = 6, theta = 0.8); beta0: initial beta; lambda_max:
 * bound of the projection of lambda; eta: line-subproblem equality tolerance
 * (inf-norm); omega_rel: line-subproblem stationarity tolerance relative to
 * max(rho.pq, rho.va); c_init_rel / c_max_rel: initial / largest
 * augmented-Lagrangian penalty of the line subproblem, relative to
 * max(rho.pq, rho.va); K_AL / K_N: iteration caps of the line subproblem's
 * multiplier and Newton loops; L_max: cap on inner sweeps per outer
 * iteration; check_every: sweeps between host convergence checks in
 * ucac_iterate; line_form: coordinates of the line subproblem solver,
 * UCAC_LINE_POLAR (default: (V_i, V_j, theta_i - theta_j), where the product
 * and angle equations hold identically) or UCAC_LINE_W (the W-form variables
 * with an augmented Lagrangian on all four equalities).  Both solve the same
 * subproblem.  uc_relax: 0 (default) solves the UC subproblem by Algorithm 2;
 * 1 replaces it by its box relaxation (u_on, u_su, u_sd in [0, 1] each, the
 * start-up/shut-down equation and the minimum up/down times dropped:
 * u = clamp(tau - c/rho_uc, 0, 1) per row), the first phase of the UC warm
 * start (ucac_uc_warm_start).  rho_every: 0 (default) keeps the penalties of
 * create; k > 0 adapts them every k sweeps by residual balancing (the
 * adaptive rules Sec. V names as future work): all three penalties are
 * multiplied by rho_tau (2) when r_p > rho_mu r_d (rho_mu = 10) and divided
 * by it when r_d > rho_mu r_p, at most 6 net steps either way from the
 * penalties of create; the current penalties are part of the state.
 * Failure detection (the library's, not the paper's): after each sweep an
 * instance whose residuals are not finite takes status UCAC_E_NAN; one whose
 * r_p or r_d exceeds div_bound (default 1e6, in the RMS units of the rows)
 * takes UCAC_E_DIVERGED; with stop_on_cap = 1 (default 0) one whose sweep
 * had a line subproblem stopped by K_N / K_AL before meeting its tolerances
 * takes UCAC_E_NEWTON_MAXIT (with 0 such solves are only counted, in
 * ucac_report.n_newton_maxit).  An instance with an error status takes no
 * further sweep (its iterate and record stay those of that sweep) while the
 * rest of a batch goes on; ucac_iterate returns the code.
 */
#define UCAC_LINE_W 0
#define UCAC_LINE_POLAR 1
typedef struct ucac_params {
  double eps_in, eps_out, tau, theta, beta0, lambda_max;
  double eta, omega_rel, c_init_rel, c_max_rel;
  double rho_mu, rho_tau;
  int32_t K_AL, K_N, L_max, check_every, line_form, uc_relax, rho_every, stop_on_cap;
  double div_bound;
} ucac_params;

/*
 * Residual record of one instance after the last sweep.
 * r_p = |Ax + Bxbar + z|_2 / sqrt(m), r_d = |B(xbar_new - xbar_old)|_2 / sqrt(m)
 * (m = number of coupling rows), z_norm = |z|_2, z_rms = z_norm / sqrt(m),
 * inf_norm_viol = |Ax + Bxbar|_inf (the primal infeasibility of Sec. IV-D),
 * objective = sum of generation, no-load, start-up and shut-down costs at the
 * current x.  newton / al = line-subproblem Newton / multiplier iterations in
 * the last sweep; n_newton_maxit = line subproblems that stopped on a cap;
 * newton_total / al_total = the same counts summed over every sweep since
 * create.  status: 0 running, 1 converged, or a negative UCAC_E_* code
 * (UCAC_E_NAN, UCAC_E_DIVERGED, UCAC_E_NEWTON_MAXIT; see ucac_params).
 */
typedef struct ucac_report {
  double r_p, r_d, z_norm, z_rms, inf_norm_viol, objective, beta;
  int64_t sweeps, outer, newton, al;
  int32_t status, n_newton_maxit;
  int64_t newton_total, al_total;
} ucac_report;

typedef struct ucac_handle ucac_handle;

/* Fills *p with the defaults listed above. */
void ucac_default_params(ucac_params *p);

/*
 * Creates a handle for one instance and applies the cold start of Sec. IV-A
 * (p, q and |V| at the middle of their bounds, angles zero, flows from the
 * initial voltages) with all units on.  horizon (1 <= horizon <= grid->T)
 * selects the first periods of Pd/Qd.  params may be NULL (defaults).
 * stream is a cudaStream_t or NULL.  Errors: UCAC_E_ARG, UCAC_E_GRID,
 * UCAC_E_CUDA; *out is NULL then.
 */
int ucac_create(const ucac_grid *grid, int32_t horizon, ucac_rho rho, const ucac_params *params,
                void *cuda_stream, ucac_handle **out);

/*
 * Same for n independent instances sharing one set of launches (batching);
 * horizons[k] and rhos[k] belong to grids[k].
 */
int ucac_create_batch(const ucac_grid *const *grids, const int32_t *horizons, const ucac_rho *rhos, int32_t n,
                      const ucac_params *params, void *cuda_stream, ucac_handle **out);

/* Number of instances in the handle. */
int32_t ucac_instances(const ucac_handle *h);

/*
 * Runs up to n_sweeps inner sweeps (Algorithm 1 inner loop body, with outer
 * updates applied when an instance's inner loop stops), checking on the host
 * every params.check_every sweeps whether every instance has converged
 * (inner residuals <= eps_in and z_rms <= eps_out).  Synchronises the
 * stream.  Returns 1 when all instances have converged, 0 otherwise, or the
 * negative status of the first instance that stopped on an error (UCAC_E_NAN,
 * UCAC_E_DIVERGED, UCAC_E_NEWTON_MAXIT; ucac_last_error names the instance).
 */
int ucac_iterate(ucac_handle *h, int32_t n_sweeps);

/*
 * Enqueues exactly n_sweeps sweeps on the handle's stream (one CUDA-graph
 * launch per sweep) and returns without synchronising or checking
 * convergence.  For timing loops.
 */
int ucac_enqueue_sweeps(ucac_handle *h, int32_t n_sweeps);

/* Copies instance `instance`'s residual record to *out (synchronises). */
int ucac_residuals(const ucac_handle *h, int32_t instance, ucac_report *out);

/*
 * The device counters of the line subproblems (Eq. acopf; the trust-region
 * Newton inside the augmented-Lagrangian loop that Sec. IV-A names): for
 * every line-period of instance `instance`, the Newton iterations (newton)
 * and multiplier rounds (al) of its solve in the last sweep the instance
 * ran, [T][n_branch] each, into caller HOST buffers (either may be NULL).
 * Counts saturate at 65535.  Their sums equal the record's newton and al.
 * Synchronises.  UCAC_E_ARG for a bad handle or instance, UCAC_E_CUDA if a
 * copy fails.
 */
int ucac_line_counts(const ucac_handle *h, int32_t instance, uint16_t *newton, uint16_t *al);

/*
 * Index-checked builds (compiled with UCAC_CHECK=1, libucac_check.so; no
 * counterpart in the paper): the sweep kernels test every index they take
 * from a table against the extent of the buffer it addresses; a failed test
 * records its site on the device and skips the access, and the next host
 * check of ucac_iterate returns UCAC_E_CUDA with "index check failed at
 * site N" (the record stays: every later call fails the same way).
 * ucac_check_inject records site (> 0) as a failed check from a device
 * thread, as a kernel's failed test would, to exercise that path; it
 * synchronises.  In a default build it returns UCAC_E_ARG.
 */
int ucac_check_inject(ucac_handle *h, int32_t site);

/*
 * Copies the solution of one instance -- the iterate Algorithm 1 returns,
 * in the variables of Sec. II (generator outputs, Eq. acopf voltages and
 * flows, the commitment of Eq. set:UC) -- into caller host buffers (any may
 * be NULL): p, q [T][n_gen] (generator x-side), w, theta [T][n_bus] (bus
 * copies: |V|^2 and the voltage angle), pf [T][n_branch][4] (p_ij, q_ij,
 * p_ji, q_ji from the line subproblems), u_on [T][n_gen] (0/1 from the UC
 * dynamic program).  The copies are queued on the handle's stream behind
 * its sweeps and the call returns once they are done; page-locked buffers
 * let them run at the copy engines' rate.  UCAC_E_ARG for a bad handle or
 * instance, UCAC_E_CUDA if a copy fails.
 */
int ucac_solution(const ucac_handle *h, int32_t instance, double *p, double *q, double *w, double *theta,
                  double *pf, uint8_t *u_on);

/*
 * Full iterate of one instance of the two-level ADMM of Sec. III-A (x, x-bar,
 * z, y, lambda, beta and the inner/outer counters of Algorithm 1; each
 * inner level starts from the previous one's iterate), in a fixed canonical
 * order of FP64 arrays
 * (all [T][n] with n the component count):
 *   17 generator fields  p q phat s_pl s_pu s_ql s_qu s_rd s_ru u_on u_su u_sd
 *                        pbar qbar ubar_on ubar_su ubar_sd
 *   y, z, lambda of the 12 generator rows  on su sd pl pu ql qu rd ru gp gq tc
 *   17 line fields       v0..v7 (w_i w_j wR wI theta_i theta_j sigma_ij
 *                        sigma_ji) mu0..mu3 c fbar0..fbar3
 *   y, z, lambda of the 8 line rows  p_ij q_ij p_ji q_ji w_i w_j th_i th_j
 *   2 bus fields         wbar thetabar
 *   12 scalars           beta, |z| at the last outer update (-1 if none),
 *                        inner sweep count, outer count, pending-outer flag,
 *                        next beta, stop flag (1 converged, 2 stopped on an
 *                        error status), the three current penalties, the
 *                        adaptive-penalty sweep counter and net step count.
 * ucac_state_size gives the number of doubles.  Export then import restores
 * the iterate bit for bit (resume / checkpoint).  buf is a caller host array
 * of n_doubles = ucac_state_size(h, instance) doubles (UCAC_E_ARG otherwise);
 * both calls synchronise the handle's stream.
 */
size_t ucac_state_size(const ucac_handle *h, int32_t instance);
int ucac_state_export(const ucac_handle *h, int32_t instance, double *buf, size_t n_doubles);
int ucac_state_import(ucac_handle *h, int32_t instance, const double *buf, size_t n_doubles);

/*
 * Runs n_sweeps sweeps with the kernels launched one by one (not from the
 * graph) and returns each kernel's average device time per sweep, timed
 * with CUDA events on the handle's stream; when n_sweeps >= 2 the first
 * sweep is untimed (it carries the first-launch costs of the one-by-one
 * launches), and each sweep is queued behind a ~0.2 ms device delay so that
 * no host launch latency enters the times.  ms[] receives UCAC_N_KERNELS values in the order of
 * ucac_kernel_name(): k_ucdp, k_gen, k_branch (the line kernel of either
 * form), k_bus, k_ucbar, k_finish, k_mlp (0 unless the learned warm start is
 * enabled).  Synchronises.
 */
#define UCAC_N_KERNELS 7
int ucac_kernel_times(ucac_handle *h, int32_t n_sweeps, double *ms);
const char *ucac_kernel_name(int32_t k);

/*
 * Autotuner (batching support; no counterpart in the paper).  Tries every
 * candidate block size of each sweep kernel in turn (32, 64, 128, 256
 * threads; the persistent line kernel 32, 64, 128) on the handle's own
 * workload: the sweep graph is re-captured with the candidate, the iterate
 * restored, and sweeps_per_trial replays after one warm-up replay are timed
 * with CUDA events on the handle's stream.  The objective is the whole
 * sweep, since the line kernel shares the GPU with the generator-side
 * branch of the graph.  Per kernel the current size is timed first and a
 * candidate replaces it only when the sweep is at least 1% faster.  Block sizes change
 * no result (work is split in warp-sized granules of one instance each), only
 * the speed.  cache_path (NULL: none) is a text file of lines
 *   <device name>|<instances>|<gen-periods>|<line-periods>|<bus-periods>|<line form> ucdp gen line bus ucbar
 * a matching entry is applied without timing; otherwise the result is
 * appended.  The iterate is unchanged on return.  Allocates a temporary copy
 * of the handle's device state.  out5 (may be NULL) receives the chosen sizes
 * {ucdp, gen, line, bus, ucbar}.  Synchronises.
 */
int ucac_autotune(ucac_handle *h, int32_t sweeps_per_trial, const char *cache_path, int32_t *out5);

/*
 * Standalone UC dynamic program (Algorithm 2) for n_gen generators over T
 * periods, on DEVICE arrays.  tau_on/tau_su/tau_sd [T][n_gen] are the targets
 * ubar - z - y/rho of the duplicate rows; c0, c_su, c_sd [n_gen]; TU, TD, u0,
 * K0 [n_gen] (K0 = forced initial periods).  Writes u_on [T][n_gen] (int8
 * 0/1) and cost [n_gen] (the optimal DP cost c_{1,u0}).  workspace is a device
 * buffer of at least ucac_ucdp_workspace_bytes(n_gen, T) bytes owned by the
 * caller (for up to 2,048 generators the kernel runs a warp per generator
 * with its scratch in shared memory and leaves the workspace untouched; the
 * results are the same bits either way).  Enqueued on cuda_stream; returns
 * without synchronising.
 */
size_t ucac_ucdp_workspace_bytes(int32_t n_gen, int32_t T);
int ucac_ucdp(int32_t n_gen, int32_t T, double rho_uc, const double *tau_on, const double *tau_su,
              const double *tau_sd, const double *c0, const double *c_su, const double *c_sd, const int32_t *TU,
              const int32_t *TD, const int32_t *u0, const int32_t *K0, int8_t *u_on, double *cost, void *workspace,
              size_t workspace_bytes, void *cuda_stream);

/*
 * Allocation-free variant of ucac_ucdp (the paper has no counterpart: this
 * is a deployment interface).  It is meant for callers that must not allocate
 * device memory on the call path -- for example a host runtime that fixes its
 * device footprint at start-up, a plugin that runs inside another
 * framework's memory pool, or a latency-critical loop where a cudaMalloc
 * would synchronise the device -- and that cannot hand over a workspace.
 * Inputs and outputs are the caller's device arrays exactly as for
 * ucac_ucdp; the scratch (stage costs, cost-to-go, decisions) lives in one
 * library-owned, statically sized device array of UCAC_UCDP_NOALLOC_MAX_BYTES
 * bytes, which every GPU that loads the library keeps until the process
 * exits.  Requests needing more than that (ucac_ucdp_workspace_bytes(n_gen,
 * T) > UCAC_UCDP_NOALLOC_MAX_BYTES) fail with UCAC_E_ARG and a message.
 * The call never allocates or frees device memory.  Its first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, once per
 * device, with that device current); make that first call before any stream
 * capture.  The address is kept for the life of the process: after
 * cudaDeviceReset (or anything else that destroys the device's primary
 * context) it is stale, and the entry point must not be called again on that
 * device.  Every call shares the one array and overwrites it; every scratch
 * entry is written before it is read within a call, so nothing needs to start
 * at zero, but two calls that overlap on the GPU (different streams, or
 * different host threads without ordering) race on the array and must be
 * serialised by the caller.
 */
#define UCAC_UCDP_NOALLOC_MAX_BYTES (16u << 20)
int ucac_ucdp_noalloc(int32_t n_gen, int32_t T, double rho_uc, const double *tau_on, const double *tau_su,
                      const double *tau_sd, const double *c0, const double *c_su, const double *c_sd,
                      const int32_t *TU, const int32_t *TD, const int32_t *u0, const int32_t *K0, int8_t *u_on,
                      double *cost, void *cuda_stream);

/*
 * UC warm start (Sec. IV-A: the UC variables start from a solve of the
 * multiperiod ACOPF, set to 0 or 1 by the generation levels).  Call right
 * after create: runs relax_sweeps sweeps with the UC subproblem relaxed to
 * the box (params.uc_relax = 1), marks unit g committed at period t when its
 * dispatch p_{t,g} >= p_frac * Pmin_g, repairs the minimum up/down times with
 * Algorithm 2 (zero costs, targets the marks and their start-up/shut-down
 * indicators: the feasible schedule nearest to the marks), and restarts every
 * instance from the cold start with that schedule as its UC variables (u and
 * its x-bar copy; y = z = lambda = 0, beta = beta0).  Sweep counters restart
 * at 0.  Synchronises.  Errors: UCAC_E_ARG, UCAC_E_CUDA.
 */
int ucac_uc_warm_start(ucac_handle *h, int32_t relax_sweeps, double p_frac);

/*
 * Learned warm start of the line subproblems (no counterpart in the paper,
 * which starts every line solve from the previous ADMM iterate).  A 12-64-64-6
 * MLP with SiLU activations maps 12 features of a line-period -- its voltage
 * magnitudes and angle difference at the previous iterate, the direction of
 * its series admittance, and the unit direction r / |r| of its target
 * residual r (flow residuals divided by |y|, w and angle residuals) -- to the
 * change of its W-form iterate (w_i, w_j, wR, wI, theta_i, theta_j) divided
 * by |r|.  Parameters are one flat FP32 vector of ucac_mlp_param_count()
 * values: W1 [64][12], b1 [64], W2 [64][64], b2 [64], W3 [6][64], b3 [6]
 * (row-major, output index first).
 *
 * ucac_mlp_forward: inference on the tensor cores (BF16 operands, FP32
 * accumulation, BF16 hidden activations) of n rows x [n][12] into y [n][6];
 * DEVICE pointers; workspace of ucac_mlp_workspace_bytes(n) bytes.
 * Synchronises; UCAC_E_CUDA if an mbarrier wait of the kernel timed out.
 * ucac_mlp_grad: FP32 loss (1/n) sum |y - labels|^2 into *loss and its
 * gradient into grad [param_count] (DEVICE pointers; sums over the batch in
 * sample order, so the result is reproducible).  Enqueued, not synchronised.
 * ucac_mlp_adam: one Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step >= 1)
 * on DEVICE params / moments m, v.  Enqueued, not synchronised.
 * ucac_line_features: features [T*n_branch][12] (FP32) and residual norms
 * |r| [T*n_branch] of instance k at the handle's current iterate, into HOST
 * buffers (training data: label = (x_after_sweep - x_before) / |r|).
 * ucac_set_warm_start: params (HOST, FP32) enable the learned start: every
 * sweep then runs the network over all line-periods before the line kernel,
 * and a line solve starts from the proposal when the proposal's objective
 * (slacks at their minimiser) is lower than the previous iterate's, as the
 * network kernel's epilogue estimates it in FP32 from the differences of the
 * objective's terms (polar form; the W-form line solver always starts from
 * the previous iterate).  NULL disables it.  Re-captures the sweep graph;
 * synchronises.
 * ucac_warm_start_stats: line solves of instance k started from the
 * proposal since the last ucac_set_warm_start; *mma_error (may be NULL) is
 * non-zero if a tensor-core wait timed out.
 */
int32_t ucac_mlp_param_count(void);
size_t ucac_mlp_workspace_bytes(int64_t n);
int ucac_mlp_forward(int64_t n, const float *params, const float *x, float *y, void *workspace,
                     size_t workspace_bytes, void *cuda_stream);
int ucac_mlp_grad(int64_t n, const float *params, const float *x, const float *labels, float *grad, float *loss,
                  void *workspace, size_t workspace_bytes, void *cuda_stream);
int ucac_mlp_adam(float *params, const float *grad, float *m, float *v, int32_t step, float lr, void *cuda_stream);
int ucac_line_features(const ucac_handle *h, int32_t instance, float *feat, double *scale);
/* Features [NBP][12], residual norms [NBP] and W-form iterates [NBP][6] of
 * every line-period of every instance (instance-major, then period, then
 * line), into HOST buffers; any of the three may be NULL.  Synchronises. */
int ucac_line_samples(const ucac_handle *h, float *feat, double *scale, double *iterate);
int ucac_set_warm_start(ucac_handle *h, const float *params);
/*
 * The same switch with the network given as a BF16 blob (no counterpart in
 * the paper): mlp_weights_bf16 holds the ucac_mlp_param_count() parameters
 * in the order above as IEEE bfloat16 bit patterns (uint16, host byte
 * order), bytes = 2 * ucac_mlp_param_count(); the library widens them to
 * FP32 exactly and proceeds as ucac_set_warm_start.  NULL with bytes = 0
 * disables the learned start.  UCAC_E_ARG for any other size.
 */
int ucac_set_warmstart(ucac_handle *h, const void *mlp_weights_bf16, size_t bytes);
int ucac_warm_start_stats(const ucac_handle *h, int32_t instance, int64_t *taken, int32_t *mma_error);

/*
 * Measures the device's FP64 fused multiply-add throughput (FLOP/s, 2 per
 * FMA) with a register-resident kernel; *flops receives the best of `reps`
 * runs.  Used as the arithmetic roofline of the FP64-bound kernels.
 */
int ucac_probe_fp64(int32_t reps, void *cuda_stream, double *flops);

/*
 * Evaluates the polar line kernel's cos/sin (double-word arithmetic: a table
 * of cos(k/256), sin(k/256) rotated by the Taylor series of the remainder) on
 * the device for n angles |d[i]| <= pi given in HOST memory (each truncated to
 * a double-word as the kernel does); c[i], s[i] (HOST) receive the results
 * widened to FP64.  For testing the kernel's trigonometry against a
 * reference.  Synchronises.  UCAC_E_ARG for n < 0 or a NULL buffer with n > 0.
 */
int ucac_probe_cossin(int32_t n, const double *d, double *c, double *s);

/*
 * Applies one double-word operation of the bus kernel (the FP32-pair
 * arithmetic that stands in for FP64 in its row updates) on the device to n
 * operand triples x[i], y[i], z[i] given in HOST memory, each first truncated
 * to a double-word: op 0 the conversion itself, 1 x + y, 2 x - y,
 * 3 x + (float)y, 4 x * y, 5 x * (float)y, 6 x^2, 7 x * y + z.  out (HOST,
 * 4 n doubles) receives per operand the result's high and low parts (op 0:
 * also their FP64 sum).  For testing the device arithmetic bit for bit
 * against the same code built for the host.  Synchronises.  UCAC_E_ARG for
 * an unknown op, n < 0 or a NULL buffer with n > 0.
 */
int ucac_probe_dw(int32_t op, int32_t n, const double *x, const double *y, const double *z, double *out);

/* Destroys the handle and frees its device memory (NULL is ignored). */
void ucac_destroy(ucac_handle *h);

/* Reason for the last error on this handle, or for the last failed create when h is NULL. */
const char *ucac_last_error(const ucac_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* UCAC_H */
