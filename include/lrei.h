/*
 * lrei.h -- C ABI of the GB300 low-rank eigenmode-integration (LREI) stepper.
 *
 * The library time-steps the quantum Landau-Lifshitz (q-LL) and quantum
 * Landau-Lifshitz-Gilbert (q-LLG) equations for a spin-1/2 system of n spins
 * (N = 2^n) with a density matrix kept in factored form rho = V Lambda_0 V^*,
 * V an N x r matrix with orthonormal columns and Lambda_0 the fixed spectrum
 * (paper: Sec. 3.1 eq. partial-eigendecom and Sec. 3.6 "Memory-efficient
 * representation").  hbar = 1 throughout.
 *
 * Conventions shared by every entry point
 *  - Complex numbers are stored as interleaved (re, im) pairs: dtype
 *    LREI_C128 = two doubles, LREI_C64 = two floats.
 *  - An N x r factor is stored row-major: element (b, c) at offset b*ld + c,
 *    ld >= r; the r columns of one basis state b are contiguous.
 *  - Basis index b: site i (0-based) is Kronecker factor i from the left
 *    (Sec. 3.6 eq. spin_op), i.e. bit n-1-i of b; bit value 0 = spin up.
 *  - "_dev" pointers are CUDA device pointers; "_host" pointers are host
 *    memory.  The library copies every input it keeps; it never frees or
 *    retains caller memory.
 *  - Every call returns an int: LREI_OK (0) or a negative lrei_status code.
 *    No C++ exception crosses the ABI.  lrei_error_string() describes a code.
 *  - All work is enqueued on the stream given to lrei_create (NULL = legacy
 *    default stream).  Calls that return host data synchronise that stream.
 *  - One context must not be used from two threads at once.
 */
#ifndef LREI_H
#define LREI_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lrei_ctx lrei_ctx; /* opaque; owns all device memory it uses */

typedef enum {
  LREI_OK = 0,
  LREI_ERR_ARG = -1,         /* invalid argument (sizes, ranges, NULL) */
  LREI_ERR_UNSUPPORTED = -2, /* valid request outside this build (an AB basis wider than 160,
                              * the BF16-split precision) */
  LREI_ERR_NONFINITE = -3,   /* NaN/Inf in an input or produced by a step */
  LREI_ERR_TRACE = -4,       /* Lambda not >= 0 or |sum(Lambda) - 1| > 1e-12 */
  LREI_ERR_RANK = -5,        /* V rank-deficient */
  LREI_ERR_EIG_NOCONV = -6,  /* small eigensolver did not converge */
  LREI_ERR_OOM = -7,         /* device allocation failed */
  LREI_ERR_CUDA = -8,        /* other CUDA runtime error */
  LREI_ERR_STATE = -9,       /* call out of order (e.g. step before set_state) */
  LREI_ERR_TIMEOUT = -10,    /* a bounded device-side wait ran out */
  LREI_ERR_STEP = -11        /* adaptive step size fell below its floor (tolerance not reachable) */
} lrei_status;

typedef enum { LREI_QLL = 0, LREI_QLLG = 1 } lrei_model;

typedef enum {
  LREI_RK1 = 0, LREI_RK2 = 1, LREI_RK3 = 2, LREI_RK4 = 3,
  LREI_AB2 = 4, LREI_AB3 = 5, LREI_AB4 = 6
} lrei_scheme;

/* Arithmetic of the N-length (bulk) work.  Small r x r / k x k solves are
 * FP64 in every mode. */
typedef enum {
  LREI_FP64 = 0,        /* complex128 storage and arithmetic */
  LREI_MIXED_C64 = 1,   /* complex64 storage and FP32 arithmetic, FP64 small solves */
  LREI_MIXED_BF16X = 2  /* BF16-split tensor-core products: declared, not built in this version;
                         * lrei_create returns LREI_ERR_UNSUPPORTED for it */
} lrei_precision;

typedef enum { LREI_C128 = 0, LREI_C64 = 1 } lrei_dtype;

/* Exchange bonds of the spin Hamiltonian, eq. H1: each bond (i, j) contributes
 * 2*jxy*(S^x_i S^x_j + S^y_i S^y_j) + 2*jz*S^z_i S^z_j, i.e. a pair-flip amplitude jxy and a
 * diagonal +-jz/2; a Dzyaloshinskii-Moriya term along z is added by lrei_set_dmi.  Host
 * arrays, copied. */
typedef struct {
  int nbonds;
  const int *site_i, *site_j;
  const double *jxy, *jz;
} lrei_bonds;

/* Observables of the current state (Sec. 3.6 eq. measuerA). */
typedef struct {
  double t;          /* simulated time */
  double energy;     /* Tr(rho H) */
  double mx, my, mz; /* Tr(rho M_v), M_v = (1/n) sum_i S_i^v */
  double purity;     /* Tr(rho^2): Tr((Lambda_0 V^*V)^2) of the stored factor (see lrei_set_werner) */
  double trace;      /* Tr(rho): Tr(Lambda_0 V^*V) of the stored factor (see lrei_set_werner) */
  double orth_err;   /* max |V^*V - I| of the stored factor */
  double herm_err;   /* max |G - G^*| / max|G|, G = V^*HV */
  double comm_norm;  /* ||[rho, H]||_F */
  int r;             /* current rank */
  double ritz[64];   /* r largest eigenvalues of the last unprojected rho_{k+1} */
  double lambda0[64];/* the conserved spectrum, decreasing */
} lrei_obs;

/* Create a context for n spins (1 <= n <= 26).
 *   J       exchange bonds (eq. H1), site indices in [0, n)
 *   B       Zeeman field (B_x, B_y, B_z): H_Z = B . sum_i S_i (eq. H1's -mu b . S with the
 *           field in energy units); B_x, B_y flip single spins
 *   lambda  damping kappa >= 0 of eqs. q-LL / q-LLG
 *   r_max   largest rank the context will hold (1..32)
 *   cuda_stream  cudaStream_t (may be NULL)
 * Allocates all device memory the context needs for ranks <= r_max. */
int lrei_create(int n, const lrei_bonds *J, const double B[3], double lambda,
                lrei_model model, lrei_precision prec, int r_max,
                void *cuda_stream, lrei_ctx **out);

/* Set rho_0 = V diag(Lambda) V^* from any full-column-rank V (N x r, device,
 * row stride ld, dtype LREI_C128 or LREI_C64) and Lambda (host, r values >= 0
 * summing to 1).  The library orthonormalises V (Cholesky QR), diagonalises
 * R Lambda R^* and stores (V~, Lambda_0) with Lambda_0 decreasing (Sec. 3.1,
 * Sec. 3.7 "Given the sparse initial density matrix ...").  Resets t to 0 and
 * clears any multistep history. */
int lrei_set_state(lrei_ctx *ctx, const void *V_dev, int r, int ld, int dtype,
                   const double *Lambda_host);

/* Copy the current factor out (N x r, row-major, ld = r, dtype of the
 * context's precision: C128 for LREI_FP64, C64 for LREI_MIXED_C64), the
 * spectrum Lambda_0 (r doubles) and t.  Any pointer may be NULL. */
int lrei_get_state(lrei_ctx *ctx, void *V_dev_out, double *Lambda_host_out,
                   double *t_out);

/* Advance nsteps fixed steps of size dt with an LREI-RK (Sec. 3.7) or LREI-AB
 * (Sec. 3.8) scheme.  AB_m takes its first m-1 steps with RK4 and keeps its
 * history across calls while scheme and dt stay the same. */
int lrei_step(lrei_ctx *ctx, double dt, lrei_scheme scheme, int nsteps);

/* Advance to t_end with RK4 and an adaptive step (the adaptive stepping Sec. 6 names as
 * future work): controller 0 = the plain rule (local error = calibrated spectral drift of
 * the unprojected rho_{k+1}, step doubling as judge every judge_every steps and after a
 * rejection, h_new = h clip(0.9 (tol/err)^(1/5), 0.2, 5)); 1 = the learned controller (the
 * attached network estimates the local error from the step's features, scaled by a factor
 * refitted at every judge; judged every 4 judge_every steps, after a rejection, and when its
 * estimate is far below the calibrated drift; a judge that finds the error more than 3x above
 * the estimate hands control to the plain rule for 16 steps).  tol bounds the relative local
 * error per step; it is raised to the
 * rounding floor of the context's precision (LREI_TOL_FLOOR_FP64,
 * LREI_TOL_FLOOR_MIXED), below which the step-doubling estimate is noise.
 * Returns LREI_ERR_STEP, with the state of the last accepted step kept, when
 * the step size falls below 1e-12 * max(1, |t_end|) or 64 steps in a row
 * are rejected. */
#define LREI_TOL_FLOOR_FP64 1e-13
#define LREI_TOL_FLOOR_MIXED 1e-6
int lrei_step_adaptive(lrei_ctx *ctx, double t_end, double tol, int controller);

/* Compute observables of the current state into a host struct (Sec. 3.6: Tr(A rho) for
 * A = H, M_x, M_y, M_z; Tr rho, Tr rho^2, ||[rho, H]||_F; the Ritz values of the last step and
 * the conserved spectrum; ||V^*V - I|| and the Hermiticity error of V^*HV as diagnostics).
 * Uses the context's step buffers as scratch (no allocation) and syncs the context's stream.
 * Returns LREI_ERR_STATE before set_state. */
int lrei_observables(lrei_ctx *ctx, lrei_obs *out);

/* Dzyaloshinskii-Moriya vectors along z (eq. H1: 2 d_ij . (S_i x S_j) with d_ij = dz[b] e_z for
 * bond b = (i, j) of lrei_create, in its order; d_ji = -d_ij).  The bond's flip part becomes
 * (jxy + i dz) S^+_i S^-_j + (jxy - i dz) S^-_i S^+_j.  nbonds must equal the bond count given
 * to lrei_create; dz = 0 everywhere restores the plain exchange.  Clears any multistep
 * history; the stored state and t are kept. */
int lrei_set_dmi(lrei_ctx *ctx, int nbonds, const double *dz);

/* Werner-state initial data (Sec. 5, eq. werner-sol).  With weight p in [0, 1) the state is
 * rho = p I/N + (1 - p) rho_hat, where rho_hat = V Lambda_0 V^* is the stored low-rank state.
 * The q-LL and q-LLG flows keep that form, rho_hat following the same equation with the
 * damping kappa replaced by (1 - p) kappa; so after this call every step uses (1 - p) kappa
 * (kappa as given to lrei_create), and lrei_observables reports the observables of rho
 * itself: energy, magnetisations and ||[rho, H]|| scaled by 1 - p (H and M_v are traceless),
 * trace p + (1 - p) Tr rho_hat, purity p^2/N + 2 p (1 - p) Tr(rho_hat)/N + (1 - p)^2 Tr rho_hat^2,
 * and ritz / lambda0 mapped to p/N + (1 - p) mu.  orth_err and herm_err stay those of the
 * stored factor.  p = 0 restores the plain problem.  Clears any multistep history; the
 * stored state and t are kept.  p outside [0, 1) or not finite returns LREI_ERR_ARG. */
int lrei_set_werner(lrei_ctx *ctx, double p);

/* Free the context and all device memory it owns. */
int lrei_destroy(lrei_ctx *ctx);

const char *lrei_error_string(int code);

/* ---- entry points exposing single steps of the hot path ---------------- */

/* Y = H V for an N x r block (matrix-free action of eq. H1 on basis
 * bitstrings; Sec. 3.3 "sparsity of H").  V_dev, Y_dev device, row-major with
 * ld = r, dtype must match the context's precision.  V_dev != Y_dev. */
int lrei_apply_h(lrei_ctx *ctx, const void *V_dev, void *Y_dev, int r);

/* Tall-skinny Gram P = [B_0, ..., B_{m-1}]^* B_{m-1} (the V^*W-type products of
 * Sec. 3.5-3.7: projections onto the current basis and the Gram of the newest
 * block), by the same fused tile pass and deterministic reduction the step uses.
 * blocks_dev: m device pointers (1 <= m <= 13), each N x r row-major with the
 * context's r and precision; G_dev: device complex128 (m r) x r, column-major,
 * written on the context's stream (no host sync).  Compensated FP32 sums in
 * mixed precision, FP64 otherwise. */
int lrei_gram(lrei_ctx *ctx, const void *const *blocks_dev, int nblocks, void *G_dev);

/* Low-rank right-hand side at the current state: f(rho) = Z V^* + V W^*
 * (Sec. 3.5 eq. q-LLG-low-rank; q-LL blocks of Sec. 4).  Writes Z and W
 * (N x r each, device, ld = r, the context's dtype) and, if G_host is not
 * NULL, G = V^*HV (r x r complex, column-major, 2*r*r doubles).
 * complement: 0 = projector form W = (I - VV^*) H V diag(conj c),
 *             1 = Householder reflectors of V applied as in Sec. 3.4
 *                 (compact WY form). */
int lrei_rhs(lrei_ctx *ctx, void *Z_dev, void *W_dev, double *G_host,
             int complement);

/* The r Householder reflectors that triangularise the current factor (Sec. 3.4,
 * eq. Householder-mat) in compact WY form Q = P_1 ... P_r = I - U T U^H:
 * U (N x r, device, row-major, context dtype, unit lower trapezoidal) into U_dev,
 * T (r x r upper triangular, complex column-major, 2 r^2 doubles) and D (r complex)
 * into host arrays, with Q[:, :r] = V diag(D), so the complement of V is Q[:, r:].
 * Requires r < N. */
int lrei_householder(lrei_ctx *ctx, void *U_dev, double *T_host, double *D_host);

/* Two-spin reduced density matrices (Sec. 3.6): for each pair (site_k[q], site_l[q]), k != l,
 * R_kl = Tr over every other spin of rho, the 4 x 4 matrix in the basis |s_k s_l> (index
 * 2 s_k + s_l, site k the first factor, s = 0 spin up), written to R_host + 32 q as complex
 * column-major (element (i, j) at 2 (4 j + i)); and, from R_kl in FP64, the concurrence
 * max(0, s1 - s2 - s3 - s4) (s_i the decreasing square roots of the eigenvalues of R Rt,
 * Rt = (Y x Y) conj(R) (Y x Y); Wootters 1998) and the negativity (minus the sum of the
 * negative eigenvalues of the partial transpose on spin l; Vidal and Werner 2002).  With a
 * Werner weight p (lrei_set_werner) the results are those of p I/N + (1 - p) rho_hat, whose
 * reduced matrix is p I/4 + (1 - p) R_hat.  Host arrays; R_host, concurrence_host and
 * negativity_host may each be NULL.  1 <= npairs <= LREI_RDM_MAX_PAIRS; sites in [0, n).
 * One pass over the factor per pair (plus one to orthonormalise it); syncs the stream. */
#define LREI_RDM_MAX_PAIRS 4096
int lrei_two_spin_rdm(lrei_ctx *ctx, int npairs, const int *site_k, const int *site_l, double *R_host,
                      double *concurrence_host, double *negativity_host);

/* Rank rule of the plain step/rank controller (the adaptive control Sec. 6 names as future
 * work): drop the trailing eigenvalues of Lambda_0 (the smallest) while their cumulative weight
 * w stays <= tol_r (at least one is kept), remove the matching columns of the factor, and
 * renormalise the kept weights to trace one.  The state changes by ||rho - rho'||_1 <= 2 w, so
 * every observable <A> moves by at most 2 w ||A||.  Lambda_0 is conserved by the q-LL and
 * q-LLG flows (Sec. 3), so the rule gives the same answer at any time and one call suffices.
 * Writes the new rank to *r_out and w to *dropped_out (either may be NULL).  Clears any
 * multistep history.  tol_r < 0 or not finite returns LREI_ERR_ARG. */
int lrei_truncate_rank(lrei_ctx *ctx, double tol_r, int *r_out, double *dropped_out);

/* Checkpoint and resume.  lrei_checkpoint_save writes into host memory everything the next steps
 * read, as stored: the factor V (not re-orthonormalised), Lambda_0, the last Ritz values, the
 * leading r x r blocks of the measured Gram V^*V and of its Cholesky factor, t, the Werner
 * weight, the adaptive controller's step and calibration, and an Adams-Bashforth history (its
 * (V_l, H V_l) pairs, scheme and dt).  lrei_checkpoint_load restores it into a context created
 * with the same n, bonds, field, kappa, model and precision (and r_max >= r); the integration
 * then continues bit for bit as in the saved context (all reductions have a fixed order).
 * lrei_checkpoint_bytes gives the size (0 without a state); a smaller buffer, another layout or
 * a mismatching context returns LREI_ERR_ARG.  Both sync. */
long long lrei_checkpoint_bytes(lrei_ctx *ctx);
int lrei_checkpoint_save(lrei_ctx *ctx, void *buf_host, long long bytes);
int lrei_checkpoint_load(lrei_ctx *ctx, const void *buf_host, long long bytes);

/* Sweep limit (1..100, default 30) of the FP64 Jacobi that finishes each partial
 * eigendecomposition (the Rayleigh-Ritz on the top-r subspace).  A step whose small eigenproblem
 * needs more sweeps, or whose eigenpair residual stays above its tolerance, returns
 * LREI_ERR_EIG_NOCONV with status bit 2 or 32 set. */
int lrei_set_eig_sweeps(lrei_ctx *ctx, int max_sweeps);

/* ---- many trajectories side by side ------------------------------------ */
/* A batch runs the RK4 steps of many contexts (trajectories of uneven n, r, kappa, model and
 * precision, each with its state set) as one CUDA graph launch per step: the graph holds every
 * context's captured step as a child graph with no edges between them, so the GPU runs the
 * trajectories side by side.  The contexts stay owned by the caller, must outlive the batch,
 * and must not be used from another thread while a batch call runs; changing a context's
 * model (lrei_set_dmi, lrei_set_werner, lrei_set_eig_sweeps) or rank requires a new batch.
 * All work runs on cuda_stream (may be NULL), ordered after each context's own stream. */
typedef struct lrei_batch lrei_batch;
int lrei_batch_create(int nctx, lrei_ctx *const *ctxs, void *cuda_stream, lrei_batch **out);
/* Advance every trajectory of the batch by nsteps RK4 steps of size dt; syncs and returns the
 * first failing trajectory's error code (each context's lrei_last_status has its own bits). */
int lrei_batch_step(lrei_batch *b, double dt, int nsteps);
/* Autotuner of the batch's launch shape: for SM shares nsm, nsm/2, nsm/4, ... (down to a few
 * SMs), every trajectory's persistent grids are sized to that share, the batch graph is rebuilt
 * and `steps` batch steps of size dt are timed; the fastest share is kept and written to
 * *nsm_out with its time per batch step (ms) to *ms_out (either may be NULL).  The timed steps
 * advance the trajectories (t included); set the states again to start over. */
int lrei_batch_autotune(lrei_batch *b, double dt, int steps, int *nsm_out, double *ms_out);
int lrei_batch_destroy(lrei_batch *b);

/* Raw device status bits of the last step / set_state call (diagnostics):
 * 1 non-finite, 2 small eigensolver sweep limit, 4 rank-deficient factor,
 * 8 bounded wait ran out, 16 trace, 32 eigenpair residual above tolerance. */
int lrei_last_status(lrei_ctx *ctx);

/* Cumulative small-eigensolver counters of this process on the current device
 * (diagnostics): FP32 Jacobi calls, their sweeps, FP64 Jacobi calls, their sweeps. Syncs. */
int lrei_debug_counters(unsigned long long *out4);

/* Number of kernels this library launched on the context's stream since the
 * last call (resets the counter). */
long long lrei_kernel_launches(lrei_ctx *ctx);

/* ---- observables without device allocation ---------------------------- */
/* For callers that cannot allocate device memory: hosts whose own allocator has reserved all of
 * it (a framework's caching pool, a fixed memory budget) and monitoring loops that must not
 * pay an allocation's latency or fragment the heap on every call.  Computes the observables of
 * rho = V diag(Lambda) V^* exactly as lrei_observables does for a context holding the same
 * factor, but without a context: n, J and B describe the Hamiltonian as in lrei_create (same
 * argument checks and error codes), V_dev is the N x r factor (row-major, ld = r, dtype
 * LREI_C128 or LREI_C64), Lambda_host its r weights.  ritz and t are left zero.
 * The paper has no counterpart: this is a deployment variant of the observable pass.
 * Scratch memory is one static device array of about 3.8 MB inside this library; nothing is
 * allocated per call.  The array is committed when the library's device code is loaded on a
 * device, which happens at the first call on that device (CUDA loads modules lazily by
 * default), so make the first call before the caller's own allocator reserves device memory,
 * and before any stream capture; the array is then held until the process exits.  Each call
 * looks the array's device address up with the device current (no caching across context
 * resets).  Every part of the array a call reads is first written by that call, so no part
 * of it has to start at zero.  All calls share the array: calls that overlap on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 * r > LREI_NOALLOC_MAX_R returns LREI_ERR_ARG.  Syncs the stream. */
#define LREI_NOALLOC_MAX_R 16
int lrei_observables_noalloc(int n, const lrei_bonds *J, const double B[3], const void *V_dev, int r,
                             int dtype, const double *Lambda_host, void *cuda_stream, lrei_obs *out);

/* ---- step/rank controller network ------------------------------------- */
/* A three-layer FP32 perceptron y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3,
 * hidden width 128, trained on the GPU by its own backward and Adam kernels.
 * It is the learned form of the adaptive time stepping the paper names as
 * future work (Sec. 6); the paper itself has no network.  Parameters are one
 * float buffer [W1 | b1 | W2 | b2 | W3 | b3], each W row-major (out x in).
 * All buffers named _dev are device float arrays, row-major (batch x features). */
typedef struct lrei_mlp lrei_mlp;

/* n_in in [1, 4096], n_out in [1, 64]; params_host may be NULL (all zero). */
int lrei_mlp_create(int n_in, int n_out, const float *params_host, void *cuda_stream, lrei_mlp **out);
int lrei_mlp_destroy(lrei_mlp *net);
int lrei_mlp_num_params(const lrei_mlp *net);
int lrei_mlp_get_params(lrei_mlp *net, float *host, int n);  /* syncs */
int lrei_mlp_set_params(lrei_mlp *net, const float *host, int n);  /* resets Adam moments; syncs */
/* Y (batch x n_out) = network(X (batch x n_in)). */
int lrei_mlp_forward(lrei_mlp *net, const float *X_dev, int batch, float *Y_dev);
/* Gradients of L = (1/2B) sum_b sum_o w_o (y_bo - t_bo)^2 into the network's gradient buffer;
 * optionally copied to grad_dev (num_params floats) and the loss to *loss_host (syncs).
 * w_host: n_out output weights or NULL (all one). */
int lrei_mlp_grads(lrei_mlp *net, const float *X_dev, const float *T_dev, const float *w_host, int batch,
                   float *grad_dev, float *loss_host);
/* One Adam update with the last computed gradients (Kingma and Ba, 2015). */
int lrei_mlp_adam(lrei_mlp *net, float lr, float beta1, float beta2, float eps);

/* ---- adaptive step controller ------------------------------------------ */
/* Features per step (LREI_CTRL_NFEAT floats): log10 of the 32 (padded) spectrum values,
 * the spectral drift of the unprojected rho_{k+1}, h, ||[rho,H]||_F^2, the stage-to-stage
 * change of G = V^*HV, kappa, the model, the tolerance and r/32 (each scaled to O(1)). */
#define LREI_CTRL_NFEAT 40

typedef struct {
  long long accepted, rejected, judged; /* steps; judged = step-doubling checks */
  long long rk4_steps;                  /* RK4 steps executed, including judges and rejects */
  double h;                             /* step proposed for the next call */
  double err_judged;                    /* last step-doubling error estimate */
  double calib;                         /* drift-to-error calibration factor */
} lrei_ctrl_stats;

/* judge_every: step-doubling period of the plain judge (>= 1); record != 0 keeps one row per
 * attempted step (features, h, drift, judged error or -1, accepted); h0 > 0 sets the first step.
 * Resets the statistics and the record. */
int lrei_controller_config(lrei_ctx *ctx, int judge_every, int record, double h0);
/* Network used by lrei_step_adaptive(..., controller = 1); output 0 is log(err / drift), the
 * natural log of the step's local error over the spectral drift of the unprojected rho_{k+1}. */
int lrei_controller_attach(lrei_ctx *ctx, lrei_mlp *net);
int lrei_controller_stats(lrei_ctx *ctx, lrei_ctrl_stats *out);
/* Copies up to max_rows rows of LREI_CTRL_NFEAT + 4 doubles; *n_rows = rows recorded. */
int lrei_controller_records(lrei_ctx *ctx, double *rows, int max_rows, int *n_rows);

#ifdef __cplusplus
}
#endif
#endif /* LREI_H */
