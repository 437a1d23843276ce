/*
 * egpe.h -- C ABI of the GB300 (sm_103a) eGPE ground-state solver hot path.
 *
 * The library evaluates and minimises the extended Gross-Pitaevskii energy of
 * a two-component dipolar Bose-Einstein condensate with Lee-Huang-Yang (LHY)
 * correction (arXiv:2510.24543, Eq. 1) on a periodic 3D grid, with the
 * preconditioned nonlinear conjugate-gradient method of its Algorithm 1.
 * Every step runs in hand-written CUDA kernels (Stockham FFTs fused with the
 * k-space multiplies, fused pointwise passes, deterministic reductions to FP64
 * values, an on-device controller).  No cuFFT and no host fallback.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Fields:  psi = (psi_1, psi_2) is one contiguous array of 2 complex fields,
 *          shape (2, nz, ny, nx), x fastest, interleaved (re, im).  Element
 *          type: complex128 (double2) for EGPE_FP64 and EGPE_MIXED handles,
 *          complex64 (float2) for EGPE_FP32 handles.  All field pointers are
 *          DEVICE pointers on the handle's device unless stated otherwise;
 *          the caller owns them; the library never frees them.
 * Grid:    periodic box [-L_a, L_a) with n_a points per axis, h_a = 2L_a/n_a,
 *          x_a[j] = -L_a + j h_a; wavenumbers k_a[j] = (pi/L_a)(j or j - n_a).
 *          Supported n_a: 16, 32, 48, 64, 80, 96, 128, 256.
 * Product: <a, b> = dV sum conj(a) b, dV = hx hy hz.
 * Model:   per-particle normalised couplings (N_i -> 1 in Eq. 1):
 *          E = sum_i <psi_i, T psi_i> + int V (n1+n2) + 1/2 int sum_ij g_ij n_i n_j
 *            + 1/2 int sum_i n_i Phi_i + int F_LHY,
 *          T = -Laplacian/2 (spectral), V = 1/2 sum_a trap_a^2 x_a^2,
 *          Phi_i = IDFT( gdd-kernel * DFT(sum_j gdd_ij n_j) ) with the k-space
 *          kernel gdd_ij (3 kz^2/|k|^2 - 1) and zero at k = 0 (dipoles along z),
 *          F_LHY = kappa eta_s^{-5/2} sum_q w_q sum_+- max(V_+-(u_q), 0)^{5/2}
 *          over a Q-point Gauss-Legendre rule on u in [0,1], with
 *          V_+- = eta11 n1 + eta22 n2 +- sqrt(delta^2 + 4 eta12 eta21 n1 n2),
 *          eta_ij(u) = g_ij + gdd_ij (3u^2 - 1)   (Sec. II, LHY branch potentials).
 * Gradient: H_i psi_i = T psi_i + (V + sum_j g_ij n_j + Phi_i + mu_LHY^(i)) psi_i
 *          (the coupled eGPE of Sec. II), so that
 *          d/de E(psi + e phi) = 2 sum_i Re <phi_i, H_i psi_i>.
 * Errors:  every function returns a status code; nothing aborts or throws.
 *          Arguments are validated before any launch (EGPE_ERR_INVALID_ARG).
 *          CUDA failures map to EGPE_ERR_CUDA (see egpe_last_error()).
 * Streams: all work is enqueued on the stream given to egpe_create; calls that
 *          return host scalars synchronise that stream before returning.  A
 *          handle created with a NULL stream works on a stream of its own and
 *          orders each call after the work already on the legacy default
 *          stream, and the legacy default stream after the call's work, so
 *          buffers written or read there by the caller need no extra
 *          synchronisation.  With a caller's stream, ordering against other
 *          streams is the caller's.
 */
#ifndef EGPE_H
#define EGPE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EGPE_OK = 0,
  EGPE_ERR_INVALID_ARG = 1,
  EGPE_ERR_CUDA = 2,
  EGPE_ERR_OOM = 3,
  EGPE_ERR_NONFINITE = 4,
  EGPE_ERR_NOT_CONVERGED = 5,
  EGPE_ERR_STAGNATED = 6,
  EGPE_ERR_TIMEOUT = 7,
  EGPE_ERR_UNSUPPORTED = 8
} egpe_status;

typedef enum { EGPE_FP64 = 0, EGPE_FP32 = 1, EGPE_MIXED = 2 } egpe_precision;

/* Preconditioner modes (Sec. IV.B). */
enum {
  EGPE_PRECOND_NONE = 0,            /* z = r                                  */
  EGPE_PRECOND_KINETIC = 1,         /* z = P_Delta^{-1} r                     */
  EGPE_PRECOND_DIAGONAL = 2,        /* z = P_V^{-1} r                         */
  EGPE_PRECOND_KINETIC_DIAGONAL = 3, /* z = P_Delta^{-1} P_V^{-1} r (formula order) */
  EGPE_PRECOND_BLEND = 4             /* z = w P_V^{-1} r + (1-w) P_Delta^{-1} r, w = pc_blend
                                        (the weighted combination of Sec. IV.B; 0.5 in
                                        egpe_precondition)                  */
};

/* Periodic box [-L_a, L_a), n_a points per axis (a = x, y, z). */
typedef struct {
  int n[3];
  double L[3];
} egpe_grid;

/* Couplings of Eq. 1 in per-particle normalised form. g and gdd must be
 * symmetric; gdd is the k-space dipolar coefficient. lhy_nodes in [1, 64]. */
typedef struct {
  double g[2][2];
  double gdd[2][2];
  double lhy_kappa;      /* kappa; the paper's literal prefactor is sqrt(2)/(15 pi^2) */
  double lhy_eta_scale;  /* eta_s > 0 (1 for the literal form)                       */
  int lhy_nodes;         /* Q                                                         */
  double trap[3];        /* (lambda_x, lambda_y, lambda_z)                            */
} egpe_params;

/* Energy terms and scalars of one evaluation (all FP64). */
typedef struct {
  double E;              /* total energy, Eq. 1                          */
  double kin[2];         /* Re <psi_i, T psi_i> (Parseval)               */
  double trap;           /* int V (n1 + n2)                              */
  double contact;        /* 1/2 int sum_ij g_ij n_i n_j                  */
  double dipolar;        /* 1/2 int sum_i n_i Phi_i                      */
  double lhy;            /* int F_LHY                                    */
  double mu[2];          /* mu_i = Re <psi_i, H_i psi_i> (Sec. III)      */
  double norm2[2];       /* ||psi_i||^2                                  */
  double shift[2];       /* alpha_i = mu_i - Re <psi_i, Phi_i psi_i>     */
} egpe_energy_terms;

/* One tuned launch shape (egpe_autotune / egpe_set_tuning). */
typedef struct {
  char key[160];            /* kernel instantiation (stable within one build)        */
  char name[48];            /* readable pass name                                   */
  int L;                    /* line length of the pass                              */
  int kind;                 /* 0 row pass: choice = rows per block; 1 column pass:
                               choice 1 = TMA-fed tile loads, 0 = plain loads;
                               2 (key "column tile row bytes"): choice = row width
                               of every column-pass tile, 64, 128 or 256 bytes     */
  int choice, default_choice;
  double ms_best, ms_default;  /* device ms of the attempt's launch sequence with the
                                  chosen and with the default choice (the earlier
                                  entries' choices applied)                         */
} egpe_tuning;

/* Options of egpe_ncg_solve (Algorithm 1 with the readings named below). */
typedef struct {
  int precond;              /* EGPE_PRECOND_*                                        */
  int beta_rule;            /* 0: Hestenes-Stiefel+, 1: Polak-Ribiere+ (Sec. IV.C)   */
  int restart_period;       /* K_r: beta = 0 when n mod K_r == 0                     */
  int max_iter;             /* accepted iterations                                   */
  int armijo_max;           /* halvings after a rejected step (Sec. V, last para.)  */
  int poll_every;           /* graph replays between host status polls              */
  int use_graph;            /* capture one attempt as a CUDA graph and replay it    */
  int psi_on_host;          /* psi_inout are HOST pointers (copied in and out)      */
  double tol_res;           /* stop when ||r|| = sqrt(sum_i <r_i, r_i>) < tol_res    */
  double tol_dE;            /* optional: stop when |E^{n+1} - E^n| < tol_dE (0 off) */
  double armijo_c1;         /* Armijo constant c1                                   */
  double theta_max;         /* cap of max_i theta_i (scales alpha)                  */
  double accept_rtol;       /* accept when E_trial < E + accept_rtol |E| (FP64)     */
  double accept_rtol_fp32;  /* the same allowance for FP32 fields                   */
  double pv_floor;          /* P_V >= pv_floor |alpha_i|                            */
  double tol_fp32_switch;   /* MIXED: FP32 phase ends when ||r|| < this             */
  int max_iter_fp32;        /* MIXED: cap of the FP32 phase                         */
  int trace_cap;            /* entries available in trace (0: no trace)             */
  void* trace;              /* HOST array of egpe_trace_entry, or NULL              */
  int batch;                /* n_inst > 1: 0 one instance after the other; 1
                               (default) all instances together, one launch per
                               pass for up to 16 instances of one grid shape, the
                               shapes' launches in sequence; 2 as 1 with the
                               launch chains of different grid shapes run as
                               concurrent branches of the replayed graph           */
  int stall_iters_fp32;     /* FP32 fields (FP32 handles, MIXED's FP32 phase): stop
                               when the best ||r|| has not dropped by 10% within this
                               many iterations (its round-off floor); 0: off       */
  double pc_blend;          /* EGPE_PRECOND_BLEND: weight w of P_V, in [0, 1]       */
} egpe_solve_opts;

/* One attempted step of the solver (accepted or rejected). */
typedef struct {
  int n;                    /* iteration index (accepted steps before this one)    */
  int kind;                 /* 0 analytic step, 1 Armijo step                       */
  int armijo;               /* halvings k for this attempt                          */
  int flags;                /* bit0 accepted, bit1 restart (beta = 0), bit2 residual
                               fallback, bit3 FP32 phase                             */
  double E, E_trial, res, beta, alpha, theta[2], Ep, Epp;
} egpe_trace_entry;

/* Result of egpe_ncg_solve, one per instance. */
typedef struct {
  int status;               /* EGPE_OK when converged                               */
  int iters;                /* accepted iterations (all phases)                     */
  int iters_fp32;           /* of which in the FP32 phase (MIXED)                   */
  int attempts;             /* trial evaluations                                    */
  int restarts;             /* iterations with beta = 0                             */
  int armijo_steps;         /* rejected trials                                      */
  int trace_len;            /* entries written to opts->trace                       */
  int graph_launches;       /* graph replays (or attempt sequences) issued          */
  double E;                 /* final energy                                         */
  double mu[2];             /* final chemical potentials                            */
  double res;               /* final ||r||                                          */
  double seconds;           /* wall time of the call                                */
  long long ffts;           /* complex 3D transforms executed                       */
  long long kernels;        /* kernel launches issued (including masked ones)       */
} egpe_report;

/* Parameters of egpe_param_grad's output, in this order: the contact couplings
 * g11, g12 (= g21, moved together), g22; the dipolar coefficients gdd11,
 * gdd12 (= gdd21), gdd22; the LHY prefactor kappa and scale eta_s; the trap
 * frequencies lambda_x, lambda_y, lambda_z. */
enum {
  EGPE_P_G11 = 0, EGPE_P_G12, EGPE_P_G22, EGPE_P_GDD11, EGPE_P_GDD12, EGPE_P_GDD22,
  EGPE_P_KAPPA, EGPE_P_ETA_S, EGPE_P_TRAP_X, EGPE_P_TRAP_Y, EGPE_P_TRAP_Z, EGPE_NPARAM
};

typedef struct egpe_handle egpe_handle;

/* Create a handle for n_inst instances (grids[i], params[i]) of the given
 * precision on the current CUDA device.  cuda_stream is a cudaStream_t, or
 * NULL for a stream owned by the handle and ordered against the legacy default
 * stream at every call (see Streams above).  Allocates every workspace up front (about 26
 * complex fields per instance and precision).  Errors: INVALID_ARG (bad sizes,
 * non-symmetric couplings, L <= 0, Q out of range), OOM, CUDA. */
egpe_status egpe_create(const egpe_grid* grids, const egpe_params* params, int n_inst,
                        egpe_precision prec, void* cuda_stream, egpe_handle** out);

/* Energy and gradient without any device allocation.  The paper has no
 * counterpart: this is a deployment variant of egpe_energy_grad for callers
 * that cannot allocate device memory -- applications whose device memory is
 * owned entirely by their own pool allocator (a cudaMalloc from a library
 * would fail or eat into a budget already handed out) and latency-sensitive
 * loops that must never enter the CUDA allocator -- and so cannot create a
 * handle (egpe_create allocates the workspaces).  Same kernels and arithmetic
 * as egpe_energy_grad on an EGPE_FP64 handle.  psi: complex128 device field
 * (2,nz,ny,nx), read only; grad: complex128 device output H_i psi_i or NULL;
 * E, mu: host outputs or NULL; cuda_stream: a cudaStream_t (NULL: the legacy
 * default stream); the call waits for its stream before returning.
 * Limit: 16 or 32 points per axis (at most 32^3 points); larger grids return
 * EGPE_ERR_INVALID_ARG with the reason in egpe_last_error().
 * Workspace: one fixed 4 MiB device array inside the library, held on every
 * GPU that loads the library until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) and
 * caches it; make that first call before any stream capture begins.  A device
 * reset (cudaDeviceReset) invalidates the cached address for the rest of the
 * process.  Every call shares the array and it keeps the last call's contents
 * (what must start at zero is cleared by each call): calls whose work overlaps
 * on the GPU race on it and must be serialised.  The call is synchronous: it
 * returns after E and mu are on the host.  The library cannot check the size
 * or element type of psi and grad: a buffer smaller than 2*nx*ny*nz complex128
 * values is read or written out of bounds. */
egpe_status egpe_energy_grad_noalloc(const egpe_grid* grid, const egpe_params* params, const void* psi,
                                     double* E, double mu[2], void* grad, void* cuda_stream);

/* Release every resource of the handle (NULL is a no-op). */
void egpe_destroy(egpe_handle* h);

/* Energy and gradient at psi (Eq. 1 and the coupled eGPE, Sec. II; mu_i of
 * Sec. III).  psi: device (2,nz,ny,nx) complex, read only.  E, mu: host
 * outputs (may be NULL).  grad: device output H_i psi_i, same layout, or NULL. */
egpe_status egpe_energy_grad(egpe_handle* h, int inst, const void* psi, double* E, double mu[2],
                             void* grad);

/* As egpe_energy_grad, returning every energy term (host struct). */
egpe_status egpe_energy_terms_eval(egpe_handle* h, int inst, const void* psi,
                                   egpe_energy_terms* terms, void* grad);

/* Partial derivatives of E (Eq. 1) with respect to its parameters at fixed
 * psi (device field of the instance's precision; the FP64 engine for MIXED
 * handles), written to dEdp[EGPE_NPARAM] (host):
 *   dE/dg_ii = 1/2 int n_i^2 + int dF/deta_ii,  dE/dg12 = int n1 n2 + int dF/deta12,
 *   dE/dgdd_ii = 1/2 int n_i (K*n_i) + int w dF/deta_ii,  dE/dgdd12 = int n1 (K*n2) + ...,
 *   dE/dkappa = E_LHY/kappa (NaN when kappa = 0), dE/deta_s = -5/2 E_LHY/eta_s,
 *   dE/dlambda_a = lambda_a int x_a^2 (n1 + n2),
 * with K the k-space dipolar kernel, w = 3u^2 - 1 and F the LHY density through
 * eta(u) = g + gdd w.  The paper has no such pass; at a normalised ground
 * state these are the derivatives of the ground-state energy
 * (Hellmann-Feynman).  Also the parameter half of the autograd binding. */
egpe_status egpe_param_grad(egpe_handle* h, int inst, const void* psi, double* dEdp);

/* Replaces the couplings, LHY constants and trap of instance inst (same grid
 * and precision; validated as in egpe_create).  Captured graphs are rebuilt;
 * the next call uses the new parameters. */
egpe_status egpe_set_params(egpe_handle* h, int inst, const egpe_params* params);

/* Coefficients of the energy along the geodesic psi_i(alpha) =
 * cos(alpha ||p_i||) psi_i + sin(alpha ||p_i||) p_i/||p_i|| (Sec. V):
 * coeffs[0] = E(psi), coeffs[1] = E'(0), coeffs[2] = E''(0).  p must be
 * tangent (Re<p_i, psi_i> = 0); it is not projected.  psi, p: device. */
egpe_status egpe_line_coeffs(egpe_handle* h, int inst, const void* psi, const void* p,
                             double coeffs[3]);

/* z = P^{-1} r at the state psi (Sec. IV.B), mode EGPE_PRECOND_*.  r == NULL
 * uses the residual r_i = H_i psi_i - mu_i psi_i of psi.  psi, r, z: device. */
egpe_status egpe_precondition(egpe_handle* h, int inst, int mode, const void* psi, const void* r,
                              void* z);

/* psi_out_i = (cos th_i psi_i + sin th_i p_i/||p_i||) / norm (Sec. III geodesic,
 * explicit renormalisation of Sec. V).  theta: host[2].  Device fields. */
egpe_status egpe_retract(egpe_handle* h, int inst, const void* psi, const void* p,
                         const double theta[2], void* psi_out);

/* Unnormalised 3D DFT (inverse: sign +, no 1/N) of nfields consecutive complex
 * fields of the instance's grid with the library's own Stockham kernels.
 * in and out may alias.  Device pointers.  A diagnostic of the transform that
 * every other entry point uses. */
egpe_status egpe_fft(egpe_handle* h, int inst, const void* in, void* out, int nfields, int inverse);

/* Diagnostic: device time of every kernel of one solver attempt
 * (precondition, line coefficients, trial evaluation: Algorithm 1 loop body),
 * measured with a CUDA event pair around each launch over `reps` attempts
 * started from psi (no graph).  engine: 0 the FP64 path (psi complex128), 1
 * the FP32 path (psi complex64); an engine the handle lacks is INVALID_ARG.
 * For each of the *count kernels (at most cap): names + 48 k holds a
 * NUL-terminated name, ms[k] the mean time per launch and bytes[k] the
 * algorithmic DRAM bytes per launch (fields read plus fields written).  All
 * output arrays are host memory owned by the caller. */
egpe_status egpe_profile_attempt(egpe_handle* h, int inst, int engine, const void* psi, int precond, int reps,
                                 int cap, char* names, double* ms, double* bytes, int* count);

/* Launch-shape autotuner (no counterpart in the paper: it picks how the
 * transforms of Sec. VI.B are tiled on this GPU).  Replays the launch sequence
 * of one attempt of the instance's engine (0 FP64, 1 FP32) from psi (device),
 * controller off, `reps` times per candidate, trying one choice at a time --
 * rows per block of each row pass, TMA-fed or plain loads of each column
 * pass, then the tile row width of all column passes -- and keeps a candidate
 * only if the sequence gets faster by more than 0.3%.  The choices stay in
 * the handle for every later call (captured graphs are rebuilt); up to cap
 * results go to out (host).  The arithmetic of each point does not change with
 * the shape (sums may regroup).  Leaves the instance's solver state reset. */
egpe_status egpe_autotune(egpe_handle* h, int inst, int engine, const void* psi, int precond, int reps,
                          egpe_tuning* out, int cap, int* count);

/* Applies tuned shapes (key and choice of each entry; host array) to the
 * instance's engine, e.g. from a cache of an earlier egpe_autotune of the same
 * build, device and grid.  Entries whose key the engine never launches are
 * ignored; out-of-range choices fall back to the untuned shape. */
egpe_status egpe_set_tuning(egpe_handle* h, int inst, int engine, const egpe_tuning* t, int count);

/* Diagnostic of the LHY interpolation tables that the energy/gradient and
 * line-search kernels use (no counterpart in the paper, which sums the
 * Gauss-Legendre rule at every point).  The LHY density is homogeneous of
 * degree 5/2 in (n1, n2), so mu_LHY,i = n^{3/2} m_i(a) and d^2F/dn_i dn_j =
 * n^{1/2} h_ij(a) with n = n1 + n2, a = sqrt(min(n1,n2)/n); the quadrature
 * sums m_i, h_ij over all but a few nodes are tabulated per parameter set as
 * piecewise polynomials in a, and the remaining nodes are evaluated exactly.
 * This host function builds the tables for params as the engine of the given
 * precision does (EGPE_FP64: degree 11, checked to 2e-15 of each function's
 * largest magnitude; EGPE_FP32: degree 7, checked to 1e-9) and evaluates
 * them from their unrounded coefficients, plus the exact nodes, in FP64 at
 * the count host points (n1[k], n2[k]) >= 0: mu (2 per point: mu_LHY,1,
 * mu_LHY,2) and hess (3 per point: d^2F/dn1^2, d^2F/dn1dn2, d^2F/dn2^2); info
 * (may be NULL) receives the intervals per half and the number of exactly
 * evaluated nodes.  All arrays are host memory.  Errors: INVALID_ARG (also
 * for a precision other than EGPE_FP64 or EGPE_FP32). */
egpe_status egpe_lhy_table_eval(const egpe_params* params, int precision, int count, const double* n1,
                                const double* n2, double* mu, double* hess, int info[2]);

/* Poll budget of the device-side waits of every engine of the handle (the
 * TMA tile loads of the column passes; default 2^20 polls, roughly a second).
 * No counterpart in the paper: a guard of this implementation.  A wait that
 * runs out of its budget lets the copies already issued land, marks the run
 * and returns; the call that launched it then reports EGPE_ERR_TIMEOUT (a
 * solve, in its report and return value), and the handle stays usable.  0
 * gives up before the first poll, which tests use to reach that path.
 * Captured graphs are rebuilt.  Errors: INVALID_ARG (NULL handle, polls < 0). */
egpe_status egpe_set_wait_limit(egpe_handle* h, long long polls);

/* Ground state by preconditioned NCG (Algorithm 1).  psi_inout[i] is the start
 * and receives the result for instance i (device pointers unless
 * opts->psi_on_host).  reports: host array of n_inst (may be NULL).
 * Returns the status of the first instance that did not converge, else OK.
 * With opts->batch and several instances, all instances advance together:
 * every pass of an attempt is one launch per group of up to 16 instances of
 * one grid shape; finished instances leave the launches at the next poll.
 * Each instance's arithmetic, controller and result are those of a solve of
 * that instance alone.  Reports then carry the shared wall time, graph
 * replays and kernel launches of the whole batch. */
egpe_status egpe_ncg_solve(egpe_handle* h, void* const* psi_inout, const egpe_solve_opts* opts,
                           egpe_report* reports);

/* Options of egpe_ite_solve. */
typedef struct {
  double dtau;              /* imaginary-time step (> 0)                             */
  double tol_dE;            /* stop once |E^{k+1} - E^k| < tol_dE (> 0)              */
  int max_steps;            /* step limit (> 0); reaching it is NOT_CONVERGED        */
  int poll_every;           /* steps enqueued between host checks of the stop flag   */
  int use_graph;            /* replay one captured step (1) or launch kernel by kernel */
  int psi_on_host;          /* psi_inout are host pointers                          */
} egpe_ite_opts;

/* Ground state by imaginary-time evolution, the baseline the paper compares
 * the NCG solver with (Sec. I; step counts and times in Sec. VI.B, stopping
 * rule |E^{k+1} - E^k| < tol of Sec. VI.A).  The paper does not state its ITE
 * scheme; this one is the Strang splitting
 *   psi <- e^{-dtau T/2} e^{-dtau U[psi']} e^{-dtau T/2} psi,  psi_i <- psi_i/||psi_i||,
 * with U_i = V + sum_j g_ij n_j + Phi_i + mu_LHY^(i) evaluated at the density
 * of psi' = e^{-dtau T/2} psi.  Runs in the handle's kernels (FP64 handles and
 * MIXED on the FP64 path, FP32 handles on the FP32 path); psi_inout[i] is the
 * start and receives the result (device pointers unless opts->psi_on_host).
 * reports (host, n_inst, may be NULL): iters = steps taken, E / mu / res of
 * the final state, ffts = 20 per step (two kinetic half steps of 4 transforms,
 * two evaluations of 6).  Errors: INVALID_ARG (dtau, tol_dE or max_steps not
 * positive), CUDA; per-instance NOT_CONVERGED / NONFINITE in the reports and
 * as the return value (first instance that failed). */
egpe_status egpe_ite_solve(egpe_handle* h, void* const* psi_inout, const egpe_ite_opts* opts,
                           egpe_report* reports);

/* Defaults: dtau 1e-3, tol_dE 1e-10, 100000 steps, poll every 32, graph on,
 * device pointers. */
void egpe_default_ite_opts(egpe_ite_opts* o);

/* Numerical continuation (named by the paper as the extension for
 * phase-diagram sweeps, Sec. VII): ground states of instance inst along a path
 * of parameter sets path[0..npoints) on its grid, each solve (as in
 * egpe_ncg_solve with opts) started from the previous ground state.
 * psi_inout: the start of the first solve; receives the last ground state.
 * psi_out: NULL, or npoints pointers (entries may be NULL) that receive each
 * point's ground state (same memory kind as psi_inout).  reports: host array
 * of npoints or NULL.  The instance keeps the last point's parameters.
 * Returns the first failing point's status (the path continues past it). */
egpe_status egpe_ncg_continuation(egpe_handle* h, int inst, const egpe_params* path, int npoints, void* psi_inout,
                                  void* const* psi_out, const egpe_solve_opts* opts, egpe_report* reports);

/* Stepping interface: the phases of egpe_ncg_solve one by one, for callers
 * that interleave their own work (event timing, checkpoints) with the solver.
 * engine: 0 the FP64 path (psi complex128), 1 the FP32 path (psi complex64;
 * the acceptance allowance is opts->accept_rtol_fp32); an engine the handle
 * lacks is EGPE_ERR_INVALID_ARG.  Options as in egpe_ncg_solve (the trace and
 * psi_on_host fields are ignored).
 * egpe_solver_start: copies psi (device) in, evaluates it and prepares the
 *   captured attempt; returns once the work is enqueued.
 * egpe_solver_step: enqueues `attempts` attempts of the loop body of
 *   Algorithm 1 (precondition, line coefficients, trial evaluation and the
 *   on-device controller); asynchronous; attempts after the solver has
 *   finished are no-ops on the device.
 * egpe_solver_read: waits for the stream, fills *report (status
 *   EGPE_ERR_NOT_CONVERGED while the solver is still running, res = ||r|| of
 *   the current point) and copies the current psi to psi_out (device; may be
 *   NULL). */
egpe_status egpe_solver_start(egpe_handle* h, int inst, int engine, const void* psi, const egpe_solve_opts* opts);
egpe_status egpe_solver_step(egpe_handle* h, int inst, int engine, int attempts);
egpe_status egpe_solver_read(egpe_handle* h, int inst, int engine, egpe_report* report, void* psi_out);

/* Defaults: kinetic preconditioner, HS+, K_r = 20, tol_res 1e-8, c1 1e-4,
 * 30 halvings, theta_max = pi/2, accept_rtol 1e-13 (FP64) / 1e-6 (FP32),
 * pv_floor 1e-2, graph replay with polls every 8 attempts, MIXED switch at
 * ||r|| < 1e-4, no FP32 stall limit, batched instances with the grid shapes'
 * launches in sequence (batch = 1). */
void egpe_default_solve_opts(egpe_solve_opts* opts);

/* Human-readable status; never NULL. */
const char* egpe_status_string(egpe_status s);

/* Message of the last CUDA error seen by this thread's calls ("" if none). */
const char* egpe_last_error(void);

/* ABI version (major * 100 + minor): 103. */
int egpe_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EGPE_H */
