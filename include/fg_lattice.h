/*
 * fg_lattice.h -- C ABI of the GB300 force-gradient Hybrid Monte Carlo library.
 *
 * The library runs the molecular-dynamics (MD) step of Hybrid Monte Carlo for
 * 4D SU(3) lattice gauge theory with the integrators of Kennedy, Clark and
 * Silva, "Force Gradient Integrators" (LAT2009):
 *
 *   - the Wilson gauge staple force and the momentum kick exp(c dt S-hat)
 *     (section 3; S-hat is "the force");
 *   - the exact link drift exp(c dt T-hat), U <- exp(i c dt P) U (section 2);
 *   - the force-gradient kick exp((48 dt S-hat - dt^3 {S,{S,T}}-hat)/72) of
 *     Table 1, evaluated as the force at links displaced along the force by
 *     dt^2/24 (section 4 gives {S,{S,T}} = e^i(S) e_i(S));
 *   - the kinetic term and the action sums behind dH (section 5, Fig. 1);
 *   - for Nf = 2 Wilson fermions: the even-odd preconditioned Wilson-Dirac
 *     operator, CG on Mhat^dagger Mhat and the pseudofermion force
 *     e_i(S) = -X^dagger e_i(M) X, X = M^{-1} phi (section 4, section 5).
 *
 * Conventions (the paper leaves them open; these are fixed here):
 *   - lattice dims {Lx, Ly, Lz, Lt}, each even and >= 2; V = Lx Ly Lz Lt;
 *     lexicographic site index i = x + Lx (y + Ly (z + Lz t)); links periodic,
 *     fermions antiperiodic in t;
 *   - Wilson gauge action S_G = beta sum_{x, mu<nu} (1 - Re Tr U_{mu nu}(x) / 3);
 *   - momenta P = sum_a p^a lambda^a / 2 (Gell-Mann), T = (1/2) sum (p^a)^2;
 *   - the force on a link is F^a = dS / d eps^a along U -> exp(i eps lambda^a/2) U;
 *     a kick is p^a <- p^a - c dt F^a, a drift is U <- exp(i c dt P) U;
 *   - Wilson-Dirac M = 1 - kappa D, D = sum_mu [(1 - gamma_mu) U_mu(x) d_{x+mu}
 *     + (1 + gamma_mu) U_mu(x-mu)^dagger d_{x-mu}], DeGrand-Rossi gammas;
 *     Mhat = 1 - kappa^2 D_eo D_oe on even sites; S_F = phi^dagger
 *     (Mhat^dagger Mhat)^{-1} phi with phi = Mhat^dagger chi.
 *
 * Host array layouts (all FP64, owned by the caller, copied by the library):
 *   gauge    double[V][4][3][3][2]  site (lexicographic), mu, row, col, re/im
 *   momenta  double[V][4][8]        Gell-Mann coefficients p^a per link
 *   force    double[V][4][8]        F^a per link
 *   spinor   double[V/2][4][3][2]   even sites in increasing lexicographic
 *                                   order (row = lexicographic index / 2),
 *                                   spin, colour, re/im
 *
 * Ownership and threading: a handle owns all of its device memory and one
 * CUDA stream (or uses the caller's stream given in fg_params.cuda_stream).
 * A handle is used by one host thread at a time; different handles are
 * independent.  Every call is stream-ordered on the handle's stream and
 * returns after the results it reports are on the host.
 *
 * Errors: every entry point returns an fg_status; nothing aborts.  On an
 * error fg_last_error() holds a one-line description.  FG_ECUDA reports a
 * CUDA runtime error (the handle should then be destroyed).
 */
#ifndef FG_LATTICE_H
#define FG_LATTICE_H

#ifdef __cplusplus
extern "C" {
#endif

#define FG_ABI_VERSION 1

typedef struct fg_lattice fg_lattice;   /* opaque handle */

typedef enum {
  FG_OK = 0,
  FG_EINVAL = 1,     /* bad argument (null pointer, odd dims, bad enum, ...) */
  FG_ENOMEM = 2,     /* device or pinned-host allocation failed */
  FG_ECUDA = 3,      /* CUDA runtime error */
  FG_ENOCONV = 4,    /* CG reached cg_maxiter without converging */
  FG_ETIMEOUT = 5,   /* a host wait exceeded its limit (fg_set_wait_limit) */
  FG_ESTATE = 6      /* call not valid in the handle's state (e.g. no pseudofermion) */
} fg_status;

/* Integrators of Table 1 / section 3.  One MD step of each, in order:
 *   FG_LEAPFROG        PQP:   kick 1/2, drift 1, kick 1/2
 *   FG_OMELYAN         PQPQP: kick a, drift 1/2, kick 1-2a, drift 1/2, kick a
 *   FG_FORCE_GRADIENT  kick 1/6, drift 1/2, force-gradient kick 2/3, drift 1/2, kick 1/6
 *   FG_CAMPOSTRINI     drift w1/2, kick w1, drift (w1+w0)/2, kick w0, drift
 *                      (w1+w0)/2, kick w1, drift w1/2; w1 = 1/(2-2^(1/3)), w0 = 1-2 w1
 *   FG_QPQ             drift 1/2, kick 1, drift 1/2
 *   FG_FORCE_GRADIENT_ANALYTIC  the FG_FORCE_GRADIENT step with G in closed form
 * (kick c means exp(c dt S-hat), drift c means exp(c dt T-hat)).  The
 * force-gradient kick of Table 1 is a kick with F - (dt^2/24) G, G the
 * derivative of the force F along the vector field e^j(S) e_j (section 4).
 * FG_FORCE_GRADIENT evaluates it as the force at links displaced along the
 * force, F(exp(-i (dt^2/24) F) U) (one extra force evaluation, equal to
 * O(dt^4)); FG_FORCE_GRADIENT_ANALYTIC computes G itself, through the
 * staples by the product rule and, with fermions, with the second solve
 * Y = -calM^{-1} F(calM) X of section 4 (one extra solve, the same count). */
typedef enum {
  FG_LEAPFROG = 0,
  FG_OMELYAN = 1,
  FG_FORCE_GRADIENT = 2,
  FG_CAMPOSTRINI = 3,
  FG_QPQ = 4,
  FG_FORCE_GRADIENT_ANALYTIC = 5
} fg_integrator;

/* Arithmetic of the bulk fields (links, momenta, forces, CG inner vectors).
 * Action, kinetic and dH sums and the CG outer residual are FP64 always.
 * FG_FP32_FP16CG is FG_FP32 whose inner CG iterates in half precision: the
 * Dslash reads a half-precision copy of the links (made at the start of
 * every solve; entries of SU(3) matrices lie in [-1, 1], so no scale is
 * needed), and the residual, search direction and Dslash temporaries are
 * stored as half precision scaled by 1/sigma, sigma^2 = |r|^2 / n reset at
 * every reliable update (the solution increment stays FP32, arithmetic is
 * FP32).  The reliable updates, on the FP32 links in double-float and FP64,
 * correct the ~5e-4 relative error of the inner operator; they come at least
 * every factor 0.1 of residual reduction, whatever cg_delta says.
 * FG_DF64 ("double-float") stores every real of the links and momenta as an
 * unevaluated sum hi + lo of two floats (about 48 significant bits, the same
 * 8 bytes as FP64) and computes the staples, force, kicks, exponential and
 * action sums in double-float arithmetic on the FP32 pipes (error-free FMA
 * products and two-sums), with no FP64 instruction in the MD step: on a
 * GB300 the FP64 unit runs at 1/64 of the FP32 rate.  It serves the dH of
 * a trajectory (section 5, Fig. 1), whose error against FP64 arithmetic
 * grows with the rounding of every MD operation: ~2^-47 relative here, 2^-24
 * with FP32 fields.  Momentum refreshes draw FP32 Gaussians (exact as
 * double-floats).  Pure gauge only: kappa must be 0.
 * FG_FP32_AUTOCG is FG_FP32_FP16CG when the FP32 inner solver's working set
 * (links and six half-lattice spinors, (4 NC 8 + 6 48) V bytes for NC
 * complex entries per link) exceeds the GPU's L2 cache, and FG_FP32
 * otherwise: below that size the fields stay in L2, half precision saves no
 * memory traffic and its extra reliable updates cost time.
 * FG_FP32_BF16CG is FG_FP32_FP16CG with bfloat16 in place of IEEE half for
 * the inner links and vectors: the same bytes, the exponent range of FP32,
 * 8 instead of 11 significant bits (unit roundoff 2^-8, ~4e-3 relative
 * error of the inner operator), so the reliable updates have more to
 * correct. */
typedef enum {
  FG_FP64 = 0,
  FG_FP32 = 1,
  FG_FP32_FP16CG = 2,
  FG_DF64 = 3,
  FG_FP32_AUTOCG = 4,
  FG_FP32_BF16CG = 5
} fg_precision;

typedef struct {
  int dims[4];             /* Lx, Ly, Lz, Lt; each even, >= 2; volume <= 2^28 sites */
  double beta;             /* gauge coupling */
  double kappa;            /* hopping parameter; 0 => pure gauge (no fermions) */
  double alpha;            /* PQPQP parameter for FG_OMELYAN (default 0.1932) */
  int precision;           /* fg_precision (default FG_FP64); FG_DF64 needs kappa == 0 */
  int link_reals;          /* 18 (full) or 12 (two rows + reconstruction); default 18 */
  int reunitarize;         /* 1: re-project links onto SU(3) after every drift;
                              default 0 for FG_FP64 and FG_DF64, 1 for FG_FP32 */
  double cg_tol;           /* relative residual |phi - M x| / |phi| for force solves (1e-10) */
  double cg_tol_action;    /* the same for the action solve at trajectory end (1e-12) */
  int cg_maxiter;          /* CG iteration cap (default 20000) */
  double cg_delta;         /* FP32 inner CG: reliable update when the iterated residual
                              |r| falls by this factor (default 0.01) */
  unsigned long long seed; /* device momentum / pseudofermion RNG and host accept RNG */
  void *cuda_stream;       /* cudaStream_t to run on; NULL => the handle creates one */
} fg_params;

/* Result of one HMC trajectory (section 5, Fig. 1: dH over a whole trajectory). */
typedef struct {
  double dH;               /* H_end - H_start, summed site by site (per-site values and block
                              sums in double-float for FP32 fields, FP64 otherwise; FP64 total) */
  double H0, H1;           /* total H at start and end */
  double S_gauge0, S_gauge1;
  double S_ferm0, S_ferm1; /* pseudofermion action (0 for pure gauge) */
  double T0, T1;           /* kinetic term */
  int accepted;            /* Metropolis outcome; on rejection the links are restored */
  int n_steps;             /* MD steps (tau / dt) */
  int n_force;             /* force evaluations (adjacent outer kicks merged) */
  int n_solves;            /* CG solves, including the action solve */
  long long cg_iters;      /* CG iterations summed over all solves */
} fg_traj_result;

typedef struct {
  int iterations;          /* inner iterations */
  int reliable_updates;    /* FP64 residual recomputations (mixed precision) */
  double true_residual;    /* |b - M x| / |b| recomputed in FP64 at exit */
} fg_cg_result;

/* Fill *p with defaults (dims 4^4, beta 6.0, pure gauge, FP64, 18 reals). */
fg_status fg_params_default(fg_params *p);

/* Measure the current device's FP32 FMA throughput: 8 blocks of 256 threads
 * per SM, each thread running 8 independent FMA chains (65,536 FMAs), timed
 * with CUDA events on a stream of its own; *tflops_out is the best of five
 * launches in TFLOP/s (2 flop per FMA).  The ceiling of an FP32 kernel bound
 * by FMA issue, measured at the clocks the GPU holds at the time.  Allocates
 * and frees 1 KiB per block of device memory.  FG_EINVAL for a NULL pointer,
 * FG_ECUDA on a CUDA error. */
fg_status fg_fp32_fma_rate(double *tflops_out);

/* Create a handle: validates *p, allocates the device fields (cold start links,
 * zero momenta).  *out is NULL on failure. */
fg_status fg_lattice_create(const fg_params *p, fg_lattice **out);
void fg_lattice_destroy(fg_lattice *h);

/* One-line description of the last error on this handle ("" if none). */
const char *fg_last_error(const fg_lattice *h);

/* Gauge field in and out (host layout above).  fg_set_gauge does not check
 * unitarity; links are stored in the handle's precision. */
fg_status fg_set_gauge(fg_lattice *h, const double *host_links);
fg_status fg_get_gauge(fg_lattice *h, double *host_links);

/* Momenta in and out (host layout above). */
fg_status fg_set_momenta(fg_lattice *h, const double *host_p8);
fg_status fg_get_momenta(fg_lattice *h, double *host_p8);

/* Draw unit-Gaussian momenta on the device (Philox-4x32-10 counter RNG keyed
 * by fg_params.seed; every call advances the counter). */
fg_status fg_refresh_momenta(fg_lattice *h);

/* Pseudofermion heat bath from a given complex Gaussian chi on even sites:
 * phi = Mhat^dagger chi (section 4's S = phi^dagger M^{-1} phi with
 * M = Mhat^dagger Mhat), and S_F = chi^dagger chi at this gauge field.
 * FG_ESTATE if the handle is pure gauge (kappa == 0). */
fg_status fg_set_pseudofermion(fg_lattice *h, const double *host_chi_even);
/* The same with chi drawn on the device (density exp(-|chi|^2)). */
fg_status fg_refresh_pseudofermion(fg_lattice *h);

/* Total force F^a = dS/d eps^a (gauge + pseudofermion) on every link, into
 * host_f8 (layout above). */
fg_status fg_force(fg_lattice *h, double *host_f8);

/* Actions at the current fields: S_G, S_F (one CG solve to cg_tol_action;
 * 0 for pure gauge) and T.  Any output pointer may be NULL. */
fg_status fg_action(fg_lattice *h, double *S_gauge, double *S_ferm, double *T_kin);

/* Mean plaquette <Re Tr U_p / 3>. */
fg_status fg_plaquette(fg_lattice *h, double *plaq);

/* One MD step of the given integrator with step dt, in place on links and
 * momenta (no kick merging across steps). */
fg_status fg_md_step(fg_lattice *h, fg_integrator integ, double dt);

/* One force-gradient PQPQP step (Table 1, last row): fg_md_step(FG_FORCE_GRADIENT). */
fg_status fg_fg_step(fg_lattice *h, double dt);

/* One HMC trajectory of length tau = n dt (section 3: (step)^(tau/dt)):
 *   refresh != 0: draw momenta (and chi, with fermions) on the device first;
 *   refresh == 0: use the momenta (and pseudofermion) already set.
 *   u_accept in [0,1): Metropolis with this uniform (accept iff u < exp(-dH));
 *   u_accept < 0: draw the uniform from the handle's host RNG.
 * Adjacent outer kicks of neighbouring steps are merged.  On rejection the
 * links are restored; momenta are left at their end-of-trajectory values.
 * *out may be NULL. */
fg_status fg_trajectory(fg_lattice *h, fg_integrator integ, double dt, double tau,
                        int refresh, double u_accept, fg_traj_result *out);

/* Two-level (Sexton-Weingarten) trajectory for Nf = 2: H = T + S_G + S_F is
 * split as (T + S_G) + S_F.  The outer integrator, with step dt, kicks with
 * the pseudofermion force alone (its force-gradient kick, for
 * FG_FORCE_GRADIENT, displaces along and kicks with that force alone); each
 * of its drifts, of length c dt, is n_inner steps of the inner integrator
 * with step c dt / n_inner on T + S_G.  Section 3 composes integrators from
 * exactly integrable flows; this nests that composition, and the outer
 * force-gradient term {S_F,{S_F,T + S_G}} reduces to {S_F,{S_F,T}} because
 * S_G and S_F depend on the links only.  Adjacent kicks (gauge and
 * pseudofermion kicks at the same links) and adjacent drifts are merged.
 * On a pure-gauge handle the outer kicks vanish and the trajectory is the
 * inner integrator's.  refresh, u_accept, *out and rejection as for
 * fg_trajectory; FG_EINVAL if n_inner < 1. */
fg_status fg_trajectory_nested(fg_lattice *h, fg_integrator outer, fg_integrator inner, int n_inner,
                               double dt, double tau, int refresh, double u_accept,
                               fg_traj_result *out);

/* n HMC trajectories whose momenta come from host memory: trajectory k
 * starts from the momenta at host_p8[k] (V x 4 x 8 doubles, layout above)
 * and takes its Metropolis uniform from u_accept[k] (u_accept NULL, or an
 * entry < 0: the handle's host RNG; every entry must be < 1).  Links, momenta,
 * pseudofermion and results are those of n calls of fg_set_momenta(host_p8[k])
 * followed by fg_trajectory(h, integ, dt, tau, 0, u_accept[k], &out[k]).
 * The upload of trajectory k+1's momenta runs on a second stream while
 * trajectory k runs on the handle's stream, so the transfers overlap the MD
 * when the host arrays are page-locked (pageable memory works, without the
 * overlap).  The two uploads in flight share the handle's canonical staging
 * buffer (4 V 18 doubles, allocated on first use as for fg_set_gauge): the
 * call needs no device buffer beyond those; the second stream and its
 * events are created on the first call.  The host
 * arrays are not read after the call returns.  out may be NULL; on an error
 * at trajectory k, out[0..k-1] hold the completed trajectories.  FG_EINVAL on
 * n < 0, a NULL array or pointer (n > 0), or u_accept[k] >= 1. */
fg_status fg_trajectories_host_momenta(fg_lattice *h, fg_integrator integ, double dt, double tau, int n,
                                       const double *const *host_p8, const double *u_accept,
                                       fg_traj_result *out);
/* The same with FP32 host momenta (canonical layout, 4 V 8 floats each):
 * half the bytes to upload.  An FP32 handle holds its momenta in FP32, so
 * its trajectories are the same bits as from the FP64 arrays rounded to
 * FP32; FP64 and double-float handles widen the FP32 values exactly. */
fg_status fg_trajectories_host_momenta_f32(fg_lattice *h, fg_integrator integ, double dt, double tau, int n,
                                           const float *const *host_p8, const double *u_accept,
                                           fg_traj_result *out);

/* Building blocks for callers and tests (even-site spinors, host layout above). */
/* out = Mhat in (dagger = 0) or Mhat^dagger in (dagger = 1). */
fg_status fg_apply_mhat(fg_lattice *h, const double *host_in_even, double *host_out_even,
                        int dagger);
/* The same operator as the inner CG iterations apply it (section 4's
 * calM = Mhat^dagger Mhat is built from it): the input rounded to the inner
 * precision, the two Dslash launches of Mhat in that precision, the output
 * widened to FP64.  Inner precision: FP32 links and spinors for FG_FP32;
 * half-precision links (a copy made for the call) and half-precision spinors
 * scaled by sigma, sigma^2 = |in|^2 / n, for FG_FP32_FP16CG; the same in
 * bfloat16 for FG_FP32_BF16CG; FP64 for FG_FP64
 * (then equal to fg_apply_mhat).  FG_ESTATE for pure-gauge handles. */
fg_status fg_apply_mhat_inner(fg_lattice *h, const double *host_in_even, double *host_out_even,
                              int dagger);
/* Solve Mhat^dagger Mhat x = b to cg_tol with x0 = 0. */
fg_status fg_cg_solve(fg_lattice *h, const double *host_b_even, double *host_x_even,
                      fg_cg_result *res);

/* Haar-random links drawn on the device (a hot start without a host
 * transfer; Philox keyed by fg_params.seed, every call draws new links). */
fg_status fg_random_gauge(fg_lattice *h);

/* Position of the handle's random streams: the next momentum refresh,
 * pseudofermion heat bath and host accept uniform all use draw `pos`.  A
 * caller that sets it to the chain's trajectory index before each trajectory
 * gets results that do not depend on what else ran in between. */
fg_status fg_set_rng_position(fg_lattice *h, unsigned long long pos);

/* Re-project every link onto SU(3) (Gram-Schmidt of rows 1-2, row 3 = (row1 x row2)^*). */
fg_status fg_reunitarize(fg_lattice *h);

/* Per-kernel timing with CUDA events on the handle's stream.  While enabled,
 * every launch of the named kernel class is bracketed by events;
 * fg_kernel_time synchronises and returns the summed device time and the
 * number of launches since the last reset.  Classes: "gauge_force",
 * "drift", "energy", "reduce", "momenta", "dslash" (Dslash in the inner
 * precision), "cg_blas", "fermion_force", "convert", "dslash_fp64" (the
 * FP64-arithmetic Dslash of the heat bath, of fg_apply_mhat and of the
 * reliable update that certifies convergence), "dslash_df" (the
 * double-float Dslash of the FP32 solver's other reliable updates). */
fg_status fg_timing_enable(fg_lattice *h, int on);
fg_status fg_timing_reset(fg_lattice *h);
fg_status fg_kernel_time(fg_lattice *h, const char *kernel_class, double *total_ms,
                         long long *launches);

/* Number of kernels this handle has launched since creation. */
long long fg_launch_count(const fg_lattice *h);

/* Block until all work queued on the handle's stream has finished. */
fg_status fg_sync(fg_lattice *h);

/* Upper limit, in seconds, on every wait of the host for this handle's GPU
 * work (0, the default: no limit).  A call whose wait would last longer
 * returns FG_ETIMEOUT and leaves its work queued on the GPU; the handle's
 * fields and results are then undefined until a later fg_sync (with a
 * larger limit, or 0) succeeds.  The copy-stream drain at the end of
 * fg_trajectories_host_momenta (the host arrays must not be read after it
 * returns) and fg_lattice_destroy wait without limit.  FG_EINVAL for a
 * negative or NaN limit. */
fg_status fg_set_wait_limit(fg_lattice *h, double seconds);

/* Device bytes held by the handle. */
unsigned long long fg_device_bytes(const fg_lattice *h);


/* ------------------------------------------------------------------------
 * Batches of independent pure-gauge chains (many small lattices at once).
 *
 * A batch holds nchains independent lattices of different volumes and
 * couplings, all advanced with the same integrator and step size.  Each MD
 * sub-step of section 3 / Table 1 (kick, drift, force-gradient displacement)
 * is one persistent launch over the links of every chain; the HMC accept /
 * reject of section 5 runs per chain on the device, so one trajectory of all
 * chains is a single CUDA graph launch (use_graphs = 1).  A chain gives the
 * same links alone (fg_lattice) and in a batch: the per-link arithmetic is
 * shared.  Pure gauge only.
 */
typedef struct fg_batch fg_batch;

typedef struct {
  int nchains;             /* number of chains, >= 1 */
  const int *dims;         /* nchains x 4 extents (Lx, Ly, Lz, Lt; even, >= 2; volume <= 2^28); copied */
  const double *beta;      /* nchains couplings; copied */
  int precision;           /* FG_FP32 (default), FG_FP64 or FG_DF64 */
  int link_reals;          /* 18 or 12 */
  int reunitarize;         /* -1: after every drift for FP32, never for FP64 and FG_DF64 */
  double alpha;            /* PQPQP parameter for FG_OMELYAN (0.1932) */
  int tile;                /* half-sites per block: 16, 32 or 64; 0 = time all three on the
                              first trajectory and keep the fastest (autotuning) */
  int use_graphs;          /* 1 (default): capture each trajectory as one CUDA graph */
  unsigned long long seed; /* device momentum and accept RNG */
  void *cuda_stream;       /* stream to run on, NULL => the batch creates one */
} fg_batch_params;

fg_status fg_batch_params_default(fg_batch_params *p);
/* Validates *p (FG_EINVAL on bad extents, couplings or tile) and allocates
 * all chains on the device with cold-start links. */
fg_status fg_batch_create(const fg_batch_params *p, fg_batch **out);
void fg_batch_destroy(fg_batch *b);
const char *fg_batch_last_error(const fg_batch *b);
/* Fields of one chain, host layouts as for fg_lattice (chain in [0, nchains)). */
fg_status fg_batch_set_gauge(fg_batch *b, int chain, const double *host_links);
fg_status fg_batch_get_gauge(fg_batch *b, int chain, double *host_links);
fg_status fg_batch_set_momenta(fg_batch *b, int chain, const double *host_p8);
fg_status fg_batch_get_momenta(fg_batch *b, int chain, double *host_p8);
/* One trajectory of length tau = n dt for every chain.  refresh != 0 draws
 * momenta on the device first; accept_mode 0 = Metropolis per chain with a
 * device uniform, 1 = accept every finite dH (thermalisation, tests).
 * out (may be NULL) receives nchains results (dH, H0, H1, action parts,
 * accepted, n_steps, n_force). */
fg_status fg_batch_trajectory(fg_batch *b, fg_integrator integ, double dt, double tau, int refresh,
                              int accept_mode, fg_traj_result *out);
/* Tile size in use (0 until the autotuner has run). */
fg_status fg_batch_tile(const fg_batch *b, int *tile);
/* Kernels launched by the batch (a graph launch counts its kernels). */
long long fg_batch_launch_count(const fg_batch *b);
/* Limit on the host waits of a batch, as fg_set_wait_limit. */
fg_status fg_batch_set_wait_limit(fg_batch *b, double seconds);

/* ------------------------------------------------------------------------
 * Allocation-free action sums (no handle).
 *
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot let this library allocate device memory: a process whose GPU memory
 * is already reserved in full by another allocator (for example the caching
 * allocator of a framework that owns the device, where an extra cudaMalloc
 * fails or fragments the pool), or a latency-critical loop in which a
 * cudaMalloc/cudaFree pair would synchronise the device.
 *
 * It computes the same two sums as fg_action,
 *   S_G = beta sum_{x, mu<nu} (1 - Re Tr U_{mu nu}(x) / 3)   -> dev_out[0]
 *   T   = (1/2) sum_{links, a} (p^a)^2                       -> dev_out[1]
 * (T = 0 if dev_momenta is NULL), in FP64, from caller-owned device arrays
 * in the canonical host layout above (gauge double[V][4][3][3][2], momenta
 * double[V][4][8]); dev_out is caller-owned device memory for two doubles.
 * Work is queued on cuda_stream (NULL = the legacy default stream) and the
 * call returns without synchronising.
 *
 * Scratch: the per-block partial sums go to one fixed 1 MiB device array
 * inside the library, sized for at most FG_NOALLOC_MAX_SITES sites; every
 * GPU that loads the library holds it until the process exits.  The call
 * itself allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).  The first call on each device looks up the array's device
 * address with that device current and caches it, so make that first call
 * before any stream capture; calls outside a capture look it up again (a
 * device reset may move the array), calls inside one use the cached value,
 * so after a device reset make one call outside capture before capturing.
 * Every call shares the array and overwrites each entry it later reads, so
 * nothing carries over from the previous call; calls whose kernels overlap
 * on the GPU (other streams or other host threads on the same device) race
 * on the array and must be serialised by the caller.
 *
 * Errors: FG_EINVAL for a null links/out/dims pointer, an odd or < 2 extent,
 * or more than FG_NOALLOC_MAX_SITES sites (nothing is queued); FG_ECUDA if
 * the address lookup or a launch fails.
 */
#define FG_NOALLOC_MAX_SITES (1LL << 24)
fg_status fg_action_sums_noalloc(const double *dev_links, const double *dev_momenta,
                                 const int dims[4], double beta, double *dev_out,
                                 void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FG_LATTICE_H */
