/*
 * sie.h -- C ABI of the GB300 MLFMM-accelerated JMCFIE surface-integral solver.
 *
 * The library computes, on one GPU, the operator of the Galerkin/RWG
 * discretisation of the JMCFIE surface integral equation for piecewise
 * homogeneous dielectric bodies (paper: "Integral Equation Formulation",
 * Eqs. 1-16; "Discretization and Iterative Solution", Eqs. 13-26) and its
 * preconditioned iterative solution (ILU, Sect. "Simulation Results"), the
 * plane-wave excitation (Eq. 30, Eqs. 20-21) and the radar cross section
 * (Eqs. 27-29).  The matrix-vector product is split into an exactly integrated
 * near field and a multilevel fast multipole (MLFMM) far field (cited by the
 * paper as its accelerator, Conclusion).
 *
 * Conventions shared by every call:
 *   - Units: SI; lambda0 is whatever freq_hz implies.  Time convention e^{+jwt}.
 *   - Unknowns: one RWG basis per edge shared by two triangles of the same
 *     interface surface (Eq. 22).  RWG numbering: lexicographic order of the
 *     (min vertex, max vertex) pair of the edge; T+ is the owning triangle of
 *     smaller index.  Two unknowns per edge, interleaved: (eta0 * c_n, v_n) --
 *     the electric-current coefficient scaled by the free-space impedance, then
 *     the magnetic-current coefficient (Eqs. 13-14 of the discretisation).
 *     Rows are (eta0 * J-row, M-row) of Eq. 14/16; every block is dimensionless.
 *   - Vectors are complex, interleaved (re, im), layout [nrhs][n_rwg][2]:
 *     complex128 (double2) unless a call says otherwise.  "_dev" pointers are
 *     device pointers on the context's device; "_host" pointers are host memory.
 *   - The caller owns every buffer it passes; the context owns everything it
 *     allocates and frees it in sie_destroy.
 *   - All calls are asynchronous on the context's stream, except those that
 *     return host data (documented per call), which synchronise it.
 *   - No call throws.  Each returns a sie_status; sie_last_error() gives the
 *     message of the last failure of that context.  A context is not thread-safe.
 *   - There is no CPU fallback: every numerical step runs in this library's
 *     CUDA kernels (sm_103a).
 */
#ifndef SIE_H
#define SIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sie_ctx sie_ctx;

typedef enum {
  SIE_OK = 0,
  SIE_EINVAL = 1,      /* invalid argument (null pointer, bad size, bad mesh) */
  SIE_ENOMEM = 2,      /* device or host allocation failed */
  SIE_ECUDA = 3,       /* a CUDA runtime call failed */
  SIE_ESTATE = 4,      /* call out of order (e.g. matvec before setup) */
  SIE_ENOTCONV = 5,    /* solver hit max_iters before the tolerance */
  SIE_EBREAKDOWN = 6,  /* Krylov breakdown or non-finite residual */
  SIE_ETIMEOUT = 7,    /* a bounded device wait gave up */
  SIE_EZEROPIVOT = 8   /* ILU(0) met a singular 2x2 diagonal block */
} sie_status;

typedef enum {
  SIE_PREC_FP64 = 0,   /* plain form: every step in FP64 */
  SIE_PREC_MIXED = 1,  /* near field, translations, patterns, ILU in FP32 complex;
                          Arnoldi, Givens, true residual in FP64 vectors */
  SIE_PREC_NEAR64 = 2  /* products only (mlfmm_matvec, sie_matvec_parts, the
                          whole-product stage timing): FP64 near field, FP32
                          far field (patterns, translations, receive sums)
                          added into the FP64 product; the true-residual
                          operator of the mixed form */
} sie_prec;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (or NULL: the context creates and owns a non-blocking stream).  */
sie_status sie_create(sie_ctx **out, int device, void *cuda_stream);
void sie_destroy(sie_ctx *ctx);
const char *sie_last_error(const sie_ctx *ctx);

/* Mesh and media (Fig. 2-3; Eqs. 12-13).
 *   verts       [nv][3] float64, metres.
 *   tris        [nt][3] int32; the normal (v1-v0)x(v2-v0) points into
 *               tri_regions[t][0] ("+" region); tri_regions[t][1] is behind.
 *   media       [nr][4] float64 = (eps_r re, eps_r im, mu_r re, mu_r im);
 *               region 0 is the host medium holding the incident wave.
 *               Passive media only (Im(eps_r mu_r) <= 0).
 *   freq_hz     frequency.
 *   n_rwg_out   receives the number of RWG edges (unknowns = 2 * n_rwg).
 * Junction edges (three or more surfaces meeting at an edge, Eq. 16's
 * multi-boundary bodies): each region touching the edge must see exactly two
 * of its triangles; the edge carries one unknown whose per-triangle
 * coefficients a_T make every region's current divergence-conforming across
 * it (s_l(T1) a_T1 = -s_l(T2) a_T2, s_l(T) = +1 when l is T's "+" region),
 * i.e. region l's basis function is an RWG function on its two triangles.
 * Errors: SIE_EINVAL for a junction edge where a region does not see two of
 * the triangles, an ordinary edge shared by triangles of different surfaces
 * or of inconsistent orientation, region indices outside [0, nr),
 * degenerate triangles, media with a zero or non-finite eps_r or mu_r,
 * active media.  Host-only work (topology); synchronous.  */
sie_status sie_build_mesh(sie_ctx *ctx, const double *verts, int64_t nv, const int32_t *tris,
                          int64_t nt, const int32_t *tri_regions, const double *media, int32_t nr,
                          double freq_hz, int64_t *n_rwg_out);

/* MLFMM options (the paper gives none; the readings adopted are stated per field). */
typedef struct {
  int32_t levels;   /* octree levels including the root, in [2, 12]; 2 puts
                       every basis pair in the near field (dense product,
                       no MLFMM).  Leaf edge =
                       D / 2^(levels-1) with D = 1.0009765625 * largest extent
                       of the vertex bounding box.  */
  double digits;    /* d0 in L = kd + 1.8 d0^(2/3) (kd)^(1/3), d = sqrt(3) * box
                       edge, k = |k_l| (the modulus, not Re k_l: in a lossy
                       medium the addition theorem converges at the rate of
                       |k| d, and a metal's k is nearly imaginary).  Typical 3. */
} sie_mlfmm_opts;

/* Octree, near-field pattern, preconditioner ordering and the far-field
 * tables of every medium: direction samples, M2L translators, exact
 * separable interpolation tables (trigonometric in phi, Lagrange in cos theta),
 * shift phases, sibling groups for the block translations.  Per medium, the
 * levels coarser than the first one with a non-empty interaction list get no
 * tables (their translations would be empty).  Requires sie_build_mesh.
 * Synchronous. */
sie_status mlfmm_setup(sie_ctx *ctx, const sie_mlfmm_opts *opts);

typedef struct {
  int32_t outer_order;  /* n of the n x n collapsed-Gauss outer rule on
                           singular / near-singular triangle pairs (4) */
  int32_t build_ilu;    /* nonzero: factor ILU(0) of the near field */
  int32_t formulation;  /* 0 JMCFIE (Eq. 14/16, the paper's); 1 CTF, 2 CNF,
                           3 PMCHWT: the variants it is compared with.  With
                           T and N the tangential and normal equations of
                           medium l (Eqs. 8-11), J-row = sum_l s_l [aTJ T-EFIE /
                           eta_l - aNJ N-MFIE], M-row = sum_l s_l [aNM N-EFIE -
                           aTM eta_l T-MFIE]; JMCFIE all weights 1, CTF only T,
                           CNF only N, PMCHWT aTJ = eta~_l, aTM = 1/eta~_l, no N.
                           4 ICTF (the improved CTF of the Fig. 6 comparison,
                           read as: CTF with each interface's tangential
                           equations normalised by the mean relative
                           impedance e = (eta~_a + eta~_b)/2 of its two media
                           instead of each medium's own), i.e. the PMCHWT rows
                           times 1/e (J-row) and e (M-row) per basis.
                           Applies to the near field, the receive patterns and
                           sie_plane_wave_rhs (ICTF: also to every product of
                           mlfmm_matvec and to the ILU(0) factors).  Other
                           values: SIE_EINVAL. */
} sie_fill_opts;

/* Near-field fill on the GPU in FP64 (Eqs. 23-26 with singularity
 * extraction; identity terms of Eqs. 8-11), leaf radiation/receive patterns
 * of every medium, FP32 copies, and (optionally) the 2x2-block ILU(0) of the
 * near field in the box-colour ordering.  Requires mlfmm_setup.  Synchronous
 * (the ILU factorisation runs on the host CPU threads). */
sie_status sie_fill_nearfield(sie_ctx *ctx, const sie_fill_opts *opts);

/* y = Z x: near-field block-sparse product plus the MLFMM far field of every
 * medium.  x_dev, y_dev: complex128 [nrhs][n_rwg][2], user (RWG) order; they
 * may not alias.  prec selects the arithmetic of the product (inputs and
 * outputs stay complex128).  Requires sie_fill_nearfield. */
sie_status mlfmm_matvec(sie_ctx *ctx, const void *x_dev, void *y_dev, int64_t nrhs, sie_prec prec);

/* Parts of the product, for testing: parts bit 1 = near field, bit 2 = far
 * field (MLFMM).  Same conventions as mlfmm_matvec. */
sie_status sie_matvec_parts(sie_ctx *ctx, const void *x_dev, void *y_dev, int64_t nrhs, sie_prec prec,
                            int32_t parts);

/* z = (L U)^-1 r with the ILU(0) factors of the near field (Sect. "Simulation
 * Results", ILU preconditioner).  Same vector conventions.  Requires
 * sie_fill_nearfield with build_ilu. */
sie_status ilu_apply(sie_ctx *ctx, const void *r_dev, void *z_dev, int64_t nrhs, sie_prec prec);

/* Allocation-free variant of ilu_apply (the paper has no counterpart; this
 * is a service of the library).  ilu_apply stages its vectors in work buffers
 * that the context allocates with cudaMalloc on first use.  Callers that must
 * not let a library allocate device memory during a step -- a host framework
 * that owns all device memory through its own pool, or a latency-critical
 * loop where cudaMalloc would synchronise the device -- call this instead: it
 * computes the same z = (L U)^-1 r, with the same conventions, and allocates
 * nothing.  Its scratch is one 16 MiB device array inside the library, which
 * every GPU that loads the library holds until the process exits.
 *   - Limit: nrhs * n_rwg <= 174762; larger requests return SIE_EINVAL
 *     before touching any buffer.
 *   - The first call on a device looks up the array's device address; make
 *     that first call before any stream capture.
 *   - All calls share the array (it keeps the last call's contents; every
 *     element is written before it is read, so nothing needs clearing).
 *     Calls whose GPU work overlaps -- on different streams, contexts or host
 *     threads -- race on it; serialise them.
 * Requires sie_fill_nearfield with build_ilu. */
sie_status ilu_apply_noalloc(sie_ctx *ctx, const void *r_dev, void *z_dev, int64_t nrhs, sie_prec prec);

/* Tested plane-wave excitation (Eqs. 20-21, Eq. 30) for nrhs incidences.
 * inc_host [nrhs][4] float64 = (theta_i, phi_i, pol, E0): the wave arrives
 * from direction (theta_i, phi_i), propagates along -r(theta_i, phi_i), with
 * E = E0 (cos(pol) theta_hat + sin(pol) phi_hat) exp(-j k0 khat.r).
 * b_dev: complex128 [nrhs][n_rwg][2], user order.  */
sie_status sie_plane_wave_rhs(sie_ctx *ctx, const double *inc_host, int64_t nrhs, void *b_dev);

typedef struct {
  int32_t restart;     /* Krylov dimension per cycle (50) */
  int32_t max_iters;   /* total inner iterations per right-hand side */
  double tol;          /* relative true residual ||b - A x|| / ||b||, A the
                          residual operator (below) */
  int32_t prec;        /* sie_prec of the inner operator and preconditioner */
  int32_t precond;     /* 0: none, 1: ILU(0), 2: ILU(0) followed by the learned
                          correction (needs nnprec_train or nnprec_params; the
                          correction is dropped for the rest of a solve as soon
                          as a restart cycle fails to reduce the true residual),
                          all as right preconditioning */
  int32_t method;      /* 0: FGMRES(restart) (default); 1: BiCGStab; 2: CGS
                          (the paper's solvers; right-preconditioned, restarted
                          from the FP64 true residual when the recurrence
                          residual reaches tol; restart and no_graphs unused) */
  int32_t no_graphs;   /* 0: each Krylov step (preconditioner + product) is
                          captured once as a CUDA graph and replayed; 1: every
                          step is launched eagerly (same kernels, same results;
                          for tools that cannot follow graph launches) */
  int32_t residual_far_fp64;  /* operator of the true residual (restarts and
                          the convergence decision) in the mixed form: 0
                          SIE_PREC_NEAR64 (FP64 near field, FP32 far field,
                          FP64 vectors) when tol >= 5e-5, the whole FP64
                          operator for smaller tol (the FP32 far field puts
                          the NEAR64 product within a few 1e-6 of the FP64
                          one, a floor for the residuals it can certify); 1
                          the whole FP64 operator.  The plain form always
                          uses the FP64 operator. */
} sie_solve_opts;

typedef struct {
  int32_t iters;        /* inner iterations used */
  int32_t restarts;     /* restart cycles (true-residual recomputations) */
  double rel_residual;  /* final true relative residual, residual operator */
  int32_t converged;    /* 1 if rel_residual <= tol */
} sie_solve_stats;

/* Right-preconditioned flexible GMRES(restart) (or BiCGStab / CGS, see
 * opts->method) for nrhs right-hand sides in lockstep (block of independent
 * Krylov spaces).  b_dev, x_dev complex128 [nrhs][n_rwg][2] user order; x_dev
 * holds the initial guess on entry and the solution on return.  stats_host
 * [nrhs] receives per-RHS results.  Synchronous.  Returns SIE_ENOTCONV if any
 * RHS did not reach tol (x_dev and the stats still hold the last iterate),
 * SIE_EBREAKDOWN on a non-finite residual or repeated breakdown, SIE_EINVAL
 * for options out of range, SIE_ESTATE when the ILU(0) factors or the
 * learned correction requested are not built. */
sie_status gmres_solve(sie_ctx *ctx, const void *b_dev, void *x_dev, int64_t nrhs,
                       const sie_solve_opts *opts, sie_solve_stats *stats_host);

/* Learned right preconditioner (not in the paper; an extension of its ILU
 * preconditioner, Sect. "Simulation Results").  One MLP 128 -> 256 -> 256 -> 128
 * with ReLU, shared by all leaf chunks (runs of <= 32 bases of one leaf box,
 * 64 complex unknowns = 128 reals); with u = ILU^-1 v,
 * z_c = u_c + |u_c| NN(u_c/|u_c|) (a learned local correction of the ILU output).
 * Weights and activations BF16, FP32 accumulation, Adam with FP32 masters.
 * Training pairs are generated by the solver itself: recording solves of
 * FGMRES(record_restart) with ILU(0) for the training incidences store the
 * iterate x_k and true residual r_k at every restart; after convergence
 * e_k = x* - x_k; with u = ILU^-1 r_k the network regresses (e_k - u)_c / |u_c|
 * on u_c / |u_c| chunk by chunk (squared error weighted by |u_c|^2, normalised
 * per pair, i.e. the error of the corrected z itself).  The last fifth of the
 * incidences is held out: the output is scaled by the least-squares factor
 * gamma (at most 1) fitted on their pairs; the correction is kept only if it
 * lowers their loss below 95 % of the loss of no correction AND the plain
 * ILU(0) solver, which decides, needs more FGMRES(50) iterations than the
 * corrected one on the last held-out incidence.  Synchronous. */
typedef struct {
  const double *train_inc;  /* host [ntrain][4] incidences, as sie_plane_wave_rhs */
  int32_t ntrain;
  int32_t record_restart;   /* restart length of the recording solves (pairs per restart) */
  int32_t max_pairs;        /* cap on recorded pairs */
  int32_t epochs;
  int32_t batch;            /* chunk samples per Adam step (>= 64) */
  double lr;                /* Adam step size */
  uint64_t seed;            /* weight initialisation and batch shuffling */
} sie_nn_opts;

typedef struct {
  int32_t pairs;            /* recorded (residual, error) pairs */
  int64_t samples;          /* chunk samples = pairs * chunks */
  double loss_first;        /* mean loss of the first and last epoch */
  double loss_last;
  double ms;                /* device time of recording + training */
  double val_loss_ratio;    /* held-out loss with the (scaled) correction / without any */
  double gamma;             /* least-squares output scale on the held-out pairs */
  int32_t enabled;          /* 1 if the correction passed both gates; otherwise
                               precond = 2 runs as plain ILU(0) */
  int32_t gate_iters_ilu;  /* FGMRES(50) iterations to 1e-4 on the last (held-out)
                               incidence with ILU(0) alone, and with the correction */
  int32_t gate_iters_nn;   /* (-1: not run, the loss gate already rejected it) */
} sie_nn_stats;

sie_status nnprec_train(sie_ctx *ctx, const sie_nn_opts *opts, sie_nn_stats *stats);

/* Get (set = 0) or set (set != 0) the network's FP32 master parameters,
 * params_host [131712] = W1 [256][128], b1 [256], W2 [256][256], b2 [256],
 * W3 [128][256], b3 [128], row-major.  Setting marks the network ready. */
sie_status nnprec_params(sie_ctx *ctx, float *params_host, int32_t set);

/* Loss and parameter gradient of the network on n given samples (for
 * verification): X_host [n][128] inputs (rounded to BF16 on the device),
 * T_host [n][128] targets; loss_out = sum (y - t)^2 / (2 n); grad_host
 * [131712] FP32, same layout as nnprec_params. */
sie_status nnprec_loss_grad(sie_ctx *ctx, const float *X_host, const float *T_host, int64_t n, double *loss_out,
                            float *grad_host);

/* Bistatic radar cross section (Eqs. 27-29) of solutions x_dev (complex128
 * [nrhs][n_rwg][2], user order) at nobs directions obs_host [nobs][2] =
 * (theta, phi) in radians.  rcs_host [nrhs][nobs][2] receives
 * (sigma_theta, sigma_phi) in m^2 for unit E0.  Synchronous. */
sie_status rcs_farfield(sie_ctx *ctx, const void *x_dev, int64_t nrhs, const double *obs_host,
                        int64_t nobs, double *rcs_host);

/* rcs_farfield with a precision: SIE_PREC_FP64 is rcs_farfield itself;
 * SIE_PREC_MIXED evaluates the radiation integrals with FP32 phases and
 * currents (positions taken relative to the octree centre, FP32 sums within
 * a slice of the quadrature points, FP64 across slices), the precision of
 * the far-field step in the mixed form; the RCS then differs from the FP64
 * one by about 1e-6 relative.  Other prec values give SIE_EINVAL. */
sie_status rcs_farfield_prec(sie_ctx *ctx, const void *x_dev, int64_t nrhs, const double *obs_host,
                             int64_t nobs, int32_t prec, double *rcs_host);

/* Export of the near-field matrix for verification.  With rows == NULL only
 * *nnzb is written.  Otherwise rows/cols [nnzb] int32 receive RWG (user)
 * indices and vals [nnzb][4][2] float64 the block (JJ, JM, MJ, MM) as
 * complex128.  Synchronous. */
sie_status sie_near_export(sie_ctx *ctx, int32_t *rows, int32_t *cols, double *vals, int64_t *nnzb);

/* Device time of one stage of the hot path, for roofline reports: launches
 * the stage `reps` times back to back on the context's stream on internal
 * work vectors and returns the mean milliseconds per launch, measured with
 * CUDA events on that stream.  stage: 0 near-field block-sparse product,
 * 1 MLFMM far field (all media, all levels), 2 ILU(0) forward + backward
 * sweeps, 3 whole product (near + far).  prec: SIE_PREC_FP64 or
 * SIE_PREC_MIXED; SIE_PREC_NEAR64 for stage 3 only (else SIE_EINVAL).
 * Synchronous.  Not a numerical operation of the method; the paper has no
 * counterpart. */
sie_status sie_stage_timing(sie_ctx *ctx, int32_t stage, int64_t nrhs, int32_t prec, int32_t reps, double *ms_out);

/* Bounded device-side waits.  The single-right-hand-side ILU(0) apply can
 * run its 15 colour steps in one cooperative launch whose steps are separated
 * by grid barriers (sie_set_param key 1 = 0); a CTA polls a barrier at most
 * `wait limit` times (about
 * 0.1-1 us per poll) before it gives up, records the failure in a device
 * flag and returns, so the launch always ends (its output is then invalid).
 * sie_device_status synchronises the context's stream and returns
 * SIE_ETIMEOUT if such a wait gave up since the last call (clearing the
 * record), SIE_OK otherwise.  gmres_solve checks the record at every restart
 * and returns SIE_ETIMEOUT.  Not a numerical operation of the method; the
 * paper has no counterpart. */
sie_status sie_device_status(sie_ctx *ctx);

/* Runtime parameters (key, value):
 *   0  wait limit: polls of a device-side barrier before it gives up
 *      (default 2^21, about a second; 0 makes every wait give up at once,
 *      for testing the failure path); in [0, 2^30].
 *   1  schedule of the single-right-hand-side ILU(0) apply: 0 one
 *      persistent cooperative launch for the 15 colour steps, with grid
 *      barriers between them; 1 (default, faster on GB300: 0.24 against
 *      0.37 ms on a 78 000-unknown case) one launch per step, chained by
 *      programmatic dependent launch.  Same results, bit for bit.
 *   2  tensor-core leaf aggregation (FP32 operator of the Krylov steps, not
 *      the true residual): used from this many right-hand sides on (default
 *      16; 0 never), in [0, 4096].
 *   3  right-hand sides per pass of the tensor-core aggregation: 0 (by the
 *      block size, default), 16, 32 or 64.
 *   4  right-hand sides per block load of the near-field product (blocks of
 *      right-hand sides): 0 (default: 8 in FP32, 4 in FP64), 4, 8 or 16.
 *   5  the same for the block ILU(0) sweeps.
 *   6  right-hand sides per pass of the leaf receive: 0 (default 4), 1, 2, 4.
 *   7  M2L form: -1 (default: sibling groups from 8 right-hand sides on,
 *      per target box below), 0 per target box, 1 sibling groups from 2 on,
 *      2 sibling groups whose union list is split over the warps of a CTA.
 *   8  tensor-core leaf receive (FP32 operator of the Krylov steps, blocks
 *      of right-hand sides): right-hand sides per pass, -1 (default: from 16
 *      right-hand sides on, 16, 32 or 64 by the block size), 0 (the SIMT
 *      receive), 16, 32 or 64.
 *   9  dense layers of the learned preconditioner with BF16 activations and
 *      weights (its forward pass): 1 (default) on the tensor cores
 *      (tcgen05, FP32 accumulation in tensor memory), 0 on the SIMT tiles.
 *   10 CTAs of the interpolation and anterpolation per (box, right-hand
 *      side): -1 (default: one per source J, M for one right-hand side on
 *      levels of fewer than 2048 boxes, one for both otherwise), 0 one for
 *      both sources in turn, 1 one per source; the same arithmetic.
 * Keys 2-10 are tile shapes: results agree to rounding (the tensor-core
 * aggregation and receive to their FP32-level split operands, the network's
 * layers to the order of their FP32 sums), speed differs.
 * Errors: SIE_EINVAL for an unknown key or a value out of range. */
sie_status sie_set_param(sie_ctx *ctx, int32_t key, int64_t value);

/* Autotuner of the tile shapes for blocks of nrhs right-hand sides (FP32
 * kernels of the mixed form): coordinate descent over the parameters of
 * sie_set_param keys 4 (near field), 5 (ILU sweeps), 2-3 (aggregation:
 * SIMT or tensor cores and their pass size), 6 (receive), 8 (receive on the
 * tensor cores, from 16 right-hand sides on), 7 (M2L form), each
 * candidate timed with CUDA events on the context's stream over `reps`
 * launches of its stage after a warm-up launch; the fastest is kept in the
 * context.  choice_out [6] receives (near RB, ILU RB, aggregation: 0 SIMT or
 * the tensor-core pass size, receive RB, M2L form, tensor-core receive pass
 * size or 0); ms_out [3] (or NULL) the
 * best near-field, ILU and far-field milliseconds.  nrhs in [2, 4096].
 * Allocates work buffers for nrhs right-hand sides.  Synchronous.  Not a
 * numerical operation of the method; the paper has no counterpart. */
sie_status sie_autotune(sie_ctx *ctx, int64_t nrhs, int32_t reps, int64_t *choice_out, double *ms_out);

/* Integer facts about the context for tests and reports: keys
 *   0 n_rwg, 1 near blocks, 2 levels, 3 regions, 4 leaf boxes (all media),
 *   5 bytes of the FP64 near field, 6 bytes of FP64 leaf patterns,
 *   7 device bytes held, 8 kernel launches so far,
 *   9 algorithmic bytes of one single-RHS FP32 ILU(0) apply (off-box factor
 *     blocks with their column indices, in-box inverse blocks, per row the
 *     colour pointers of both sweeps and the source and result vectors; 0
 *     without ILU factors),
 *   10 Krylov step graphs of the last FGMRES solve: 1 captured and replayed,
 *     0 capture failed and the steps ran eagerly, -1 none captured,
 *   100 + 16*l + j: K (directions) of medium l at level j (0 at levels
 *     coarser than the medium's coarsest level with a non-empty interaction
 *     list: they translate nothing and are skipped). */
sie_status sie_query(const sie_ctx *ctx, int32_t key, int64_t *value);

#ifdef __cplusplus
}
#endif
#endif /* SIE_H */
