/*
 * nlpot — NUFFT evaluation of nonlocal potentials phi = U * rho on one GB300 (sm_103a).
 *
 * Method: Bao, Jiang, Tang & Zhang, "Computing the ground state and dynamics of the
 * nonlinear Schroedinger equation with nonlocal interactions via the nonuniform FFT"
 * (arXiv:1410.3584).  Given rho on a uniform grid, phi = U * rho (Sec. 2, Eq. (nonlocal53))
 * is evaluated in Fourier space on a spherical (3D) or polar (2D) quadrature grid whose
 * Jacobian cancels the singularity of U-hat (Sec. 2.1, Eq. (ifft)): a type-2 NUFFT gives
 * rho-hat at the nodes, each node is scaled by its weight times |k|^{d-1} U-hat(k), and a
 * type-1 NUFFT returns phi to the grid.  The 2D Laplace kernel 1/|k|^2 uses the paper's
 * Gaussian subtraction (Sec. 2.2, Algorithm 1).  The ground-state step is the backward-Euler
 * normalized gradient flow (Sec. 3.1) and the dynamics step is time splitting (Sec. 4.1).
 *
 * Conventions for every entry point:
 *  - Grid: per axis a, n[a] points on [-L[a], L[a]), h[a] = 2 L[a] / n[a],
 *    x_m = -L + m h (m = 0..n-1; the origin is m = n/2).  Arrays are C order with the last
 *    axis fastest: a[i][j][k] = f(x_i, y_j, z_k).
 *  - Real arrays hold the plan precision (double for NLP_FP64, float for NLP_FP32); complex
 *    arrays are interleaved (re, im) pairs of that type.
 *  - Pointers named *_dev are device pointers owned by the caller; the plan owns every
 *    workspace it allocates and frees it in nlp_plan_destroy.  *_host pointers are host
 *    memory owned by the caller.
 *  - All device work is enqueued on the plan's stream (the stream given at creation;
 *    NULL = legacy default stream).  Calls return once the work is enqueued unless stated.
 *  - Errors are return codes; nothing throws across this boundary.  Invalid arguments
 *    are rejected with NLP_ERR_INVALID_ARG before any launch.  After NLP_ERR_CUDA the
 *    plan should be destroyed.
 *  - A plan is not thread-safe: calls on one plan must not overlap.
 */
#ifndef NLPOT_H
#define NLPOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NLP_OK = 0,
    NLP_ERR_INVALID_ARG = 1,
    NLP_ERR_UNSUPPORTED = 2,
    NLP_ERR_OOM = 3,
    NLP_ERR_CUDA = 4,
    NLP_ERR_TIMEOUT = 5,
    NLP_ERR_DIVERGED = 6,
    NLP_ERR_NOT_CONVERGED = 7
} nlp_status;

/* Interaction kernels (Sec. 1, Eqs. (Kernal), (Kernal21d)):
 *   NLP_COULOMB_3D  U = 1/(4 pi |x|),      U-hat = 1/|k|^2
 *   NLP_DIPOLE_3D   U-hat = 3 (n.k)^2/|k|^2 - 1 for dipole axis n (the paper names the
 *                   dipolar kernel without writing it; this is the standard form)
 *   NLP_COULOMB_2D  U = 1/(2 pi |x|),      U-hat = 1/|k|
 *   NLP_POISSON_2D  U = -ln|x| / (2 pi),   U-hat = 1/|k|^2 (Algorithm 1)
 *   NLP_CONFINED_2D the 2D confined Coulomb kernel of Eq. (Kernal124d) with parameter
 *                   eps = nlp_opts.confine_eps >= 0: |k| U-hat = W_1(|k|) of Eq. (2Dw1),
 *                   = exp(a) erfc(sqrt a), a = eps^2 |k|^2 / 2 (eps = 0: NLP_COULOMB_2D)
 *   NLP_POISSON_1D  U = -|x|/2 in 1D (Sec. 2.2, the 1D case), FP64 plans only: the Gaussian
 *                   G_1 carrying rho-hat(0) and (x rho)-hat(0) is split off, its potential
 *                   u_1 = rho-hat(0) u_{1,1} - (x rho)-hat(0) u_{1,2} is taken in closed form
 *                   (Eq. (1DPois)), and u_2 = (1/2pi) int_{-P}^{P} W(k) e^{ikx} dk with
 *                   W(k) = (rho-hat(k) - G_1-hat(k)) / k^2, W(0) = -(x^2 rho)-hat(0)/2 +
 *                   sigma^2 rho-hat(0)/2, by the rectangle rule on the frequencies
 *                   k_l = l pi/(n h), l = -n..n-1, of the zero-padded 2n-point grid, rho-hat by
 *                   the trapezoid sum; sigma = 6 sqrt(2)/P, P = min(kmax, pi/h) (default pi/h).
 *                   The nodes, tiles and quadrature counts of nlp_opts do not apply.        */
typedef enum {
    NLP_COULOMB_3D = 0,
    NLP_DIPOLE_3D = 1,
    NLP_COULOMB_2D = 2,
    NLP_POISSON_2D = 3,
    NLP_CONFINED_2D = 4,
    NLP_POISSON_1D = 5
} nlp_kernel;

typedef enum { NLP_FP64 = 0, NLP_FP32 = 1 } nlp_precision;

typedef struct {
    int dim;        /* 1, 2 or 3 (must match the kernel) */
    int n[3];       /* points per axis: even, 8..1024, of the form 2^a 3^b 5^c; 3D: n <= 256 */
    double L[3];    /* half-widths, > 0 */
} nlp_grid;

typedef struct {
    double kmax;            /* truncation radius P of the Fourier ball (Sec. 2.1); 0 -> pi / max h */
    int n_r, n_theta, n_phi;/* quadrature counts (radial GL, GL in cos(theta), trapezoid in phi);
                               0 -> n_r = n_theta = roundup16(P R/2 + 16), n_phi = roundup16(P Rp + 32)
                               with R, Rp the half-diagonals of the box and of its first two axes.
                               n_theta and n_phi must be even (k -> -k symmetry). */
    double dipole_axis[3];  /* NLP_DIPOLE_3D: unit vector (normalised here; zero vector -> z) */
    double nufft_tol;       /* NUFFT tolerance, 1e-14..1e-2; 0 -> 1e-12 (FP64) / 1e-6 (FP32) */
    int tile;               /* spread/interp tile edge in fine cells: 0 = default, else 2..32 */
    int spread_variant;     /* 0 = default (3D: register-column kernels where the width is supported),
                               1 = the generic one-warp-per-node kernel everywhere */
    int method;             /* 0 = NUFFT per evaluation (default).  1 = precomputed discrete kernel:
                               the quadrature sum of Eq. (ifft) equals sum_i' K(i - i') rho_i' with
                               K(m) = sum_j w_j |k_j|^{d-1} U-hat(k_j) cos(k_j . m h) h^d / (2 pi)^d;
                               the plan computes K once (type-1 NUFFT of the weights onto the doubled
                               grid) and each evaluation is an aperiodic convolution by FFT on the
                               2n grid.  Not for NLP_POISSON_2D (its operator is not translation
                               invariant): NLP_ERR_UNSUPPORTED.
                               2 = the improved algorithm (Sec. 2.1, Eq. (3.9); Fig. 3.1): with a
                               partition of unity p(k), phi = I_1 + I_2 where I_1 takes (1 - p) U-hat
                               by the rectangle rule on the 2n grid's frequencies (an FFT convolution
                               with an analytic multiplier over the whole frequency box) and I_2 takes
                               p U-hat by the quadrature of Eq. (ifft) on the ball |k| <= k2 where
                               p >= eps (NUFFT with few nodes).  (kappa, eps) = (5.5, 1e-16) for FP64
                               and (3.8, 1e-8) for FP32 plans; default counts follow from k2.
                               NLP_COULOMB_3D, NLP_DIPOLE_3D: p = exp(-|k|^2/a), a = (kappa/min L)^2,
                                 k2 = min(P, sqrt(a ln 1/eps)).
                               NLP_COULOMB_2D: p = erfc(|k|/l), l = kappa/min L (w = erf(|k|/l)/|k| is
                                 smooth at k = 0, which no Gaussian p gives for U-hat = 1/|k|),
                                 k2 = min(P, l erfc^-1(eps)).
                               NLP_POISSON_2D: p = exp(-|k|^2/a) (w = (1 - p)/|k|^2 is smooth); I_2 is
                                 Algorithm 1 on the small ball with the integrand of u_2 times p and
                                 u_1 taken with the width sqrt(sigma^2 + 2/a), sigma = 6 sqrt(2)/k2.
                               NLP_CONFINED_2D and 1D plans: NLP_ERR_UNSUPPORTED. */
    int reserved[5];        /* must be zero */
    double confine_eps;     /* NLP_CONFINED_2D: the confinement ratio eps >= 0 (else ignored) */
} nlp_opts;

typedef struct nlp_plan_s *nlp_plan;

/* Plan facts for tests and roofline accounting. */
typedef struct {
    int dim, kernel, precision;
    int n[3], nf[3];        /* grid and oversampled (2n) fine grid */
    int width;              /* spreading-function width w (fine cells) */
    double beta_es;         /* shape parameter of the exp-of-semicircle function */
    double kmax;            /* P */
    int n_r, n_theta, n_phi;
    int64_t nodes_total;    /* full symmetric node count M */
    int64_t nodes_half;     /* nodes processed (k -> -k half) */
    int64_t tiles, chunks;  /* non-empty tiles; work items of the interp/spread kernel */
    int tile;
    size_t workspace_bytes; /* device memory owned by the plan */
    double sigma_poisson;   /* NLP_POISSON_2D: width of the auxiliary Gaussian */
    int sub_tile;           /* register-column kernel sub-tile edge (0: the generic one-warp-per-node kernel) */
    int64_t segments;       /* register kernel work units (node runs of one sub-tile) */
    double split_a;         /* method 2: partition parameter, a (Gaussian p) or l (erfc p); 0 otherwise */
    double split_radius;    /* method 2: radius k2 of the NUFFT ball of I_2 (0 otherwise) */
    int64_t combine_entries;/* window slots summed by the combine pass, over all tiles of G */
} nlp_plan_info;

/* Create a plan: quadrature nodes and weights (FP64), their binning by fine-grid tile,
 * the spreading-function tables, FFT twiddles and all workspace.  Synchronous.
 * stream: a cudaStream_t (NULL = legacy default stream).  opts may be NULL (defaults). */
nlp_status nlp_plan_create(const nlp_grid *grid, nlp_kernel kernel, nlp_precision prec,
                           const nlp_opts *opts, void *stream, nlp_plan *out);

void nlp_plan_destroy(nlp_plan plan);

nlp_status nlp_plan_get_info(nlp_plan plan, nlp_plan_info *out);

/* phi = U * rho (Sec. 2.1 Eq. (ifft); Sec. 2.2 Algorithm 1 for NLP_POISSON_2D).
 * rho_dev, phi_dev: device arrays of prod(n) reals in the plan precision (may not alias).
 * Steps: deconvolve + zero-pad + forward FFT (type 2), interpolate at the nodes, scale by
 * the weights and |k|^{d-1} U-hat, spread (type 1), inverse FFT, deconvolve + crop. */
nlp_status nlp_eval_potential(nlp_plan plan, const void *rho_dev, void *phi_dev);

/* Same operation on HOST arrays: copies rho to plan-owned device memory, evaluates, copies
 * phi back and synchronizes the plan stream before returning. */
nlp_status nlp_eval_potential_host(nlp_plan plan, const void *rho_host, void *phi_host);

/* One step of the backward-Euler normalized gradient flow (Sec. 3.1, Eqs. (gf-eq2)-(gffg33)):
 *   b = V + g |phi^n|^2 + beta (U * |phi^n|^2),
 *   solve (1/tau - Delta/2 + b) phi^(1) = phi^n / tau, phi^{n+1} = phi^(1)/||phi^(1)||.
 * The linear solve (omitted in the paper) is the stabilised Fourier fixed point
 *   (1/tau + alpha + |mu|^2/2) phi^(m+1) = F[phi^n/tau + (alpha - b) phi^(m)],
 *   alpha = (max b + min b)/2, iterated until max|phi^(m+1) - phi^(m)| <= inner_tol or
 *   max_inner iterations (NLP_ERR_NOT_CONVERGED if the cap is hit).
 * phi_dev: real, normalised (h^d sum phi^2 = 1), updated in place; V_dev: real trap.
 * Norms, min/max and energies are reduced in FP64 for both precisions.
 * Outputs (host, may be NULL): *max_change = max|phi^{n+1} - phi^n| / tau (stopping rule of
 * Sec. 3.2), *inner_iters, energies[5] = {E, E_kin, E_pot, E_int, mu} of phi^{n+1}.
 * Synchronizes the plan stream.  NLP_ERR_DIVERGED if a non-finite value appears.
 * All kernels of 2D and 3D grids, NLP_POISSON_2D included (its potential through
 * Algorithm 1); NLP_POISSON_1D plans: NLP_ERR_UNSUPPORTED (as for nlp_gf_solve,
 * nlp_energies, nlp_energies_noalloc and nlp_ts_step). */
nlp_status nlp_gf_step(nlp_plan plan, void *phi_dev, const void *V_dev, double beta, double g,
                       double tau, double inner_tol, int max_inner, double *max_change,
                       int *inner_iters, double *energies);

/* The gradient flow run to convergence: nlp_gf_step repeated until
 * max|phi^{n+1} - phi^n| / tau <= stop_tol (the stopping rule of Sec. 3.2, epsilon_0 = 1e-10
 * there) or max_steps steps.  A step whose inner solve hits max_inner is kept (the iterate is
 * normalised) and the flow continues.  Outputs (host, may be NULL): *steps taken,
 * *max_change of the last step, energies[5] of the final phi.  NLP_ERR_NOT_CONVERGED if
 * max_steps ran out.  Synchronizes the plan stream. */
nlp_status nlp_gf_solve(nlp_plan plan, void *phi_dev, const void *V_dev, double beta, double g,
                        double tau, double stop_tol, int max_steps, double inner_tol, int max_inner,
                        int *steps, double *max_change, double *energies);

/* Energies {E, E_kin, E_pot, E_int, mu} of a real phi (Sec. 3.2), FP64 reductions.
 * Synchronizes the plan stream. */
nlp_status nlp_energies(nlp_plan plan, const void *phi_dev, const void *V_dev, double beta,
                        double g, double *energies);

/* Energies as nlp_energies, for callers that cannot let the library allocate device memory.
 * nlp_energies allocates the plan's gradient-flow workspace (cudaMalloc) on its first use.
 * A process whose device memory is already reserved by another allocator (a framework's
 * caching pool, an arena sized at start-up) may see that cudaMalloc fail or fragment its
 * pool, and a latency-bound loop may not accept the device-wide synchronisation that
 * cudaMalloc / cudaFree can imply.  This entry point calls no cudaMalloc, cudaFree or other
 * allocating routine: its buffers (density, potential, spectrum, FFT tables, FP64 partial
 * sums) live in one file-scope static device array of 1 MiB, which every GPU that loads the
 * library holds until the process exits.  The potential evaluation inside uses the spectra
 * that nlp_plan_create allocated.  (The paper has no counterpart: this is a deployment
 * variant of nlp_energies.)
 *  - Limit: grids of at most 32768 points (e.g. 32^3, 128 x 256); larger grids return
 *    NLP_ERR_INVALID_ARG before any launch.  NLP_POISSON_2D plans: NLP_ERR_UNSUPPORTED.
 *  - The first call on each device looks up the array's device address there
 *    (cudaGetSymbolAddress, with that device current); make that first call before any
 *    stream capture.
 *  - All calls share the array and it keeps the last call's contents; every value a call
 *    reads it first writes.  Calls that overlap on the GPU (other streams, other host
 *    threads) race on the array and must not be issued.
 *  - The energies are returned in host memory: the call synchronizes the plan stream. */
nlp_status nlp_energies_noalloc(nlp_plan plan, const void *phi_dev, const void *V_dev, double beta,
                                double g, double *energies);

/* One time step of the time-splitting Fourier pseudospectral method (Sec. 4.1):
 * order 2: K(tau/2) P(tau) K(tau/2) with the kinetic flow K solved exactly in Fourier space
 * and P(s): psi <- exp(-i (V + g|psi|^2 + beta U*|psi|^2) s) psi (Eq. (sps-eq68));
 * order 4: Yoshida's composition of three order-2 steps.  psi_dev: complex, in place. */
nlp_status nlp_ts_step(nlp_plan plan, void *psi_dev, const void *V_dev, double beta, double g,
                       double tau, int order);

/* ---------------------------------------------------------------- batched evaluation
 * Many FP32 plans (any mix of grids and of the NLP_COULOMB_3D / NLP_DIPOLE_3D /
 * NLP_COULOMB_2D kernels) evaluated by one replay of a CUDA graph, in one of two forms:
 *
 * NLP_BATCH_PERSISTENT (the default at creation): the graph holds ONE persistent kernel
 * launch.  Work items are (plan, stage, block) tasks taken in a fixed order from a device
 * ticket counter, stage-major (every plan's stage k before any plan's stage k + 1; the
 * default) or item-major (plan by plan); a stage of one plan starts when the previous stage
 * of the same plan has completed, which the device checks with a bounded number of polls
 * (NLP_ERR_TIMEOUT if a limit runs out; the batch stays usable).  Every stage runs at the one
 * CTA shape (256 threads, the largest stage's shared memory) of the persistent kernel.
 *
 * NLP_BATCH_GRAPH: the graph holds every plan's own stage launches (the kernels of
 * nlp_eval_potential, each at its own CTA shape), the plans spread over B parallel branches
 * (largest fine grid first, each to the branch with the least work so far); plans of one
 * branch run one after another.  The launches carry the rho / phi pointers, so an evaluation
 * with other pointers than the previous one captures the graph again first (the
 * instantiated graph is updated in place; a few milliseconds for 64 plans).
 *
 * nlp_batch_autotune times both forms and keeps the faster.  The batch uses the plans' own
 * workspaces: the plans must outlive the batch and must not be evaluated while a batch
 * evaluation is in flight.  Not thread-safe. */
typedef struct nlp_batch_s *nlp_batch;

/* plans: count FP32 plans of method 0 (NLP_POISSON_2D or another method: NLP_ERR_UNSUPPORTED).  stream: cudaStream_t
 * for all batch work (must not be the legacy NULL stream: graph capture). */
nlp_status nlp_batch_create(const nlp_plan *plans, int count, void *stream, nlp_batch *out);

/* phi_i = U_i * rho_i for every plan i: rho_dev[i], phi_dev[i] device arrays as for
 * nlp_eval_potential.  Asynchronous (one graph launch); call nlp_batch_sync for the result
 * status.  The pointer arrays are copied before return. */
nlp_status nlp_batch_eval(nlp_batch batch, const void *const *rho_dev, void *const *phi_dev);

/* Waits for the last nlp_batch_eval; NLP_ERR_TIMEOUT if a dependency poll ran out. */
nlp_status nlp_batch_sync(nlp_batch batch);

/* Persistent form: tasks, persistent CTAs and dynamic shared memory per CTA (any may be NULL). */
nlp_status nlp_batch_get_info(nlp_batch batch, int *tasks, int *grid_ctas, size_t *smem_bytes);

enum { NLP_BATCH_PERSISTENT = 0, NLP_BATCH_GRAPH = 1 };

/* Selects the form of the next nlp_batch_eval: mode NLP_BATCH_PERSISTENT or NLP_BATCH_GRAPH,
 * branches (graph form: 1..64, capped at the number of plans; ignored for the persistent
 * form).  Waits for an evaluation in flight.  NLP_ERR_INVALID_ARG for another mode or, in the
 * graph form, another branch count. */
nlp_status nlp_batch_set_mode(nlp_batch batch, int mode, int branches);

/* The form in use and the graph form's branch count (branches may be NULL). */
nlp_status nlp_batch_get_mode(nlp_batch batch, int *mode, int *branches);

/* The task order in use: *item_major = 0 (stage-major) or 1 (item-major). */
nlp_status nlp_batch_get_order(nlp_batch batch, int *item_major);

/* Autotuner of the batch's own launch: times the graph (4 replays, the first a warm-up) of
 * the persistent form for both task orders and the persistent grid at 1, 2, ... up to the
 * occupancy limit of CTAs per SM, and of the graph form at 1, 2, 4 and 8 branches, on these
 * inputs, and keeps the fastest form with its settings (the persistent form's best order and
 * grid are kept as well).  Outputs (may be NULL): *best_grid = the persistent CTAs, or 0 when
 * the graph form won; *best_ms per evaluation of the batch; nlp_batch_get_mode and
 * nlp_batch_get_order report what was kept.  Synchronous; the outputs phi_dev are
 * overwritten. */
nlp_status nlp_batch_autotune(nlp_batch batch, const void *const *rho_dev, void *const *phi_dev,
                              int *best_grid, double *best_ms);

/* Test hook: set the poll limit of the dependency waits and, if block_item and block_stage
 * are >= 0, make that stage of that item never count as complete, so the stages after it
 * run out of polls (failure injection on the host; the device only sees an unreachable
 * count).  Pass -1, -1 to restore normal operation.  Re-captures the graph.  Persistent form
 * only (the graph form has no polls). */
nlp_status nlp_batch_set_wait_limit(nlp_batch batch, long long polls, int block_item, int block_stage);

void nlp_batch_destroy(nlp_batch batch);

/* Spread-tile autotuner (2D and 3D grids; 1D: NLP_ERR_UNSUPPORTED): times complete evaluations of plans built with each candidate
 * tile edge (FP32 3D: 4, 8, 16; FP64 3D: 2, 4, 6; 2D: 8, 16, 32) on zero input (the work is
 * data independent) and returns the fastest in *best_tile with its time.  If cache_path
 * is not NULL the choice is looked up in / appended to that text file (one line per
 * configuration).  Allocates plan workspaces temporarily; synchronous. */
nlp_status nlp_autotune_tile(const nlp_grid *grid, nlp_kernel kernel, nlp_precision prec,
                             const nlp_opts *base, void *stream, const char *cache_path,
                             int *best_tile, double *best_ms);

/* Stage timers for measurement (not part of the method).  When enabled, each evaluation
 * records CUDA events on the plan stream between its stages; nlp_get_stage_times then
 * synchronizes on the last event and returns, for the most recent evaluation, up to max
 * (stage id, milliseconds) pairs in execution order.  Stage ids: */
enum {
    NLP_STAGE_FWD_LAST = 0,   /* deconvolve + zero-pad + R2C FFT along the last axis */
    NLP_STAGE_FWD_MID = 1,    /* forward FFT along axis 1 (3D) / axis 0 (2D) */
    NLP_STAGE_FWD_FIRST = 2,  /* forward FFT along axis 0 (3D only) */
    NLP_STAGE_COMBINE = 3,    /* sum the chunks' windows into the spreading target (writes all of it) */
    NLP_STAGE_SPREAD = 4,     /* interpolate -> scale -> spread (chunk windows to scratch) */
    NLP_STAGE_INV_FIRST = 5,  /* inverse FFT along axis 0 (3D only) */
    NLP_STAGE_INV_MID = 6,    /* inverse FFT along axis 1 (3D) / axis 0 (2D) */
    NLP_STAGE_INV_LAST = 7,   /* C2R FFT along the last axis + deconvolve + crop */
    NLP_STAGE_POISSON = 8,    /* 2D Poisson FP64 parts (moments, rho-hat(0), u_1) */
    NLP_STAGE_WINDOW_SUM = 9, /* sum the windows of tiles split into several chunks (before the combine) */
    NLP_STAGE_INTERP = 10     /* FP32 plans of the default 3D kernels: interpolation and scaling; the
                                 spreading follows as NLP_STAGE_SPREAD */
};
nlp_status nlp_set_stage_timing(nlp_plan plan, int on);
nlp_status nlp_get_stage_times(nlp_plan plan, int *stage_ids, double *ms, int max, int *count);

/* ---------------------------------------------------------------------------------------
 * Learned initial guess for the gradient flow (the paper has no counterpart; the flow it
 * starts is unchanged and still decides the ground state).  A network maps the features
 *   f = [log10(beta)/3, (gamma - 1)/3, kernel == NLP_COULOMB_3D, kernel == NLP_DIPOLE_3D]
 * (beta: interaction strength, gamma: trap anisotropy of V = (x^2 + y^2 + gamma^2 z^2)/2) to
 * a ground-state amplitude on a 48^3 grid over [-box_L, box_L)^3 (point j at
 * -box_L + j * 2 box_L / 48):
 *   MLP 64 -> 512 -> 512 -> 512 -> 512 (SiLU; f zero-padded to 64) -> 1792 (linear; the
 *   first 1728 outputs are 8 channels of 6^3), then [nearest x2, 3^3 conv 8->8, SiLU] at 12^3
 *   and 24^3, nearest x2 and a 3^3 conv 8->1 at 48^3 (zero padding).
 * Parameters are one FP32 vector, in this order: for l = 0..4, W_l [out][in] row-major then
 * b_l [out] (sizes 512x64, 512x512 (3x), 1792x512); then for each conv layer w [co][ci][27]
 * (tap d = 9 dz + 3 dy + dx for offsets (dz, dy, dx) - 1 in {-1, 0, 1}, input position
 * p + offset) then bias [co].  Padding entries (W_0 columns >= 4, W_4 rows >= 1728, b_4
 * entries >= 1728) start at zero and receive zero gradient.
 * mode 0: dense layers as BF16 tensor-core GEMMs (tcgen05, FP32 accumulation) on BF16
 * copies of the weights; mode 1: the same on FP32 CUDA cores (gradient checks).
 * Batches hold 1..128 samples: features [B][4] and targets [B][48^3] FP32 on the device.
 * All calls run on the given stream and are not thread-safe per object. */
typedef struct nlp_surrogate_s *nlp_surrogate;

/* Feature vector for (beta, gamma, kernel) as defined above (host). */
void nlp_surrogate_features(double beta, double gamma, nlp_kernel kernel, float *feat4);

/* Allocates the network (about 1.7 GB of device memory for batches up to 128) and
 * initialises W ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from seed, biases zero.  Synchronous. */
nlp_status nlp_surrogate_create(double box_L, unsigned long long seed, int mode, void *stream,
                                nlp_surrogate *out);
int64_t nlp_surrogate_num_params(nlp_surrogate s);
nlp_status nlp_surrogate_get_params(nlp_surrogate s, float *params_host);
nlp_status nlp_surrogate_set_params(nlp_surrogate s, const float *params_host);

/* out_dev [B][48^3] = network(feat_dev [B][4]).  Synchronizes; NLP_ERR_TIMEOUT if a
 * tensor-core wait ran out. */
nlp_status nlp_surrogate_forward(nlp_surrogate s, const float *feat_dev, int B, float *out_dev);

/* Loss = mean over B x 48^3 of (out - target)^2 and its gradient with respect to every
 * parameter, copied to grads_host (may be NULL) in the parameter layout.  Synchronizes. */
nlp_status nlp_surrogate_gradients(nlp_surrogate s, const float *feat_dev, const float *target_dev,
                                   int B, double *loss, float *grads_host);

/* One AdamW step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, decoupled weight
 * decay) on that loss.  Synchronizes only when loss is not NULL. */
nlp_status nlp_surrogate_train_step(nlp_surrogate s, const float *feat_dev, const float *target_dev,
                                    int B, float lr, float weight_decay, double *loss);

/* The network learns the correction to the beta = 0 ground state of the trap,
 *   b(x) = gamma^{1/4} pi^{-3/4} exp(-(x^2 + y^2 + gamma z^2)/2):
 * training targets are (ground state - b) on the 48^3 cube.  out_dev [B][48^3] = b on the
 * cube for gamma_dev [B] (device FP32).  Asynchronous. */
nlp_status nlp_surrogate_base(nlp_surrogate s, const float *gamma_dev, int B, float *out_dev);

/* Initial guess for nlp_gf_step / nlp_gf_solve on a 3D grid:
 *   phi = S[max(0, b(x) + c(x))] normalised to h^3 sum phi^2 = 1 (FP64 reductions),
 * c = the network output for (beta, gamma, kernel) sampled trilinearly at the grid points
 * (zero outside the 48^3 cube), S = the average over the 8 reflections x_a -> -x_a of the
 * grid (index i -> (n - i) mod n on each axis): the trap and both kernels are even under
 * each reflection, and so is the ground state.  Written in the given precision.
 * kernel: NLP_COULOMB_3D or NLP_DIPOLE_3D.  Synchronizes. */
nlp_status nlp_surrogate_initial_guess(nlp_surrogate s, double beta, double gamma, nlp_kernel kernel,
                                       const nlp_grid *grid, nlp_precision prec, void *phi_dev);

void nlp_surrogate_destroy(nlp_surrogate s);

/* Kernel classes of a training step, for the per-class timers below. */
enum {
    NLP_SK_GEMM = 0,        /* dense layers: the tensor-core GEMM (mode 1: the FP32 one) */
    NLP_SK_CONV_FWD = 1,    /* 3^3 convolutions, forward */
    NLP_SK_CONV_BWD_IN = 2, /* 3^3 convolutions, gradient of the input */
    NLP_SK_CONV_BWD_W = 3,  /* 3^3 convolutions, gradient of the weights (both stages) */
    NLP_SK_ELEMENTWISE = 4, /* bias/activation, upsampling, BF16 conversion, packing */
    NLP_SK_LOSS = 5,        /* mean squared error and its gradient */
    NLP_SK_ADAMW = 6,       /* the optimizer step */
    NLP_SK_COUNT = 7
};

/* Per-class kernel timers of nlp_surrogate_train_step (measurement, not part of the method).
 * on != 0: every later training step records a CUDA event after each of its launches on the
 * object's stream and, at its end, waits for the last event and adds each interval to the
 * class of the launch that ended it (so an interval also holds the launch gap before that
 * kernel).  Enabling or disabling resets the totals.  The first enable creates the events. */
nlp_status nlp_surrogate_set_timing(nlp_surrogate s, int on);

/* ms[NLP_SK_COUNT]: milliseconds per class summed since the timers were enabled;
 * launches[NLP_SK_COUNT] (may be NULL): timed intervals per class (one per launch, except the
 * two-stage weight gradient of a convolution, timed as one interval). */
nlp_status nlp_surrogate_get_kernel_times(nlp_surrogate s, double *ms, int64_t *launches);

/* Test hook for the tensor-core GEMM of the network: C[M x N] (FP32) = A[M x K] B[N x K]^T,
 * A and B BF16 row-major device arrays; M % 128 == 0, K % 64 == 0, N % 64 == 0.
 * Synchronizes; NLP_ERR_TIMEOUT if a tensor-core wait ran out. */
nlp_status nlp_gemm_bf16(const void *A_dev, const void *B_dev, float *C_dev, int M, int N, int K,
                         void *stream);

/* Measured FMA throughput of the GPU in flop/s for the given precision (a microbenchmark of
 * independent FMA chains over all SMs, best of 3 timed runs); the denominator of the ALU
 * roofline of the interpolation/spreading kernel.  Allocates 64 bytes; synchronizes. */
nlp_status nlp_measure_alu_peak(int precision, void *stream, double *flops_per_s);

const char *nlp_status_string(nlp_status s);

/* Library version string. */
const char *nlp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NLPOT_H */
