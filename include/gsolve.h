/*
 * gsolve — C-ABI of the GB300 solver for plane-wave scattering by a three-layer periodic
 * dielectric grating whose middle layer holds M disk inclusions (Lai, Kobayashi, Barnett,
 * arXiv:1412.7466).
 *
 * All functions return an int status (GS_OK == 0 on success) and never throw across the ABI.
 * Host arrays passed to gs_set_* are copied; the library keeps no pointer to them.  Device
 * pointers passed to the compute calls are owned by the caller, must hold the stated number of
 * complex128 values (interleaved re, im) and must be valid on the context's device; the library
 * owns and frees (in gs_destroy) every buffer it allocates.  Every kernel runs on the stream given
 * to gs_create (the legacy default stream when NULL).  Calls on one context are not thread-safe.
 *
 * Paper notation used throughout: period d, interfaces Gamma1 (top) and Gamma2, wavenumbers
 * k1, k2, k3 of the three layers and kp inside a disk, incidence angle theta with
 * u_inc = exp(i k1 (cos(theta) x + sin(theta) y)) (sin(theta) < 0, downward), Bloch phase
 * alpha = exp(i k1 cos(theta) d), multipole order p (2p+1 coefficients per disk).
 */
#ifndef GSOLVE_H
#define GSOLVE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------------- */
#define GS_OK 0
#define GS_ERR_ARG 1             /* a null pointer, a size out of range, an angle index out of range */
#define GS_ERR_STATE 2           /* calls out of order (e.g. gs_solve before gs_factor)             */
#define GS_ERR_CUDA 3            /* a CUDA runtime call failed; gs_last_error() has the message      */
#define GS_ERR_OOM 4             /* device allocation failed                                         */
#define GS_ERR_GEOMETRY 5        /* overlapping disks (minimum-image), disk crossing an interface    */
#define GS_ERR_NOT_CONVERGED 6   /* GMRES hit maxit; the iterate and its residual remain readable    */
#define GS_ERR_NUMERIC 7         /* a NaN or Inf appeared in a result                                */
#define GS_ERR_TIMEOUT 8         /* a device-side wait gave up (bounded); the result is not valid   */

typedef struct gs_ctx gs_ctx;
typedef struct { double re, im; } gs_c128;

/* Precision of the inclusion-to-inclusion translation inside the matrix-vector product. */
#define GS_FP64 0                /* complex128 throughout                                            */
#define GS_C64 1                 /* complex64 translation with order rescaling, FP32 accumulation    */
#define GS_MIXED_BF16 3          /* gs_solve_angles: inner translation on the tensor cores (bfloat16 parts) */

/*
 * Layered grating (Sec. 2 "Problem formulation"; Sec. 3 discretisation; Sec. 6 parameters).
 * Interface j is the graph y = h_j(x) = hj_0 + sum_{m=1..n_fourier} (hj_cos[m-1] cos(2 pi m x/d)
 * + hj_sin[m-1] sin(2 pi m x/d)), x in [-d/2, d/2].  N equispaced parameter nodes per interface,
 * J-expansions of orders -Qj..Qj about the layer centres (0,(h1_0+y0)/2), (0,(h1_0+h2_0)/2),
 * (0,(h2_0-y0)/2) (Eq. qGreen2, repre1-repre3), Rayleigh-Bloch orders -K_rb..K_rb (Eqs. rad1,
 * rad2), n_wallj Gauss-Legendre nodes on the walls of layer j, n_bound equispaced nodes on
 * Gamma_u (y = y0) and Gamma_d (y = -y0), pseudo-inverse regularisation eps_pinv (Sec. 5).
 */
typedef struct {
    double d;
    double h1_0, h2_0;
    int n_fourier;
    const double *h1_cos, *h1_sin, *h2_cos, *h2_sin;   /* host, length n_fourier (NULL if 0) */
    double k1, k2, k3;
    int N;
    double y0;
    int Q1, Q2, Q3;
    int K_rb;
    int n_wall1, n_wall2, n_wall3;
    int n_bound;
    double eps_pinv;
} gs_layers;

/* Inclusions of one general shape (Sec. 4.1, 4.2): the star r(t) = a1 + a2 cos(a3 t), t in
 * [0, 2 pi) (Eq. par1), rotated counter-clockwise by phi[i] about the centre xy[2i], xy[2i+1] (host
 * arrays, copied), interior wavenumber kp (real), multipole order p.  gs_factor then computes the
 * star's (2p+1) x (2p+1) scattering matrix s_ln on the GPU from the second-kind boundary integral
 * equation of Eqs. intg1-intg2 on n_nodes equispaced boundary nodes (Kress's product rule for the
 * log-singular kernel differences; TE scales the interior potentials by (kp/k2)^2), solved by
 * Gaussian elimination with partial pivoting for the 2p+1 incident orders J_n(k2 r) e^{i n theta},
 * and the moment integral s_ln = (i/4) int [J_l(k2 r) e^{-i l theta} sigma_n + d_n(J_l(k2 r)
 * e^{-i l theta}) mu_n] ds; inclusion i gets e^{i phi_i (n - l)} s_ln (a counter-clockwise rotation;
 * the paper prints e^{i phi (l - n)} with the angle measured the other way).  The preconditioner S
 * becomes block diagonal (these blocks) in every single-geometry solve (FP64, mixed, many angles).
 * The geometry checks and the multipole expansions use the enclosing disks of radius a1 + |a2|,
 * which must not overlap (Sec. 4.2).  GS_ERR_ARG unless a1 > |a2|, 0 <= a3 <= 64, kp > 0 and
 * n_nodes even in [16, 1024]; GS_ERR_GEOMETRY as gs_set_inclusions.  Batched solves and the
 * learned warm start take disks only. */
typedef struct {
    int M;
    int p;
    const double *xy;
    const double *phi;
    double a1, a2;
    int a3;
    double kp;
    int n_nodes;
} gs_star_inclusions;
int gs_set_inclusions_star(gs_ctx *ctx, const gs_star_inclusions *inc);
/* The preconditioner's blocks S_i (M x (2p+1) x (2p+1), [i][l][n], device, caller-owned): the
 * rotated star matrices, or the diagonal disk coefficients for disks.  Needs gs_factor. */
int gs_get_scattering_blocks(gs_ctx *ctx, gs_c128 *S_dev);

/* Polarisation (Sec. 2): GS_TM (default, u the electric field; [u] = [d_n u] = 0 on the interfaces)
 * or GS_TE (u the magnetic field; [u] = [(1/eps) d_n u] = 0, eps_j proportional to k_j^2 for a
 * constant permeability; Sec. 7 leaves it to future work).  TE scales each layer's potentials by its
 * permittivity relative to the middle layer, w_j = (k_j/k_2)^2 (which keeps the system of the second
 * kind), the flux rows by 1/w_j, uses the TE disk coefficients and the TE energy identity
 * sum k_{1,n}|c_n|^2/w1 + sum k_{3,n}|d_n|^2/w3 = k1|sin theta|/w1 for gs_bragg's flux error.
 * Changing it discards every factorisation; kept across gs_set_layers. */
#define GS_TM 0
#define GS_TE 1
int gs_set_polarization(gs_ctx *ctx, int pol);

/* Disk inclusions (Sec. 4): M centres xy[2*i], xy[2*i+1] (host, unit cell x in [-d/2, d/2)),
 * radii and interior wavenumbers kp (host, length M), multipole order p (1 <= p <= 16). */
typedef struct {
    int M;
    int p;
    const double *xy;
    const double *radius;
    const double *kp;
} gs_inclusions;

typedef struct {
    double tol;       /* stop when ||b - L beta|| <= tol ||b|| (relative residual, Sec. 5)            */
    int maxit;        /* total iteration cap                                                          */
    int restart;      /* Krylov dimension before restart (capped at 512; the workspace grows on demand) */
    int precision;    /* GS_FP64: GMRES on the FP64 operator.  GS_C64: iterative refinement -- FP64
                         residual b - L beta, inner GMRES on the operator with the complex64
                         translation to relative residual inner_tol, FP64 correction; repeated until
                         the FP64 residual meets tol                                                 */
    double inner_tol; /* GS_C64: tightest inner GMRES tolerance; each correction is solved to
                         max(inner_tol, tol / (2 * current relative residual)); <= 0 means 1e-6     */
    int max_sweeps;   /* GS_C64: cap on the inner solves (1 = one complex64 solve from zero with no
                         FP64 correction, the pre-refinement iterate); <= 0 means 30                 */
} gs_solve_opts;

/* ---- context --------------------------------------------------------------------------------- */
/* Creates a context on CUDA device `device`; cuda_stream is a cudaStream_t (may be NULL). */
int gs_create(gs_ctx **out, int device, void *cuda_stream);
void gs_destroy(gs_ctx *ctx);
const char *gs_strerror(int status);
/* Detail of the last failure on this context (static storage owned by the context). */
const char *gs_last_error(gs_ctx *ctx);

/* ---- problem definition ---------------------------------------------------------------------- */
/* Sets the grating; invalidates any factorisation.  GS_ERR_ARG on non-positive sizes or
 * wavenumbers, N odd, N > 4096, or Q, K_rb, n_wall, n_bound outside [1, 1024]. */
int gs_set_layers(gs_ctx *ctx, const gs_layers *layers);
/* Incidence angles (host array of n_angles values, paper convention, sin(theta) < 0). */
int gs_set_incidence(gs_ctx *ctx, int n_angles, const double *theta);
/* Disks; GS_ERR_GEOMETRY if two disks overlap (minimum image in x) or a disk touches an
 * interface's extreme height band.  Requires gs_set_layers first. */
int gs_set_inclusions(gs_ctx *ctx, const gs_inclusions *inc);

/* Lossy inclusions (complex permittivity, Sec. 7): kp_im (host, length M of the current inclusions,
 * >= 0) is the imaginary part of each disk's interior wavenumber kp + i kp_im; NULL makes all disks
 * lossless again.  The disk coefficients then use J_n of complex argument (power series, for
 * |kp R| <= 12; GS_ERR_ARG beyond).  gs_bragg's flux error then measures the absorbed fraction.
 * Invalidates the inclusion part of the factorisation (call gs_factor again); gs_set_inclusions
 * resets the disks to lossless.  The batched solves take lossless disks. */
int gs_set_inclusion_loss(gs_ctx *ctx, const double *kp_im);

/* Builds, on the GPU in FP64, what the solve needs (Sec. 3 and Sec. 5).  Per incidence angle, once
 * for the grating: assembles the empty-grating matrix A (Eq. matA) and right-hand side f (Eq. Arhs),
 * rescales its J-expansion columns to unit 2-norm and takes the SVD A D = U Sigma V^* (pivoted
 * Householder QR, then one-sided Jacobi on R^*).  For the current disks: the scattering diagonal S
 * (Sec. 4.1), B_phys (Eq. matB, physical sign) and C (Eq. matC).  The grating part is kept until
 * gs_set_layers or gs_set_incidence; gs_set_inclusions only invalidates the disk part, so a new
 * geometry on the same grating re-runs only the coupling.  Must follow gs_set_layers,
 * gs_set_incidence and gs_set_inclusions. */
int gs_factor(gs_ctx *ctx);

/* The FP64 translation reads its coefficients H_q(k2 R) e^{i q Th} (all pairs and images) from a
 * table built by gs_factor for each geometry, 3 M^2 (4p+1) complex128 values, when that fits the
 * budget (default: half of the free device memory at gs_factor); otherwise it recomputes them in
 * the kernel.  The complex64 translation reads a complex64 copy of the same coefficients, built on
 * the geometry's first complex64 use under the same budget (else it too recomputes them).
 * budget_gb < 0 restores the default, 0 disables the tables built after the call. */
int gs_set_table_budget(gs_ctx *ctx, double budget_gb);

/* ---- sizes ----------------------------------------------------------------------------------- */
/* rows, cols of A; n = M (2p+1) unknowns; nB = columns of B_phys (4N + 2 Q2 + 1); nC = rows of C
 * (4N + 2 n_wall2).  Any output pointer may be NULL. */
int gs_dims(gs_ctx *ctx, int *rows, int *cols, int *n, int *nB, int *nC);

/* ---- parity / inspection (device outputs, caller-owned) -------------------------------------- */
/* A (unscaled) column-major rows x cols, lda = rows (Eq. matA), for angle index `angle`. */
int gs_get_A(gs_ctx *ctx, int angle, gs_c128 *A_dev);
/* f (Eq. Arhs), length rows. */
int gs_get_f(gs_ctx *ctx, int angle, gs_c128 *f_dev);
/* B_phys row-major n x nB and C row-major nC x n (Eqs. matB, matC; B carries the physical sign,
 * so the paper's B equals -B_phys).  Either pointer may be NULL. */
int gs_get_coupling(gs_ctx *ctx, int angle, gs_c128 *B_dev, gs_c128 *C_dev);
/* Disk scattering diagonal s, M x (2p+1), order index fastest (Sec. 4.1). */
int gs_get_scattering(gs_ctx *ctx, gs_c128 *s_dev);
/* x = A^+ g = D V Sigma^+ U^* g with Sigma^+ = min(1/sigma_j, 1/eps) (Eq. applypA); g length rows,
 * x length cols. */
int gs_pinv_apply(gs_ctx *ctx, int angle, const gs_c128 *g_dev, gs_c128 *x_dev);

/* ---- hot path (device vectors of length n, layout beta[i*(2p+1) + (m+p)]) ------------------- */
/* alpha = T beta: all-pairs Graf translation including the +-d images, self term (i, l=0) left
 * out (Sec. 4.2 Eq. trans, Sec. 5 Eq. repre3_mod).  precision GS_FP64 or GS_C64.  GS_C64 (also in
 * gs_apply and the mixed gs_solve) returns GS_ERR_ARG when the geometry's largest Hankel value,
 * |H_2p(k2 R_min)| with R_min the smallest centre distance, would exceed 1e36 (FP32 range). */
int gs_translate(gs_ctx *ctx, int angle, const gs_c128 *beta_dev, gs_c128 *alpha_dev, int precision);
/* y = L x = x - S T x + S B_phys A^+ C x (the preconditioned Schur operator, Sec. 5).  GS_FP64:
 * FP64 throughout.  GS_C64 (the inner operator of the mixed solve): complex64 translation and
 * complex64 B_phys; C x in double-float arithmetic (C and x as complex64 (hi, lo) pairs, 48-bit
 * significands; C is copied to that form on first use, or kept FP64 if an entry exceeds 1e30);
 * A^+ in FP64. */
int gs_apply(gs_ctx *ctx, int angle, const gs_c128 *x_dev, gs_c128 *y_dev, int precision);
/* b = S B_phys A^+ f (right-hand side of the preconditioned Schur system, Sec. 5). */
int gs_rhs(gs_ctx *ctx, int angle, gs_c128 *b_dev);
/* Solves L beta = b by restarted GMRES on the device (Sec. 5); beta0_dev (nullable) is the start.
 * Returns GS_ERR_NOT_CONVERGED if maxit is reached (the iterate stays readable). */
int gs_solve(gs_ctx *ctx, int angle, const gs_solve_opts *opts, const gs_c128 *beta0_dev);
/* Copies the last solution of `angle` into beta_dev (length n). */
int gs_get_beta(gs_ctx *ctx, int angle, gs_c128 *beta_dev);
/* Iterations and final relative residual ||b - L beta||/||b|| (recomputed in FP64) of the last solve;
 * for GS_C64 solves, iters counts all inner GMRES iterations. */
int gs_stats(gs_ctx *ctx, int angle, int *iters, double *relres);
/* Number of FP64 refinement sweeps of the last GS_C64 solve (0 after an FP64 solve). */
int gs_stats_refinement(gs_ctx *ctx, int angle, int *outer);
/* Statistics of the angle's factorisation of the empty grating (Sec. 5 "We precompute A = U Sigma
 * V^*"): the FP32 and FP64 one-sided Jacobi sweeps it took and, in phase_ms[6] (host, nullable),
 * the device time in ms of its phases: assembly of A and f, pivoted QR, FP32 sweeps, orthogonal
 * polar step and R^* V, FP64 sweeps, U = Q V_x and V Sigma; in rot32[32], rot64[32] (host,
 * nullable) the pair rotations applied in each sweep (0 past the last); in *ns_steps and ns_defect[6]
 * (host, nullable) the FP64 Newton-Schulz steps of the polar step and the measured max |V^H V - I|
 * before each of them and at the stop; where the last step was taken because the Frobenius norm x of
 * V^H V - I before it lay below 1e-7, the value after it is the bound (3/4) x^2 + x^3/4 and not a
 * measurement.  GS_ERR_STATE before the grating is factored (gs_factor or
 * gs_factor_batch), GS_ERR_ARG for a bad angle.  Host-only. */
int gs_factor_stats(gs_ctx *ctx, int angle, int *sweeps32, int *sweeps64, double *phase_ms, long long *rot32,
                    long long *rot64, int *ns_steps, double *ns_defect);
/* Bragg amplitudes of the propagating orders (Sec. 2 rad1/rad2; Sec. 5 alpha = A^+(f - C beta)),
 * written to HOST arrays: orders_top[*n_top], c[*n_top], orders_bot[*n_bot], d[*n_bot], each of
 * capacity >= 2 K_rb + 1, and the relative flux error
 * |sum k_{1,n}|c_n|^2 + sum k_{3,n}|d_n|^2 - k1|sin theta|| / (k1 |sin theta|)  (Sec. 6). */
int gs_bragg(gs_ctx *ctx, int angle, int *n_top, int *orders_top, gs_c128 *c,
             int *n_bot, int *orders_bot, gs_c128 *d, double *flux_err);

/* Allocation-free translation, for callers that cannot allocate device memory where they need it
 * (a framework whose pool owns the device heap, a real-time loop that allows no allocation after
 * start-up, code that runs without a gs_ctx).  The paper has no counterpart: it is the operation
 * of gs_translate (alpha = T beta over all pairs and the +-d images) without a context.  Inputs and
 * outputs are the caller's device buffers on the current device: xy_dev holds the M centres
 * (x, y interleaved, FP64), beta_dev and alpha_dev hold M (2p+1) complex128 values each (layout
 * of gs_translate; alpha_dev must not overlap the inputs), k2 is the middle-layer wavenumber, d
 * the period, alpha_re + i alpha_im the Bloch phase exp(i k1 cos(theta) d); precision GS_FP64 or
 * GS_C64; work is queued on cuda_stream (NULL = legacy default stream).  GS_FP64 is asynchronous.
 * GS_C64 first finds the smallest image distance R_min on the device and reads it back (one wait
 * for cuda_stream), then refuses with GS_ERR_ARG, as gs_translate does, a geometry whose largest
 * Hankel value |H_2p(k2 R_min)| would exceed 1e36 (FP32 range); the translation itself is then
 * queued asynchronously.
 * Nothing is allocated: the chunk partials live in a fixed device array of 2^19 complex128 values
 * (8 MiB) compiled into the library, which every GPU that loads the library holds until exit.
 * Sizes: M (2p+1) must not exceed 2^19 (524288) for GS_FP64; for GS_C64, whose complex64 copy of
 * beta, float image coordinates and R_min share the array, M (2p+1) + ceil(M (2p+1) / 2) + 3M + 1
 * must not exceed 2^19 (M <= 12945 at p = 12); else GS_ERR_ARG is returned before any device
 * work; GS_ERR_ARG also for M < 1, null or aliased pointers, k2 <= 0, d <= 0, an unsupported p or
 * precision; GS_ERR_CUDA if a launch fails.  The first call on a device looks up the array's
 * device address (once per device, with that device current); make that first call before any
 * stream capture.  All calls share the one array and it keeps the last call's contents: every
 * value a call reads there is written by that same call (R_min's slot is reset first), so nothing
 * needs clearing, but calls whose work overlaps on the GPU (other streams, other host threads)
 * race on the array and must be serialised by the caller. */
int gs_translate_noalloc(int M, int p, const double *xy_dev, double k2, double d, double alpha_re,
                         double alpha_im, const gs_c128 *beta_dev, gs_c128 *alpha_dev, int precision,
                         void *cuda_stream);

/* ---- batched solves (many geometries on one grating) ----------------------------------------- */
/* Batched form: G geometries of uneven size, all with the same multipole
 * order, share the per-angle grating factorisation; their translations run as one persistent launch
 * (an atomic work queue over (geometry, 4 targets, chunk of source images) items, largest geometries
 * first, chunk length and blocks per SM picked by timing candidates on the first factorisation),
 * the low-rank products are grouped over the geometries, and GMRES advances all of them in
 * lockstep, one CUDA-graph replay per Arnoldi step (the step reads its index from device memory).
 * Host arrays are copied; each geometry is validated as by gs_set_inclusions.  The batch replaces
 * the single-geometry inclusions of the context; gs_set_layers and gs_set_incidence discard it. */
int gs_set_inclusions_batch(gs_ctx *ctx, int G, const gs_inclusions *geos);
/* Grating factorisation (if not built) and S, B_phys, C of every geometry at every angle. */
int gs_factor_batch(gs_ctx *ctx);
/* y_g = L_g x_g for all g; x and y concatenate the geometries' vectors (geometry order). */
int gs_apply_batch(gs_ctx *ctx, int angle, const gs_c128 *x_dev, gs_c128 *y_dev, int precision);
/* Solves all geometries at `angle` (GS_FP64: lockstep GMRES; GS_C64: lockstep mixed refinement).
 * GS_ERR_NOT_CONVERGED if any geometry misses tol; per-geometry results stay readable. */
int gs_solve_batch(gs_ctx *ctx, int angle, const gs_solve_opts *opts);
int gs_batch_stats(gs_ctx *ctx, int angle, int g, int *iters, double *relres);
int gs_get_beta_batch(gs_ctx *ctx, int angle, int g, gs_c128 *beta_dev);
/* Bragg amplitudes of geometry g (host outputs as in gs_bragg). */
int gs_bragg_batch(gs_ctx *ctx, int angle, int g, int *n_top, int *orders_top, gs_c128 *c, int *n_bot,
                   int *orders_bot, gs_c128 *d, double *flux_err);
/* The autotuned source-image chunk length and blocks per SM of the batched translation. */
int gs_batch_tuning(gs_ctx *ctx, int *chunk, int *blocks_per_sm);

/* ---- many incidence angles of one geometry ---------------------------------------------------- */
/* Solves the current geometry at every incidence angle of the context (R = the n_angles given to
 * gs_set_incidence, 1 <= R <= 256) together, in a mixed form (the other fields of opts as for
 * gs_solve): per angle, FP64 residuals b_r - L_r beta_r and refinement to the relative residual tol
 * (Sec. 5, each angle its own quasi-periodic problem, Sec. 2 Eqs. quasi, rad1-rad2); the inner GMRES
 * advances all open angles in lockstep, each Arnoldi step of the R angles one CUDA-graph replay; the
 * low-rank part runs per angle (complex64 B_phys, double-float C x, FP64 A^+).  opts->precision
 * selects the inner translation:
 *   GS_MIXED_BF16: the geometry's operator [T_-1 T_0 T_1] applied to all R angles' vectors at once on
 *     the tensor cores (three bfloat16 parts of the operator and of the coefficients, the six products
 *     of parts whose orders add up to at most 2 accumulated in FP32, single-precision accuracy; the
 *     three operator parts take 3 x 2n x 6n x 2 bytes, 45 GB at M = 1000, p = 12; GS_ERR_OOM if they
 *     do not fit);
 *   GS_C64: each angle's translation from the geometry's complex64 pair table (as gs_translate with
 *     GS_C64; GS_ERR_OOM if the table does not fit; GS_ERR_ARG under the complex64 range check).
 * Needs gs_factor (all angles).  Per-angle results are read with gs_get_beta, gs_stats,
 * gs_stats_refinement and gs_bragg at that angle.  GS_ERR_NOT_CONVERGED if an angle misses tol
 * within maxit inner iterations (its iterate stays readable); GS_ERR_TIMEOUT if a device wait gave
 * up.  Synchronous. */
int gs_solve_angles(gs_ctx *ctx, const gs_solve_opts *opts);

/* ---- instrumentation (not part of the method) ------------------------------------------------ */
/* Kernel launches issued by this context since gs_create (all calls). */
int gs_launch_count(gs_ctx *ctx, unsigned long long *count);
/* enable != 0 starts CUDA-event timing of every launch of the translation kernel (the events are
 * recorded on the context's stream around the launch); any call resets the accumulated record. */
int gs_profile(gs_ctx *ctx, int enable);
/* Number of timed translation launches of the given precision (GS_FP64 or GS_C64) and their
 * summed device time in ms (synchronises). */
int gs_profile_read(gs_ctx *ctx, int precision, int *launches, double *total_ms);
/* Measures the FMA throughput of this GPU with independent multiply-add chains (precision GS_FP64,
 * GS_C64 for scalar FP32, or GS_PROBE_F32X2 for packed two-wide FP32 multiply-adds) over all SMs;
 * writes the achieved TFLOP/s (2 flops per FMA). */
#define GS_PROBE_F32X2 2
int gs_probe_fma(gs_ctx *ctx, int precision, double *tflops);

/* Total field at npts points of one period, in all three layers (the paper's field plots; Sec. 3
 * Eqs. repre1-repre3 and Sec. 5 Eq. repre3_mod with the last solution at `angle`): in the middle
 * layer the interface potentials at k2 (+-d copies), the far-copy J-expansion and the inclusions'
 * outgoing fields (+-d copies); in the top layer the incident wave, the potentials of Gamma1's
 * densities at k1 and the J-expansion about the top layer's centre, and above Gamma_u (y >= y0) the
 * incident wave plus the Rayleigh-Bloch expansion with the amplitudes c_n (Eq. rad1); in the bottom
 * layer the potentials of Gamma2's densities at k3 and the J-expansion about the bottom layer's
 * centre, and below Gamma_d (y <= -y0) the Rayleigh-Bloch expansion with d_n (Eq. rad2).
 * xy_dev holds (x, y) pairs, u_dev receives complex128 values (device arrays, caller-owned).
 * Points outside one period (|x| > d/2), exactly on an interface, or inside an inclusion give NaN;
 * accuracy is that of the trapezoid rule, i.e. a few node spacings (d/N) away from the interfaces.
 * Needs gs_solve at this angle (GS_ERR_STATE). */
int gs_field(gs_ctx *ctx, int angle, long npts, const double *xy_dev, gs_c128 *u_dev);

/* alpha_r = T(theta_r) beta_r for R right-hand sides at once (R incidence angles of the current
 * geometry; Sec. 4.2 Eq. trans with each angle's image phase a_r = exp(i k1 cos(theta_r) d), passed
 * in alpha_host[r]).  beta_dev and out_dev hold R consecutive vectors of length n (caller-owned
 * device memory).  The translation runs on the tensor cores in bfloat16 with FP32 accumulation:
 * the operator [T_-1 T_0 T_1] is built once per geometry in real 2x2 form (2n x 6n bfloat16,
 * 15 GB at M = 1000, p = 12; GS_ERR_OOM if it does not fit) and kept until the geometry changes.
 * Relative accuracy ~3e-3 (bfloat16 operands) -- an inner operator, not a final one.  Needs
 * gs_factor; GS_ERR_TIMEOUT if a device wait gave up.  Synchronous. */
int gs_translate_multi(gs_ctx *ctx, int R, const gs_c128 *alpha_host, const gs_c128 *beta_dev, gs_c128 *out_dev);
/* The operator of gs_solve_angles' inner solves: as gs_translate_multi, with the operator and the
 * coefficients each split into three bfloat16 parts (~24 significant bits together; the six
 * products of parts whose orders add up to at most 2 accumulated in FP32, single-precision accuracy;
 * three times the operator memory of gs_translate_multi).  Synchronous. */
int gs_translate_multi_split(gs_ctx *ctx, int R, const gs_c128 *alpha_host, const gs_c128 *beta_dev,
                             gs_c128 *out_dev);
#define GS_TC_BF16 3             /* gs_profile_read tag of the tensor-core product in gs_translate_multi
                                    (the same value as GS_MIXED_BF16) */

/* ---- tensor-core product ---------------------------------------------------------------------
 * C[M][N] = A[M][K] B[N][K]^T with A, B bfloat16 (row-major, K contiguous) and C FP32 (row-major),
 * accumulated in FP32 on the tensor cores (tcgen05).  The paper has no such routine: it is the dense
 * contraction under the multi-right-hand-side translation (Sec. 4.2 Eq. trans applied to many
 * angles at once).  M % 128 == 0, N % 256 == 0, K % 64 == 0, 16-byte aligned device pointers
 * (caller-owned), else GS_ERR_ARG; GS_ERR_TIMEOUT if a device wait gave up.  Synchronous. */
int gs_tc_gemm_bf16(gs_ctx *ctx, const void *A_dev, const void *B_dev, float *C_dev, long M, long N, long K);

/* ---- learned warm start ----------------------------------------------------------------------
 * The paper has no learned component: this is an addition to the iterative solve of Sec. 5 that
 * only chooses where GMRES starts; the converged answer is that of the zero start.
 * A per-inclusion network with weights shared by all inclusions maps 64 features to the part of the
 * incoming coefficients (Sec. 4.1: beta_i = s_i (.) alpha_i) that the empty grating's field
 * w = B_phys A^+ f does not give:
 *   features X[i][0..63] (FP32): x_i, y_i, sin and cos(2 pi j x_i / d) for j = 1..4 (in that
 *     order), theta, k1, Re and Im of w_i at order 0 (the empty grating's field at the centre),
 *     zeros;
 *   network: x0 = (X - mu) / sd, then Linear 64->128, SiLU, Linear 128->128, SiLU,
 *     Linear 128->2(2p+1); weights and activations in bfloat16, products accumulated in FP32;
 *     output row [Re of orders -p..p, Im of orders -p..p];
 *   start: beta_0 = s (.) (w + scale (.) (Re + i Im)), used only if ||b - L beta_0|| < ||b||.
 * Parameter vector (FP32, host, in this order): W1[64][128], b1[128], W2[128][128], b2[128],
 * W3[128][2(2p+1)], b3[2(2p+1)] (the trained weights, W[in][out] row-major), then mu[64], sd[64]
 * (feature standardisation, sd > 0) and scale[2p+1] (>= 0, per order; 0 leaves that order to the
 * empty grating's field and makes its target 0).  Device row arrays are row-major FP32 and
 * caller-owned. */
/* Length of the parameter vector for multipole order p, or -1 for an unsupported p. */
int gs_mlp_param_count(int p);
/* Loads the network for order p (copies the host vector; resets the Adam state).  GS_ERR_ARG for a
 * wrong length, non-finite values, sd <= 0 or scale < 0. */
int gs_mlp_set_params(gs_ctx *ctx, int p, const float *params, long n);
/* Copies the current parameters (trained weights + the fixed mu, sd, scale) to a host vector. */
int gs_mlp_get_params(gs_ctx *ctx, float *params, long n);
/* Y_dev[rows][2(2p+1)] = network(X_dev[rows][64]). */
int gs_mlp_forward(gs_ctx *ctx, const float *X_dev, long rows, float *Y_dev);
/* Mean squared error of network(X) against Y over all rows and outputs, and (grad_dev non-null)
 * its gradient with respect to the trained weights, in the parameter order (FP32 device vector of
 * the weights' length, caller-owned). */
int gs_mlp_loss_grad(gs_ctx *ctx, const float *X_dev, const float *Y_dev, long rows, float *grad_dev,
                     double *loss);
/* One full-batch Adam step (Kingma & Ba; beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on
 * the FP32 master weights; *loss is the loss before the step. */
int gs_mlp_train_step(gs_ctx *ctx, const float *X_dev, const float *Y_dev, long rows, double lr, double *loss);
/* Features of the current geometry at `angle` into X_dev[M][64] (needs gs_factor and a network of
 * the context's order). */
int gs_ws_features(gs_ctx *ctx, int angle, float *X_dev);
/* Fixes the network's normalisations from the current geometry and its last solution at `angle`
 * (run once, after the first solved sweep point), in place of the mu, sd and scale loaded by
 * gs_mlp_set_params (the trained weights are kept): mu and sd of each feature over the M inclusions
 * (mean and population standard deviation), except theta and k1, which take the sweep's uniform
 * ranges [theta_lo, theta_hi] and [k_lo, k_hi] (mean (lo + hi)/2, sd (hi - lo)/sqrt(12)); a constant
 * feature gets sd = 1.  scale[n] = rms over the inclusions of t_n (as in gs_ws_targets), or 0 where
 * the order's share of beta, rms(s_n t_n), is at most `share` times the largest order's (such orders
 * are left to the empty grating's field).  GS_ERR_ARG for lo >= hi, non-finite ranges or share < 0. */
int gs_ws_normalise(gs_ctx *ctx, int angle, double theta_lo, double theta_hi, double k_lo, double k_hi,
                    double share);
/* Training targets from the last solution at `angle`: Y_dev[M][2(2p+1)] = t / scale split as
 * [Re, Im], t = T beta - B_phys A^+ C beta (the incoming field from the other inclusions, their
 * images and the layers' response; equal to beta/s - w at a converged beta). */
int gs_ws_targets(gs_ctx *ctx, int angle, float *Y_dev);
/* From the last solution at `angle`, per order n (t as for gs_ws_targets): ms_host[n] = mean over
 * the inclusions of |t_n|^2 and ms_host[2p+1 + n] = mean of |s_n t_n|^2 (the order's share of
 * beta), 2(2p+1) values, to choose `scale`. */
int gs_ws_moments(gs_ctx *ctx, int angle, double *ms_host);
/* The warm start at `angle`: writes beta_0 (or zeros when ||b - L beta_0|| >= ||b||, FP64 check)
 * to beta0_dev (n complex128, caller-owned), its relative residual to *relres0 and 1/0 to *used.
 * Pass beta0_dev to gs_solve. */
int gs_warm_start(gs_ctx *ctx, int angle, gs_c128 *beta0_dev, double *relres0, int *used);

#ifdef __cplusplus
}
#endif
#endif /* GSOLVE_H */
