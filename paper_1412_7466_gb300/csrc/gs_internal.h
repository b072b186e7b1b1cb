// Internal context of the gsolve library (not part of the ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/gsolve.h"
#include "gs_common.cuh"

// complex64 pair table h[i][q][s] of one geometry (s = (l+1) M + j fastest, row stride sp = 3M rounded
// up to 32 images) and its TMA map (boxes of 32 images x (4p+1) orders)
struct gs_tab32 {
    float2 *h = nullptr;
    long sp = 0;
    CUtensorMap map;
};

// Row and column blocks of A (Eq. matA): unknowns [mu1, sigma1, mu2, sigma2, a2, a1, a3, c, d];
// rows [Gamma1 value, Gamma1 normal, Gamma2 value, Gamma2 normal, middle walls (value, x-deriv),
// upper walls, lower walls, Gamma_u (value, y-deriv), Gamma_d (value, y-deriv)].
struct Layout {
    int N, Q1, Q2, Q3, K, nw1, nw2, nw3, nb;
    int col_mu1, col_sig1, col_mu2, col_sig2, col_a2, col_a1, col_a3, col_c, col_d, cols;
    int row_g1v, row_g1n, row_g2v, row_g2n, row_w2v, row_w2n, row_w1v, row_w1n, row_w3v, row_w3n,
        row_uv, row_un, row_dv, row_dn, rows;
    int nB() const { return col_a1; }     // columns of B_phys: mu1..a2
    int nC() const { return row_w1v; }    // rows of C: Gamma1, Gamma2, middle walls
};

// largest |entry| of C held in double-float form: products with the inner operator's input (|x| of
// order 1) and their sums over up to ~1e6 columns stay inside the FP32 exponent range
#define GS_DF_LIMIT 1e30
// inner products of the complex64 Arnoldi step: at most this many blocks share one basis vector
#define GS_DOT_SPLIT 32
// partial squared norms of the Arnoldi vector (one per block of the second Gram-Schmidt pass)
#define GS_NORM_PARTS 4096

struct AngleData {
    double theta = 0, kappa0 = 0;
    cplx alpha = {1, 0};
    double *kappa = nullptr;     // 2K+1
    cplx *k1n = nullptr;         // 2K+1, k_{1,n}
    cplx *k3n = nullptr;         // 2K+1, k_{3,n}
    cplx *f = nullptr;           // rows
    cplx *W = nullptr;           // rows x cols column-major U (orthonormal left singular vectors)
    cplx *Vr = nullptr;          // cols x cols row-major V Sigma (= P W_x)
    double *dscale = nullptr;    // cols, column scaling D
    double *coef = nullptr;      // cols, 1/(sigma max(sigma, eps)) (0 for sigma = 0)
    double *sigma = nullptr;     // cols
    cplx *B = nullptr;           // n x nB row-major (physical sign)
    cplx *Cm = nullptr;          // nC x n row-major
    mutable float2 *B32 = nullptr;   // complex64 copy of B for the mixed inner operator (on first use)
    mutable float4 *C2 = nullptr;    // double-float (hi, lo) copy of C for the mixed inner operator
    mutable bool C2_off = false;     // C has entries beyond GS_DF_LIMIT (or no memory for the copy):
                                     // the inner operator keeps the FP64 product
    mutable bool C2_ready = false;   // C2 holds the split of the current C
    mutable float4 *WH2 = nullptr;   // double-float U^H rows (cols x nC row-major) for the mixed inner operator
    mutable float4 *Vr2 = nullptr;   // double-float rows of V Sigma diag(coef) (nB x cols row-major)
    mutable bool A2_off = false;     // no memory for them, or an entry beyond GS_DF_LIMIT: FP64 products
    mutable bool A2_ready = false;   // WH2 and Vr2 hold the split of the current factorisation
    cplx *beta = nullptr;        // n, last solution
    int sweeps = 0;              // FP64 Jacobi sweeps of the grating factorisation
    int sweeps32 = 0;            // FP32-guided sweeps before them
    double phase_ms[6] = {};     // factorisation phases: assembly, QR, FP32 sweeps, polar step, FP64 sweeps, U/V
    long long rot32[32] = {}, rot64[32] = {};   // rotations applied in each FP32 / FP64 sweep
    double ns_defect[6] = {};    // measured max |V^H V - I| before each Newton-Schulz step
    int ns_iters = 0;            // Newton-Schulz steps taken
    int iters = 0;               // GMRES iterations (all inner iterations for the mixed solve)
    int outer = 0;               // refinement sweeps of the mixed solve (0 for FP64)
    double relres = -1.0;
};

struct gs_batch;   // batched solves over many geometries (gs_batch.cu)
struct gs_angles;  // lockstep solves of one geometry at many angles (gs_angles.cu)
struct gs_mlp;     // network of the learned warm start (gs_warm.cu)

struct gs_ctx {
    int device = 0;
    int sms = 1;                  // streaming multiprocessors of the device (queried at gs_create)
    cudaStream_t stream = nullptr;
    std::string err;

    // layers
    bool have_layers = false;
    gs_layers L{};
    std::vector<double> four[4];   // h1_cos, h1_sin, h2_cos, h2_sin
    Layout lay{};
    double *curve[2] = {nullptr, nullptr};   // per interface: 7 arrays of N (x, px, py, nx, ny, speed, w)
    double *wall_y[3] = {nullptr, nullptr, nullptr};
    double *bound_x = nullptr;
    double *kress = nullptr;
    double *four_dev = nullptr;              // device copy of the Fourier coefficients
    double yL1 = 0, yL2 = 0;                 // interface heights at the walls
    double h1_min = 0, h2_max = 0;

    // polarisation (GS_TM or GS_TE)
    int pol = 0;

    // incidence
    std::vector<double> thetas;

    // inclusions
    bool have_inc = false;
    int M = 0, p = 0, nc = 0;
    double *xy = nullptr, *radius = nullptr, *kp = nullptr;
    double *kp_im = nullptr;                 // Im kp of lossy inclusions (null: all lossless)
    std::vector<double> radius_h, kp_h;      // host copies of the radii and Re kp
    // general inclusion shape (gs_set_inclusions_star): one star, rotated per inclusion
    bool is_star = false;
    struct {
        double a1 = 0, a2 = 0, kp = 0;
        int a3 = 0, n_nodes = 0;
    } star;
    double *star_phi = nullptr;              // M rotation angles
    cplx *S0 = nullptr;                      // nc x nc scattering matrix of the unrotated star
    cplx *Sblk = nullptr;                    // M x nc x nc rotated blocks (the preconditioner)
    cplx *s = nullptr;                       // M x nc

    bool grating_ready = false;   // per-angle factorisation of the empty grating is built
    bool factored = false;        // ... and the inclusion coupling for the current disks
    std::vector<AngleData> ang;

    // scratch
    cplx *v1 = nullptr, *v2 = nullptr, *v3 = nullptr;   // n each
    cplx *v4 = nullptr, *v5 = nullptr;                  // n each (refinement residual, correction)
    cplx *v6 = nullptr;                                 // n, block preconditioner scratch (general shapes)
    cplx *g = nullptr;                                  // rows
    cplx *w = nullptr, *x = nullptr;                     // cols
    float2 *x32 = nullptr;                               // cols, complex64 copy of x (B_phys input, mixed form)
    cplx *Vtmp = nullptr;                                // rows x cols, QR workspace
    cplx *Xtmp = nullptr, *Vxtmp = nullptr;              // cols x cols, Jacobi on R^*
    float2 *X32tmp = nullptr;                            // 2 x cols x cols: FP32 copy of R^* and its rotations
    double *nrm2 = nullptr;                              // cols, trailing column norms
    int *perm = nullptr;                                 // cols, column pivots
    cplx *tau = nullptr;                                 // cols, reflector scalars
    cplx *part = nullptr;                                // translation partials
    float2 *b32 = nullptr;                               // n, complex64 copy of the source coefficients
    float4 *img32 = nullptr;                             // 3M, (hi, lo) float image coordinates
    float4 *xdf = nullptr;                               // n, double-float split of the operator input
    float4 *adf = nullptr;                               // adf_n, double-float split of A^+'s vectors
    long adf_n = 0;
    int *iflag = nullptr;                                // one int, device-side flag
    cplx *htab = nullptr;                                // pair table of translation coefficients (optional)
    gs_tab32 tab32;                                      // its complex64 copy (on first complex64 use)
    bool tab32_off = false;                              // no room for it: complex64 recomputes the coefficients
    float2 *b3pad = nullptr;                             // complex64 phased source coefficients, 32-image tiles
    int *terr = nullptr;                                 // device flag: a bounded wait of the table kernel gave up
    void *tcA = nullptr;                                 // bfloat16 [T_-1 T_0 T_1] in real 2x2 form (on demand)
    long tcA_rows = 0, tcA_cols = 0;
    double tc_gamma = 1.0;                               // order rescaling of tcA (min(1, k2 r_min))
    void *tcA_sp[2] = {nullptr, nullptr};                // second and third bfloat16 parts of the same operator
    void *sp_scratch = nullptr;                          // scratch of the three-part multi-right-hand-side product
    size_t sp_scratch_bytes = 0;
    long sp_zeroed_R = -1;                               // R whose scratch padding is already zero
    void *tc_scratch = nullptr;                          // multi-right-hand-side scratch
    size_t tc_scratch_bytes = 0;
    long tc_zeroed_rp = -1, tc_zeroed_k = -1, tc_zeroed_R = -1;   // padding of the scratch already zero
    double table_budget_gb = -1.0;                       // < 0: half of the free device memory
    size_t part_elems = 0;
    // GMRES workspace
    int kdim = 0;
    cplx *Vk = nullptr;                                  // (kdim+1) x n (complex64 basis: reinterpreted)
    cplx *kv1 = nullptr, *kv2 = nullptr;                 // n each: complex64-basis GMRES work vectors
    float2 *kw32 = nullptr;                              // n, complex64 copy of the Arnoldi vector
    cplx *dpart = nullptr;                               // GS_DOT_SPLIT x 513 partial inner products
    double *npart = nullptr;                             // GS_NORM_PARTS partial squared norms
    cplx *Hh = nullptr;                                  // (kdim+1) x kdim column-major
    cplx *cs = nullptr, *sn = nullptr, *gg = nullptr, *yy = nullptr;
    double *dscal = nullptr;                             // device scalars
    double *hscal = nullptr;                             // pinned host scalars
    unsigned long long *dcount = nullptr;               // two device counters (rotations; Gram defect)
    unsigned *bar = nullptr;                             // grid barrier (count, generation) of cooperative kernels

    // instrumentation: kernel launches issued, optional event timing of the translation kernel
    unsigned long long nlaunch = 0;
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;   // start/stop pairs, reused
    std::vector<int> prof_prec;         // precision of each timed launch
    size_t prof_used = 0;               // events used since the last reset

    gs_batch *batch = nullptr;
    gs_angles *angles = nullptr;
    gs_mlp *mlp = nullptr;
    double min_center_dist = 0.0;   // smallest inclusion centre distance (minimum image), set_inclusions

    int n() const { return M * nc; }
};

// TE weights w1 = (k1/k2)^2, w3 = (k3/k2)^2 of the top and bottom layers (1, 1 for TM)
inline void gs_layer_weights(const gs_ctx *c, double *w1, double *w3) {
    const bool te = c->pol != 0;
    *w1 = te ? (c->L.k1 / c->L.k2) * (c->L.k1 / c->L.k2) : 1.0;
    *w3 = te ? (c->L.k3 / c->L.k2) * (c->L.k3 / c->L.k2) : 1.0;
}

void gs_batch_destroy(gs_ctx *c);
void gs_angles_destroy(gs_ctx *c);
void gs_mlp_destroy(gs_ctx *c);

#define GS_COUNT_LAUNCH(ctx) ((ctx)->nlaunch++)
// returns a (start, stop) event pair for timing one launch, or false when profiling is off
bool gs_prof_pair(gs_ctx *c, cudaEvent_t *e0, cudaEvent_t *e1, int precision);

// error helpers (defined in gs_api.cu)
int gs_fail(gs_ctx *c, int code, const std::string &msg);
#define GS_CUDA(ctx, call)                                                                       \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return gs_fail((ctx), e_ == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,     \
                           std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    } while (0)
#define GS_CHECK_LAUNCH(ctx) GS_CUDA(ctx, cudaGetLastError())
#define GS_TRY(expr)                \
    do {                            \
        int st_ = (expr);           \
        if (st_ != GS_OK) return st_; \
    } while (0)

// assembly (gs_assemble.cu)
int gs_build_geometry(gs_ctx *c);
int gs_assemble_A(gs_ctx *c, const AngleData &a, cplx *A, int lda);
int gs_assemble_f(gs_ctx *c, const AngleData &a, cplx *f);
int gs_angle_scalars(gs_ctx *c, AngleData &a);
int gs_mie(gs_ctx *c);
int gs_assemble_B(gs_ctx *c, const AngleData &a, cplx *B);
int gs_assemble_C(gs_ctx *c, const AngleData &a, cplx *Cm);
// the same for an explicit geometry (M disks at xy; the multipole order is the context's)
int gs_mie_geo(gs_ctx *c, int M, const double *radius, const double *kp, const double *kp_im, cplx *s);
int gs_assemble_B_geo(gs_ctx *c, const AngleData &a, int M, const double *xy, cplx *B);
int gs_assemble_C_geo(gs_ctx *c, const AngleData &a, int M, const double *xy, cplx *Cm);
// per-angle grating factorisation if not built yet (gs_api.cu)
int gs_ensure_grating(gs_ctx *c);
// factorisation (gs_svd.cu)
int gs_factor_angle(gs_ctx *c, AngleData &a);
// translation (gs_translate.cu)
int gs_translate_impl(gs_ctx *c, const AngleData &a, const cplx *beta, cplx *out, int precision);
// GS_OK when the complex64 translation's Hankel values stay inside the FP32 range for this geometry
// (|H_2p(k2 R_min)| <= 1e36), else GS_ERR_ARG with a message
int gs_c64_range(gs_ctx *c);
size_t gs_pair_table_elems(int M, int p);
int gs_build_pair_table(gs_ctx *c);
// complex64 pair table for the complex64 translation, built on first use when it fits (gs_translate.cu)
int gs_ensure_table32(gs_ctx *c);
size_t gs_tab32_bytes(int M, int p);
// allocates and builds the complex64 table of M inclusions at xy (rounded from htab when given)
int gs_tab32_build(gs_ctx *c, const double *xy, int M, int p, const cplx *htab, gs_tab32 *t, cudaStream_t st);
// out = T beta for one geometry from its complex64 table (b3: 32-image tiles of phased coefficients,
// part: partial sums, at least 64 M (2p+1)); active (nullable device flag): 0 -> out = 0, no work
int gs_tab32_translate(gs_ctx *c, const gs_tab32 &t, int M, int p, const cplx *beta, cplx alpha, float2 *b3,
                       cplx *part, size_t part_elems, cplx *out, const int *active, cudaStream_t st);
// GS_ERR_TIMEOUT if a bounded wait of that kernel gave up since the last check (synchronises)
int gs_check_table_wait(gs_ctx *c);
// plain (unswizzled) 2-D tensor map over a row-major rows x cols array (gs_tc.cu)
int gs_make_map_plain(gs_ctx *c, CUtensorMap *m, CUtensorMapDataType dt, const void *base, long rows, long cols,
                      long row_bytes, int box_cols, int box_rows);
// (hi, lo) float coordinates of the 3M images of M inclusions (complex64 translation), on stream st
int gs_build_images_c64(gs_ctx *c, const double *xy, int M, float4 *img, cudaStream_t st);
// Tensor-core translation of R concatenated coefficient vectors (R angles of the current geometry,
// image phases alpha_dev[r]) with the operator and the coefficients each split into three bfloat16
// parts (gs_tc.cu).  _prepare builds the three operator parts and the scratch for R (allocates: call
// it before any stream capture); _translate only launches kernels (capturable) and sets *err_dev if
// a device wait gave up.
int gs_tc_split_prepare(gs_ctx *c, int R);
int gs_tc_split_translate(gs_ctx *c, int R, const cplx *alpha_dev, const cplx *x, cplx *out, int *err_dev,
                          cudaStream_t st);
// general inclusion shapes (gs_shape.cu): scattering matrix of the star and its rotated blocks
int gs_star_blocks(gs_ctx *c);
void gs_kress_weights(int N, double *R, cudaStream_t st);
// tensor-core product C[M][N] = A[M][K] B[N][K]^T, bfloat16 in, FP32 out (gs_tc.cu)
int gs_tc_gemm_impl(gs_ctx *c, const void *A, const void *B, float *C, long M, long N, long K, int *err_dev,
                    cudaStream_t st, int kslices = 1);
// low-rank, operator, GMRES, Bragg (gs_solve.cu)
int gs_pinv_impl(gs_ctx *c, const AngleData &a, const cplx *g, cplx *x);
int gs_apply_impl(gs_ctx *c, const AngleData &a, const cplx *x, cplx *y, int precision);
// the mixed inner operator in two parts: copies of B_phys (complex64) and C (double-float) made once
// per geometry and angle (allocates), then y = x - s t + s B_phys A^+ C x for a given t = T x
// (launches only; uses the context's scratch vectors g, w, x, xdf)
int gs_prepare_c64(gs_ctx *c, const AngleData &a);
int gs_prepare_apinv_df(gs_ctx *c, const AngleData &a);
int gs_lowrank_c64(gs_ctx *c, const AngleData &a, const cplx *x, const cplx *t, cplx *y);
int gs_rhs_impl(gs_ctx *c, const AngleData &a, cplx *b);
// w = B_phys A^+ f: incoming coefficients of the empty grating's field about every centre
int gs_incoming_impl(gs_ctx *c, const AngleData &a, cplx *w);
// z = B_phys A^+ C x: the layer response to the inclusions' field (no scattering diagonal)
int gs_layer_response_impl(gs_ctx *c, const AngleData &a, const cplx *x, cplx *z);
int gs_solve_impl(gs_ctx *c, AngleData &a, const gs_solve_opts &o, const cplx *x0);
int gs_bragg_impl(gs_ctx *c, const AngleData &a, cplx *cd_host, double *flux);
// a = A^+ (f - C beta) for the last solution at this angle (cols)
int gs_layer_unknowns_impl(gs_ctx *c, const AngleData &a, cplx *x);
