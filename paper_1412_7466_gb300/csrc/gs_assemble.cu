// Assembly on the GPU (FP64): discretisation of the empty grating, the block matrix A and the
// right-hand side f (Sec. 3: Eqs. repre1-repre3, slp, dlp, jr1-jr4, bound1-bound3, matA, Arhs),
// the disk scattering diagonal (Sec. 4.1) and the coupling matrices B_phys, C (Sec. 5: Eqs.
// repre3_mod, matB, matC and Remark "cancel").
//
// Discretisation: N equispaced parameter nodes x_i = -d/2 + (i+1/2) d/N per interface with
// periodic trapezoid weights; near copies l = -1, 0, 1 with Bloch phases alpha^l (Eq. qGreen2,
// P = 1).  Self blocks use the periodic log-singular product rule of Kress (1991) on a windowed
// log coefficient (in place of the paper's Alpert corrections), with the Bloch phase applied to
// neighbours across the period end.  Wall rows use the cancelled form alpha^2 u_{+1}(L) -
// alpha^{-1} u_{-2}(L).
#include "gs_internal.h"
#include "gs_kernels.cuh"

namespace {

constexpr int TPB = 256;
inline int nblk(long n, int t = TPB) { return (int)((n + t - 1) / t); }

struct Curve {
    const double *x, *px, *py, *nx, *ny, *sp, *w, *curv;
};
Curve curve_of(const double *base, int N) {
    return Curve{base, base + N, base + 2 * N, base + 3 * N, base + 4 * N, base + 5 * N, base + 6 * N, base + 7 * N};
}

// ---- geometry -------------------------------------------------------------------------------

__global__ void k_curve_nodes(int N, double d, double h0, int nf, const double *ca, const double *sa,
                              double *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double x = -0.5 * d + (i + 0.5) * d / N;
    double h = h0, hp = 0.0, hpp = 0.0;
    for (int m = 1; m <= nf; ++m) {
        double om = 2.0 * GS_PI * m / d, s, c;
        sincos(om * x, &s, &c);
        h += ca[m - 1] * c + sa[m - 1] * s;
        hp += -ca[m - 1] * om * s + sa[m - 1] * om * c;
        hpp += -(ca[m - 1] * c + sa[m - 1] * s) * om * om;
    }
    double sp = sqrt(1.0 + hp * hp);
    out[i] = x;
    out[N + i] = x;
    out[2 * N + i] = h;
    out[3 * N + i] = -hp / sp;
    out[4 * N + i] = 1.0 / sp;
    out[5 * N + i] = sp;
    out[6 * N + i] = sp * d / N;
    out[7 * N + i] = hpp / (sp * sp * sp);   // signed curvature with respect to the upward normal
}

// Gauss-Legendre nodes on [lo, hi], ascending, by Newton iteration on P_n.
__global__ void k_gauss_legendre(int n, double lo, double hi, double *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int ir = n - 1 - i;   // descending root index -> ascending output
    double x = cos(GS_PI * (ir + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double pn = (n == 1) ? x : p1, pnm1 = (n == 1) ? 1.0 : p0;
        double dp = n * (x * pn - pnm1) / (x * x - 1.0);
        double dx = pn / dp;
        x -= dx;
        if (fabs(dx) < 1e-17) break;
    }
    out[i] = 0.5 * (hi + lo) + 0.5 * (hi - lo) * x;
}

__global__ void k_linspace_mid(int n, double lo, double hi, double *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = lo + (i + 0.5) * (hi - lo) / n;
}

// Kress weights R_m (m = 0..N-1) of int_0^{2pi} log(4 sin^2((t-s)/2)) f(s) ds on N nodes.
__global__ void k_kress(int N, double *R) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    double acc = 0.0;
    for (int q = N / 2 - 1; q >= 1; --q) acc += cos(2.0 * GS_PI * (double)((long)q * m % N) / N) / q;
    R[m] = -(4.0 * GS_PI / N) * acc - (4.0 * GS_PI / ((double)N * N)) * ((m & 1) ? -1.0 : 1.0);
}

// Kress weights for the closed-curve equations of general inclusion shapes (gs_shape.cu)
}  // namespace
void gs_kress_weights(int N, double *R, cudaStream_t st) { k_kress<<<nblk(N), TPB, 0, st>>>(N, R); }
namespace {

// Self blocks of one interface: differences of the ka and kb operators, wa S_ka - wb S_kb,
// wa D_ka - wb D_kb, N_ka - N_kb, T_ka - T_kb (the weights are the TE permittivity ratios of the two
// sides, 1 for TM), near copies with Bloch phases, Kress-corrected.  Writes A11-type blocks:
//   [row_v, col_mu] = (wa + wb)/2 I + D,  [row_v, col_sig] = S,  [row_n, col_mu] = T,
//   [row_n, col_sig] = -I + N.
__global__ void k_self_ops(int N, double d, Curve cv, cplx alpha, double ka, double kb, double wa, double wb,
                           const double *R, cplx *A, int lda, int row_v, int row_n, int col_mu,
                           int col_sig) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)N * N) return;
    int i = (int)(t / N), j = (int)(t % N);
    double h = d / N;
    cplx F[4] = {C(0, 0), C(0, 0), C(0, 0), C(0, 0)};
    cplx ainv = cconj(alpha);   // |alpha| = 1
    for (int l = -1; l <= 1; ++l) {
        if (l == 0 && i == j) continue;
        double Rx = cv.px[i] - (cv.px[j] + l * d), Ry = cv.py[i] - cv.py[j];
        K4 a = layer_kernels(Rx, Ry, cv.nx[i], cv.ny[i], cv.nx[j], cv.ny[j], ka);
        K4 b = layer_kernels(Rx, Ry, cv.nx[i], cv.ny[i], cv.nx[j], cv.ny[j], kb);
        cplx ph = (l == 0) ? C(1, 0) : (l == 1 ? alpha : ainv);
        F[0] = cadd(F[0], cmul(ph, csub(cscale(a.S, wa), cscale(b.S, wb))));
        F[1] = cadd(F[1], cmul(ph, csub(cscale(a.D, wa), cscale(b.D, wb))));
        F[2] = cadd(F[2], cmul(ph, csub(a.N, b.N)));
        F[3] = cadd(F[3], cmul(ph, csub(a.T, b.T)));
    }
    double hw = h * cv.sp[j];
    cplx out[4];
    double W = d / (2.0 * GS_PI) * R[((i - j) % N + N) % N];
    if (i != j) {
        double dx = (cv.x[j] - cv.x[i]) / d;
        double lstar = -rint(dx);
        double u = dx + lstar;
        double psi = gs_window(u);
        double L[4] = {0, 0, 0, 0};
        cplx ph = C(1, 0);
        if (psi > 0.0) {
            double Rx = cv.px[i] - (cv.px[j] + lstar * d), Ry = cv.py[i] - cv.py[j];
            double la[4], lb[4];
            log_coeffs(Rx, Ry, cv.nx[i], cv.ny[i], cv.nx[j], cv.ny[j], ka, la);
            log_coeffs(Rx, Ry, cv.nx[i], cv.ny[i], cv.nx[j], cv.ny[j], kb, lb);
            for (int q = 0; q < 4; ++q) {
                const double w_a = q < 2 ? wa : 1.0, w_b = q < 2 ? wb : 1.0;
                L[q] = psi * 0.5 * (w_a * la[q] - w_b * lb[q]) * cv.sp[j];
            }
            ph = (lstar == 0.0) ? C(1, 0) : (lstar > 0.0 ? alpha : ainv);
        }
        double s = sin(GS_PI * (double)(i - j) / N);
        double corr = W - h * log(4.0 * s * s);
        for (int q = 0; q < 4; ++q) out[q] = cadd(cscale(F[q], hw), cscale(ph, corr * L[q]));
    } else {
        // diagonal: limits of the kernel differences (log r coefficient K1, remainder Krest): for S
        // from (i/4) H0(kr) = -log(r)/(2 pi) + i/4 - (log(k/2) + gamma)/(2 pi) + o(1); for D the
        // Laplace double layer's limit kappa/(4 pi) (kappa the curvature), which cancels unless the
        // weights differ; N's curvature term and T's hypersingular part cancel in the differences
        double sp = cv.sp[i];
        double lg = log(sp * sp * d * d / (4.0 * GS_PI * GS_PI));
        double dk2 = ka * ka - kb * kb;
        double la = log(ka / 2.0), lb = log(kb / 2.0);
        double K1[4] = {-(wa - wb) / (2.0 * GS_PI), 0.0, 0.0, -dk2 / (4.0 * GS_PI)};
        cplx Kr[4] = {C(-(wa * (la + GS_EULER) - wb * (lb + GS_EULER)) / (2.0 * GS_PI), 0.25 * (wa - wb)),
                      C((wa - wb) * cv.curv[i] / (4.0 * GS_PI), 0.0), C(0, 0),
                      C(-(ka * ka * la - kb * kb * lb) / (4.0 * GS_PI) +
                            dk2 * (1.0 - 2.0 * GS_EULER) / (8.0 * GS_PI),
                        dk2 / 8.0)};
        for (int q = 0; q < 4; ++q) {
            cplx v = cscale(F[q], hw);
            v.x += W * 0.5 * K1[q] * sp + h * sp * (0.5 * K1[q] * lg + Kr[q].x);
            v.y += h * sp * Kr[q].y;
            out[q] = v;
        }
        out[1].x += 0.5 * (wa + wb);   // (wa + wb)/2 I + D
        out[2].x -= 1.0;   // -I + N
    }
    A[(size_t)(col_sig + j) * lda + row_v + i] = out[0];
    A[(size_t)(col_mu + j) * lda + row_v + i] = out[1];
    A[(size_t)(col_sig + j) * lda + row_n + i] = out[2];
    A[(size_t)(col_mu + j) * lda + row_n + i] = out[3];
}

// Plain-trapezoid layer potentials of a curve (copies with given x-shifts and phases) at targets:
// adds sign * (D mu + S sigma) to value rows and sign * (T mu + N sigma) to derivative rows.
struct Targets {
    const double *x, *y, *nx, *ny;   // nx/ny may be null: then (cnx, cny) for all
    double cnx, cny, cx, cy;         // constant normal; x or y constant when the pointer is null
    int T;
};
__device__ __forceinline__ void target_at(const Targets &tg, int t, double &x, double &y, double &nx,
                                          double &ny) {
    x = tg.x ? tg.x[t] : tg.cx;
    y = tg.y ? tg.y[t] : tg.cy;
    nx = tg.nx ? tg.nx[t] : tg.cnx;
    ny = tg.ny ? tg.ny[t] : tg.cny;
}

__global__ void k_potentials(Targets tg, Curve cv, int S, double k, int nsh, double sh0, double sh1,
                             double sh2, cplx ph0, cplx ph1, cplx ph2, double sign, cplx *A, int lda,
                             int row_v, int row_n, int col_mu, int col_sig) {
    long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)tg.T * S) return;
    int t = (int)(id / S), s = (int)(id % S);
    double x, y, nx, ny;
    target_at(tg, t, x, y, nx, ny);
    double shs[3] = {sh0, sh1, sh2};
    cplx phs[3] = {ph0, ph1, ph2};
    cplx aS = C(0, 0), aD = C(0, 0), aN = C(0, 0), aT = C(0, 0);
    for (int q = 0; q < nsh; ++q) {
        K4 kk = layer_kernels(x - (cv.px[s] + shs[q]), y - cv.py[s], nx, ny, cv.nx[s], cv.ny[s], k);
        aS = cadd(aS, cmul(phs[q], kk.S));
        aD = cadd(aD, cmul(phs[q], kk.D));
        aN = cadd(aN, cmul(phs[q], kk.N));
        aT = cadd(aT, cmul(phs[q], kk.T));
    }
    double f = sign * cv.w[s];
    size_t rv = row_v + t, rn = row_n + t;
    cplx *p;
    p = &A[(size_t)(col_mu + s) * lda + rv];  *p = cadd(*p, cscale(aD, f));
    p = &A[(size_t)(col_sig + s) * lda + rv]; *p = cadd(*p, cscale(aS, f));
    p = &A[(size_t)(col_mu + s) * lda + rn];  *p = cadd(*p, cscale(aT, f));
    p = &A[(size_t)(col_sig + s) * lda + rn]; *p = cadd(*p, cscale(aN, f));
}

// J-expansion columns: coef * J_n(k|x-x0|) e^{in theta} in the value rows and coef_n * its normal
// derivative in the derivative rows, n = -Q..Q, using d_x f_n = (k/2)(f_{n-1} - f_{n+1}),
// d_y f_n = (ik/2)(f_{n-1} + f_{n+1}).
__global__ void k_jexp(Targets tg, double cx, double cy, double k, int Q, cplx coef, cplx coef_n, cplx *A, int lda,
                       int row_v, int row_n, int col0) {
    long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    int nq = 2 * Q + 1;
    if (id >= (long)tg.T * nq) return;
    int t = (int)(id / nq), n = (int)(id % nq) - Q;
    double x, y, nx, ny;
    target_at(tg, t, x, y, nx, ny);
    double Rx = x - cx, Ry = y - cy;
    double rho = hypot(Rx, Ry), th = atan2(Ry, Rx);
    cplx f[3];
    for (int q = -1; q <= 1; ++q) f[q + 1] = cscale(cexpi((n + q) * th), besselj_int(n + q, k * rho));
    cplx fx = cscale(csub(f[0], f[2]), 0.5 * k);
    cplx fy = cscale(cmuli(cadd(f[0], f[2])), 0.5 * k);
    cplx dn = cadd(cscale(fx, nx), cscale(fy, ny));
    cplx *p;
    p = &A[(size_t)(col0 + n + Q) * lda + row_v + t];  *p = cadd(*p, cmul(coef, f[1]));
    p = &A[(size_t)(col0 + n + Q) * lda + row_n + t];  *p = cadd(*p, cmul(coef_n, dn));
}

// Rayleigh-Bloch columns on Gamma_u (top=1) or Gamma_d (top=0):
// value rows -e^{i kappa_n x}; derivative rows -i k_{1,n} e^{..} (top) or +i k_{3,n} e^{..} (bottom).
__global__ void k_rb(int nb, const double *bx, int K, const double *kappa, const cplx *kv, int top,
                     cplx *A, int lda, int row_v, int row_n, int col0) {
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    int nq = 2 * K + 1;
    if (id >= nb * nq) return;
    int t = id / nq, n = id % nq;
    cplx e = cexpi(kappa[n] * bx[t]);
    A[(size_t)(col0 + n) * lda + row_v + t] = cscale(e, -1.0);
    cplx ike = cmuli(cmul(kv[n], e));
    A[(size_t)(col0 + n) * lda + row_n + t] = top ? cscale(ike, -1.0) : ike;
}

// f = -u_inc on the Gamma1 value rows and -(1/w1) d_n u_inc on its flux rows (w1 = 1 for TM)
__global__ void k_rhs(int N, Curve cv, double kx, double ky, double inv_w1, cplx *f, int row_v, int row_n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    cplx u = cexpi(kx * cv.px[i] + ky * cv.py[i]);
    f[row_v + i] = cscale(u, -1.0);
    f[row_n + i] = cscale(cmuli(u), -inv_w1 * (kx * cv.nx[i] + ky * cv.ny[i]));
}

__global__ void k_angle_scalars(int K, double k1, double k3, double kappa0, double d, double *kappa,
                                cplx *k1n, cplx *k3n) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= 2 * K + 1) return;
    double kap = kappa0 + 2.0 * GS_PI * (n - K) / d;
    kappa[n] = kap;
    double kj[2] = {k1, k3};
    cplx *o[2] = {k1n, k3n};
    for (int q = 0; q < 2; ++q) {
        double s = kj[q] * kj[q] - kap * kap;
        cplx v = (s >= 0.0) ? C(sqrt(s), 0.0) : C(0.0, sqrt(-s));
        if (fabs(s) < 1e-12 * kj[q] * kj[q]) v = C(0.0, 0.0);   // Wood anomaly snapping
        o[q][n] = v;
    }
}

// ---- disks ----------------------------------------------------------------------------------

// s_n = [wp J_n'(b) J_n(a) - w2 J_n(b) J_n'(a)] / [w2 J_n(b) H_n'(a) - wp J_n'(b) H_n(a)],
// a = k2 R, b = kp R: continuity of u and of w d_r u at the disk boundary (Sec. 4.1), the radial
// derivative weights (wp, w2) = (kp, k2) for TM and (1/kp, 1/k2) for TE (1/eps ~ 1/k^2 times
// d_r J_n(k r) = k J_n').  kp_im (nullable) holds Im kp of lossy inclusions: then J_n(b) is
// complex (power series).
__global__ void k_mie(int M, int p, const double *radius, const double *kp, const double *kp_im, double k2, int te,
                      cplx *s) {
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    int nc = 2 * p + 1;
    if (id >= M * nc) return;
    int i = id / nc, n = id % nc - p;
    const double R = radius[i], a = k2 * R;
    const cplx kpc = C(kp[i], kp_im ? kp_im[i] : 0.0);
    const double Ja = besselj_int(n, a);
    const double Jpa = 0.5 * (besselj_int(n - 1, a) - besselj_int(n + 1, a));
    cplx Jb, Jpb;
    if (kpc.y != 0.0) {
        const cplx b = cscale(kpc, R);
        Jb = besselj_cplx(n, b);
        Jpb = cscale(csub(besselj_cplx(n - 1, b), besselj_cplx(n + 1, b)), 0.5);
    } else {
        const double b = kpc.x * R;
        Jb = C(besselj_int(n, b), 0.0);
        Jpb = C(0.5 * (besselj_int(n - 1, b) - besselj_int(n + 1, b)), 0.0);
    }
    cplx Ha = C(Ja, bessely_int(n, a));
    cplx Hpa = C(Jpa, 0.5 * (bessely_int(n - 1, a) - bessely_int(n + 1, a)));
    const cplx wp = te ? cdiv(C(1.0, 0.0), kpc) : kpc;
    const double w2 = te ? 1.0 / k2 : k2;
    const cplx num = csub(cscale(cmul(wp, Jpb), Ja), cscale(Jb, w2 * Jpa));
    const cplx den = csub(cscale(cmul(Hpa, Jb), w2), cmul(cmul(wp, Jpb), Ha));
    s[id] = cdiv(num, den);
}

#define GS_PMAX 16

// B_phys layer columns: particle i, node s of a curve; incoming coefficients (m = -p..p)
//   single layer (i/4) H_m(k|y-c|) e^{-im phi} w, double layer (i/4) n_y . grad_y[...] w,
// summed over the copies l = -1, 0, 1 with alpha^l.
__global__ void k_B_layer(int M, int p, const double *xy, Curve cv, int S, double k, double d,
                          cplx alpha, cplx *B, int nB, int col_mu, int col_sig) {
    long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)M * S) return;
    int i = (int)(id / S), s = (int)(id % S);
    int nc = 2 * p + 1;
    cplx accS[2 * GS_PMAX + 1], accD[2 * GS_PMAX + 1];
    for (int m = 0; m < nc; ++m) accS[m] = accD[m] = C(0, 0);
    cplx g[2 * GS_PMAX + 3];   // g_m, m = -p-1..p+1
    cplx H[GS_PMAX + 2];
    for (int l = -1; l <= 1; ++l) {
        double Rx = cv.px[s] + l * d - xy[2 * i], Ry = cv.py[s] - xy[2 * i + 1];
        double rho = hypot(Rx, Ry);
        double z = k * rho;
        hankel01(z, H[0], H[1]);
        for (int q = 1; q <= p; ++q) H[q + 1] = csub(cscale(H[q], 2.0 * q / z), H[q - 1]);
        cplx e = C(Rx / rho, -Ry / rho);   // e^{-i phi}
        cplx ep = C(1, 0);
        for (int q = 0; q <= p + 1; ++q) {
            g[p + 1 + q] = cmul(H[q], ep);                                        // H_q e^{-iq phi}
            cplx neg = cmul(H[q], cconj(ep));                                      // H_q e^{iq phi}
            g[p + 1 - q] = (q & 1) ? cscale(neg, -1.0) : neg;                      // H_{-q} e^{iq phi}
            ep = cmul(ep, e);
        }
        cplx ph = (l == 0) ? C(1, 0) : (l == 1 ? alpha : cconj(alpha));
        ph = cscale(cmuli(ph), 0.25 * cv.w[s]);
        for (int m = -p; m <= p; ++m) {
            cplx gm1 = g[p + 1 + m - 1], g0 = g[p + 1 + m], gp1 = g[p + 1 + m + 1];
            cplx gx = cscale(csub(gm1, gp1), 0.5 * k);
            cplx gy = cscale(cmuli(cadd(gm1, gp1)), -0.5 * k);
            cplx gn = cadd(cscale(gx, cv.nx[s]), cscale(gy, cv.ny[s]));
            accS[m + p] = cadd(accS[m + p], cmul(ph, g0));
            accD[m + p] = cadd(accD[m + p], cmul(ph, gn));
        }
    }
    for (int m = 0; m < nc; ++m) {
        size_t r = (size_t)(i * nc + m) * nB;
        B[r + col_sig + s] = accS[m];
        B[r + col_mu + s] = accD[m];
    }
}

// B_phys a2 columns: J_{n-m}(k|c-x2|) e^{i(n-m) Th}, (R, Th) = polar(c_i - x2) (Graf for J).
__global__ void k_B_a2(int M, int p, const double *xy, double x2, double y2, double k, int Q2,
                       cplx *B, int nB, int col0) {
    long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    int nq = 2 * Q2 + 1;
    if (id >= (long)M * nq) return;
    int i = (int)(id / nq), n = (int)(id % nq) - Q2;
    int nc = 2 * p + 1;
    double Rx = xy[2 * i] - x2, Ry = xy[2 * i + 1] - y2;
    double R = hypot(Rx, Ry), Th = atan2(Ry, Rx);
    for (int m = -p; m <= p; ++m) {
        int q = n - m;
        B[(size_t)(i * nc + m + p) * nB + col0 + n + Q2] = cscale(cexpi(q * Th), besselj_int(q, k * R));
    }
}

// C: outgoing waves H_n(k|x-c_j-l d|) e^{in theta} (n = -p..p) of every particle copy at targets,
// value and normal derivative, times sign * phase_l, added to rows (row_v, row_n).
__global__ void k_C(Targets tg, int M, int p, const double *xy, double k, int nsh, double sh0,
                    double sh1, double sh2, cplx ph0, cplx ph1, cplx ph2, double sign, cplx *Cm,
                    int ldc, int row_v, int row_n) {
    long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)tg.T * M) return;
    int t = (int)(id / M), j = (int)(id % M);
    int nc = 2 * p + 1;
    double x, y, nx, ny;
    target_at(tg, t, x, y, nx, ny);
    double shs[3] = {sh0, sh1, sh2};
    cplx phs[3] = {ph0, ph1, ph2};
    cplx accV[2 * GS_PMAX + 1], accN[2 * GS_PMAX + 1];
    for (int m = 0; m < nc; ++m) accV[m] = accN[m] = C(0, 0);
    cplx f[2 * GS_PMAX + 3];
    cplx H[GS_PMAX + 2];
    for (int q = 0; q < nsh; ++q) {
        double Rx = x - (xy[2 * j] + shs[q]), Ry = y - xy[2 * j + 1];
        double rho = hypot(Rx, Ry), z = k * rho;
        hankel01(z, H[0], H[1]);
        for (int m = 1; m <= p; ++m) H[m + 1] = csub(cscale(H[m], 2.0 * m / z), H[m - 1]);
        cplx e = C(Rx / rho, Ry / rho);
        cplx ep = C(1, 0);
        for (int m = 0; m <= p + 1; ++m) {
            f[p + 1 + m] = cmul(H[m], ep);
            cplx neg = cmul(H[m], cconj(ep));
            f[p + 1 - m] = (m & 1) ? cscale(neg, -1.0) : neg;
            ep = cmul(ep, e);
        }
        cplx ph = cscale(phs[q], sign);
        for (int m = -p; m <= p; ++m) {
            cplx fm1 = f[p + m], f0 = f[p + 1 + m], fp1 = f[p + 2 + m];
            cplx fx = cscale(csub(fm1, fp1), 0.5 * k);
            cplx fy = cscale(cmuli(cadd(fm1, fp1)), 0.5 * k);
            cplx dn = cadd(cscale(fx, nx), cscale(fy, ny));
            accV[m + p] = cadd(accV[m + p], cmul(ph, f0));
            accN[m + p] = cadd(accN[m + p], cmul(ph, dn));
        }
    }
    for (int m = 0; m < nc; ++m) {
        size_t col = (size_t)j * nc + m;
        cplx *pv = &Cm[(size_t)(row_v + t) * ldc + col];
        cplx *pn = &Cm[(size_t)(row_n + t) * ldc + col];
        *pv = cadd(*pv, accV[m]);
        *pn = cadd(*pn, accN[m]);
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------------

int gs_build_geometry(gs_ctx *c) {
    const gs_layers &L = c->L;
    const Layout &ly = c->lay;
    int N = L.N, nf = L.n_fourier;
    // Fourier coefficients: [h1_cos, h1_sin, h2_cos, h2_sin] each of length max(nf,1)
    int nfa = nf > 0 ? nf : 1;
    std::vector<double> four(4 * nfa, 0.0);
    for (int q = 0; q < 4; ++q)
        for (int m = 0; m < nf; ++m) four[q * nfa + m] = c->four[q][m];
    GS_CUDA(c, cudaMemcpyAsync(c->four_dev, four.data(), sizeof(double) * four.size(),
                               cudaMemcpyHostToDevice, c->stream));
    GS_COUNT_LAUNCH(c);
    k_curve_nodes<<<nblk(N), TPB, 0, c->stream>>>(N, L.d, L.h1_0, nf, c->four_dev, c->four_dev + nfa,
                                                   c->curve[0]);
    GS_COUNT_LAUNCH(c);
    k_curve_nodes<<<nblk(N), TPB, 0, c->stream>>>(N, L.d, L.h2_0, nf, c->four_dev + 2 * nfa,
                                                   c->four_dev + 3 * nfa, c->curve[1]);
    GS_COUNT_LAUNCH(c);
    k_gauss_legendre<<<nblk(ly.nw1), TPB, 0, c->stream>>>(ly.nw1, c->yL1, L.y0, c->wall_y[0]);
    GS_COUNT_LAUNCH(c);
    k_gauss_legendre<<<nblk(ly.nw2), TPB, 0, c->stream>>>(ly.nw2, c->yL2, c->yL1, c->wall_y[1]);
    GS_COUNT_LAUNCH(c);
    k_gauss_legendre<<<nblk(ly.nw3), TPB, 0, c->stream>>>(ly.nw3, -L.y0, c->yL2, c->wall_y[2]);
    GS_COUNT_LAUNCH(c);
    k_linspace_mid<<<nblk(ly.nb), TPB, 0, c->stream>>>(ly.nb, -0.5 * L.d, 0.5 * L.d, c->bound_x);
    GS_COUNT_LAUNCH(c);
    k_kress<<<nblk(N), TPB, 0, c->stream>>>(N, c->kress);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

int gs_angle_scalars(gs_ctx *c, AngleData &a) {
    a.kappa0 = c->L.k1 * cos(a.theta);
    a.alpha = C(cos(a.kappa0 * c->L.d), sin(a.kappa0 * c->L.d));
    int K = c->lay.K;
    GS_COUNT_LAUNCH(c);
    k_angle_scalars<<<nblk(2 * K + 1), TPB, 0, c->stream>>>(K, c->L.k1, c->L.k3, a.kappa0, c->L.d,
                                                            a.kappa, a.k1n, a.k3n);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

static Targets curve_targets(const Curve &cv, int N) {
    Targets t{};
    t.x = cv.px;
    t.y = cv.py;
    t.nx = cv.nx;
    t.ny = cv.ny;
    t.T = N;
    return t;
}
static Targets wall_targets(const double *ys, int n, double x) {
    Targets t{};
    t.x = nullptr;
    t.cx = x;
    t.y = ys;
    t.nx = t.ny = nullptr;
    t.cnx = 1.0;
    t.cny = 0.0;
    t.T = n;
    return t;
}
static Targets bound_targets(const double *bx, int n, double y) {
    Targets t{};
    t.x = bx;
    t.y = nullptr;
    t.cy = y;
    t.nx = t.ny = nullptr;
    t.cnx = 0.0;
    t.cny = 1.0;
    t.T = n;
    return t;
}

int gs_assemble_A(gs_ctx *c, const AngleData &a, cplx *A, int lda) {
    const gs_layers &L = c->L;
    const Layout &ly = c->lay;
    cudaStream_t st = c->stream;
    int N = L.N;
    double d = L.d;
    GS_CUDA(c, cudaMemsetAsync(A, 0, sizeof(cplx) * (size_t)lda * ly.cols, st));
    Curve c1 = curve_of(c->curve[0], N), c2 = curve_of(c->curve[1], N);
    cplx al = a.alpha, ai = cconj(a.alpha);
    cplx one = C(1, 0);
    cplx al2 = cmul(al, al), mai = cscale(ai, -1.0);
    double x1c = 0.0, y1c = 0.5 * (L.h1_0 + L.y0), y2c = 0.5 * (L.h1_0 + L.h2_0), y3c = 0.5 * (L.h2_0 - L.y0);
    // TE: the top and bottom layers' potentials carry w1, w3 and their flux rows 1/w1, 1/w3
    double w1, w3;
    gs_layer_weights(c, &w1, &w3);

    // Gamma1 rows: u1 - u2 = -u_inc (Eq. bound1)
    GS_COUNT_LAUNCH(c);
    k_self_ops<<<nblk((long)N * N), TPB, 0, st>>>(N, d, c1, al, L.k1, L.k2, w1, 1.0, c->kress, A, lda,
                                                   ly.row_g1v, ly.row_g1n, ly.col_mu1, ly.col_sig1);
    Targets t1 = curve_targets(c1, N), t2 = curve_targets(c2, N);
    GS_COUNT_LAUNCH(c);
    k_potentials<<<nblk((long)N * N), TPB, 0, st>>>(t1, c2, N, L.k2, 3, -d, 0.0, d, ai, one, al, -1.0,
                                                     A, lda, ly.row_g1v, ly.row_g1n, ly.col_mu2,
                                                     ly.col_sig2);
    GS_COUNT_LAUNCH(c);
    k_jexp<<<nblk((long)N * (2 * ly.Q2 + 1)), TPB, 0, st>>>(t1, x1c, y2c, L.k2, ly.Q2, C(-1, 0), C(-1, 0), A, lda,
                                                            ly.row_g1v, ly.row_g1n, ly.col_a2);
    GS_COUNT_LAUNCH(c);
    k_jexp<<<nblk((long)N * (2 * ly.Q1 + 1)), TPB, 0, st>>>(t1, x1c, y1c, L.k1, ly.Q1, one, C(1.0 / w1, 0), A, lda,
                                                            ly.row_g1v, ly.row_g1n, ly.col_a1);
    // Gamma2 rows: u2 - u3 = 0
    GS_COUNT_LAUNCH(c);
    k_self_ops<<<nblk((long)N * N), TPB, 0, st>>>(N, d, c2, al, L.k2, L.k3, 1.0, w3, c->kress, A, lda,
                                                   ly.row_g2v, ly.row_g2n, ly.col_mu2, ly.col_sig2);
    GS_COUNT_LAUNCH(c);
    k_potentials<<<nblk((long)N * N), TPB, 0, st>>>(t2, c1, N, L.k2, 3, -d, 0.0, d, ai, one, al, 1.0, A,
                                                     lda, ly.row_g2v, ly.row_g2n, ly.col_mu1,
                                                     ly.col_sig1);
    GS_COUNT_LAUNCH(c);
    k_jexp<<<nblk((long)N * (2 * ly.Q2 + 1)), TPB, 0, st>>>(t2, x1c, y2c, L.k2, ly.Q2, one, one, A, lda,
                                                            ly.row_g2v, ly.row_g2n, ly.col_a2);
    GS_COUNT_LAUNCH(c);
    k_jexp<<<nblk((long)N * (2 * ly.Q3 + 1)), TPB, 0, st>>>(t2, x1c, y3c, L.k3, ly.Q3, C(-1, 0), C(-1.0 / w3, 0), A,
                                                            lda, ly.row_g2v, ly.row_g2n, ly.col_a3);
    // walls (Eq. bound2, cancelled form for the layer potentials)
    struct WallJob {
        int nw;
        const double *ys;
        int rv, rn;
        double k, cy;
        int Q, col;
        double w;   // TE weight of the layer's potentials
    };
    WallJob wj[3] = {{ly.nw2, c->wall_y[1], ly.row_w2v, ly.row_w2n, L.k2, y2c, ly.Q2, ly.col_a2, 1.0},
                     {ly.nw1, c->wall_y[0], ly.row_w1v, ly.row_w1n, L.k1, y1c, ly.Q1, ly.col_a1, w1},
                     {ly.nw3, c->wall_y[2], ly.row_w3v, ly.row_w3n, L.k3, y3c, ly.Q3, ly.col_a3, w3}};
    for (int q = 0; q < 3; ++q) {
        const WallJob &w = wj[q];
        Targets TL = wall_targets(w.ys, w.nw, -0.5 * d), TR = wall_targets(w.ys, w.nw, 0.5 * d);
        bool has1 = (q == 0 || q == 1), has2 = (q == 0 || q == 2);
        if (has1) {
            GS_COUNT_LAUNCH(c);
            k_potentials<<<nblk((long)w.nw * N), TPB, 0, st>>>(TL, c1, N, w.k, 2, d, -2.0 * d, 0.0, al2,
                                                                mai, one, w.w, A, lda, w.rv, w.rn,
                                                                ly.col_mu1, ly.col_sig1);
        }
        if (has2) {
            GS_COUNT_LAUNCH(c);
            k_potentials<<<nblk((long)w.nw * N), TPB, 0, st>>>(TL, c2, N, w.k, 2, d, -2.0 * d, 0.0, al2,
                                                                mai, one, w.w, A, lda, w.rv, w.rn,
                                                                ly.col_mu2, ly.col_sig2);
        }
        GS_COUNT_LAUNCH(c);
        k_jexp<<<nblk((long)w.nw * (2 * w.Q + 1)), TPB, 0, st>>>(TL, x1c, w.cy, w.k, w.Q, al, al, A, lda, w.rv,
                                                                 w.rn, w.col);
        GS_COUNT_LAUNCH(c);
        k_jexp<<<nblk((long)w.nw * (2 * w.Q + 1)), TPB, 0, st>>>(TR, x1c, w.cy, w.k, w.Q, C(-1, 0), C(-1, 0), A,
                                                                 lda, w.rv, w.rn, w.col);
    }
    // Gamma_u / Gamma_d (Eq. bound3)
    Targets tu = bound_targets(c->bound_x, ly.nb, L.y0), td = bound_targets(c->bound_x, ly.nb, -L.y0);
    GS_COUNT_LAUNCH(c);
    k_potentials<<<nblk((long)ly.nb * N), TPB, 0, st>>>(tu, c1, N, L.k1, 3, -d, 0.0, d, ai, one, al, w1,
                                                         A, lda, ly.row_uv, ly.row_un, ly.col_mu1,
                                                         ly.col_sig1);
    GS_COUNT_LAUNCH(c);
    k_jexp<<<nblk((long)ly.nb * (2 * ly.Q1 + 1)), TPB, 0, st>>>(tu, x1c, y1c, L.k1, ly.Q1, one, one, A, lda,
                                                                ly.row_uv, ly.row_un, ly.col_a1);
    GS_COUNT_LAUNCH(c);
    k_rb<<<nblk(ly.nb * (2 * ly.K + 1)), TPB, 0, st>>>(ly.nb, c->bound_x, ly.K, a.kappa, a.k1n, 1, A, lda,
                                                      ly.row_uv, ly.row_un, ly.col_c);
    GS_COUNT_LAUNCH(c);
    k_potentials<<<nblk((long)ly.nb * N), TPB, 0, st>>>(td, c2, N, L.k3, 3, -d, 0.0, d, ai, one, al, w3,
                                                         A, lda, ly.row_dv, ly.row_dn, ly.col_mu2,
                                                         ly.col_sig2);
    GS_COUNT_LAUNCH(c);
    k_jexp<<<nblk((long)ly.nb * (2 * ly.Q3 + 1)), TPB, 0, st>>>(td, x1c, y3c, L.k3, ly.Q3, one, one, A, lda,
                                                                ly.row_dv, ly.row_dn, ly.col_a3);
    GS_COUNT_LAUNCH(c);
    k_rb<<<nblk(ly.nb * (2 * ly.K + 1)), TPB, 0, st>>>(ly.nb, c->bound_x, ly.K, a.kappa, a.k3n, 0, A, lda,
                                                      ly.row_dv, ly.row_dn, ly.col_d);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

int gs_assemble_f(gs_ctx *c, const AngleData &a, cplx *f) {
    const Layout &ly = c->lay;
    GS_CUDA(c, cudaMemsetAsync(f, 0, sizeof(cplx) * ly.rows, c->stream));
    Curve c1 = curve_of(c->curve[0], c->L.N);
    GS_COUNT_LAUNCH(c);
    double w1, w3;
    gs_layer_weights(c, &w1, &w3);
    k_rhs<<<nblk(c->L.N), TPB, 0, c->stream>>>(c->L.N, c1, a.kappa0, c->L.k1 * sin(a.theta), 1.0 / w1, f, ly.row_g1v,
                                                ly.row_g1n);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

int gs_mie_geo(gs_ctx *c, int M, const double *radius, const double *kp, const double *kp_im, cplx *s) {
    GS_COUNT_LAUNCH(c);
    k_mie<<<nblk(M * c->nc), TPB, 0, c->stream>>>(M, c->p, radius, kp, kp_im, c->L.k2, c->pol != 0, s);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

int gs_mie(gs_ctx *c) { return gs_mie_geo(c, c->M, c->radius, c->kp, c->kp_im, c->s); }

int gs_assemble_B_geo(gs_ctx *c, const AngleData &a, int M, const double *xy, cplx *B) {
    const Layout &ly = c->lay;
    int N = c->L.N, nB = ly.nB();
    Curve c1 = curve_of(c->curve[0], N), c2 = curve_of(c->curve[1], N);
    GS_COUNT_LAUNCH(c);
    k_B_layer<<<nblk((long)M * N, 128), 128, 0, c->stream>>>(M, c->p, xy, c1, N, c->L.k2, c->L.d,
                                                               a.alpha, B, nB, ly.col_mu1, ly.col_sig1);
    GS_COUNT_LAUNCH(c);
    k_B_layer<<<nblk((long)M * N, 128), 128, 0, c->stream>>>(M, c->p, xy, c2, N, c->L.k2, c->L.d,
                                                               a.alpha, B, nB, ly.col_mu2, ly.col_sig2);
    GS_COUNT_LAUNCH(c);
    k_B_a2<<<nblk((long)M * (2 * ly.Q2 + 1), 128), 128, 0, c->stream>>>(
        M, c->p, xy, 0.0, 0.5 * (c->L.h1_0 + c->L.h2_0), c->L.k2, ly.Q2, B, nB, ly.col_a2);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

int gs_assemble_B(gs_ctx *c, const AngleData &a, cplx *B) { return gs_assemble_B_geo(c, a, c->M, c->xy, B); }

int gs_assemble_C_geo(gs_ctx *c, const AngleData &a, int M, const double *xy, cplx *Cm) {
    const Layout &ly = c->lay;
    int N = c->L.N, n = M * c->nc;
    double d = c->L.d;
    GS_CUDA(c, cudaMemsetAsync(Cm, 0, sizeof(cplx) * (size_t)ly.nC() * n, c->stream));
    Curve c1 = curve_of(c->curve[0], N), c2 = curve_of(c->curve[1], N);
    cplx al = a.alpha, ai = cconj(a.alpha), one = C(1, 0);
    Targets t1 = curve_targets(c1, N), t2 = curve_targets(c2, N);
    Targets tw = wall_targets(c->wall_y[1], ly.nw2, -0.5 * d);
    GS_COUNT_LAUNCH(c);
    k_C<<<nblk((long)N * M, 128), 128, 0, c->stream>>>(t1, M, c->p, xy, c->L.k2, 3, -d, 0.0, d, ai,
                                                         one, al, -1.0, Cm, n, ly.row_g1v, ly.row_g1n);
    GS_COUNT_LAUNCH(c);
    k_C<<<nblk((long)N * M, 128), 128, 0, c->stream>>>(t2, M, c->p, xy, c->L.k2, 3, -d, 0.0, d, ai,
                                                         one, al, 1.0, Cm, n, ly.row_g2v, ly.row_g2n);
    GS_COUNT_LAUNCH(c);
    k_C<<<nblk((long)ly.nw2 * M, 128), 128, 0, c->stream>>>(tw, M, c->p, xy, c->L.k2, 2, d,
                                                              -2.0 * d, 0.0, cmul(al, al),
                                                              cscale(ai, -1.0), one, 1.0, Cm, n,
                                                              ly.row_w2v, ly.row_w2n);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

int gs_assemble_C(gs_ctx *c, const AngleData &a, cplx *Cm) { return gs_assemble_C_geo(c, a, c->M, c->xy, Cm); }
