// Total field at given points of one period, in all three layers (the paper's field plots, Sec. 6
// Figs.), from the layer unknowns a = A^+ (f - C beta) of the converged solution:
//   middle (Sec. 3 Eq. repre3, Sec. 5 Eq. repre3_mod):
//     u = sum over both interfaces and their +-d copies of alpha^l [S sigma + D mu](x)      (k2)
//       + sum_q a2_q J_q(k2 |x - x2|) e^{i q theta}                                        (far copies)
//       + sum_j sum_l alpha^l sum_n beta^j_n H_n(k2 |x - c_j - l d|) e^{i n theta}          (inclusions)
//   top, below Gamma_u (Eq. repre1): u_inc + the potentials of Gamma1's densities at k1 (near
//     copies; times w1 = (k1/k2)^2 in TE polarisation) + sum_q a1_q J_q(k1 |x - x1|) e^{i q theta};
//     above (Eq. rad1):
//     u_inc + sum_n c_n e^{i (kappa_n x + k_{1,n} (y - y0))}
//   bottom, above Gamma_d (Eq. repre2): the potentials of Gamma2's densities at k3 (times w3 in TE) +
//     sum_q a3_q J_q(k3 |x - x3|) e^{i q theta};  below (Eq. rad2): sum_n d_n e^{i (kappa_n x - k_{3,n} (y + y0))}
// One thread per point, FP64 throughout: interface sums by the plain trapezoid rule (accurate a few
// node spacings away from the interfaces), J_q by Miller's backward recurrence accumulated on the
// fly (no per-order storage), H_n by upward recurrence from H_0, H_1.  Points outside one period
// (|x| > d/2), on an interface, or inside an inclusion give NaN.
#include <cmath>

#include "gs_internal.h"

namespace {

struct FieldArgs {
    const double *c1, *c2;        // curve arrays: x, px, py, nx, ny, speed, w (N each)
    int N;
    const double *four;           // [h1_cos, h1_sin, h2_cos, h2_sin], nfa each
    int nf, nfa;
    double h1_0, h2_0, d, k1, k2, k3, y0, ycen, ycen1, ycen3, kx, ky;   // kx, ky: incident wave vector
    double w1, w3;                // TE weights of the top and bottom layers' potentials (1 for TM)
    cplx alpha;
    const cplx *a;                // layer unknowns (cols)
    int col_mu1, col_sig1, col_mu2, col_sig2, col_a2, Q2, col_a1, Q1, col_a3, Q3, col_c, col_d, K;
    const double *kappa;          // 2K+1 Bloch wavenumbers kappa_n
    const cplx *k1n, *k3n;        // 2K+1 vertical wavenumbers of the top and bottom layers
    const double *xy, *radius;    // inclusions
    const cplx *beta;
    int M, p;
};

__device__ double iface_h(double h0, const double *ca, const double *sa, int nf, double d, double x) {
    double h = h0;
    for (int m = 1; m <= nf; ++m) {
        double s, c;
        sincos(2.0 * GS_PI * m * x / d, &s, &c);
        h += ca[m - 1] * c + sa[m - 1] * s;
    }
    return h;
}

// sum_{q=-Q..Q} a[q+Q] J_q(z) e^{i q th}, J_q by Miller's backward recurrence from an order well
// above max(Q, z), normalised with J_0 + 2 sum_k J_2k = 1 (J_-q = (-1)^q J_q)
__device__ cplx jexp_sum(const cplx *a, int Q, double z, double th) {
    if (z < 1e-300) return a[Q];
    const double big = fmax((double)Q, z);
    int m = 2 * (((int)big + 16 + (int)sqrt(40.0 * big)) / 2);
    double jp = 0.0, jc = 1e-200, norm = 0.0;   // J_{k+1}, J_k (unnormalised)
    cplx acc = C(0.0, 0.0);
    for (int k = m; k >= 0; --k) {
        if (k <= Q) {
            cplx t;
            if (k == 0) {
                t = a[Q];
            } else {
                double s, c;
                sincos(k * th, &s, &c);
                const cplx ep = C(c, s), em = C(c, -s);
                const cplx pos = cmul(a[Q + k], ep), neg = cmul(a[Q - k], em);
                t = (k & 1) ? csub(pos, neg) : cadd(pos, neg);
            }
            acc = cadd(acc, cscale(t, jc));
        }
        norm += (k == 0) ? jc : ((k & 1) ? 0.0 : 2.0 * jc);
        if (k > 0) {
            const double jm = (2.0 * k / z) * jc - jp;
            jp = jc;
            jc = jm;
        }
        if (fabs(jc) > 1e200) {   // rescale the recurrence and what it has accumulated
            jc *= 1e-200;
            jp *= 1e-200;
            norm *= 1e-200;
            acc = cscale(acc, 1e-200);
        }
    }
    return cscale(acc, 1.0 / norm);
}

// sum over the +-d copies of alpha^l [S sigma + D mu](x, y) for interface q's densities at wavenumber k
__device__ cplx layer_potentials(const FieldArgs &A, int q, double k, double x, double y) {
    const double *cv = q == 0 ? A.c1 : A.c2;
    const double *px = cv + A.N, *py = cv + 2 * A.N, *nx = cv + 3 * A.N, *ny = cv + 4 * A.N, *w = cv + 6 * A.N;
    const cplx *mu = A.a + (q == 0 ? A.col_mu1 : A.col_mu2), *sg = A.a + (q == 0 ? A.col_sig1 : A.col_sig2);
    const cplx ai = cconj(A.alpha);
    cplx acc = C(0.0, 0.0);
    for (int l = -1; l <= 1; ++l) {
        const cplx ph = l == 0 ? C(1.0, 0.0) : (l == 1 ? A.alpha : ai);
        cplx s = C(0.0, 0.0);
        for (int j = 0; j < A.N; ++j) {
            const double Rx = x - (px[j] + l * A.d), Ry = y - py[j];
            const double r = hypot(Rx, Ry);
            cplx H0, H1;
            hankel01(k * r, H0, H1);
            // S = (i/4) H0, D = (i k/4) H1 (R . n_y) / r
            const cplx Sk = cmuli(cscale(H0, 0.25 * w[j]));
            const cplx Dk = cmuli(cscale(H1, 0.25 * k * (Rx * nx[j] + Ry * ny[j]) / r * w[j]));
            s = cadd(s, cadd(cmul(Sk, sg[j]), cmul(Dk, mu[j])));
        }
        acc = cadd(acc, cmul(ph, s));
    }
    return acc;
}

// sum_n amp_n e^{i (kappa_n x + kv_n dy)} over the 2K+1 Rayleigh-Bloch orders (kv complex: the
// evanescent orders decay away from the layer)
__device__ cplx rayleigh_bloch(const FieldArgs &A, const cplx *amp, const cplx *kv, double x, double dy) {
    cplx acc = C(0.0, 0.0);
    for (int n = 0; n < 2 * A.K + 1; ++n) {
        const double ph = A.kappa[n] * x + kv[n].x * dy, damp = exp(-kv[n].y * dy);
        double s, c;
        sincos(ph, &s, &c);
        acc = cadd(acc, cmul(amp[n], C(damp * c, damp * s)));
    }
    return acc;
}

__global__ void k_field(FieldArgs A, long npts, const double *__restrict__ pts, cplx *__restrict__ u) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts) return;
    const double x = pts[2 * t], y = pts[2 * t + 1];
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (!(fabs(x) <= 0.5 * A.d)) {
        u[t] = C(nan, nan);
        return;
    }
    const double top = iface_h(A.h1_0, A.four, A.four + A.nfa, A.nf, A.d, x);
    const double bot = iface_h(A.h2_0, A.four + 2 * A.nfa, A.four + 3 * A.nfa, A.nf, A.d, x);
    double si, co;
    sincos(A.kx * x + A.ky * y, &si, &co);
    const cplx uinc = C(co, si);
    if (y >= A.y0) {
        u[t] = cadd(uinc, rayleigh_bloch(A, A.a + A.col_c, A.k1n, x, y - A.y0));
        return;
    }
    if (y <= -A.y0) {
        u[t] = rayleigh_bloch(A, A.a + A.col_d, A.k3n, x, -(y + A.y0));
        return;
    }
    if (y > top) {
        const double Ry = y - A.ycen1;
        cplx acc = cadd(uinc, cscale(layer_potentials(A, 0, A.k1, x, y), A.w1));
        u[t] = cadd(acc, jexp_sum(A.a + A.col_a1, A.Q1, A.k1 * hypot(x, Ry), atan2(Ry, x)));
        return;
    }
    if (y < bot) {
        const double Ry = y - A.ycen3;
        const cplx acc = cscale(layer_potentials(A, 1, A.k3, x, y), A.w3);
        u[t] = cadd(acc, jexp_sum(A.a + A.col_a3, A.Q3, A.k3 * hypot(x, Ry), atan2(Ry, x)));
        return;
    }
    if (!(y > bot && y < top)) {   // on an interface
        u[t] = C(nan, nan);
        return;
    }
    const cplx ai = cconj(A.alpha);
    cplx acc = cadd(layer_potentials(A, 0, A.k2, x, y), layer_potentials(A, 1, A.k2, x, y));
    // far copies: J-expansion about the layer's centre
    {
        const double Rx = x, Ry = y - A.ycen;
        acc = cadd(acc, jexp_sum(A.a + A.col_a2, A.Q2, A.k2 * hypot(Rx, Ry), atan2(Ry, Rx)));
    }
    // inclusions with their near copies
    const int nc = 2 * A.p + 1;
    for (int j = 0; j < A.M; ++j) {
        const cplx *b = A.beta + (size_t)j * nc;
        for (int l = -1; l <= 1; ++l) {
            const double Rx = x - (A.xy[2 * j] + l * A.d), Ry = y - A.xy[2 * j + 1];
            const double R = hypot(Rx, Ry);
            if (R < A.radius[j]) {
                u[t] = C(nan, nan);
                return;
            }
            const double z = A.k2 * R, twoz = 2.0 / z;
            const cplx u1 = C(Rx / R, Ry / R);
            cplx Hm1, Hc;
            hankel01(z, Hm1, Hc);
            cplx s = cmul(Hm1, b[A.p]);
            cplx up = u1;
            for (int n = 1; n <= A.p; ++n) {
                // H_n e^{i n th} b_n + (-1)^n H_n e^{-i n th} b_-n
                const cplx pos = cmul(cmul(Hc, up), b[A.p + n]);
                const cplx neg = cmul(cmul(Hc, cconj(up)), b[A.p - n]);
                s = cadd(s, (n & 1) ? csub(pos, neg) : cadd(pos, neg));
                const cplx Hn = csub(cscale(Hc, n * twoz), Hm1);
                Hm1 = Hc;
                Hc = Hn;
                up = cmul(up, u1);
            }
            const cplx ph = l == 0 ? C(1.0, 0.0) : (l == 1 ? A.alpha : ai);
            acc = cadd(acc, cmul(ph, s));
        }
    }
    u[t] = acc;
}

}  // namespace

extern "C" int gs_field(gs_ctx *c, int angle, long npts, const double *xy_dev, gs_c128 *u_dev) {
    if (!c) return GS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, "cudaSetDevice");
    if (!c->factored) return gs_fail(c, GS_ERR_STATE, "gs_factor has not run");
    if (angle < 0 || angle >= (int)c->ang.size()) return gs_fail(c, GS_ERR_ARG, "angle index out of range");
    if (npts < 0 || (npts > 0 && (!xy_dev || !u_dev))) return gs_fail(c, GS_ERR_ARG, "bad point arrays");
    const AngleData &a = c->ang[angle];
    if (a.relres < 0.0) return gs_fail(c, GS_ERR_STATE, "gs_solve has not run for this angle");
    if (npts == 0) return GS_OK;
    const Layout &ly = c->lay;
    // a = A^+ (f - C beta) into c->x (cols), as for the Bragg amplitudes
    GS_TRY(gs_layer_unknowns_impl(c, a, c->x));
    FieldArgs A;
    A.c1 = c->curve[0];
    A.c2 = c->curve[1];
    A.N = c->L.N;
    A.four = c->four_dev;
    A.nf = c->L.n_fourier;
    A.nfa = c->L.n_fourier > 0 ? c->L.n_fourier : 1;
    A.h1_0 = c->L.h1_0;
    A.h2_0 = c->L.h2_0;
    A.d = c->L.d;
    A.k1 = c->L.k1;
    A.k2 = c->L.k2;
    A.k3 = c->L.k3;
    A.y0 = c->L.y0;
    A.ycen = 0.5 * (c->L.h1_0 + c->L.h2_0);
    A.ycen1 = 0.5 * (c->L.h1_0 + c->L.y0);
    A.ycen3 = 0.5 * (c->L.h2_0 - c->L.y0);
    gs_layer_weights(c, &A.w1, &A.w3);
    A.kx = a.kappa0;
    A.ky = c->L.k1 * std::sin(a.theta);
    A.col_a1 = ly.col_a1;
    A.Q1 = ly.Q1;
    A.col_a3 = ly.col_a3;
    A.Q3 = ly.Q3;
    A.col_c = ly.col_c;
    A.col_d = ly.col_d;
    A.K = ly.K;
    A.kappa = a.kappa;
    A.k1n = a.k1n;
    A.k3n = a.k3n;
    A.alpha = a.alpha;
    A.a = c->x;
    A.col_mu1 = ly.col_mu1;
    A.col_sig1 = ly.col_sig1;
    A.col_mu2 = ly.col_mu2;
    A.col_sig2 = ly.col_sig2;
    A.col_a2 = ly.col_a2;
    A.Q2 = ly.Q2;
    A.xy = c->xy;
    A.radius = c->radius;
    A.beta = a.beta;
    A.M = c->M;
    A.p = c->p;
    GS_COUNT_LAUNCH(c);
    k_field<<<(int)((npts + 127) / 128), 128, 0, c->stream>>>(A, npts, xy_dev, (cplx *)u_dev);
    GS_CHECK_LAUNCH(c);
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}
