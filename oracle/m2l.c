/* Oracle-only direct-sum translation (Sec. 4.2, Eq. trans; Sec. 5, Eq. repre3_mod).
 *
 * TEST INFRASTRUCTURE: built and loaded only by the oracle package.
 *
 * out[i][m] = sum_{l=-1..1} alpha^l sum_{j, (j,l) != (i,0)} sum_n H_{n-m}(k R) e^{i(n-m) Th} beta[j][n],
 * (R, Th) = polar(c_i - c_j - l d x).  H_0, H_1 from the C library's Bessel functions j0, j1, y0,
 * y1; higher orders by the upward recurrence H_{q+1}(z) = (2q/z) H_q(z) - H_{q-1}(z) (DLMF 10.6.1);
 * H_{-q} = (-1)^q H_q; e^{i q Th} as powers of (dx + i dy)/R.  Plain loops, FP64, OpenMP over i.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>

void oracle_m2l_apply(int M, int p, const double *xy, double k, double d, double alpha_re,
                      double alpha_im, const double complex *beta, double complex *out)
{
    const int nc = 2 * p + 1, nq = 4 * p + 1;
    const double complex alpha = alpha_re + I * alpha_im;
#pragma omp parallel
    {
        double complex *Hq = malloc(sizeof(double complex) * nq);
        double complex *Hp = malloc(sizeof(double complex) * (2 * p + 1));
#pragma omp for schedule(dynamic, 4)
        for (int i = 0; i < M; ++i) {
            for (int m = 0; m < nc; ++m) out[(size_t)i * nc + m] = 0;
            for (int l = -1; l <= 1; ++l) {
                const double complex ph = (l == 0) ? 1.0 : (l == 1 ? alpha : 1.0 / alpha);
                for (int j = 0; j < M; ++j) {
                    if (l == 0 && j == i) continue;
                    const double dx = xy[2 * i] - (xy[2 * j] + l * d);
                    const double dy = xy[2 * i + 1] - xy[2 * j + 1];
                    const double R = hypot(dx, dy);
                    const double z = k * R;
                    Hp[0] = j0(z) + I * y0(z);
                    Hp[1] = j1(z) + I * y1(z);
                    for (int q = 1; q < 2 * p; ++q) Hp[q + 1] = (2.0 * q / z) * Hp[q] - Hp[q - 1];
                    const double complex u = (dx + I * dy) / R;
                    /* Hq[q + 2p] = H_q e^{iq Th}, q = -2p..2p */
                    double complex up = 1.0;
                    for (int q = 0; q <= 2 * p; ++q) {
                        Hq[2 * p + q] = Hp[q] * up;
                        /* H_{-q} e^{-iq Th} = (-1)^q H_q conj(u)^q */
                        Hq[2 * p - q] = ((q & 1) ? -1.0 : 1.0) * Hp[q] * conj(up);
                        up *= u;
                    }
                    const double complex *b = beta + (size_t)j * nc;
                    for (int m = 0; m < nc; ++m) {
                        double complex acc = 0;
                        for (int n = 0; n < nc; ++n) acc += Hq[n - m + 2 * p] * b[n];
                        out[(size_t)i * nc + m] += ph * acc;
                    }
                }
            }
        }
        free(Hq);
        free(Hp);
    }
}
