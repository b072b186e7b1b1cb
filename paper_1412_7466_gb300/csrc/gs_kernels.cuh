// Kernels of the layer potentials shared by the interface assembly (gs_assemble.cu) and the
// boundary integral equation of general inclusion shapes (gs_shape.cu): G = (i/4) H0(k r).
#pragma once
#include "gs_internal.h"

namespace {

// ---- kernels of the layer potentials ----------------------------------------------------------

struct K4 {
    cplx S, D, N, T;
};

// S = (i/4) H0(kr); D = (ik/4) H1 R.ny/r; N = -(ik/4) H1 R.nx/r;
// T = (ik/4)[k H0 R.nx R.ny/r^2 - 2 H1 R.nx R.ny/r^3 + H1 nx.ny/r], R = x - y.
__device__ __forceinline__ K4 layer_kernels(double Rx, double Ry, double tnx, double tny, double snx,
                                            double sny, double k) {
    double r = hypot(Rx, Ry);
    cplx H0, H1;
    hankel01(k * r, H0, H1);
    double Rnx = Rx * tnx + Ry * tny, Rny = Rx * snx + Ry * sny, nn = tnx * snx + tny * sny;
    double ir = 1.0 / r;
    K4 o;
    o.S = cscale(cmuli(H0), 0.25);
    o.D = cscale(cmuli(H1), 0.25 * k * Rny * ir);
    o.N = cscale(cmuli(H1), -0.25 * k * Rnx * ir);
    cplx t = cadd(cscale(H0, k * Rnx * Rny * ir * ir),
                  cscale(H1, (-2.0 * Rnx * Rny * ir * ir + nn) * ir));
    o.T = cscale(cmuli(t), 0.25 * k);
    return o;
}

// coefficient of log r in each kernel (H_n -> (2i/pi) J_n)
__device__ __forceinline__ void log_coeffs(double Rx, double Ry, double tnx, double tny, double snx,
                                           double sny, double k, double out[4]) {
    double r = hypot(Rx, Ry);
    double J0 = j0(k * r), J1 = j1(k * r);
    double Rnx = Rx * tnx + Ry * tny, Rny = Rx * snx + Ry * sny, nn = tnx * snx + tny * sny;
    double ir = 1.0 / r;
    const double c = -1.0 / (2.0 * GS_PI);
    out[0] = c * J0;
    out[1] = c * k * J1 * Rny * ir;
    out[2] = -c * k * J1 * Rnx * ir;
    out[3] = c * k * (k * J0 * Rnx * Rny * ir * ir - 2.0 * J1 * Rnx * Rny * ir * ir * ir + J1 * nn * ir);
}

}  // namespace
