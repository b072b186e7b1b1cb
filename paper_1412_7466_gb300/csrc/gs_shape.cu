// General inclusion shapes on the GPU (Sec. 4.1 Eqs. rep1-rep2, intg1-intg2 and the moment
// integral; Sec. 4.2 rotations), FP64: the scattering matrix of one star r(t) = a1 + a2 cos(a3 t)
// (Eq. par1) from its boundary integral equation, then one rotated copy per inclusion.
//
//  * Nodes t_j = 2 pi j / N on the closed curve; outward normal; the Laplace double layer's
//    curvature term gamma''.n / |gamma'|^2.
//  * The 2N x 2N second-kind system [[(1 + wp)/2 I + D2 - wp Dp, S2 - wp Sp], [T2 - Tp, -I + N2 - Np]]
//    (wp = 1 for TM, (kp/k2)^2 for TE) by Kress's product rule on the log-singular part of the
//    kernel differences and the trapezoid rule on the rest, with the 2p+1 right-hand sides
//    -(J_n(k2 r) e^{i n th}, d_n of it) appended as extra columns.
//  * Gaussian elimination with partial pivoting, one launch pair per column (pivot, swap and scale
//    in one block; the trailing update over a grid), then back substitution per right-hand side.
//  * Moments s_ln = (i/4) sum_j w_j [J_l(k2 r_j) e^{-i l th_j} sigma_n(y_j) + d_n(J_l e^{-i l th}) mu_n(y_j)]
//    and the rotated copies (counter-clockwise phi): e^{i phi (n - l)} s_ln.
#include <cmath>
#include <string>
#include <vector>

#include "gs_internal.h"
#include "gs_kernels.cuh"

namespace {

inline int nblk(long n, int t = 256) { return (int)((n + t - 1) / t); }

// node arrays: x, y, nx, ny, speed, kappa (N each)
__global__ void k_star_nodes(int N, double a1, double a2, int a3, double *out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double t = 2.0 * GS_PI * j / N;
    double s3, c3, s, c;
    sincos(a3 * t, &s3, &c3);
    sincos(t, &s, &c);
    const double r = a1 + a2 * c3, rp = -a2 * a3 * s3, rpp = -a2 * a3 * a3 * c3;
    const double d1x = rp * c - r * s, d1y = rp * s + r * c;
    const double d2x = rpp * c - 2.0 * rp * s - r * c, d2y = rpp * s + 2.0 * rp * c - r * s;
    const double sp = hypot(d1x, d1y);
    const double nx = d1y / sp, ny = -d1x / sp;
    out[j] = r * c;
    out[N + j] = r * s;
    out[2 * N + j] = nx;
    out[3 * N + j] = ny;
    out[4 * N + j] = sp;
    out[5 * N + j] = (d2x * nx + d2y * ny) / (sp * sp);
}

// augmented matrix G (column-major, ld = 2N): columns 0..2N-1 the system, 2N..2N+nc-1 the
// right-hand sides; one thread per (row, source node) fills the four operator blocks
__global__ void k_star_system(int N, const double *nd, const double *R, double k2, double kp, double wp, cplx *G,
                              int ld) {
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)N * N) return;
    const int i = (int)(id / N), j = (int)(id % N);
    const double *x = nd, *y = nd + N, *nx = nd + 2 * N, *ny = nd + 3 * N, *sp = nd + 4 * N, *kap = nd + 5 * N;
    const double h = 2.0 * GS_PI / N;
    const double W = R[((i - j) % N + N) % N];
    cplx out[4];   // S, D, N, T of the differences (S and D weighted: 1 and wp)
    const double w_a[4] = {1.0, 1.0, 1.0, 1.0}, w_b[4] = {wp, wp, 1.0, 1.0};
    if (i != j) {
        const double Rx = x[i] - x[j], Ry = y[i] - y[j];
        const K4 a = layer_kernels(Rx, Ry, nx[i], ny[i], nx[j], ny[j], k2);
        const K4 b = layer_kernels(Rx, Ry, nx[i], ny[i], nx[j], ny[j], kp);
        double la[4], lb[4];
        log_coeffs(Rx, Ry, nx[i], ny[i], nx[j], ny[j], k2, la);
        log_coeffs(Rx, Ry, nx[i], ny[i], nx[j], ny[j], kp, lb);
        const cplx Ka[4] = {a.S, a.D, a.N, a.T}, Kb[4] = {b.S, b.D, b.N, b.T};
        const double s = sin(GS_PI * (double)(i - j) / N);
        const double lg = log(4.0 * s * s);
        for (int q = 0; q < 4; ++q) {
            const cplx K = cscale(csub(cscale(Ka[q], w_a[q]), cscale(Kb[q], w_b[q])), sp[j]);
            const double K1 = 0.5 * (w_a[q] * la[q] - w_b[q] * lb[q]) * sp[j];   // coefficient of log(4 sin^2)
            out[q] = cadd(C(W * K1, 0.0), cscale(csub(K, C(K1 * lg, 0.0)), h));
        }
    } else {
        // limits at coincidence (per unit length: K = K1 log r + Krest), log r = log(4 sin^2)/2 + log|gamma'|
        const double s_ = sp[i], ls = log(s_);
        const double l2 = log(k2 / 2.0), lp = log(kp / 2.0), dk2 = k2 * k2 - kp * kp;
        const double K1d[4] = {-(1.0 - wp) / (2.0 * GS_PI), 0.0, 0.0, -dk2 / (4.0 * GS_PI)};
        const cplx Kr[4] = {C(-((l2 + GS_EULER) - wp * (lp + GS_EULER)) / (2.0 * GS_PI), 0.25 * (1.0 - wp)),
                            C((1.0 - wp) * kap[i] / (4.0 * GS_PI), 0.0), C(0.0, 0.0),
                            C(-(k2 * k2 * l2 - kp * kp * lp) / (4.0 * GS_PI) + dk2 * (1.0 - 2.0 * GS_EULER) / (8.0 * GS_PI),
                              dk2 / 8.0)};
        for (int q = 0; q < 4; ++q)
            out[q] = C(W * 0.5 * K1d[q] * s_ + h * s_ * (K1d[q] * ls + Kr[q].x), h * s_ * Kr[q].y);
        out[1].x += 0.5 * (1.0 + wp);   // (1 + wp)/2 I + D
        out[2].x -= 1.0;                // -I + N
    }
    // rows 0..N-1: value equation [D, S]; rows N..2N-1: flux equation [T, N]
    G[(size_t)j * ld + i] = out[1];
    G[(size_t)(N + j) * ld + i] = out[0];
    G[(size_t)j * ld + N + i] = out[3];
    G[(size_t)(N + j) * ld + N + i] = out[2];
}

// right-hand sides: column 2N + (n + p) holds -(J_n(k2 r) e^{i n th}) and -d_n of it at the nodes
__global__ void k_star_rhs(int N, int p, const double *nd, double k2, cplx *G, int ld) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    const int nc = 2 * p + 1;
    if (id >= N * nc) return;
    const int i = id / nc, n = id % nc - p;
    const double x = nd[i], y = nd[N + i], nx = nd[2 * N + i], ny = nd[3 * N + i];
    const double rho = hypot(x, y), th = atan2(y, x);
    cplx f[3];
    for (int q = -1; q <= 1; ++q) f[q + 1] = cscale(cexpi((n + q) * th), besselj_int(n + q, k2 * rho));
    const cplx fx = cscale(csub(f[0], f[2]), 0.5 * k2);
    const cplx fy = cscale(cmuli(cadd(f[0], f[2])), 0.5 * k2);
    const cplx dn = cadd(cscale(fx, nx), cscale(fy, ny));
    const size_t col = (size_t)(2 * N + n + p) * ld;
    G[col + i] = cscale(f[1], -1.0);
    G[col + N + i] = cscale(dn, -1.0);
}

// elimination step k: pivot row (largest |G[i][k]|, i >= k), swap rows k and the pivot over all
// ncol columns, multipliers G[i][k] /= G[k][k] below the diagonal (one block)
__global__ void k_lu_pivot(cplx *G, int ld, int n, int ncol, int k, int *singular) {
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    double best = -1.0;
    int arg = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
        const double v = cabs2(G[(size_t)k * ld + i]);
        if (v > best) {
            best = v;
            arg = i;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = arg;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s && (bv[threadIdx.x + s] > bv[threadIdx.x] ||
                                (bv[threadIdx.x + s] == bv[threadIdx.x] && bi[threadIdx.x + s] < bi[threadIdx.x]))) {
            bv[threadIdx.x] = bv[threadIdx.x + s];
            bi[threadIdx.x] = bi[threadIdx.x + s];
        }
        __syncthreads();
    }
    const int pr = bi[0];
    if (!(bv[0] > 0.0)) {
        if (threadIdx.x == 0) *singular = 1;
        return;
    }
    if (pr != k)
        for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
            const cplx t = G[(size_t)c * ld + k];
            G[(size_t)c * ld + k] = G[(size_t)c * ld + pr];
            G[(size_t)c * ld + pr] = t;
        }
    __syncthreads();
    const cplx inv = cdiv(C(1.0, 0.0), G[(size_t)k * ld + k]);
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) G[(size_t)k * ld + i] = cmul(G[(size_t)k * ld + i], inv);
}

// trailing update G[i][c] -= G[i][k] G[k][c] for i > k, k < c < ncol (right-hand sides included)
__global__ void k_lu_update(cplx *G, int ld, int n, int ncol, int k) {
    const long rows = n - k - 1;
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= rows * (ncol - k - 1)) return;
    const int i = k + 1 + (int)(id % rows), c = k + 1 + (int)(id / rows);
    G[(size_t)c * ld + i] = csub(G[(size_t)c * ld + i], cmul(G[(size_t)k * ld + i], G[(size_t)c * ld + k]));
}

// back substitution U x = y for each right-hand-side column (one block per column), in place
__global__ void k_lu_backsolve(cplx *G, int ld, int n, int nrhs) {
    const int r = blockIdx.x;
    if (r >= nrhs) return;
    cplx *b = G + (size_t)(n + r) * ld;
    __shared__ cplx xi;
    for (int i = n - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            xi = cdiv(b[i], G[(size_t)i * ld + i]);
            b[i] = xi;
        }
        __syncthreads();
        const cplx v = xi;
        for (int q = threadIdx.x; q < i; q += blockDim.x) b[q] = csub(b[q], cmul(G[(size_t)i * ld + q], v));
        __syncthreads();
    }
}

// S0[(l+p) nc + (n+p)] = s_ln (row l: outgoing order, column n: incident order), one block per (l, n)
__global__ void k_star_moments(int N, int p, const double *nd, double k2, const cplx *G, int ld, cplx *S0) {
    const int nc = 2 * p + 1;
    const int l = blockIdx.x / nc - p, n = blockIdx.x % nc - p;
    const cplx *mu = G + (size_t)(2 * N + n + p) * ld, *sg = mu + N;
    double re = 0.0, im = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double x = nd[j], y = nd[N + j], nx = nd[2 * N + j], ny = nd[3 * N + j], sp = nd[4 * N + j];
        const double rho = hypot(x, y), th = atan2(y, x);
        cplx g[3];   // J_q e^{-i q th}, q = l-1, l, l+1
        for (int q = -1; q <= 1; ++q) g[q + 1] = cscale(cexpi(-(l + q) * th), besselj_int(l + q, k2 * rho));
        const cplx gx = cscale(csub(g[0], g[2]), 0.5 * k2);
        const cplx gy = cscale(cmuli(cadd(g[0], g[2])), -0.5 * k2);
        const cplx gn = cadd(cscale(gx, nx), cscale(gy, ny));
        const cplx t = cscale(cadd(cmul(g[1], sg[j]), cmul(gn, mu[j])), (2.0 * GS_PI / N) * sp);
        re += t.x;
        im += t.y;
    }
    __shared__ double sh[32];
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) S0[(size_t)(l + p) * nc + n + p] = cmuli(C(0.25 * re, 0.25 * im));
}

// Sblk[i][l][n] = e^{i phi_i (n - l)} s_ln
__global__ void k_star_rotate(int M, int p, const double *phi, const cplx *S0, cplx *Sblk) {
    const int nc = 2 * p + 1;
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)M * nc * nc) return;
    const int i = (int)(id / (nc * nc)), e = (int)(id % (nc * nc));
    const int l = e / nc - p, n = e % nc - p;
    Sblk[id] = cmul(cexpi(phi[i] * (n - l)), S0[e]);
}

}  // namespace

// the scattering matrix of the context's star (at k2 and the polarisation) into c->S0, then the
// rotated blocks into c->Sblk
int gs_star_blocks(gs_ctx *c) {
    const int N = c->star.n_nodes, p = c->p, nc = c->nc, n = 2 * N, ncol = n + nc;
    cudaStream_t st = c->stream;
    const double k2 = c->L.k2, kp = c->star.kp;
    const double wp = c->pol ? (kp / k2) * (kp / k2) : 1.0;
    double *nd = nullptr, *R = nullptr;
    cplx *G = nullptr;
    int *sing = nullptr;
    int rc = GS_OK;
    auto cleanup = [&]() {
        if (nd) cudaFree(nd);
        if (R) cudaFree(R);
        if (G) cudaFree(G);
        if (sing) cudaFree(sing);
    };
    if (cudaMalloc((void **)&nd, sizeof(double) * 6 * N) != cudaSuccess ||
        cudaMalloc((void **)&R, sizeof(double) * N) != cudaSuccess ||
        cudaMalloc((void **)&G, sizeof(cplx) * (size_t)n * ncol) != cudaSuccess ||
        cudaMalloc((void **)&sing, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return gs_fail(c, GS_ERR_OOM, "cudaMalloc (inclusion shape system)");
    }
    cudaMemsetAsync(sing, 0, sizeof(int), st);
    GS_COUNT_LAUNCH(c);
    k_star_nodes<<<nblk(N), 256, 0, st>>>(N, c->star.a1, c->star.a2, c->star.a3, nd);
    GS_COUNT_LAUNCH(c);
    gs_kress_weights(N, R, st);
    GS_COUNT_LAUNCH(c);
    k_star_system<<<nblk((long)N * N), 256, 0, st>>>(N, nd, R, k2, kp, wp, G, n);
    GS_COUNT_LAUNCH(c);
    k_star_rhs<<<nblk(N * nc), 256, 0, st>>>(N, p, nd, k2, G, n);
    for (int k = 0; k < n; ++k) {
        GS_COUNT_LAUNCH(c);
        k_lu_pivot<<<1, 1024, 0, st>>>(G, n, n, ncol, k, sing);
        if (k + 1 < n) {
            GS_COUNT_LAUNCH(c);
            k_lu_update<<<nblk((long)(n - k - 1) * (ncol - k - 1)), 256, 0, st>>>(G, n, n, ncol, k);
        }
    }
    GS_COUNT_LAUNCH(c);
    k_lu_backsolve<<<nc, 256, 0, st>>>(G, n, n, nc);
    if (!c->S0) rc = cudaMalloc((void **)&c->S0, sizeof(cplx) * nc * nc) == cudaSuccess ? GS_OK : GS_ERR_OOM;
    if (rc == GS_OK) {
        GS_COUNT_LAUNCH(c);
        k_star_moments<<<nc * nc, 128, 0, st>>>(N, p, nd, k2, G, n, c->S0);
        GS_COUNT_LAUNCH(c);
        k_star_rotate<<<nblk((long)c->M * nc * nc), 256, 0, st>>>(c->M, p, c->star_phi, c->S0, c->Sblk);
    }
    int hs = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, std::string("inclusion shape system: ") + cudaGetErrorString(e));
    if (rc != GS_OK) return gs_fail(c, rc, "cudaMalloc (inclusion scattering matrix)");
    if (hs) return gs_fail(c, GS_ERR_NUMERIC, "inclusion shape system is singular");
    return GS_OK;
}
