// Factorisation of the empty-grating block on the GPU (FP64, Sec. 5 "We precompute A = U Sigma V^*").
//
// The J-expansion columns of A are rescaled to unit 2-norm (Sec. 3, Fig. 2a remark), then the
// SVD of the scaled matrix is taken by one-sided (Hestenes) Jacobi: pairs of columns of W = A D
// are rotated until every pair is orthogonal to relative precision tol; then W = U Sigma and the
// accumulated rotations form V.  Column pairs follow the round-robin (circle) schedule, so each
// launch rotates n/2 disjoint pairs, one thread block per pair.  The pseudo-inverse is applied as
// A^+ g = D V Sigma^+ U^* g with Sigma^+ = min(1/sigma, 1/eps) (Eq. applypA), stored as
// coef_j = 1/(sigma_j max(sigma_j, eps)) acting on W^* g.
#include "gs_internal.h"

namespace {

constexpr int JTPB = 256;

__global__ void k_colnorm_scale(cplx *A, int lda, int rows, int c0, int c1, double *dscale) {
    int col = c0 + blockIdx.x;
    if (col >= c1) return;
    __shared__ double sh[32];
    cplx *a = A + (size_t)col * lda;
    double s = 0.0;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) s += cabs2(a[i]);
    s = block_sum(s, sh);
    double sc = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
    if (threadIdx.x == 0) dscale[col] = sc;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) a[i] = cscale(a[i], sc);
}

__global__ void k_fill(double *x, int n, double v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

__global__ void k_identity(cplx *V, int n) {
    long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)n * n) return;
    int r = (int)(id % n), c = (int)(id / n);
    V[id] = C(r == c ? 1.0 : 0.0, 0.0);
}

// One round of the circle schedule: block k rotates the pair (player(k), player(npad-1-k)).
__global__ void __launch_bounds__(JTPB) k_jacobi_round(cplx *W, int m, cplx *V, int n, int r, int npad,
                                                       double tol, unsigned long long *nrot) {
    int k = blockIdx.x;
    auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + r) % (npad - 1)) + 1; };
    int a = player(k), b = player(npad - 1 - k);
    if (a >= n || b >= n) return;
    int pc = a < b ? a : b, qc = a < b ? b : a;
    cplx *wp = W + (size_t)pc * m, *wq = W + (size_t)qc * m;
    __shared__ double sh[32];
    __shared__ double rot[4];
    double al = 0, be = 0, gr = 0, gi = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        cplx x = wp[i], y = wq[i];
        al += cabs2(x);
        be += cabs2(y);
        gr += x.x * y.x + x.y * y.y;   // conj(x) y
        gi += x.x * y.y - x.y * y.x;
    }
    al = block_sum(al, sh);
    be = block_sum(be, sh);
    gr = block_sum(gr, sh);
    gi = block_sum(gi, sh);
    if (threadIdx.x == 0) {
        double g = hypot(gr, gi);
        if (g == 0.0 || g <= tol * sqrt(al * be)) {
            rot[0] = 0.0;
        } else {
            double zeta = (be - al) / (2.0 * g);
            double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            double cc = 1.0 / sqrt(1.0 + t * t);
            rot[0] = 1.0;
            rot[1] = cc;
            rot[2] = cc * t;
            rot[3] = atan2(gi, gr);
            atomicAdd(nrot, 1ull);
        }
    }
    __syncthreads();
    if (rot[0] == 0.0) return;
    double cc = rot[1], ss = rot[2];
    cplx e = cexpi(-rot[3]);   // e^{-i phi}, phi = arg(conj(w_p) w_q)
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        cplx x = wp[i], y = cmul(wq[i], e);
        wp[i] = csub(cscale(x, cc), cscale(y, ss));
        wq[i] = cadd(cscale(x, ss), cscale(y, cc));
    }
    cplx *vp = V + (size_t)pc * n, *vq = V + (size_t)qc * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        cplx x = vp[i], y = cmul(vq[i], e);
        vp[i] = csub(cscale(x, cc), cscale(y, ss));
        vq[i] = cadd(cscale(x, ss), cscale(y, cc));
    }
}

__global__ void k_sigma(const cplx *W, int m, int n, double eps, double *sigma, double *coef) {
    int col = blockIdx.x;
    if (col >= n) return;
    __shared__ double sh[32];
    const cplx *a = W + (size_t)col * m;
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s += cabs2(a[i]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        double sg = sqrt(s);
        sigma[col] = sg;
        coef[col] = sg > 0.0 ? 1.0 / (sg * fmax(sg, eps)) : 0.0;
    }
}

// row-major copy of the column-major V
__global__ void k_transpose(const cplx *V, int n, cplx *Vr) {
    __shared__ cplx tile[32][33];
    int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    int tx = threadIdx.x, ty = threadIdx.y;
    for (int j = ty; j < 32; j += blockDim.y) {
        int r = bx + tx, c = by + j;   // element V[r + c n] = V(r, c)
        if (r < n && c < n) tile[j][tx] = V[(size_t)c * n + r];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += blockDim.y) {
        int r = bx + j, c = by + tx;
        if (r < n && c < n) Vr[(size_t)r * n + c] = tile[tx][j];
    }
}

}  // namespace

int gs_factor_angle(gs_ctx *c, AngleData &a) {
    const Layout &ly = c->lay;
    int m = ly.rows, n = ly.cols;
    cudaStream_t st = c->stream;
    GS_TRY(gs_assemble_A(c, a, a.W, m));
    GS_TRY(gs_assemble_f(c, a, a.f));
    k_fill<<<(n + 255) / 256, 256, 0, st>>>(a.dscale, n, 1.0);
    k_colnorm_scale<<<ly.col_c - ly.col_a2, 256, 0, st>>>(a.W, m, m, ly.col_a2, ly.col_c, a.dscale);
    // V (column-major) accumulates the rotations; a.Vr receives its row-major copy at the end
    cplx *V = c->Vtmp;   // cols x cols, allocated by gs_factor
    k_identity<<<(int)(((long)n * n + 255) / 256), 256, 0, st>>>(V, n);
    GS_CHECK_LAUNCH(c);
    int npad = n + (n & 1);
    const double tol = 1e-14;
    a.sweeps = 0;
    for (int sweep = 0; sweep < 40; ++sweep) {
        GS_CUDA(c, cudaMemsetAsync(c->dcount, 0, sizeof(unsigned long long), st));
        for (int r = 0; r < npad - 1; ++r)
            k_jacobi_round<<<npad / 2, JTPB, 0, st>>>(a.W, m, V, n, r, npad, tol, c->dcount);
        GS_CHECK_LAUNCH(c);
        unsigned long long h = 0;
        GS_CUDA(c, cudaMemcpyAsync(&h, c->dcount, sizeof(h), cudaMemcpyDeviceToHost, st));
        GS_CUDA(c, cudaStreamSynchronize(st));
        a.sweeps = sweep + 1;
        if (h == 0) break;
    }
    k_sigma<<<n, 256, 0, st>>>(a.W, m, n, c->L.eps_pinv, a.sigma, a.coef);
    dim3 tb(32, 8), tg((n + 31) / 32, (n + 31) / 32);
    k_transpose<<<tg, tb, 0, st>>>(V, n, a.Vr);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}
