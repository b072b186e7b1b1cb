// Schur-complement low-rank apply, preconditioned operator, right-hand side, GMRES and Bragg
// recovery on the GPU (FP64; Sec. 4.2 preconditioner, Sec. 5 Eqs. applypA, schur and the
// preconditioned system, Sec. 6 flux).
//
//   L x = x - S (T x) + S B_phys A^+ C x,   A^+ g = D V Sigma^+ U^* g   (never formed)
// The low-rank term is four matrix-vector products (HBM-bound): g = C x (C rows only),
// w = coef .* (W^* g), v = D .* (V w) restricted to the columns of B_phys, and z = B_phys v, whose
// epilogue fuses the preconditioner and the combination y = x - s .* (T x) + s .* z.
#include <algorithm>
#include <vector>

#include "gs_internal.h"

size_t gs_translate_scratch_elems(int M, int p);

namespace {

// y[r] = scale[r] * sum_c A[r, c] x[c]   (A row-major, warp per row)
__global__ void k_gemv_rows(const cplx *__restrict__ A, int nrows, int ncols, long lda,
                            const cplx *__restrict__ x, const double *__restrict__ scale,
                            cplx *__restrict__ y, float2 *__restrict__ y32 = nullptr) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= nrows) return;
    const cplx *a = A + (size_t)warp * lda;
    cplx s = C(0, 0);
    for (int c = lane; c < ncols; c += 32) cfma(s, a[c], __ldg(&x[c]));
    s.x = warp_sum(s.x);
    s.y = warp_sum(s.y);
    if (lane == 0) {
        const cplx r = scale ? cscale(s, scale[warp]) : s;
        y[warp] = r;
        if (y32) y32[warp] = make_float2((float)r.x, (float)r.y);   // y32: complex64 copy (nullable)
    }
}

// y[r] = sum_c A[r, c] x[c] for few long rows (C: ~1300 rows of M (2p+1) columns), FP64: one block
// of GEMV_BLK_THREADS per row, two independent accumulators per thread.  With a warp per row only
// ~8 warps per SM would be in flight for C, about half of what the FP64 pipe needs.
constexpr int GEMV_BLK_THREADS = 128;
__global__ void __launch_bounds__(GEMV_BLK_THREADS) k_gemv_rows_blk(const cplx *__restrict__ A, int nrows, long ncols,
                                                                   const cplx *__restrict__ x,
                                                                   cplx *__restrict__ y) {
    const int r = blockIdx.x;
    if (r >= nrows) return;
    const cplx *a = A + (size_t)r * ncols;
    cplx s0 = C(0, 0), s1 = C(0, 0);
    long c = threadIdx.x;
    for (; c + GEMV_BLK_THREADS < ncols; c += 2 * GEMV_BLK_THREADS) {
        cfma(s0, __ldcs(&a[c]), __ldg(&x[c]));
        cfma(s1, __ldcs(&a[c + GEMV_BLK_THREADS]), __ldg(&x[c + GEMV_BLK_THREADS]));
    }
    if (c < ncols) cfma(s0, __ldcs(&a[c]), __ldg(&x[c]));
    s0 = cadd(s0, s1);
    s0.x = warp_sum(s0.x);
    s0.y = warp_sum(s0.y);
    __shared__ cplx part[GEMV_BLK_THREADS / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s0;
    __syncthreads();
    if (threadIdx.x == 0) {
        cplx t = part[0];
        for (int k = 1; k < GEMV_BLK_THREADS / 32; ++k) t = cadd(t, part[k]);
        y[r] = t;
    }
}

// y[j] = coef[j] * sum_{i < nr} conj(W[i, j]) g[i]   (W column-major, warp per column)
__global__ void k_gemv_colsH(const cplx *__restrict__ W, int m, int nr, int ncols, const cplx *__restrict__ g,
                             const double *__restrict__ coef, cplx *__restrict__ y) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= ncols) return;
    const cplx *a = W + (size_t)warp * m;
    cplx s = C(0, 0);
    for (int i = lane; i < nr; i += 32) cfma(s, cconj(a[i]), __ldg(&g[i]));
    s.x = warp_sum(s.x);
    s.y = warp_sum(s.y);
    if (lane == 0) y[warp] = cscale(s, coef[warp]);
}

// y[r] = x[r] - s[r] * t[r] + s[r] * (B v)[r]   (B row-major n x nB, warp per row)
__global__ void k_B_combine(const cplx *__restrict__ B, int n, int nB, const cplx *__restrict__ v,
                            const cplx *__restrict__ x, const cplx *__restrict__ t,
                            const cplx *__restrict__ s, cplx *__restrict__ y) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const cplx *b = B + (size_t)warp * nB;
    cplx acc = C(0, 0);
    for (int c = lane; c < nB; c += 32) cfma(acc, b[c], __ldg(&v[c]));
    acc.x = warp_sum(acc.x);
    acc.y = warp_sum(acc.y);
    if (lane == 0) {
        cplx r = x ? x[warp] : C(0, 0);
        if (t) r = csub(r, cmul(s[warp], t[warp]));
        r = cadd(r, s ? cmul(s[warp], acc) : acc);
        y[warp] = r;
    }
}

// ---- complex64 low rank (inner operator of the mixed solve) ----------------------------------------
// A complex FP64 matrix-vector product needs 0.5 flop per byte, above the GB300's FP64 ridge
// (1.26 TFLOP/s / 6.7 TB/s = 0.19): the FP64 products with B_phys and C are bound by the FP64
// pipe.  The inner operator of the mixed solve (whose translation is complex64 anyway) reads a
// complex64 copy of B_phys instead: half the bytes, FP32 arithmetic, HBM-bound.  B_phys acts last
// (after A^+), so its FP32 rounding is not amplified.  C x feeds A^+, whose clipped Sigma^+ (up to
// 1/eps = 1e10 in the near-null directions) would amplify FP32 rounding of C x into the whole
// correction: the inner operator forms it in double-float arithmetic (C and x as complex64 (hi, lo)
// pairs, 48-bit significands), as accurate as the FP64 sum at the FP32 pipe's rate, and as
// bytes-bound as the FP64 form would be with an FP64 pipe 64 times faster.

__global__ void k_to_c64_vec(const cplx *__restrict__ a, long n, float2 *__restrict__ b) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

// complex128 -> (hi, lo) complex64 pairs; flag set if some |entry| exceeds lim (beyond it, sums of
// products could leave the FP32 exponent range) or is not finite
__global__ void k_split_df(const cplx *__restrict__ a, long n, float4 *__restrict__ b, double lim,
                           int *__restrict__ flag) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const cplx v = a[e];
    b[e] = df_split(v.x, v.y);
    if (flag && !(fabs(v.x) <= lim && fabs(v.y) <= lim)) *flag = 1;
}

// y[r] = (C x)[r] in double-float arithmetic, C (nrows x ncols row-major) and x as (hi, lo)
// complex64 pairs; one block of GEMV_DF_THREADS per row, the FP64 result hi + lo
constexpr int GEMV_DF_THREADS = 128;
__global__ void __launch_bounds__(GEMV_DF_THREADS) k_gemv_rows_df(const float4 *__restrict__ C2, int nrows, long ncols,
                                                                 const float4 *__restrict__ x2,
                                                                 cplx *__restrict__ y,
                                                                 const double *__restrict__ scale = nullptr,
                                                                 float2 *__restrict__ y32 = nullptr) {
    const int r = blockIdx.x;
    if (r >= nrows) return;
    const float4 *a = C2 + (size_t)r * ncols;
    dfc s = {0.f, 0.f, 0.f, 0.f};
    dfc_row_dot<GEMV_DF_THREADS>(s, a, x2, ncols, threadIdx.x);
    dfc_warp_sum(s);
    __shared__ dfc part[GEMV_DF_THREADS / 32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) part[w] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        dfc t = part[0];
        for (int k = 1; k < GEMV_DF_THREADS / 32; ++k) dfc_add(t, part[k]);
        cplx v = C((double)t.rh + (double)t.rl, (double)t.ih + (double)t.il);
        if (scale) v = cscale(v, scale[r]);   // scale, y32: optional row scale and complex64 copy
        y[r] = v;
        if (y32) y32[r] = make_float2((float)v.x, (float)v.y);
    }
}

// WH2[j][i] = split(conj(W[i][j])) for i < nr, j < ncols (W column-major with leading dimension m):
// the rows of U^H restricted to C's rows, for k_gemv_rows_df
__global__ void k_split_df_conjT(const cplx *__restrict__ W, int m, int nr, int ncols, float4 *__restrict__ WH2) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)nr * ncols) return;
    const int j = (int)(e / nr), i = (int)(e % nr);
    const cplx v = W[(size_t)j * m + i];
    WH2[e] = df_split(v.x, -v.y);
}

// Vr2[r][j] = split(Vr[r][j] coef[j]) (row-major nrows x ncols); flag set beyond lim
__global__ void k_split_df_colscale(const cplx *__restrict__ Vr, int nrows, int ncols, const double *__restrict__ coef,
                                    float4 *__restrict__ Vr2, double lim, int *__restrict__ flag) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)nrows * ncols) return;
    const cplx v = cscale(Vr[e], coef[e % ncols]);
    Vr2[e] = df_split(v.x, v.y);
    if (!(fabs(v.x) <= lim && fabs(v.y) <= lim)) *flag = 1;
}

// y[r] = x[r] - s[r] t[r] + s[r] (B v)[r] with B and v complex64 (FP32 products), warp per row.  v
// arrives as complex64 (converted once by its producer): an FP64 -> FP32 conversion per entry of B
// would run at the FP64 pipe's rate and bound the kernel, not HBM.  Two accumulator pairs per lane
// keep two loads of each row in flight.
__global__ void k_B_combine32(const float2 *__restrict__ B, int n, int nB, const float2 *__restrict__ v,
                              const cplx *__restrict__ x, const cplx *__restrict__ t, const cplx *__restrict__ s,
                              cplx *__restrict__ y) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const float2 *b = B + (size_t)warp * nB;
    float re0 = 0.f, im0 = 0.f, re1 = 0.f, im1 = 0.f;
    int c = lane;
    for (; c + 32 < nB; c += 64) {
        const float2 m0 = __ldcs(&b[c]), m1 = __ldcs(&b[c + 32]);
        const float2 w0 = __ldg(&v[c]), w1 = __ldg(&v[c + 32]);
        re0 = fmaf(m0.x, w0.x, fmaf(-m0.y, w0.y, re0));
        im0 = fmaf(m0.x, w0.y, fmaf(m0.y, w0.x, im0));
        re1 = fmaf(m1.x, w1.x, fmaf(-m1.y, w1.y, re1));
        im1 = fmaf(m1.x, w1.y, fmaf(m1.y, w1.x, im1));
    }
    if (c < nB) {
        const float2 m0 = __ldcs(&b[c]), w0 = __ldg(&v[c]);
        re0 = fmaf(m0.x, w0.x, fmaf(-m0.y, w0.y, re0));
        im0 = fmaf(m0.x, w0.y, fmaf(m0.y, w0.x, im0));
    }
    float re = re0 + re1, im = im0 + im1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) y[warp] = cadd(csub(x[warp], cmul(s[warp], t[warp])), cmul(s[warp], C(re, im)));
}

// ---- general inclusion shapes: the block preconditioner (Sec. 4.2, S = diag(S_p^(m))) -------------

// u[r] = (B v)[r] - t[r] (t nullable), B row-major FP64 (TB = cplx) or complex64 (TB = float2), warp
// per row; u may alias t
template <typename TB>
__global__ void k_B_minus_t(const TB *__restrict__ B, int n, int nB, const cplx *__restrict__ v, const cplx *t,
                            cplx *u) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const TB *b = B + (size_t)warp * nB;
    cplx acc = C(0, 0);
    for (int c = lane; c < nB; c += 32) {
        const TB m = b[c];
        cfma(acc, C((double)m.x, (double)m.y), __ldg(&v[c]));
    }
    acc.x = warp_sum(acc.x);
    acc.y = warp_sum(acc.y);
    if (lane == 0) u[warp] = t ? csub(acc, t[warp]) : acc;
}

// y[i nc + m] = x[i nc + m] + sum_n S_i[m][n] u[i nc + n] (x nullable), one thread per row
__global__ void k_apply_blocks(const cplx *__restrict__ S, int M, int nc, const cplx *__restrict__ u,
                               const cplx *__restrict__ x, cplx *__restrict__ y) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)M * nc) return;
    const int i = (int)(e / nc), m = (int)(e % nc);
    const cplx *Sr = S + ((size_t)i * nc + m) * nc;
    const cplx *ui = u + (size_t)i * nc;
    cplx acc = x ? x[e] : C(0, 0);
    for (int n = 0; n < nc; ++n) cfma(acc, Sr[n], ui[n]);
    y[e] = acc;
}

// g[r] = f[r] - (C x)[r] for r < nC, and f[r] for nC <= r < rows
__global__ void k_f_minus_Cx(const cplx *__restrict__ Cm, int nC, int n, const cplx *__restrict__ x,
                             const cplx *__restrict__ f, int rows, cplx *__restrict__ g) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= rows) return;
    if (warp >= nC) {
        if (lane == 0) g[warp] = f[warp];
        return;
    }
    const cplx *a = Cm + (size_t)warp * n;
    cplx s = C(0, 0);
    for (int c = lane; c < n; c += 32) cfma(s, a[c], __ldg(&x[c]));
    s.x = warp_sum(s.x);
    s.y = warp_sum(s.y);
    if (lane == 0) g[warp] = csub(f[warp], s);
}

// ---- GMRES helpers ------------------------------------------------------------------------------

// h[i] (+)= V_i^* w for i < cnt (block per basis vector)
__global__ void k_dots(const cplx *__restrict__ Vb, long n, const cplx *__restrict__ w, int cnt,
                       cplx *__restrict__ h, int accumulate) {
    int i = blockIdx.x;
    if (i >= cnt) return;
    __shared__ double sh[32];
    const cplx *v = Vb + (size_t)i * n;
    double re = 0, im = 0;
    for (long e = threadIdx.x; e < n; e += blockDim.x) {
        cplx a = v[e], b = w[e];
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
    }
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) {
        cplx r = C(re, im);
        h[i] = accumulate ? cadd(h[i], r) : r;
    }
}

// w -= sum_{i < cnt} coef[i] V_i
__global__ void k_sub_combo(cplx *__restrict__ w, const cplx *__restrict__ Vb, long n,
                            const cplx *__restrict__ coef, int cnt) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    cplx s = w[e];
    for (int i = 0; i < cnt; ++i) s = csub(s, cmul(coef[i], Vb[(size_t)i * n + e]));
    w[e] = s;
}

// x += sum_{i < cnt} y[i] V_i
__global__ void k_add_combo(cplx *__restrict__ x, const cplx *__restrict__ Vb, long n,
                            const cplx *__restrict__ y, int cnt) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    cplx s = x[e];
    for (int i = 0; i < cnt; ++i) s = cadd(s, cmul(y[i], Vb[(size_t)i * n + e]));
    x[e] = s;
}

// out[0] = ||w||_2 (single block)
__global__ void k_norm(const cplx *__restrict__ w, long n, double *out) {
    __shared__ double sh[32];
    double s = 0;
    for (long e = threadIdx.x; e < n; e += blockDim.x) s += cabs2(w[e]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[0] = sqrt(s);
}

// dst = src * (1 / norm[0]); also records norm into Hsub (complex) if given
__global__ void k_scale_by_inv(const cplx *src, long n, const double *norm, cplx *dst,
                               cplx *Hsub) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double nv = norm[0];
    if (e == 0 && Hsub) *Hsub = C(nv, 0.0);
    if (e >= n) return;
    dst[e] = nv > 0.0 ? cscale(src[e], 1.0 / nv) : C(0, 0);
}

__global__ void k_add_vec(cplx *h, const cplx *v, int cnt) {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) h[i] = cadd(h[i], v[i]);
}

__global__ void k_sub(const cplx *a, const cplx *b, long n, cplx *y) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) y[e] = csub(a[e], b[e]);
}

// Givens step for Hessenberg column j (column-major, leading dimension ld): applies the previous
// rotations, forms the new one, updates g and writes the residual estimate |g[j+1]| to res.
// Applying rotations 0..j-1 in turn to the column is a linear recurrence in the value carried down
// it: with carry_0 = h_0,
//   h'_i = c_i carry_i + s_i h_{i+1},   carry_{i+1} = -conj(s_i) carry_i + c_i h_{i+1},
// so carry_{i+1} = A_i h_0 + B_i with (A_i, B_i) the composition of the affine maps
// x -> -conj(s_k) x + c_k h_{k+1}, k <= i; the block forms all compositions by an inclusive scan
// (|s_k| <= 1, so the products stay bounded) instead of j dependent steps on one thread.  Launch
// with GS_KMAX threads (j < GS_KMAX).
constexpr int GS_KMAX = 512;
__global__ void __launch_bounds__(GS_KMAX) k_givens(cplx *H, int ld, int j, cplx *cs, cplx *sn, cplx *g,
                                                   double *res) {
    __shared__ cplx mA[GS_KMAX], mB[GS_KMAX];
    cplx *col = H + (size_t)j * ld;
    const int t = threadIdx.x;
    const cplx h0 = col[0], hj1 = col[j + 1];
    cplx ct = C(1, 0), st = C(0, 0), hn = C(0, 0), a = C(1, 0), b = C(0, 0);
    if (t < j) {
        ct = cs[t];
        st = sn[t];
        hn = col[t + 1];
        a = cscale(cconj(st), -1.0);
        b = cmul(ct, hn);
    }
    mA[t] = a;
    mB[t] = b;
    __syncthreads();
    for (int off = 1; off < GS_KMAX; off <<= 1) {
        cplx pa = C(1, 0), pb = C(0, 0);
        if (t >= off) {
            pa = mA[t - off];
            pb = mB[t - off];
        }
        __syncthreads();
        if (t >= off) {   // (a, b) after (pa, pb): x -> a (pa x + pb) + b
            const cplx na = cmul(mA[t], pa), nb = cadd(cmul(mA[t], pb), mB[t]);
            mA[t] = na;
            mB[t] = nb;
        }
        __syncthreads();
    }
    if (t < j) {
        const cplx carry = t == 0 ? h0 : cadd(cmul(mA[t - 1], h0), mB[t - 1]);
        col[t] = cadd(cmul(ct, carry), cmul(st, hn));
    }
    if (t == 0) {
        const cplx av = j == 0 ? h0 : cadd(cmul(mA[j - 1], h0), mB[j - 1]), bv = hj1;
        const double aa = sqrt(cabs2(av)), bb = sqrt(cabs2(bv));
        const double rr = hypot(aa, bb);
        cplx c, s;
        if (rr == 0.0) {
            c = C(1, 0);
            s = C(0, 0);
        } else if (aa == 0.0) {
            c = C(0, 0);
            s = cscale(cconj(bv), 1.0 / bb);
        } else {
            c = C(aa / rr, 0.0);
            s = cmul(cscale(av, 1.0 / aa), cscale(cconj(bv), 1.0 / rr));
        }
        cs[j] = c;
        sn[j] = s;
        col[j] = cadd(cmul(c, av), cmul(s, bv));
        col[j + 1] = C(0, 0);
        const cplx gj = g[j];
        g[j + 1] = cmul(cscale(cconj(s), -1.0), gj);
        g[j] = cmul(c, gj);
        res[0] = sqrt(cabs2(g[j + 1]));
    }
}

// back substitution H[0:k,0:k] y = g[0:k] (upper triangular), column-oriented: one thread divides,
// the block updates the remaining right-hand side
__global__ void k_backsolve(const cplx *H, int ld, int kk, const cplx *g, cplx *y) {
    __shared__ cplx r[GS_KMAX];
    __shared__ cplx yi;
    for (int i = threadIdx.x; i < kk; i += blockDim.x) r[i] = g[i];
    __syncthreads();
    for (int i = kk - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            yi = cdiv(r[i], H[(size_t)i * ld + i]);
            y[i] = yi;
        }
        __syncthreads();
        const cplx v = yi;
        for (int q = threadIdx.x; q < i; q += blockDim.x) r[q] = csub(r[q], cmul(H[(size_t)i * ld + q], v));
        __syncthreads();
    }
}

__global__ void k_set_g0(cplx *g, int len, const double *beta) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) g[i] = C(i == 0 ? beta[0] : 0.0, 0.0);
}

// Bragg amplitudes and flux error (single block): c_n = x_c[n], d_n = x_d[n] for propagating orders;
// the vertical energy fluxes carry 1/w1, 1/w3 in TE (w = 1 for TM), inc = k1 |sin theta| / w1.
__global__ void k_flux(int K, const cplx *cd, const cplx *k1n, const cplx *k3n, double inv_w1, double inv_w3,
                       double inc, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int n = 0; n < 2 * K + 1; ++n) {
        if (k1n[n].y == 0.0 && k1n[n].x > 0.0) s += inv_w1 * k1n[n].x * cabs2(cd[n]);
        if (k3n[n].y == 0.0 && k3n[n].x > 0.0) s += inv_w3 * k3n[n].x * cabs2(cd[2 * K + 1 + n]);
    }
    out[0] = fabs(s - inc) / inc;
}

inline int warps_blocks(long nwarps) { return (int)((nwarps * 32 + 255) / 256); }

}  // namespace

// x = A^+ g (full): w = coef .* W^* g; x = D .* V w
int gs_pinv_impl(gs_ctx *c, const AngleData &a, const cplx *g, cplx *x) {
    const Layout &ly = c->lay;
    GS_COUNT_LAUNCH(c);
    k_gemv_colsH<<<warps_blocks(ly.cols), 256, 0, c->stream>>>(a.W, ly.rows, ly.rows, ly.cols, g, a.coef, c->w);
    GS_COUNT_LAUNCH(c);
    k_gemv_rows<<<warps_blocks(ly.cols), 256, 0, c->stream>>>(a.Vr, ly.cols, ly.cols, ly.cols, c->w, a.dscale, x);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

// double-float copies of U^H (C's rows) and of V Sigma diag(coef) for the mixed inner operator's A^+,
// once per factorisation (allocates: not inside a stream capture); a.A2_ready tells whether they hold
int gs_prepare_apinv_df(gs_ctx *c, const AngleData &a) {
    const Layout &ly = c->lay;
    const int nB = ly.nB(), nC = ly.nC();
    // the vectors go through the context's scratch adf, which geometry changes free
    const long need = std::max((long)nC, (long)ly.cols);
    if (!a.A2_off && c->adf_n < need) {
        if (c->adf) cudaFree(c->adf);
        c->adf = nullptr;
        c->adf_n = 0;
        if (cudaMalloc((void **)&c->adf, sizeof(float4) * need) != cudaSuccess) {
            cudaGetLastError();   // no room: the FP64 products stay
            c->adf = nullptr;
            a.A2_off = true;
        } else {
            c->adf_n = need;
        }
    }
    if (!a.A2_off && !c->iflag && cudaMalloc((void **)&c->iflag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        c->iflag = nullptr;
        a.A2_off = true;
    }
    if (!a.A2_ready && !a.A2_off) {
        const long nw = (long)ly.cols * nC, nv = (long)nB * ly.cols;
        if (!a.WH2 && (cudaMalloc((void **)&a.WH2, sizeof(float4) * nw) != cudaSuccess ||
                       cudaMalloc((void **)&a.Vr2, sizeof(float4) * nv) != cudaSuccess)) {
            cudaGetLastError();   // no room: the FP64 products stay
            if (a.WH2) cudaFree(a.WH2);
            a.WH2 = nullptr;
            a.Vr2 = nullptr;
            a.A2_off = true;
        }
        if (a.WH2 && !a.A2_off) {
            GS_CUDA(c, cudaMemsetAsync(c->iflag, 0, sizeof(int), c->stream));
            GS_COUNT_LAUNCH(c);
            k_split_df_conjT<<<(int)((nw + 255) / 256), 256, 0, c->stream>>>(a.W, ly.rows, nC, ly.cols, a.WH2);
            GS_COUNT_LAUNCH(c);
            k_split_df_colscale<<<(int)((nv + 255) / 256), 256, 0, c->stream>>>(a.Vr, nB, ly.cols, a.coef, a.Vr2,
                                                                                GS_DF_LIMIT, c->iflag);
            GS_CHECK_LAUNCH(c);
            int big = 0;
            GS_CUDA(c, cudaMemcpyAsync(&big, c->iflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            GS_CUDA(c, cudaStreamSynchronize(c->stream));
            if (big) a.A2_off = true;
            else a.A2_ready = true;
        }
    }
    return GS_OK;
}

// complex64 copy of B_phys and double-float copy of C for the mixed inner operator, once per
// geometry and angle (allocates: not inside a stream capture)
int gs_prepare_c64(gs_ctx *c, const AngleData &a) {
    const Layout &ly = c->lay;
    const int n = c->n(), nB = ly.nB(), nC = ly.nC();
    if (!a.B32) {
        const long nb = (long)n * nB;
        GS_CUDA(c, cudaMalloc((void **)&a.B32, sizeof(float2) * nb));
        GS_COUNT_LAUNCH(c);
        k_to_c64_vec<<<(int)((nb + 255) / 256), 256, 0, c->stream>>>(a.B, nb, a.B32);
    }
    if (!a.C2 && !a.C2_off) {
        const long nc2 = (long)nC * n;
        if (cudaMalloc((void **)&a.C2, sizeof(float4) * nc2) != cudaSuccess) {
            cudaGetLastError();   // no room for the copy: the FP64 product stays
            a.C2 = nullptr;
            a.C2_off = true;
        }
    }
    GS_TRY(gs_prepare_apinv_df(c, a));
    if (a.C2 && !a.C2_ready) {
        const long nc2 = (long)nC * n;
        GS_CUDA(c, cudaMemsetAsync(c->iflag, 0, sizeof(int), c->stream));
        GS_COUNT_LAUNCH(c);
        k_split_df<<<(int)((nc2 + 255) / 256), 256, 0, c->stream>>>(a.Cm, nc2, a.C2, GS_DF_LIMIT, c->iflag);
        GS_CHECK_LAUNCH(c);
        int big = 0;
        GS_CUDA(c, cudaMemcpyAsync(&big, c->iflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        if (big) {   // entries beyond the double-float range: keep the FP64 product
            cudaFree(a.C2);
            a.C2 = nullptr;
            a.C2_off = true;
        } else {
            a.C2_ready = true;
        }
    }
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

// y = x - s .* t + s .* (B_phys A^+ C x) for the mixed inner operator, t = T x given: C x and A^+
// in double-float arithmetic (each in FP64 when its copies are off), B_phys in complex64.  Only
// launches kernels (after gs_prepare_c64).
int gs_lowrank_c64(gs_ctx *c, const AngleData &a, const cplx *x, const cplx *t, cplx *y) {
    const Layout &ly = c->lay;
    const int n = c->n(), nB = ly.nB(), nC = ly.nC();
    if (!a.B32 || (!a.C2 && !a.C2_off)) return gs_fail(c, GS_ERR_STATE, "gs_prepare_c64 has not run");
    GS_COUNT_LAUNCH(c);
    if (a.C2) {
        k_split_df<<<(int)((n + 255) / 256), 256, 0, c->stream>>>(x, n, c->xdf, 0.0, nullptr);
        GS_COUNT_LAUNCH(c);
        k_gemv_rows_df<<<nC, GEMV_DF_THREADS, 0, c->stream>>>(a.C2, nC, n, c->xdf, c->g);
    } else {
        k_gemv_rows_blk<<<nC, GEMV_BLK_THREADS, 0, c->stream>>>(a.Cm, nC, n, x, c->g);
    }
    if (a.A2_ready && a.WH2 && a.Vr2 && c->adf && c->adf_n >= std::max((long)nC, (long)ly.cols)) {
        // A^+ g in double-float: U^H g, then (V Sigma diag(coef)) (U^H g), scaled by D
        GS_COUNT_LAUNCH(c);
        k_split_df<<<(nC + 255) / 256, 256, 0, c->stream>>>(c->g, nC, c->adf, 0.0, nullptr);
        GS_COUNT_LAUNCH(c);
        k_gemv_rows_df<<<ly.cols, GEMV_DF_THREADS, 0, c->stream>>>(a.WH2, ly.cols, nC, c->adf, c->w);
        GS_COUNT_LAUNCH(c);
        k_split_df<<<(ly.cols + 255) / 256, 256, 0, c->stream>>>(c->w, ly.cols, c->adf, 0.0, nullptr);
        GS_COUNT_LAUNCH(c);
        k_gemv_rows_df<<<nB, GEMV_DF_THREADS, 0, c->stream>>>(a.Vr2, nB, ly.cols, c->adf, c->x, a.dscale, c->x32);
    } else {
        GS_COUNT_LAUNCH(c);
        k_gemv_colsH<<<warps_blocks(ly.cols), 256, 0, c->stream>>>(a.W, ly.rows, nC, ly.cols, c->g, a.coef, c->w);
        GS_COUNT_LAUNCH(c);
        k_gemv_rows<<<warps_blocks(nB), 256, 0, c->stream>>>(a.Vr, nB, ly.cols, ly.cols, c->w, a.dscale, c->x,
                                                             c->x32);
    }
    GS_COUNT_LAUNCH(c);
    if (c->Sblk) {   // general shapes: y = x + S (B v - t), in two steps through the scratch c->v6
        k_B_minus_t<float2><<<warps_blocks(n), 256, 0, c->stream>>>(a.B32, n, nB, c->x, t, c->v6);
        GS_COUNT_LAUNCH(c);
        k_apply_blocks<<<(n + 255) / 256, 256, 0, c->stream>>>(c->Sblk, c->M, c->nc, c->v6, x, y);
    } else {
        k_B_combine32<<<warps_blocks(n), 256, 0, c->stream>>>(a.B32, n, nB, c->x32, x, t, c->s, y);
    }
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

// y = x - s .* T x + s .* (B_phys A^+ C x)
int gs_apply_impl(gs_ctx *c, const AngleData &a, const cplx *x, cplx *y, int precision) {
    const Layout &ly = c->lay;
    int n = c->n(), nB = ly.nB(), nC = ly.nC();
    cplx *tx = c->v3;
    GS_TRY(gs_translate_impl(c, a, x, tx, precision));
    if (precision == GS_C64) {
        GS_TRY(gs_prepare_c64(c, a));
        return gs_lowrank_c64(c, a, x, tx, y);
    }
    GS_COUNT_LAUNCH(c);
    k_gemv_rows_blk<<<nC, GEMV_BLK_THREADS, 0, c->stream>>>(a.Cm, nC, n, x, c->g);
    GS_COUNT_LAUNCH(c);
    k_gemv_colsH<<<warps_blocks(ly.cols), 256, 0, c->stream>>>(a.W, ly.rows, nC, ly.cols, c->g, a.coef, c->w);
    GS_COUNT_LAUNCH(c);
    k_gemv_rows<<<warps_blocks(nB), 256, 0, c->stream>>>(a.Vr, nB, ly.cols, ly.cols, c->w, a.dscale, c->x);
    GS_COUNT_LAUNCH(c);
    if (c->Sblk) {   // general shapes: y = x + S (B v - T x), B v - T x in place of T x
        k_B_minus_t<cplx><<<warps_blocks(n), 256, 0, c->stream>>>(a.B, n, nB, c->x, tx, tx);
        GS_COUNT_LAUNCH(c);
        k_apply_blocks<<<(n + 255) / 256, 256, 0, c->stream>>>(c->Sblk, c->M, c->nc, tx, x, y);
    } else {
        k_B_combine<<<warps_blocks(n), 256, 0, c->stream>>>(a.B, n, nB, c->x, x, tx, c->s, y);
    }
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

// z = B_phys A^+ C x (the layer response to the inclusions' field, without the diagonal s)
int gs_layer_response_impl(gs_ctx *c, const AngleData &a, const cplx *x, cplx *z) {
    const Layout &ly = c->lay;
    int n = c->n(), nB = ly.nB(), nC = ly.nC();
    GS_COUNT_LAUNCH(c);
    k_gemv_rows_blk<<<nC, GEMV_BLK_THREADS, 0, c->stream>>>(a.Cm, nC, n, x, c->g);
    GS_COUNT_LAUNCH(c);
    k_gemv_colsH<<<warps_blocks(ly.cols), 256, 0, c->stream>>>(a.W, ly.rows, nC, ly.cols, c->g, a.coef, c->w);
    GS_COUNT_LAUNCH(c);
    k_gemv_rows<<<warps_blocks(nB), 256, 0, c->stream>>>(a.Vr, nB, ly.cols, ly.cols, c->w, a.dscale, c->x);
    GS_COUNT_LAUNCH(c);
    k_B_combine<<<warps_blocks(n), 256, 0, c->stream>>>(a.B, n, nB, c->x, nullptr, nullptr, nullptr, z);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

// b = s .* (B_phys A^+ f); f vanishes outside the Gamma1 rows
namespace {
// y = [s (.)] B_phys A^+ f (s null: no scattering diagonal)
int incoming_f(gs_ctx *c, const AngleData &a, const cplx *s, cplx *y) {
    const Layout &ly = c->lay;
    int n = c->n(), nB = ly.nB();
    GS_COUNT_LAUNCH(c);
    k_gemv_colsH<<<warps_blocks(ly.cols), 256, 0, c->stream>>>(a.W, ly.rows, ly.row_g2v, ly.cols, a.f, a.coef, c->w);
    GS_COUNT_LAUNCH(c);
    k_gemv_rows<<<warps_blocks(nB), 256, 0, c->stream>>>(a.Vr, nB, ly.cols, ly.cols, c->w, a.dscale, c->x);
    GS_COUNT_LAUNCH(c);
    k_B_combine<<<warps_blocks(n), 256, 0, c->stream>>>(a.B, n, nB, c->x, nullptr, nullptr, s, y);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}
}  // namespace

int gs_rhs_impl(gs_ctx *c, const AngleData &a, cplx *b) {
    if (!c->Sblk) return incoming_f(c, a, c->s, b);
    // general shapes: b = S w, w = B_phys A^+ f
    GS_TRY(incoming_f(c, a, nullptr, c->v3));
    GS_COUNT_LAUNCH(c);
    k_apply_blocks<<<(c->n() + 255) / 256, 256, 0, c->stream>>>(c->Sblk, c->M, c->nc, c->v3, nullptr, b);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

int gs_incoming_impl(gs_ctx *c, const AngleData &a, cplx *w) { return incoming_f(c, a, nullptr, w); }

namespace {

__global__ void k_axpy_inplace(cplx *x, const cplx *y, long n) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) x[e] = cadd(x[e], y[e]);
}

// ---- complex64 Krylov basis (inner GMRES of the mixed solve) ---------------------------------------
// The CGS2 products with j basis vectors cost 16 j n flops per iteration; in FP64 they are bound by
// the FP64 pipe (0.5 flop per byte).  The inner solves of the mixed form, solved to >= 1e-6 and
// checked against their true residual, keep the basis in complex64 and do these products in FP32
// (block sums in FP64); the operator still takes and returns FP64 vectors.

// Partial inner products part[q ld + i] = V_i^* w over the q-th of Q element ranges, V and w complex64
// (FP32 products, FP64 block sums); grid (cnt, Q).  With Q = 1 the sum goes straight to h[i].  A
// block per basis vector alone leaves most SMs idle early in a cycle (few vectors), so short
// cycles split each vector over Q blocks; k_dots_reduce adds the Q partials in a fixed order.
__global__ void k_dots32(const float2 *__restrict__ Vb, long n, const float2 *__restrict__ w, int cnt,
                         cplx *__restrict__ out, int ld, int accumulate) {
    const int i = blockIdx.x, q = blockIdx.y, Q = gridDim.y;
    if (i >= cnt) return;
    __shared__ double sh[32];
    const float2 *v = Vb + (size_t)i * n;
    const long e0 = n * q / Q, e1 = n * (q + 1) / Q;
    float re = 0.f, im = 0.f, re1 = 0.f, im1 = 0.f;
    long e = e0 + threadIdx.x;
    for (; e + blockDim.x < e1; e += 2 * blockDim.x) {
        const float2 a = v[e], b = w[e], a1 = v[e + blockDim.x], b1 = w[e + blockDim.x];
        re = fmaf(a.x, b.x, fmaf(a.y, b.y, re));   // conj(a) b
        im = fmaf(a.x, b.y, fmaf(-a.y, b.x, im));
        re1 = fmaf(a1.x, b1.x, fmaf(a1.y, b1.y, re1));
        im1 = fmaf(a1.x, b1.y, fmaf(-a1.y, b1.x, im1));
    }
    if (e < e1) {
        const float2 a = v[e], b = w[e];
        re = fmaf(a.x, b.x, fmaf(a.y, b.y, re));
        im = fmaf(a.x, b.y, fmaf(-a.y, b.x, im));
    }
    const double R = block_sum((double)re + (double)re1, sh), I = block_sum((double)im + (double)im1, sh);
    if (threadIdx.x == 0) {
        const cplx r = C(R, I);
        if (Q == 1)
            out[i] = accumulate ? cadd(out[i], r) : r;
        else
            out[(size_t)q * ld + i] = r;
    }
}

// h[i] (+)= sum_q part[q ld + i], q = 0..Q-1 in order
__global__ void k_dots_reduce(const cplx *__restrict__ part, int Q, int ld, int cnt, cplx *__restrict__ h,
                              int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    cplx r = C(0, 0);
    for (int q = 0; q < Q; ++q) r = cadd(r, part[(size_t)q * ld + i]);
    h[i] = accumulate ? cadd(h[i], r) : r;
}

// w (+/-)= sum_{i < cnt} coef[i] V_i, products in FP32; cnt <= GS_KMAX + 1.  A block takes
// COMBO_E = 64 consecutive elements with four thread groups, group g summing the basis vectors
// i = g, g + 4, ... (four loads in flight per thread); the four partial sums are added in shared
// memory in a fixed order.  With one thread per element the ~25 000-element vectors left about five
// warps per SM, too few to cover the basis loads.  Optionally writes the complex64 copy w32 of the
// result and, per block, the partial squared norm of the result to npart[blockIdx.x].
constexpr int COMBO_E = 64;
__global__ void __launch_bounds__(256) k_combo32(cplx *__restrict__ w, const float2 *__restrict__ Vb, long n,
                                                 const cplx *__restrict__ coef, int cnt, float sign,
                                                 float2 *__restrict__ w32, double *__restrict__ npart) {
    __shared__ float2 cf[513];
    __shared__ float2 part[4][COMBO_E];
    __shared__ double sh[32];
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) cf[i] = make_float2((float)coef[i].x, (float)coef[i].y);
    __syncthreads();
    const int le = threadIdx.x % COMBO_E, grp = threadIdx.x / COMBO_E;
    const long e = (long)blockIdx.x * COMBO_E + le;
    if (e < n) {
        float sr[4] = {0.f, 0.f, 0.f, 0.f}, si[4] = {0.f, 0.f, 0.f, 0.f};
        int i = grp;
        for (; i + 12 < cnt; i += 16) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 v = Vb[(size_t)(i + 4 * u) * n + e], c = cf[i + 4 * u];
                sr[u] = fmaf(c.x, v.x, fmaf(-c.y, v.y, sr[u]));
                si[u] = fmaf(c.x, v.y, fmaf(c.y, v.x, si[u]));
            }
        }
        for (; i < cnt; i += 4) {
            const float2 v = Vb[(size_t)i * n + e], c = cf[i];
            sr[0] = fmaf(c.x, v.x, fmaf(-c.y, v.y, sr[0]));
            si[0] = fmaf(c.x, v.y, fmaf(c.y, v.x, si[0]));
        }
        part[grp][le] = make_float2((sr[0] + sr[1]) + (sr[2] + sr[3]), (si[0] + si[1]) + (si[2] + si[3]));
    }
    __syncthreads();
    double nrm = 0.0;
    if (grp == 0 && e < n) {
        const float tr = (part[0][le].x + part[1][le].x) + (part[2][le].x + part[3][le].x);
        const float ti = (part[0][le].y + part[1][le].y) + (part[2][le].y + part[3][le].y);
        const cplx r = cadd(w[e], C((double)(sign * tr), (double)(sign * ti)));
        w[e] = r;
        if (w32) w32[e] = make_float2((float)r.x, (float)r.y);
        nrm = cabs2(r);
    }
    if (npart) {
        nrm = block_sum(nrm, sh);
        if (threadIdx.x == 0) npart[blockIdx.x] = nrm;
    }
}

// dst = src / nv in complex64, nv = norm[0], or nv = sqrt(sum of np partials npart[0..np-1]) when
// npart is given (added in the same order by every block); records nv into Hsub (complex) if given
__global__ void k_store32(const cplx *__restrict__ src, long n, const double *norm, float2 *__restrict__ dst,
                          cplx *Hsub, const double *__restrict__ npart = nullptr, int np = 0) {
    __shared__ double sh[32];
    double nv;
    if (npart) {
        double t = 0.0;
        for (int k = threadIdx.x; k < np; k += blockDim.x) t += npart[k];
        nv = sqrt(block_sum(t, sh));
    } else {
        nv = norm[0];
    }
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e == 0 && Hsub) *Hsub = C(nv, 0.0);
    if (e >= n) return;
    const double inv = nv > 0.0 ? 1.0 / nv : 0.0;
    dst[e] = make_float2((float)(src[e].x * inv), (float)(src[e].y * inv));
}

__global__ void k_load64(const float2 *__restrict__ v, long n, cplx *__restrict__ out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = C((double)v[e].x, (double)v[e].y);
}

// Restarted GMRES (Saad-Schultz) with classical Gram-Schmidt applied twice and Givens rotations on
// the device; the host reads one residual estimate per iteration.  Solves L_prec x = b from the
// start x (zero when x_zero) until ||b - L_prec x|| <= tol * bnorm; the true residual is checked
// at the end of each cycle.  Uses v2 (residual), v3 (translation output) and the Krylov workspace.
int gmres_core(gs_ctx *c, const AngleData &a, const cplx *b, double bnorm, cplx *x, bool x_zero, double tol,
               int maxit, int restart, int precision, int *iters, double *relres) {
    const long n = c->n();
    cudaStream_t st = c->stream;
    const int kd = std::min(restart, c->kdim);
    const int ld = c->kdim + 1;
    const int eb = (int)((n + 255) / 256);
    cplx *r = c->v2;
    double *ds = c->dscal;   // [1] = ||r||, [2] = residual estimate, [3] = scratch
    int it = 0;
    bool first = x_zero;
    double est = 1.0;
    if (x_zero) GS_CUDA(c, cudaMemsetAsync(x, 0, sizeof(cplx) * n, st));
    while (it < maxit) {
        if (first) {
            GS_CUDA(c, cudaMemcpyAsync(r, b, sizeof(cplx) * n, cudaMemcpyDeviceToDevice, st));
        } else {
            GS_TRY(gs_apply_impl(c, a, x, r, precision));
            GS_COUNT_LAUNCH(c);
            k_sub<<<eb, 256, 0, st>>>(b, r, n, r);
        }
        first = false;
        GS_COUNT_LAUNCH(c);
        k_norm<<<1, 1024, 0, st>>>(r, n, ds + 1);
        GS_CUDA(c, cudaMemcpyAsync(c->hscal + 1, ds + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
        GS_CUDA(c, cudaStreamSynchronize(st));
        est = c->hscal[1] / bnorm;
        if (est <= tol) break;
        GS_COUNT_LAUNCH(c);
        k_scale_by_inv<<<eb, 256, 0, st>>>(r, n, ds + 1, c->Vk, nullptr);
        GS_COUNT_LAUNCH(c);
        k_set_g0<<<(ld + 255) / 256, 256, 0, st>>>(c->gg, ld, ds + 1);
        GS_CUDA(c, cudaMemsetAsync(c->Hh, 0, sizeof(cplx) * (size_t)ld * c->kdim, st));
        int j = 0, kk = 0;
        for (; j < kd && it < maxit; ++j) {
            cplx *vj = c->Vk + (size_t)j * n;
            cplx *w = c->Vk + (size_t)(j + 1) * n;
            GS_TRY(gs_apply_impl(c, a, vj, w, precision));
            ++it;
            cplx *h = c->Hh + (size_t)j * ld;
            // CGS2
            GS_COUNT_LAUNCH(c);
            k_dots<<<j + 1, 256, 0, st>>>(c->Vk, n, w, j + 1, h, 0);
            GS_COUNT_LAUNCH(c);
            k_sub_combo<<<eb, 256, 0, st>>>(w, c->Vk, n, h, j + 1);
            GS_COUNT_LAUNCH(c);
            k_dots<<<j + 1, 256, 0, st>>>(c->Vk, n, w, j + 1, c->yy, 0);
            GS_COUNT_LAUNCH(c);
            k_sub_combo<<<eb, 256, 0, st>>>(w, c->Vk, n, c->yy, j + 1);
            GS_COUNT_LAUNCH(c);
            k_add_vec<<<1, 256, 0, st>>>(h, c->yy, j + 1);   // h += second-pass coefficients
            GS_COUNT_LAUNCH(c);
            k_norm<<<1, 1024, 0, st>>>(w, n, ds + 3);
            GS_COUNT_LAUNCH(c);
            k_scale_by_inv<<<eb, 256, 0, st>>>(w, n, ds + 3, w, h + j + 1);
            GS_COUNT_LAUNCH(c);
            k_givens<<<1, GS_KMAX, 0, st>>>(c->Hh, ld, j, c->cs, c->sn, c->gg, ds + 2);
            GS_CHECK_LAUNCH(c);
            GS_CUDA(c, cudaMemcpyAsync(c->hscal + 2, ds + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
            GS_CUDA(c, cudaStreamSynchronize(st));
            est = c->hscal[2] / bnorm;
            kk = j + 1;
            if (est <= tol) break;
        }
        GS_COUNT_LAUNCH(c);
        k_backsolve<<<1, 256, 0, st>>>(c->Hh, ld, kk, c->gg, c->yy);
        GS_COUNT_LAUNCH(c);
        k_add_combo<<<eb, 256, 0, st>>>(x, c->Vk, n, c->yy, kk);
        GS_CHECK_LAUNCH(c);
        if (est <= tol) {
            // confirm with the true residual of this operator
            GS_TRY(gs_apply_impl(c, a, x, r, precision));
            GS_COUNT_LAUNCH(c);
            k_sub<<<eb, 256, 0, st>>>(b, r, n, r);
            GS_COUNT_LAUNCH(c);
            k_norm<<<1, 1024, 0, st>>>(r, n, ds + 1);
            GS_CUDA(c, cudaMemcpyAsync(c->hscal + 1, ds + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
            GS_CUDA(c, cudaStreamSynchronize(st));
            est = c->hscal[1] / bnorm;
            if (est <= 10.0 * tol) break;
        }
    }
    *iters = it;
    *relres = est;
    return GS_OK;
}

// The same restarted GMRES with a complex64 basis (the inner solves of the mixed form): the basis
// lives in Vk reinterpreted as complex64, the current vector and the operator output in kv1, kv2.
int gmres_core32(gs_ctx *c, const AngleData &a, const cplx *b, double bnorm, cplx *x, double tol, int maxit,
                 int restart, int *iters, double *relres) {
    const long n = c->n();
    cudaStream_t st = c->stream;
    const int kd = std::min(restart, c->kdim);
    const int ld = c->kdim + 1;
    const int eb = (int)((n + 255) / 256);
    float2 *V = (float2 *)c->Vk;
    cplx *r = c->v2, *vj = c->kv1, *w = c->kv2;
    double *ds = c->dscal;
    const int ebc = (int)((n + COMBO_E - 1) / COMBO_E);   // blocks of k_combo32
    const bool fused_norm = ebc <= GS_NORM_PARTS;          // the second CGS pass leaves the norm partials
    // h[0..cnt) = V^* w32, split over up to GS_DOT_SPLIT blocks per basis vector early in a cycle
    auto dots = [&](int cnt, cplx *dst) -> int {
        const int Q = std::min(GS_DOT_SPLIT, std::max(1, (2 * c->sms + cnt - 1) / cnt));
        GS_COUNT_LAUNCH(c);
        k_dots32<<<dim3(cnt, Q), 256, 0, st>>>(V, n, c->kw32, cnt, Q == 1 ? dst : c->dpart, 513, 0);
        if (Q > 1) {
            GS_COUNT_LAUNCH(c);
            k_dots_reduce<<<(cnt + 255) / 256, 256, 0, st>>>(c->dpart, Q, 513, cnt, dst, 0);
        }
        GS_CHECK_LAUNCH(c);
        return GS_OK;
    };
    int it = 0;
    bool first = true;
    double est = 1.0;
    GS_CUDA(c, cudaMemsetAsync(x, 0, sizeof(cplx) * n, st));
    while (it < maxit) {
        if (first) {
            GS_CUDA(c, cudaMemcpyAsync(r, b, sizeof(cplx) * n, cudaMemcpyDeviceToDevice, st));
        } else {
            GS_TRY(gs_apply_impl(c, a, x, r, GS_C64));
            GS_COUNT_LAUNCH(c);
            k_sub<<<eb, 256, 0, st>>>(b, r, n, r);
        }
        first = false;
        GS_COUNT_LAUNCH(c);
        k_norm<<<1, 1024, 0, st>>>(r, n, ds + 1);
        GS_CUDA(c, cudaMemcpyAsync(c->hscal + 1, ds + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
        GS_CUDA(c, cudaStreamSynchronize(st));
        est = c->hscal[1] / bnorm;
        if (est <= tol) break;
        GS_COUNT_LAUNCH(c);
        k_store32<<<eb, 256, 0, st>>>(r, n, ds + 1, V, nullptr);
        GS_COUNT_LAUNCH(c);
        k_set_g0<<<(ld + 255) / 256, 256, 0, st>>>(c->gg, ld, ds + 1);
        GS_CUDA(c, cudaMemsetAsync(c->Hh, 0, sizeof(cplx) * (size_t)ld * c->kdim, st));
        int j = 0, kk = 0;
        for (; j < kd && it < maxit; ++j) {
            GS_COUNT_LAUNCH(c);
            k_load64<<<eb, 256, 0, st>>>(V + (size_t)j * n, n, vj);
            GS_TRY(gs_apply_impl(c, a, vj, w, GS_C64));
            ++it;
            cplx *h = c->Hh + (size_t)j * ld;
            // CGS2 on the complex64 basis: w32 = complex64 copy of w for the inner products; the
            // second pass also leaves the partial squared norms of the new vector
            GS_COUNT_LAUNCH(c);
            k_to_c64_vec<<<eb, 256, 0, st>>>(w, n, c->kw32);
            GS_TRY(dots(j + 1, h));
            GS_COUNT_LAUNCH(c);
            k_combo32<<<ebc, 256, 0, st>>>(w, V, n, h, j + 1, -1.f, c->kw32, nullptr);
            GS_TRY(dots(j + 1, c->yy));
            GS_COUNT_LAUNCH(c);
            k_combo32<<<ebc, 256, 0, st>>>(w, V, n, c->yy, j + 1, -1.f, nullptr, fused_norm ? c->npart : nullptr);
            GS_COUNT_LAUNCH(c);
            k_add_vec<<<1, 256, 0, st>>>(h, c->yy, j + 1);
            if (fused_norm) {
                GS_COUNT_LAUNCH(c);
                k_store32<<<eb, 256, 0, st>>>(w, n, nullptr, V + (size_t)(j + 1) * n, h + j + 1, c->npart, ebc);
            } else {
                GS_COUNT_LAUNCH(c);
                k_norm<<<1, 1024, 0, st>>>(w, n, ds + 3);
                GS_COUNT_LAUNCH(c);
                k_store32<<<eb, 256, 0, st>>>(w, n, ds + 3, V + (size_t)(j + 1) * n, h + j + 1);
            }
            GS_COUNT_LAUNCH(c);
            k_givens<<<1, GS_KMAX, 0, st>>>(c->Hh, ld, j, c->cs, c->sn, c->gg, ds + 2);
            GS_CHECK_LAUNCH(c);
            GS_CUDA(c, cudaMemcpyAsync(c->hscal + 2, ds + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
            GS_CUDA(c, cudaStreamSynchronize(st));
            est = c->hscal[2] / bnorm;
            kk = j + 1;
            if (est <= tol) break;
        }
        GS_COUNT_LAUNCH(c);
        k_backsolve<<<1, 256, 0, st>>>(c->Hh, ld, kk, c->gg, c->yy);
        GS_COUNT_LAUNCH(c);
        k_combo32<<<ebc, 256, 0, st>>>(x, V, n, c->yy, kk, 1.f, nullptr, nullptr);
        GS_CHECK_LAUNCH(c);
        if (est <= tol) {
            GS_TRY(gs_apply_impl(c, a, x, r, GS_C64));
            GS_COUNT_LAUNCH(c);
            k_sub<<<eb, 256, 0, st>>>(b, r, n, r);
            GS_COUNT_LAUNCH(c);
            k_norm<<<1, 1024, 0, st>>>(r, n, ds + 1);
            GS_CUDA(c, cudaMemcpyAsync(c->hscal + 1, ds + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
            GS_CUDA(c, cudaStreamSynchronize(st));
            est = c->hscal[1] / bnorm;
            if (est <= 10.0 * tol) break;
        }
    }
    *iters = it;
    *relres = est;
    return GS_OK;
}

}  // namespace

// FP64: GMRES on L.  GS_C64: iterative refinement with FP64 residuals and inner GMRES on the
// operator whose translation runs in complex64 (the correction equation L d = r is solved to
// inner_tol, x += d), until the FP64 relative residual meets tol.
int gs_ensure_krylov(gs_ctx *c, int restart);

int gs_solve_impl(gs_ctx *c, AngleData &a, const gs_solve_opts &o, const cplx *x0) {
    GS_TRY(gs_ensure_krylov(c, o.restart));
    const long n = c->n();
    cudaStream_t st = c->stream;
    const int eb = (int)((n + 255) / 256);
    cplx *b = c->v1;
    cplx *x = a.beta;
    GS_TRY(gs_rhs_impl(c, a, b));
    GS_COUNT_LAUNCH(c);
    k_norm<<<1, 1024, 0, st>>>(b, n, c->dscal);
    if (x0) GS_CUDA(c, cudaMemcpyAsync(x, x0, sizeof(cplx) * n, cudaMemcpyDeviceToDevice, st));
    GS_CUDA(c, cudaMemcpyAsync(c->hscal, c->dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
    GS_CUDA(c, cudaStreamSynchronize(st));
    const double bnorm = c->hscal[0];
    a.iters = 0;
    a.outer = 0;
    a.relres = 0.0;
    if (bnorm == 0.0) {
        GS_CUDA(c, cudaMemsetAsync(x, 0, sizeof(cplx) * n, st));
        return GS_OK;
    }
    if (o.precision == GS_FP64) {
        int its = 0;
        double rr = 1.0;
        GS_TRY(gmres_core(c, a, b, bnorm, x, x0 == nullptr, o.tol, o.maxit, o.restart, GS_FP64, &its, &rr));
        a.iters = its;
        a.relres = rr;
        return rr <= 10.0 * o.tol ? GS_OK : GS_ERR_NOT_CONVERGED;
    }
    // mixed precision refinement
    cplx *r = c->v4, *dx = c->v5;
    if (!x0) GS_CUDA(c, cudaMemsetAsync(x, 0, sizeof(cplx) * n, st));
    // inner tolerance: each correction only needs to bring the residual from rel down to tol, but
    // no tighter than inner_tol (the accuracy the complex64 operator can support)
    const double floor_tol = o.inner_tol > 0 ? o.inner_tol : 1e-6;
    double rel = 1.0;
    int total = 0;
    const int max_sweeps = o.max_sweeps > 0 ? o.max_sweeps : 30;
    for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
        if (sweep == 0 && !x0) {
            GS_CUDA(c, cudaMemcpyAsync(r, b, sizeof(cplx) * n, cudaMemcpyDeviceToDevice, st));
        } else {
            GS_TRY(gs_apply_impl(c, a, x, r, GS_FP64));
            GS_COUNT_LAUNCH(c);
            k_sub<<<eb, 256, 0, st>>>(b, r, n, r);
        }
        GS_COUNT_LAUNCH(c);
        k_norm<<<1, 1024, 0, st>>>(r, n, c->dscal + 5);
        GS_CUDA(c, cudaMemcpyAsync(c->hscal + 5, c->dscal + 5, sizeof(double), cudaMemcpyDeviceToHost, st));
        GS_CUDA(c, cudaStreamSynchronize(st));
        const double rnorm = c->hscal[5];
        rel = rnorm / bnorm;
        a.outer = sweep;
        if (rel <= o.tol || total >= o.maxit || sweep == max_sweeps) break;
        int its = 0;
        double rr = 1.0;
        const double itol = std::max(floor_tol, 0.5 * o.tol / rel);
        GS_TRY(gmres_core32(c, a, r, rnorm, dx, itol, o.maxit - total, o.restart, &its, &rr));
        total += its;
        GS_COUNT_LAUNCH(c);
        k_axpy_inplace<<<eb, 256, 0, st>>>(x, dx, n);
        GS_CHECK_LAUNCH(c);
    }
    a.iters = total;
    a.relres = rel;
    if (o.precision == GS_C64 && c->tab32.h) GS_TRY(gs_check_table_wait(c));
    return rel <= o.tol ? GS_OK : GS_ERR_NOT_CONVERGED;
}

// Bragg amplitudes: x_cd = D_cd .* V[cd rows] (coef .* W^* (f - C beta)); flux error on the device.
// a = A^+ (f - C beta): every layer unknown of the last solution (cols)
int gs_layer_unknowns_impl(gs_ctx *c, const AngleData &a, cplx *x) {
    const Layout &ly = c->lay;
    GS_COUNT_LAUNCH(c);
    k_f_minus_Cx<<<warps_blocks(ly.rows), 256, 0, c->stream>>>(a.Cm, ly.nC(), c->n(), a.beta, a.f, ly.rows, c->g);
    GS_CHECK_LAUNCH(c);
    return gs_pinv_impl(c, a, c->g, x);
}

int gs_bragg_impl(gs_ctx *c, const AngleData &a, cplx *cd_host, double *flux) {
    const Layout &ly = c->lay;
    int n = c->n();
    int ncd = 2 * (2 * ly.K + 1);
    GS_COUNT_LAUNCH(c);
    k_f_minus_Cx<<<warps_blocks(ly.rows), 256, 0, c->stream>>>(a.Cm, ly.nC(), n, a.beta, a.f, ly.rows, c->g);
    GS_COUNT_LAUNCH(c);
    k_gemv_colsH<<<warps_blocks(ly.cols), 256, 0, c->stream>>>(a.W, ly.rows, ly.rows, ly.cols, c->g, a.coef, c->w);
    GS_COUNT_LAUNCH(c);
    k_gemv_rows<<<warps_blocks(ncd), 256, 0, c->stream>>>(a.Vr + (size_t)ly.col_c * ly.cols, ncd, ly.cols, ly.cols,
                                                          c->w, a.dscale + ly.col_c, c->x);
    double w1, w3;
    gs_layer_weights(c, &w1, &w3);
    double inc = c->L.k1 * fabs(sin(a.theta)) / w1;
    GS_COUNT_LAUNCH(c);
    k_flux<<<1, 1, 0, c->stream>>>(ly.K, c->x, a.k1n, a.k3n, 1.0 / w1, 1.0 / w3, inc, c->dscal + 4);
    GS_CHECK_LAUNCH(c);
    GS_CUDA(c, cudaMemcpyAsync(cd_host, c->x, sizeof(cplx) * ncd, cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaMemcpyAsync(flux, c->dscal + 4, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}
