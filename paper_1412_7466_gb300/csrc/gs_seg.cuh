// Segmented restarted-GMRES kernels shared by the lockstep solvers (many geometries at one angle,
// gs_batch.cu; one geometry at many angles, gs_angles.cu).  A batch of G independent systems is
// stored as one concatenated vector: segment g has M targets of (2p+1) unknowns starting at element
// noff; gid maps each target of the concatenation to its segment.  Every kernel reads the Arnoldi
// step index j from device memory, so one Arnoldi step can be captured once as a CUDA graph and
// replayed; `active` masks segments that have converged.
#pragma once
#include <type_traits>

#include "gs_internal.h"

namespace {

struct Geo {
    int M, moff, noff;
};

// ---- segmented GMRES kernels (step index j read from device memory) --------------------------------
// Templated on the basis type: complex128 (FP64 solves) or complex64 (the inner solves of the mixed
// form: FP32 products, FP64 block sums -- the FP64 products are bound by GB300's FP64 pipe).

__device__ __forceinline__ cplx bget(const cplx *V, size_t i) { return V[i]; }
__device__ __forceinline__ cplx bget(const float2 *V, size_t i) { const float2 v = V[i]; return C(v.x, v.y); }
__device__ __forceinline__ void bput(cplx *V, size_t i, cplx v) { V[i] = v; }
__device__ __forceinline__ void bput(float2 *V, size_t i, cplx v) { V[i] = make_float2((float)v.x, (float)v.y); }

// re/im of sum_e conj(V[e]) w[e] over a thread's elements (FP64 basis: FP64; complex64: FP32)
template <typename TB>
__device__ __forceinline__ void seg_dot_part(const TB *v, const cplx *ww, size_t n, double &re, double &im) {
    if constexpr (std::is_same<TB, cplx>::value) {
        for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
            const cplx a = v[e], b = ww[e];
            re += a.x * b.x + a.y * b.y;
            im += a.x * b.y - a.y * b.x;
        }
    } else {
        float fr = 0.f, fi = 0.f;
        for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
            const float2 a = v[e];
            const cplx b = ww[e];
            const float br = (float)b.x, bi = (float)b.y;
            fr = fmaf(a.x, br, fmaf(a.y, bi, fr));
            fi = fmaf(a.x, bi, fmaf(-a.y, br, fi));
        }
        re = fr;
        im = fi;
    }
}

// X = V_j
template <typename TB>
__global__ void k_seg_fetch(const TB *__restrict__ Vb, long Ntot, const int *jdev, cplx *__restrict__ X) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < Ntot) X[e] = bget(Vb, (size_t)(*jdev) * Ntot + e);
}

// h[g][i] (+)= V_i[g]^* w[g], i <= j, blocks (i, g); written into column j of H_g (ld = kdim+1)
template <typename TB>
__global__ void k_seg_dots(const TB *__restrict__ Vb, long Ntot, const cplx *__restrict__ w, const Geo *__restrict__ geo,
                           int nc, const int *jdev, const int *__restrict__ active, cplx *__restrict__ H, int ld,
                           int kdim, int second) {
    const int i = blockIdx.x, g = blockIdx.y, j = *jdev;
    if (i > j || (active && !active[g])) return;
    __shared__ double sh[32];
    const size_t off = (size_t)geo[g].noff, n = (size_t)geo[g].M * nc;
    double re = 0, im = 0;
    seg_dot_part(Vb + (size_t)i * Ntot + off, w + off, n, re, im);
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) {
        cplx *h = H + ((size_t)g * kdim + j) * ld + i;
        *h = second ? cadd(*h, C(re, im)) : C(re, im);
    }
}

// per-geometry copy of the CGS coefficients of the current pass: hp[g][i] = value just written
// (the second pass accumulates into H and subtracts only its own contribution, so the pass-2
// coefficients are staged separately)
template <typename TB>
__global__ void k_seg_dots2(const TB *__restrict__ Vb, long Ntot, const cplx *__restrict__ w, const Geo *__restrict__ geo,
                            int nc, const int *jdev, const int *__restrict__ active, cplx *__restrict__ hp, int ldh) {
    const int i = blockIdx.x, g = blockIdx.y, j = *jdev;
    if (i > j || (active && !active[g])) return;
    __shared__ double sh[32];
    const size_t off = (size_t)geo[g].noff, n = (size_t)geo[g].M * nc;
    double re = 0, im = 0;
    seg_dot_part(Vb + (size_t)i * Ntot + off, w + off, n, re, im);
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) hp[(size_t)g * ldh + i] = C(re, im);
}

// w[e] -= sum_{i <= j} coef_g[i] V_i[e], coef_g = column j of H_g (pass 1) or hp[g] (pass 2)
template <typename TB>
__global__ void k_seg_sub(cplx *__restrict__ w, const TB *__restrict__ Vb, long Ntot, const int *__restrict__ gid,
                          int nc, const int *jdev, const int *__restrict__ active, const cplx *__restrict__ H, int ld,
                          int kdim, const cplx *__restrict__ hp, int ldh) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Ntot) return;
    const int g = gid[e / nc], j = *jdev;
    if (active && !active[g]) return;
    const cplx *coef = hp ? hp + (size_t)g * ldh : H + ((size_t)g * kdim + j) * ld;
    if constexpr (std::is_same<TB, cplx>::value) {
        cplx s = w[e];
        for (int i = 0; i <= j; ++i) s = csub(s, cmul(coef[i], Vb[(size_t)i * Ntot + e]));
        w[e] = s;
    } else {
        float sr = 0.f, si = 0.f;
        for (int i = 0; i <= j; ++i) {
            const float2 v = Vb[(size_t)i * Ntot + e];
            const cplx cf = coef[i];
            const float cr = (float)cf.x, ci = (float)cf.y;
            sr = fmaf(cr, v.x, fmaf(-ci, v.y, sr));
            si = fmaf(cr, v.y, fmaf(ci, v.x, si));
        }
        w[e] = csub(w[e], C((double)sr, (double)si));
    }
}

// H_g[:, j] += hp[g]
__global__ void k_seg_addh(cplx *H, int ld, int kdim, const cplx *hp, int ldh, const int *jdev, const int *active, int G) {
    const int g = blockIdx.x, j = *jdev;
    if (g >= G || (active && !active[g])) return;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        cplx *h = H + ((size_t)g * kdim + j) * ld + i;
        *h = cadd(*h, hp[(size_t)g * ldh + i]);
    }
}

// nrm[g] = ||w_g||; with H given, also H_g[j+1, j] = nrm[g]
__global__ void k_seg_norm(const cplx *__restrict__ w, const Geo *__restrict__ geo, int nc, const int *__restrict__ active,
                           double *__restrict__ nrm, cplx *H, int ld, int kdim, const int *jdev) {
    const int g = blockIdx.x;
    if (active && !active[g]) return;
    __shared__ double sh[32];
    const size_t off = (size_t)geo[g].noff, n = (size_t)geo[g].M * nc;
    double s = 0;
    for (size_t e = threadIdx.x; e < n; e += blockDim.x) s += cabs2(w[off + e]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        nrm[g] = sqrt(s);
        if (H) {
            const int j = *jdev;
            H[((size_t)g * kdim + j) * ld + j + 1] = C(sqrt(s), 0.0);
        }
    }
}

// V_{j+1}[e] = w[e] / nrm[g]
template <typename TB>
__global__ void k_seg_scale(const cplx *__restrict__ w, TB *__restrict__ Vb, long Ntot, const int *__restrict__ gid,
                            int nc, const int *jdev, const int *__restrict__ active, const double *__restrict__ nrm) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Ntot) return;
    const int g = gid[e / nc], j = *jdev;
    if (active && !active[g]) return;
    const double nv = nrm[g];
    bput(Vb, (size_t)(j + 1) * Ntot + e, nv > 0.0 ? cscale(w[e], 1.0 / nv) : C(0, 0));
}

// Givens step of column j of H_g for every active geometry (block per geometry); res[g] = |g_g[j+1]|
__global__ void k_seg_givens(cplx *H, int ld, int kdim, const int *jdev, const int *active, cplx *cs, cplx *sn,
                             cplx *gg, double *res, int G) {
    const int g = blockIdx.x, j = *jdev;
    if (g >= G || (active && !active[g])) return;
    __shared__ cplx h[512 + 1];
    cplx *col = H + ((size_t)g * kdim + j) * ld;
    cplx *c_ = cs + (size_t)g * ld, *s_ = sn + (size_t)g * ld, *gv = gg + (size_t)g * ld;
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) h[i] = col[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < j; ++i) {
            cplx t = cadd(cmul(c_[i], h[i]), cmul(s_[i], h[i + 1]));
            h[i + 1] = cadd(cmul(cscale(cconj(s_[i]), -1.0), h[i]), cmul(c_[i], h[i + 1]));
            h[i] = t;
        }
        cplx a = h[j], b = h[j + 1];
        double aa = sqrt(cabs2(a)), bb = sqrt(cabs2(b)), rr = hypot(aa, bb);
        cplx c, s;
        if (rr == 0.0) {
            c = C(1, 0);
            s = C(0, 0);
        } else if (aa == 0.0) {
            c = C(0, 0);
            s = cscale(cconj(b), 1.0 / bb);
        } else {
            c = C(aa / rr, 0.0);
            s = cmul(cscale(a, 1.0 / aa), cscale(cconj(b), 1.0 / rr));
        }
        c_[j] = c;
        s_[j] = s;
        h[j] = cadd(cmul(c, a), cmul(s, b));
        h[j + 1] = C(0, 0);
        cplx gj = gv[j];
        gv[j + 1] = cmul(cscale(cconj(s), -1.0), gj);
        gv[j] = cmul(c, gj);
        res[g] = sqrt(cabs2(gv[j + 1]));
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) col[i] = h[i];
}

__global__ void k_inc(int *jdev) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *jdev += 1;
}

// per geometry: y_g = H_g[0:kk,0:kk]^{-1} g_g[0:kk] (block per geometry, column-oriented)
__global__ void k_seg_backsolve(const cplx *H, int ld, int kdim, const int *kk, const cplx *gg, cplx *yy, int G) {
    const int g = blockIdx.x;
    if (g >= G) return;
    const int n = kk[g];
    __shared__ cplx r[512];
    __shared__ cplx yi;
    const cplx *Hg = H + (size_t)g * kdim * ld;
    for (int i = threadIdx.x; i < n; i += blockDim.x) r[i] = gg[(size_t)g * ld + i];
    __syncthreads();
    for (int i = n - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            yi = cdiv(r[i], Hg[(size_t)i * ld + i]);
            yy[(size_t)g * ld + i] = yi;
        }
        __syncthreads();
        const cplx v = yi;
        for (int q = threadIdx.x; q < i; q += blockDim.x) r[q] = csub(r[q], cmul(Hg[(size_t)i * ld + q], v));
        __syncthreads();
    }
}

// x[e] += sum_{i < kk[g]} yy[g][i] V_i[e]
template <typename TB>
__global__ void k_seg_update(cplx *__restrict__ x, const TB *__restrict__ Vb, long Ntot, const int *__restrict__ gid,
                             int nc, const int *__restrict__ kk, const cplx *__restrict__ yy, int ld) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Ntot) return;
    const int g = gid[e / nc];
    cplx s = x[e];
    for (int i = 0; i < kk[g]; ++i) s = cadd(s, cmul(yy[(size_t)g * ld + i], bget(Vb, (size_t)i * Ntot + e)));
    x[e] = s;
}

// V_0 = r / nrm[g]; gg[g] = (nrm[g], 0, ...)
template <typename TB>
__global__ void k_seg_start(const cplx *__restrict__ r, TB *__restrict__ V0, long Ntot, const int *__restrict__ gid,
                            int nc, const double *__restrict__ nrm, const int *__restrict__ active) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Ntot) return;
    const int g = gid[e / nc];
    const double nv = nrm[g];
    bput(V0, (size_t)e, (active[g] && nv > 0.0) ? cscale(r[e], 1.0 / nv) : C(0, 0));
}

__global__ void k_seg_g0(cplx *gg, int ld, const double *nrm, int G) {
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= G * ld) return;
    int g = id / ld, i = id % ld;
    gg[id] = C(i == 0 ? nrm[g] : 0.0, 0.0);
}

__global__ void k_vsub(const cplx *a, const cplx *b, long n, cplx *y) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) y[e] = csub(a[e], b[e]);
}
__global__ void k_vadd(cplx *x, const cplx *y, long n) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) x[e] = cadd(x[e], y[e]);
}

}  // namespace
