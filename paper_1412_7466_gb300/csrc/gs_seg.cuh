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

// re/im of sum_e conj(V[e]) w[e] over a thread's elements (FP64 basis: FP64 with w; complex64
// basis: FP32 with w32, the complex64 copy of w, so that no FP64 -> FP32 conversion runs per entry)
template <typename TB>
__device__ __forceinline__ void seg_dot_part(const TB *v, const cplx *ww, const float2 *ww32, size_t n, double &re,
                                             double &im) {
    if constexpr (std::is_same<TB, cplx>::value) {
        for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
            const cplx a = v[e], b = ww[e];
            re += a.x * b.x + a.y * b.y;
            im += a.x * b.y - a.y * b.x;
        }
    } else {
        float fr = 0.f, fi = 0.f, fr1 = 0.f, fi1 = 0.f;
        size_t e = threadIdx.x;
        for (; e + blockDim.x < n; e += 2 * blockDim.x) {
            const float2 a = v[e], b = ww32[e], a1 = v[e + blockDim.x], b1 = ww32[e + blockDim.x];
            fr = fmaf(a.x, b.x, fmaf(a.y, b.y, fr));
            fi = fmaf(a.x, b.y, fmaf(-a.y, b.x, fi));
            fr1 = fmaf(a1.x, b1.x, fmaf(a1.y, b1.y, fr1));
            fi1 = fmaf(a1.x, b1.y, fmaf(-a1.y, b1.x, fi1));
        }
        if (e < n) {
            const float2 a = v[e], b = ww32[e];
            fr = fmaf(a.x, b.x, fmaf(a.y, b.y, fr));
            fi = fmaf(a.x, b.y, fmaf(-a.y, b.x, fi));
        }
        re = (double)fr + (double)fr1;
        im = (double)fi + (double)fi1;
    }
}

// complex64 copy of w
__global__ void k_seg_to32(const cplx *__restrict__ w, long n, float2 *__restrict__ w32) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) w32[e] = make_float2((float)w[e].x, (float)w[e].y);
}

// X = V_j
template <typename TB>
__global__ void k_seg_fetch(const TB *__restrict__ Vb, long Ntot, const int *jdev, cplx *__restrict__ X) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < Ntot) X[e] = bget(Vb, (size_t)(*jdev) * Ntot + e);
}

// h[g][i] (+)= V_i[g]^* w[g], i <= j, blocks (i, g); written into column j of H_g (ld = kdim+1)
template <typename TB>
__global__ void k_seg_dots(const TB *__restrict__ Vb, long Ntot, const cplx *__restrict__ w, const float2 *__restrict__ w32,
                           const Geo *__restrict__ geo, int nc, const int *jdev, const int *__restrict__ active,
                           cplx *__restrict__ H, int ld, int kdim, int second) {
    const int i = blockIdx.x, g = blockIdx.y, j = *jdev;
    if (i > j || (active && !active[g])) return;
    __shared__ double sh[32];
    const size_t off = (size_t)geo[g].noff, n = (size_t)geo[g].M * nc;
    double re = 0, im = 0;
    seg_dot_part(Vb + (size_t)i * Ntot + off, w + off, w32 ? w32 + off : nullptr, n, re, im);
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
__global__ void k_seg_dots2(const TB *__restrict__ Vb, long Ntot, const cplx *__restrict__ w, const float2 *__restrict__ w32,
                            const Geo *__restrict__ geo, int nc, const int *jdev, const int *__restrict__ active,
                            cplx *__restrict__ hp, int ldh) {
    const int i = blockIdx.x, g = blockIdx.y, j = *jdev;
    if (i > j || (active && !active[g])) return;
    __shared__ double sh[32];
    const size_t off = (size_t)geo[g].noff, n = (size_t)geo[g].M * nc;
    double re = 0, im = 0;
    seg_dot_part(Vb + (size_t)i * Ntot + off, w + off, w32 ? w32 + off : nullptr, n, re, im);
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) hp[(size_t)g * ldh + i] = C(re, im);
}

// cf32[g][i] = coef_g[i] in complex64, i <= j: column j of H_g (hp null) or hp[g] (block per segment)
__global__ void k_seg_coef32(const cplx *__restrict__ H, int ld, int kdim, const cplx *__restrict__ hp, int ldh,
                             const int *jdev, const int *__restrict__ active, int G, float2 *__restrict__ cf32) {
    const int g = blockIdx.x, j = *jdev;
    if (g >= G || (active && !active[g])) return;
    const cplx *coef = hp ? hp + (size_t)g * ldh : H + ((size_t)g * kdim + j) * ld;
    for (int i = threadIdx.x; i <= j; i += blockDim.x)
        cf32[(size_t)g * ld + i] = make_float2((float)coef[i].x, (float)coef[i].y);
}

// w[e] -= sum_{i <= j} coef_g[i] V_i[e], coef_g = column j of H_g (pass 1) or hp[g] (pass 2).  The
// complex64 basis takes the coefficients from cf32 (k_seg_coef32; stride ld per segment), eight basis
// vectors per pass so eight loads are in flight, and writes the complex64 copy w32 of the result
// when given.
template <typename TB>
__global__ void k_seg_sub(cplx *__restrict__ w, const TB *__restrict__ Vb, long Ntot, const int *__restrict__ gid,
                          int nc, const int *jdev, const int *__restrict__ active, const cplx *__restrict__ H, int ld,
                          int kdim, const cplx *__restrict__ hp, int ldh, const float2 *__restrict__ cf32,
                          float2 *__restrict__ w32) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Ntot) return;
    const int g = gid[e / nc], j = *jdev;
    if (active && !active[g]) return;
    if constexpr (std::is_same<TB, cplx>::value) {
        const cplx *coef = hp ? hp + (size_t)g * ldh : H + ((size_t)g * kdim + j) * ld;
        cplx s = w[e];
        for (int i = 0; i <= j; ++i) s = csub(s, cmul(coef[i], Vb[(size_t)i * Ntot + e]));
        w[e] = s;
    } else {
        const float2 *cf = cf32 + (size_t)g * ld;
        float sr[8], si[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) sr[u] = si[u] = 0.f;
        int i = 0;
        for (; i + 8 <= j + 1; i += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float2 v = Vb[(size_t)(i + u) * Ntot + e], c = cf[i + u];
                sr[u] = fmaf(c.x, v.x, fmaf(-c.y, v.y, sr[u]));
                si[u] = fmaf(c.x, v.y, fmaf(c.y, v.x, si[u]));
            }
        }
        for (; i <= j; ++i) {
            const float2 v = Vb[(size_t)i * Ntot + e], c = cf[i];
            sr[0] = fmaf(c.x, v.x, fmaf(-c.y, v.y, sr[0]));
            si[0] = fmaf(c.x, v.y, fmaf(c.y, v.x, si[0]));
        }
        float tr = 0.f, ti = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            tr += sr[u];
            ti += si[u];
        }
        const cplx r = csub(w[e], C((double)tr, (double)ti));
        w[e] = r;
        if (w32) w32[e] = make_float2((float)r.x, (float)r.y);
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

// nrm[g] = ||w_g||; with H given, also H_g[j+1, j] = nrm[g] (block per segment; used outside the
// Arnoldi step)
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

// the same in two steps with SEG_NQ blocks per segment: partial sums, then their sum in a fixed order
constexpr int SEG_NQ = 16;
__global__ void k_seg_norm_part(const cplx *__restrict__ w, const Geo *__restrict__ geo, int nc,
                                const int *__restrict__ active, double *__restrict__ npart) {
    const int q = blockIdx.x, g = blockIdx.y;
    if (active && !active[g]) return;
    __shared__ double sh[32];
    const size_t off = (size_t)geo[g].noff, n = (size_t)geo[g].M * nc;
    const size_t e0 = n * q / SEG_NQ, e1 = n * (q + 1) / SEG_NQ;
    double s = 0;
    for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) s += cabs2(w[off + e]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) npart[(size_t)g * SEG_NQ + q] = s;
}
__global__ void k_seg_norm_fin(const double *__restrict__ npart, const int *__restrict__ active, int G,
                               double *__restrict__ nrm, cplx *H, int ld, int kdim, const int *jdev) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G || (active && !active[g])) return;
    double s = 0;
    for (int q = 0; q < SEG_NQ; ++q) s += npart[(size_t)g * SEG_NQ + q];
    nrm[g] = sqrt(s);
    if (H) H[((size_t)g * kdim + *jdev) * ld + *jdev + 1] = C(sqrt(s), 0.0);
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

// Givens step of column j of H_g for every active geometry (block of SEG_GIVENS_THREADS per
// geometry, j < SEG_GIVENS_THREADS); res[g] = |g_g[j+1]|.  The previous rotations act on the column
// as a linear recurrence in the value carried down it (carry_{i+1} = -conj(s_i) carry_i + c_i h_{i+1},
// h'_i = c_i carry_i + s_i h_{i+1}, carry_0 = h_0): the block forms all prefix compositions of these
// affine maps by an inclusive scan instead of applying the j rotations one after another.
constexpr int SEG_GIVENS_THREADS = 512;
__global__ void __launch_bounds__(SEG_GIVENS_THREADS) k_seg_givens(cplx *H, int ld, int kdim, const int *jdev,
                                                                   const int *active, cplx *cs, cplx *sn, cplx *gg,
                                                                   double *res, int G) {
    const int g = blockIdx.x, j = *jdev, t = threadIdx.x;
    if (g >= G || (active && !active[g])) return;
    __shared__ cplx mA[SEG_GIVENS_THREADS], mB[SEG_GIVENS_THREADS];
    cplx *col = H + ((size_t)g * kdim + j) * ld;
    cplx *c_ = cs + (size_t)g * ld, *s_ = sn + (size_t)g * ld, *gv = gg + (size_t)g * ld;
    const cplx h0 = col[0], hj1 = col[j + 1];
    cplx ct = C(1, 0), st = C(0, 0), hn = C(0, 0), a = C(1, 0), b = C(0, 0);
    if (t < j) {
        ct = c_[t];
        st = s_[t];
        hn = col[t + 1];
        a = cscale(cconj(st), -1.0);
        b = cmul(ct, hn);
    }
    mA[t] = a;
    mB[t] = b;
    __syncthreads();
    for (int off = 1; off < SEG_GIVENS_THREADS; off <<= 1) {
        cplx pa = C(1, 0), pb = C(0, 0);
        if (t >= off) {
            pa = mA[t - off];
            pb = mB[t - off];
        }
        __syncthreads();
        if (t >= off) {
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
        const double aa = sqrt(cabs2(av)), bb = sqrt(cabs2(bv)), rr = hypot(aa, bb);
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
        c_[j] = c;
        s_[j] = s;
        col[j] = cadd(cmul(c, av), cmul(s, bv));
        col[j + 1] = C(0, 0);
        const cplx gj = gv[j];
        gv[j + 1] = cmul(cscale(cconj(s), -1.0), gj);
        gv[j] = cmul(c, gj);
        res[g] = sqrt(cabs2(gv[j + 1]));
    }
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

// Scratch and state of one segmented Arnoldi step (device pointers; w32: Ntot complex64, cf32:
// G x ld complex64, npart: G x SEG_NQ)
struct SegStep {
    const Geo *geo;
    const int *gid, *active, *jdev;
    cplx *H, *hp, *cs, *sn, *gg;
    double *nrm, *res, *npart;
    float2 *w32, *cf32;
    long N;
    int G, kdim, nc;
};

// Y <- the next orthonormal basis vector of every active segment from the operator output Y: CGS2
// against V_0..V_j, H_g[:, j], V_{j+1}, the Givens update; j read from s.jdev (graph-capturable)
template <typename TB>
int seg_cgs2(gs_ctx *c, const SegStep &s, TB *V, cplx *Y, cudaStream_t st) {
    const int ld = s.kdim + 1;
    const int eb = (int)((s.N + 255) / 256);
    const bool f32 = std::is_same<TB, float2>::value;
    const dim3 gd(s.kdim, s.G);
    if (f32) {
        GS_COUNT_LAUNCH(c);
        k_seg_to32<<<eb, 256, 0, st>>>(Y, s.N, s.w32);
    }
    GS_COUNT_LAUNCH(c);
    k_seg_dots<TB><<<gd, 256, 0, st>>>(V, s.N, Y, f32 ? s.w32 : nullptr, s.geo, s.nc, s.jdev, s.active, s.H, ld,
                                        s.kdim, 0);
    if (f32) {
        GS_COUNT_LAUNCH(c);
        k_seg_coef32<<<s.G, 256, 0, st>>>(s.H, ld, s.kdim, nullptr, ld, s.jdev, s.active, s.G, s.cf32);
    }
    GS_COUNT_LAUNCH(c);
    k_seg_sub<TB><<<eb, 256, 0, st>>>(Y, V, s.N, s.gid, s.nc, s.jdev, s.active, s.H, ld, s.kdim, nullptr, 0, s.cf32,
                                       f32 ? s.w32 : nullptr);
    GS_COUNT_LAUNCH(c);
    k_seg_dots2<TB><<<gd, 256, 0, st>>>(V, s.N, Y, f32 ? s.w32 : nullptr, s.geo, s.nc, s.jdev, s.active, s.hp, ld);
    if (f32) {
        GS_COUNT_LAUNCH(c);
        k_seg_coef32<<<s.G, 256, 0, st>>>(s.H, ld, s.kdim, s.hp, ld, s.jdev, s.active, s.G, s.cf32);
    }
    GS_COUNT_LAUNCH(c);
    k_seg_sub<TB><<<eb, 256, 0, st>>>(Y, V, s.N, s.gid, s.nc, s.jdev, s.active, s.H, ld, s.kdim, s.hp, ld, s.cf32,
                                       nullptr);
    GS_COUNT_LAUNCH(c);
    k_seg_addh<<<s.G, 256, 0, st>>>(s.H, ld, s.kdim, s.hp, ld, s.jdev, s.active, s.G);
    GS_COUNT_LAUNCH(c);
    k_seg_norm_part<<<dim3(SEG_NQ, s.G), 256, 0, st>>>(Y, s.geo, s.nc, s.active, s.npart);
    GS_COUNT_LAUNCH(c);
    k_seg_norm_fin<<<(s.G + 127) / 128, 128, 0, st>>>(s.npart, s.active, s.G, s.nrm, s.H, ld, s.kdim, s.jdev);
    GS_COUNT_LAUNCH(c);
    k_seg_scale<TB><<<eb, 256, 0, st>>>(Y, V, s.N, s.gid, s.nc, s.jdev, s.active, s.nrm);
    GS_COUNT_LAUNCH(c);
    k_seg_givens<<<s.G, SEG_GIVENS_THREADS, 0, st>>>(s.H, ld, s.kdim, s.jdev, s.active, s.cs, s.sn, s.gg, s.res, s.G);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

}  // namespace
