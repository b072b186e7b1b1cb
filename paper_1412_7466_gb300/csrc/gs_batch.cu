// Batched solves: many inclusion geometries of uneven size on one factored grating, solved in
// lockstep by GMRES (FP64) or by the mixed refinement (complex64 inner solves, FP64 residuals).
//
//  * Translation: one persistent launch for the whole batch.  The (geometry, group of 4 targets,
//    chunk of source images) work items are taken from an atomic counter by a fixed grid of
//    SMs x blocks-per-SM blocks, largest geometries first; each item writes its partial sums to its
//    own slot, and a second kernel adds each target's slots in a fixed order (deterministic).
//    The chunk length and the blocks per SM are picked by timing candidates on first use (autotuner).
//  * Low rank: the grating factorisation (U, V Sigma, D, coef) is shared by all geometries, so the
//    four products become grouped kernels over a geometry table (C_g x_g for all g, U^* g for all g,
//    V w for all g, B_g v_g + preconditioner + combination for all rows).
//  * GMRES: all geometries advance one Arnoldi step together; the step (operator, CGS2, norm,
//    Givens) reads the step index from device memory, so it is captured once as a CUDA graph and
//    replayed; the host reads one residual estimate per geometry per step.  Converged geometries are
//    masked out of the translation and the low-rank products.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "gs_internal.h"
#include "gs_seg.cuh"
#include "gs_pair.cuh"

namespace {

constexpr int BW = 4;          // targets (warps) per block in the batched translation
constexpr int TILE = 32;       // source images per shared-memory tile

struct Item {
    int g, i0, s0, s1;         // geometry, first target of the group, source-image range
};

inline int nblk(long n, int t = 256) { return (int)((n + t - 1) / t); }
inline int wblk(long nwarps) { return (int)((nwarps * 32 + 255) / 256); }

template <typename T>
int dalloc_b(gs_ctx *c, T **p, size_t n) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * n);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return gs_fail(c, GS_ERR_OOM, std::string("cudaMalloc (batch): ") + cudaGetErrorString(e));
    }
    return GS_OK;
}
template <typename T>
void dfree_b(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// ---- batched translation ------------------------------------------------------------------------

__global__ void k_b_to_c64(const cplx *__restrict__ b, long n, float2 *__restrict__ b32) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b32[e] = make_float2((float)b[e].x, (float)b[e].y);
}

template <int P, bool C64>
__global__ void __launch_bounds__(BW * 32, (C64 && P <= 12) ? 3 : 1)
k_batch_translate(const Item *__restrict__ items, int n_items, int *counter, const Geo *__restrict__ geo,
                  const int *__restrict__ active, const double *__restrict__ xy, const float4 *__restrict__ img,
                  const cplx *__restrict__ beta, const float2 *__restrict__ beta32, double k, double d, cplx alpha,
                  cplx *__restrict__ part) {
    constexpr int NC = 2 * P + 1;
    typedef typename std::conditional<C64, cplxf_t, cplx>::type T;
    __shared__ T sb[NC][TILE + 1];   // +1: the [n][u] stores of the staging loop spread over the banks
    __shared__ double sx[TILE], sy[TILE];
    __shared__ float4 sg[TILE];
    __shared__ int sid[TILE];
    __shared__ int cur;
    __shared__ float2 sphf[3];   // complex64 image phases alpha^l, l = -1, 0, 1 (once per launch)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const cplx ainv = cconj(alpha);
    const float kf = (float)k;
    if (threadIdx.x == 0) {
        sphf[0] = make_float2((float)alpha.x, (float)-alpha.y);
        sphf[1] = make_float2(1.f, 0.f);
        sphf[2] = make_float2((float)alpha.x, (float)alpha.y);
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
        __syncthreads();
        const int it = cur;
        if (it >= n_items) break;
        const Item w = items[it];
        const Geo G = geo[w.g];
        cplx *slot = part + ((size_t)it * BW + warp) * NC;
        if (active && !active[w.g]) {
            if (lane < NC) slot[lane] = C(0.0, 0.0);
            if (lane + 32 < NC) slot[lane + 32] = C(0.0, 0.0);
            continue;
        }
        const int i = w.i0 + warp;
        const double *gxy = xy + 2 * (size_t)G.moff;
        const float4 *gimg = img + 3 * (size_t)G.moff;    // (hi, lo) float image coordinates (C64)
        double xi = 0.0, yi = 0.0;
        float4 gi = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < G.M) {
            if constexpr (C64) {
                gi = gimg[G.M + i];
            } else {
                xi = gxy[2 * i];
                yi = gxy[2 * i + 1];
            }
        }
        T acc[NC], Qa[NC];   // complex64: acc and Qa are the packed accumulators of gs_pair_c64x2
#pragma unroll
        for (int m = 0; m < NC; ++m) acc[m] = Qa[m] = T{0, 0};
        for (int t0 = w.s0; t0 < w.s1; t0 += TILE) {
            __syncthreads();
            for (int e = threadIdx.x; e < TILE * NC; e += BW * 32) {
                int u = e / NC, n = e - u * NC;
                int s = t0 + u;
                T v{0, 0};
                if (s < w.s1) {
                    const int l = (s >= G.M) + (s >= 2 * G.M) - 1;   // source image s = (l+1) M + j
                    const int j = s - (l + 1) * G.M;
                    if constexpr (C64) {
                        v = gs_cmulf(sphf[l + 1], beta32[(size_t)G.noff + (size_t)j * NC + n]);
                    } else {
                        const cplx ph = (l == 0) ? C(1.0, 0.0) : (l == 1 ? alpha : ainv);
                        v = cmul(ph, beta[(size_t)G.noff + (size_t)j * NC + n]);
                    }
                }
                sb[n][u] = v;
            }
            for (int u = threadIdx.x; u < TILE; u += BW * 32) {
                int s = t0 + u;
                if (s < w.s1) {
                    const int l = (s >= G.M) + (s >= 2 * G.M) - 1;
                    const int j = s - (l + 1) * G.M;
                    if constexpr (C64) {
                        sg[u] = gimg[s];
                    } else {
                        sx[u] = gxy[2 * j] + l * d;
                        sy[u] = gxy[2 * j + 1];
                    }
                    sid[u] = (l == 0) ? j : -1;
                } else {
                    sid[u] = -2;
                    sx[u] = sy[u] = 0.0;
                    sg[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            __syncthreads();
            if (i >= G.M) continue;
            const int s = t0 + lane;
            if (s >= w.s1 || sid[lane] == i) continue;
            T b[NC];
#pragma unroll
            for (int n = 0; n < NC; ++n) b[n] = sb[n][lane];
            if constexpr (C64) {
                const float4 gs = sg[lane];
                gs_pair_c64x2<P>((gi.x - gs.x) + (gi.y - gs.y), (gi.z - gs.z) + (gi.w - gs.w), kf, b, acc, Qa);
            } else {
                gs_pair_f64<P>(xi - sx[lane], yi - sy[lane], k, b, acc);
            }
        }
        if constexpr (C64) {
            __shared__ float red[BW][2 * NC * 33];
            T sum[NC];
            gs_pq_combine<NC>(acc, Qa, sum);
            gs_warp_sum_c64<NC>(sum, red[warp], lane, (double *)slot, true);
        } else {
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                acc[m].x = warp_sum(acc[m].x);
                acc[m].y = warp_sum(acc[m].y);
            }
#pragma unroll
            for (int m = 0; m < NC; ++m)
                if (lane == (m & 31)) slot[m] = acc[m];
        }
    }
}

// out[row] = sum of the target's item slots; row = (target, order), target t has chunks
// tchunks[t] starting at item tbase[t], warp tw[t] within the item
__global__ void k_batch_reduce(const cplx *__restrict__ part, long Ntot, int nc, const int *__restrict__ tbase,
                               const int *__restrict__ tchunks, const int *__restrict__ tw, cplx *__restrict__ out) {
    long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Ntot) return;
    int t = (int)(r / nc), m = (int)(r % nc);
    cplx s = C(0.0, 0.0);
    const int b = tbase[t], nch = tchunks[t], w = tw[t];
    for (int q = 0; q < nch; ++q) s = cadd(s, part[((size_t)(b + q) * BW + w) * nc + m]);
    out[r] = s;
}

// ---- grouped low-rank products --------------------------------------------------------------------

// gC[g][r] = sum_c C_g[r, c] x_g[c]
__global__ void k_batch_C(const cplx *__restrict__ Call, const size_t *__restrict__ coff, const Geo *__restrict__ geo,
                          int G, int nC, int nc, const int *__restrict__ active, const cplx *__restrict__ x,
                          cplx *__restrict__ gC) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= G * nC) return;
    int g = warp / nC, r = warp % nC;
    if (active && !active[g]) return;
    const int n = geo[g].M * nc;
    const cplx *a = Call + coff[g] + (size_t)r * n;
    const cplx *xv = x + geo[g].noff;
    cplx s = C(0, 0);
    for (int c = lane; c < n; c += 32) cfma(s, a[c], __ldg(&xv[c]));
    s.x = warp_sum(s.x);
    s.y = warp_sum(s.y);
    if (lane == 0) gC[(size_t)g * nC + r] = s;
}

// w[g][j] = coef[j] sum_{i < nr} conj(U[i, j]) gv[g][i]  (U column-major m x cols; gv leading dim ldg)
__global__ void k_batch_UH(const cplx *__restrict__ U, int m, int nr, int cols, const cplx *__restrict__ gv, int ldg,
                           const double *__restrict__ coef, int G, const int *__restrict__ active, cplx *__restrict__ w) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= G * cols) return;
    int j = warp / G, g = warp % G;   // g fastest: neighbouring warps read the same column of U
    if (active && !active[g]) return;
    const cplx *a = U + (size_t)j * m;
    const cplx *v = gv + (size_t)g * ldg;
    cplx s = C(0, 0);
    for (int i = lane; i < nr; i += 32) cfma(s, cconj(a[i]), __ldg(&v[i]));
    s.x = warp_sum(s.x);
    s.y = warp_sum(s.y);
    if (lane == 0) w[(size_t)g * cols + j] = cscale(s, coef[j]);
}

// xo[g][i] = dscale[i] sum_j Vr[i, j] w[g][j] for i < nrow
__global__ void k_batch_V(const cplx *__restrict__ Vr, int nrow, int cols, const cplx *__restrict__ w,
                          const double *__restrict__ dscale, int G, const int *__restrict__ active, cplx *__restrict__ xo,
                          float2 *__restrict__ xo32 = nullptr) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= G * nrow) return;
    int i = warp / G, g = warp % G;
    if (active && !active[g]) return;
    const cplx *a = Vr + (size_t)i * cols;
    const cplx *v = w + (size_t)g * cols;
    cplx s = C(0, 0);
    for (int j = lane; j < cols; j += 32) cfma(s, a[j], __ldg(&v[j]));
    s.x = warp_sum(s.x);
    s.y = warp_sum(s.y);
    if (lane == 0) {
        const cplx r = cscale(s, dscale[i]);
        xo[(size_t)g * nrow + i] = r;
        if (xo32) xo32[(size_t)g * nrow + i] = make_float2((float)r.x, (float)r.y);   // complex64 copy
    }
}

// y[r] = x[r] - s[r] t[r] + s[r] (B_g v_g)[r]  (x, t nullable); v_g = vv + g * ldv
__global__ void k_batch_Bcombine(const cplx *__restrict__ Ball, long Ntot, int nB, const int *__restrict__ gid, int nc,
                                 const int *__restrict__ active, const cplx *__restrict__ vv, int ldv,
                                 const cplx *__restrict__ x, const cplx *__restrict__ t, const cplx *__restrict__ s,
                                 cplx *__restrict__ y) {
    long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= Ntot) return;
    const int g = gid[warp / nc];
    if (active && !active[g]) return;
    const cplx *b = Ball + (size_t)warp * nB;
    const cplx *v = vv + (size_t)g * ldv;
    cplx acc = C(0, 0);
    for (int c = lane; c < nB; c += 32) cfma(acc, b[c], __ldg(&v[c]));
    acc.x = warp_sum(acc.x);
    acc.y = warp_sum(acc.y);
    if (lane == 0) {
        cplx r = x ? x[warp] : C(0, 0);
        if (t) r = csub(r, cmul(s[warp], t[warp]));
        y[warp] = cadd(r, cmul(s[warp], acc));
    }
}

// complex64 copy of B_g (FP32 products) for the mixed form's inner operator: B acts after A^+, so its
// rounding is not amplified; C_g x stays FP64 (it feeds A^+, whose clipped Sigma^+ would)
__global__ void k_batch_Bcombine32(const float2 *__restrict__ Ball, long Ntot, int nB, const int *__restrict__ gid,
                                   int nc, const int *__restrict__ active, const float2 *__restrict__ vv, int ldv,
                                   const cplx *__restrict__ x, const cplx *__restrict__ t, const cplx *__restrict__ s,
                                   cplx *__restrict__ y) {
    long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= Ntot) return;
    const int g = gid[warp / nc];
    if (active && !active[g]) return;
    const float2 *b = Ball + (size_t)warp * nB;
    const float2 *v = vv + (size_t)g * ldv;   // complex64 (no per-entry FP64 -> FP32 conversion)
    float re = 0.f, im = 0.f, re1 = 0.f, im1 = 0.f;
    int c = lane;
    for (; c + 32 < nB; c += 64) {
        const float2 m0 = __ldcs(&b[c]), m1 = __ldcs(&b[c + 32]);
        const float2 w0 = __ldg(&v[c]), w1 = __ldg(&v[c + 32]);
        re = fmaf(m0.x, w0.x, fmaf(-m0.y, w0.y, re));
        im = fmaf(m0.x, w0.y, fmaf(m0.y, w0.x, im));
        re1 = fmaf(m1.x, w1.x, fmaf(-m1.y, w1.y, re1));
        im1 = fmaf(m1.x, w1.y, fmaf(m1.y, w1.x, im1));
    }
    if (c < nB) {
        const float2 m0 = __ldcs(&b[c]), w0 = __ldg(&v[c]);
        re = fmaf(m0.x, w0.x, fmaf(-m0.y, w0.y, re));
        im = fmaf(m0.x, w0.y, fmaf(m0.y, w0.x, im));
    }
    re += re1;
    im += im1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) y[warp] = cadd(csub(x[warp], cmul(s[warp], t[warp])), cmul(s[warp], C(re, im)));
}

__global__ void k_to_c64_b(const cplx *__restrict__ a, long n, float2 *__restrict__ b) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

// complex128 -> double-float (hi, lo) complex64 pairs; flag set if some |entry| exceeds lim or is
// not finite
__global__ void k_b_split_df(const cplx *__restrict__ a, long n, float4 *__restrict__ b, double lim,
                             int *__restrict__ flag) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const cplx v = a[e];
    b[e] = df_split(v.x, v.y);
    if (flag && !(fabs(v.x) <= lim && fabs(v.y) <= lim)) *flag = 1;
}

// gC[g][r] = (C_g x_g)[r] for the mixed inner operator, in double-float arithmetic (C_g and x_g as
// (hi, lo) complex64 pairs, 48-bit significands: C x feeds A^+, whose clipped Sigma^+ amplifies
// rounding in its near-null directions); one block of BATCH_DF_THREADS per (geometry, row)
constexpr int BATCH_DF_THREADS = 128;
__global__ void __launch_bounds__(BATCH_DF_THREADS)
    k_batch_C_df(const float4 *__restrict__ C2all, const size_t *__restrict__ coff, const Geo *__restrict__ geo,
                 int nC, int nc, const int *__restrict__ active, const float4 *__restrict__ x2,
                 cplx *__restrict__ gC) {
    const int g = blockIdx.x / nC, r = blockIdx.x % nC;
    if (active && !active[g]) return;
    const long n = (long)geo[g].M * nc;
    const float4 *a = C2all + coff[g] + (size_t)r * n;
    const float4 *xv = x2 + geo[g].noff;
    dfc s = {0.f, 0.f, 0.f, 0.f};
    dfc_row_dot<BATCH_DF_THREADS>(s, a, xv, n, threadIdx.x);
    dfc_warp_sum(s);
    __shared__ dfc part[BATCH_DF_THREADS / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        dfc t = part[0];
        for (int k = 1; k < BATCH_DF_THREADS / 32; ++k) dfc_add(t, part[k]);
        gC[(size_t)g * nC + r] = C((double)t.rh + (double)t.rl, (double)t.ih + (double)t.il);
    }
}

// y[g][r] = scale[r] (A2 x2_g)[r] for every active geometry g, in double-float arithmetic (A2 rows x
// ncols row-major, x2_g = x2 + g ldx, both (hi, lo) complex64 pairs); the A^+ products of the mixed
// inner operator, whose matrices (the angle's U^H and V Sigma diag(coef)) all geometries share.  One
// block per (row, geometry), the geometry fastest so that neighbouring blocks read the same row.
__global__ void __launch_bounds__(BATCH_DF_THREADS)
    k_batch_gemv_df(const float4 *__restrict__ A2, int nrows, int ncols, const float4 *__restrict__ x2, int ldx, int G,
                    const int *__restrict__ active, cplx *__restrict__ y, int ldy, const double *__restrict__ scale,
                    float2 *__restrict__ y32) {
    const int r = blockIdx.x / G, g = blockIdx.x % G;
    if (r >= nrows || (active && !active[g])) return;
    dfc s = {0.f, 0.f, 0.f, 0.f};
    dfc_row_dot<BATCH_DF_THREADS>(s, A2 + (size_t)r * ncols, x2 + (size_t)g * ldx, ncols, threadIdx.x);
    dfc_warp_sum(s);
    __shared__ dfc part[BATCH_DF_THREADS / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        dfc t = part[0];
        for (int k = 1; k < BATCH_DF_THREADS / 32; ++k) dfc_add(t, part[k]);
        cplx v = C((double)t.rh + (double)t.rl, (double)t.ih + (double)t.il);
        if (scale) v = cscale(v, scale[r]);
        y[(size_t)g * ldy + r] = v;
        if (y32) y32[(size_t)g * ldy + r] = make_float2((float)v.x, (float)v.y);
    }
}

// Bragg: gfull = f - C_g beta_g on the C rows, f elsewhere (one geometry)
__global__ void k_b_f_minus_Cx(const cplx *__restrict__ Cg, int nC, int n, const cplx *__restrict__ x,
                               const cplx *__restrict__ f, int rows, cplx *__restrict__ gout) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= rows) return;
    if (warp >= nC) {
        if (lane == 0) gout[warp] = f[warp];
        return;
    }
    const cplx *a = Cg + (size_t)warp * n;
    cplx s = C(0, 0);
    for (int c = lane; c < n; c += 32) cfma(s, a[c], __ldg(&x[c]));
    s.x = warp_sum(s.x);
    s.y = warp_sum(s.y);
    if (lane == 0) gout[warp] = csub(f[warp], s);
}

// relative flux error of one geometry's Bragg amplitudes (TE weights 1/w1, 1/w3; 1 for TM)
__global__ void k_b_flux(int K, const cplx *cd, const cplx *k1n, const cplx *k3n, double inv_w1, double inv_w3,
                         double inc, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int n = 0; n < 2 * K + 1; ++n) {
        if (k1n[n].y == 0.0 && k1n[n].x > 0.0) s += inv_w1 * k1n[n].x * cabs2(cd[n]);
        if (k3n[n].y == 0.0 && k3n[n].x > 0.0) s += inv_w3 * k3n[n].x * cabs2(cd[2 * K + 1 + n]);
    }
    out[0] = fabs(s - inc) / inc;
}

}  // namespace

// ==== host side =======================================================================================

struct gs_batch {
    int G = 0, p = 0, nc = 0, Mtot = 0;
    long Ntot = 0;
    std::vector<int> M, moff;
    std::vector<long> noff;
    double *xy = nullptr, *radius = nullptr, *kp = nullptr;
    cplx *s = nullptr;
    int *gid = nullptr;            // geometry of each target (Mtot)
    Geo *geo = nullptr;
    size_t *coff = nullptr;        // offset of C_g in Call
    std::vector<size_t> coffh;     // host copy
    cudaStream_t bst = nullptr;    // the batch's own (capturable) stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<cplx *> B, Cm, beta;   // per angle
    std::vector<float2 *> B32;         // per angle: complex64 copy of B (mixed inner operator)
    std::vector<float4 *> C2;          // per angle: double-float copy of C (mixed inner operator;
                                       // null when an entry exceeds GS_DF_LIMIT: FP64 C kept)
    size_t call_elems = 0;
    // translation work list
    Item *items = nullptr;
    int n_items = 0;
    int *counter = nullptr;
    cplx *part = nullptr;
    int *tbase = nullptr, *tchunks = nullptr, *tw = nullptr;
    int chunk = 1024, bpsm = 4;
    bool tuned = false;
    // scratch
    cplx *X = nullptr, *Y = nullptr, *T = nullptr, *b = nullptr, *r = nullptr, *dx = nullptr, *xr = nullptr;
    float2 *b32 = nullptr;
    float4 *img32 = nullptr;       // (hi, lo) float image coordinates, 3 M_g per geometry at 3 moff_g
    float4 *xdf = nullptr;         // Ntot: double-float split of the operator input
    float4 *adf = nullptr;         // G max(nC, cols): double-float split of A^+'s vectors
    int *dflag = nullptr;          // range flag of the double-float split of C
    cplx *gC = nullptr, *w = nullptr, *xv = nullptr;   // G nC, G cols, G cols
    float2 *xv32 = nullptr;        // G cols: complex64 copy of xv (the B_phys input of the mixed operator)
    float2 *w32 = nullptr, *cf32 = nullptr;   // Ntot; G x (kdim+1): complex64 CGS2 operands
    double *npart = nullptr;       // G x SEG_NQ partial squared norms
    int *active = nullptr;
    // GMRES
    int kdim = 0;
    cplx *Vk = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *gg = nullptr, *yy = nullptr, *hp = nullptr;
    double *nrm = nullptr, *res = nullptr;
    int *jdev = nullptr, *kk = nullptr;
    double *hbuf = nullptr;        // pinned host, G values
    // graphs of one Arnoldi step, per precision, for one angle
    cudaGraphExec_t step_exec[2] = {nullptr, nullptr};
    int step_angle[2] = {-1, -1};
    // complex64 pair tables of all geometries (mixed inner translation; empty when they do not all
    // fit the table budget, and the persistent recomputing kernel runs instead), with the scratch of
    // one geometry's table translation (largest geometry)
    std::vector<gs_tab32> tab32;
    float2 *b3 = nullptr;
    cplx *tpart = nullptr;
    size_t tpart_elems = 0;
    // per-geometry statistics (per angle)
    std::vector<std::vector<int>> iters;
    std::vector<std::vector<double>> relres;
    bool factored = false;
};

namespace {

void batch_free(gs_batch *b) {
    if (!b) return;
    dfree_b(b->xy);
    dfree_b(b->radius);
    dfree_b(b->kp);
    dfree_b(b->s);
    dfree_b(b->gid);
    dfree_b(b->geo);
    dfree_b(b->coff);
    for (auto &p : b->B) dfree_b(p);
    for (auto &p : b->B32) dfree_b(p);
    for (auto &p : b->C2) dfree_b(p);
    for (auto &p : b->Cm) dfree_b(p);
    for (auto &p : b->beta) dfree_b(p);
    for (auto &t : b->tab32) dfree_b(t.h);
    dfree_b(b->b3);
    dfree_b(b->tpart);
    dfree_b(b->items);
    dfree_b(b->counter);
    dfree_b(b->part);
    dfree_b(b->tbase);
    dfree_b(b->tchunks);
    dfree_b(b->tw);
    dfree_b(b->X);
    dfree_b(b->Y);
    dfree_b(b->T);
    dfree_b(b->b);
    dfree_b(b->r);
    dfree_b(b->dx);
    dfree_b(b->xr);
    dfree_b(b->b32);
    dfree_b(b->img32);
    dfree_b(b->xdf);
    dfree_b(b->adf);
    dfree_b(b->dflag);
    dfree_b(b->gC);
    dfree_b(b->w);
    dfree_b(b->xv);
    dfree_b(b->xv32);
    dfree_b(b->w32);
    dfree_b(b->cf32);
    dfree_b(b->npart);
    dfree_b(b->active);
    dfree_b(b->Vk);
    dfree_b(b->H);
    dfree_b(b->cs);
    dfree_b(b->sn);
    dfree_b(b->gg);
    dfree_b(b->yy);
    dfree_b(b->hp);
    dfree_b(b->nrm);
    dfree_b(b->res);
    dfree_b(b->jdev);
    dfree_b(b->kk);
    if (b->hbuf) cudaFreeHost(b->hbuf);
    for (int q = 0; q < 2; ++q)
        if (b->step_exec[q]) cudaGraphExecDestroy(b->step_exec[q]);
    if (b->bst) cudaStreamDestroy(b->bst);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    delete b;
}

// work list: per geometry (largest first), target groups of BW, source-image chunks of `chunk`
int build_items(gs_ctx *c, gs_batch *b, int chunk) {
    std::vector<int> order(b->G);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->M[x] > b->M[y]; });
    std::vector<Item> it;
    std::vector<int> tbase(b->Mtot), tch(b->Mtot), tw(b->Mtot);
    for (int g : order) {
        const int M = b->M[g], S = 3 * M;
        const int nch = (S + chunk - 1) / chunk;
        for (int i0 = 0; i0 < M; i0 += BW) {
            const int base = (int)it.size();
            for (int q = 0; q < nch; ++q) it.push_back(Item{g, i0, q * chunk, std::min(S, (q + 1) * chunk)});
            for (int w = 0; w < BW && i0 + w < M; ++w) {
                int t = b->moff[g] + i0 + w;
                tbase[t] = base;
                tch[t] = nch;
                tw[t] = w;
            }
        }
    }
    b->n_items = (int)it.size();
    b->chunk = chunk;
    GS_TRY(dalloc_b(c, &b->items, it.size()));
    GS_TRY(dalloc_b(c, &b->part, (size_t)it.size() * BW * b->nc));
    GS_CUDA(c, cudaMemcpy(b->items, it.data(), sizeof(Item) * it.size(), cudaMemcpyHostToDevice));
    GS_CUDA(c, cudaMemcpy(b->tbase, tbase.data(), sizeof(int) * b->Mtot, cudaMemcpyHostToDevice));
    GS_CUDA(c, cudaMemcpy(b->tchunks, tch.data(), sizeof(int) * b->Mtot, cudaMemcpyHostToDevice));
    GS_CUDA(c, cudaMemcpy(b->tw, tw.data(), sizeof(int) * b->Mtot, cudaMemcpyHostToDevice));
    return GS_OK;
}

template <int P>
int launch_batch_translate(gs_ctx *c, gs_batch *b, const AngleData &a, const cplx *x, cplx *out, int precision,
                           const int *active) {
    cudaStream_t st = c->stream;
    const int sms = c->sms;
    if (precision == GS_C64 && !b->tab32.empty()) {
        // one table-driven launch per geometry (masked ones return at once)
        for (int g = 0; g < b->G; ++g)
            GS_TRY(gs_tab32_translate(c, b->tab32[g], b->M[g], b->p, x + b->noff[g], a.alpha, b->b3, b->tpart,
                                      b->tpart_elems, out + b->noff[g], active ? active + g : nullptr, st));
        return GS_OK;
    }
    if (precision == GS_C64) {
        GS_COUNT_LAUNCH(c);
        k_b_to_c64<<<nblk(b->Ntot), 256, 0, st>>>(x, b->Ntot, b->b32);
    }
    GS_CUDA(c, cudaMemsetAsync(b->counter, 0, sizeof(int), st));
    GS_COUNT_LAUNCH(c);
    if (precision == GS_C64)
        k_batch_translate<P, true><<<sms * b->bpsm, BW * 32, 0, st>>>(b->items, b->n_items, b->counter, b->geo, active,
                                                                      b->xy, b->img32, x, b->b32, c->L.k2, c->L.d, a.alpha,
                                                                      b->part);
    else
        k_batch_translate<P, false><<<sms * b->bpsm, BW * 32, 0, st>>>(b->items, b->n_items, b->counter, b->geo, active,
                                                                       b->xy, b->img32, x, b->b32, c->L.k2, c->L.d, a.alpha,
                                                                       b->part);
    GS_COUNT_LAUNCH(c);
    k_batch_reduce<<<nblk(b->Ntot), 256, 0, st>>>(b->part, b->Ntot, b->nc, b->tbase, b->tchunks, b->tw, out);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

int batch_translate(gs_ctx *c, gs_batch *b, const AngleData &a, const cplx *x, cplx *out, int precision,
                    const int *active) {
    switch (b->p) {
        case 1: return launch_batch_translate<1>(c, b, a, x, out, precision, active);
        case 2: return launch_batch_translate<2>(c, b, a, x, out, precision, active);
        case 3: return launch_batch_translate<3>(c, b, a, x, out, precision, active);
        case 4: return launch_batch_translate<4>(c, b, a, x, out, precision, active);
        case 5: return launch_batch_translate<5>(c, b, a, x, out, precision, active);
        case 6: return launch_batch_translate<6>(c, b, a, x, out, precision, active);
        case 7: return launch_batch_translate<7>(c, b, a, x, out, precision, active);
        case 8: return launch_batch_translate<8>(c, b, a, x, out, precision, active);
        case 10: return launch_batch_translate<10>(c, b, a, x, out, precision, active);
        case 12: return launch_batch_translate<12>(c, b, a, x, out, precision, active);
        default: return gs_fail(c, GS_ERR_ARG, "batched solves support p in 1-8, 10, 12");
    }
}

// y = x - s T x + s B A^+ C x for every geometry (masked by active)
int batch_apply(gs_ctx *c, gs_batch *b, int angle, const cplx *x, cplx *y, int precision, const int *active) {
    const AngleData &a = c->ang[angle];
    const Layout &ly = c->lay;
    const int nC = ly.nC(), nB = ly.nB(), cols = ly.cols;
    cudaStream_t st = c->stream;
    GS_TRY(batch_translate(c, b, a, x, b->T, precision, active));
    GS_COUNT_LAUNCH(c);
    if (precision == GS_C64 && b->C2[angle]) {
        k_b_split_df<<<nblk(b->Ntot), 256, 0, st>>>(x, b->Ntot, b->xdf, 0.0, nullptr);
        GS_COUNT_LAUNCH(c);
        k_batch_C_df<<<b->G * nC, BATCH_DF_THREADS, 0, st>>>(b->C2[angle], b->coff, b->geo, nC, b->nc, active, b->xdf,
                                                             b->gC);
    } else {
        k_batch_C<<<wblk((long)b->G * nC), 256, 0, st>>>(b->Cm[angle], b->coff, b->geo, b->G, nC, b->nc, active, x,
                                                         b->gC);
    }
    if (precision == GS_C64 && a.A2_ready && a.WH2 && a.Vr2 && b->adf) {
        // A^+ in double-float: U^H gC_g, then (V Sigma diag(coef)) w_g, scaled by D
        GS_COUNT_LAUNCH(c);
        k_b_split_df<<<nblk((long)b->G * nC), 256, 0, st>>>(b->gC, (long)b->G * nC, b->adf, 0.0, nullptr);
        GS_COUNT_LAUNCH(c);
        k_batch_gemv_df<<<b->G * cols, BATCH_DF_THREADS, 0, st>>>(a.WH2, cols, nC, b->adf, nC, b->G, active, b->w, cols,
                                                                    nullptr, nullptr);
        GS_COUNT_LAUNCH(c);
        k_b_split_df<<<nblk((long)b->G * cols), 256, 0, st>>>(b->w, (long)b->G * cols, b->adf, 0.0, nullptr);
        GS_COUNT_LAUNCH(c);
        k_batch_gemv_df<<<b->G * nB, BATCH_DF_THREADS, 0, st>>>(a.Vr2, nB, cols, b->adf, cols, b->G, active, b->xv, nB,
                                                                  a.dscale, b->xv32);
    } else {
        GS_COUNT_LAUNCH(c);
        k_batch_UH<<<wblk((long)b->G * cols), 256, 0, st>>>(a.W, ly.rows, nC, cols, b->gC, nC, a.coef, b->G, active,
                                                            b->w);
        GS_COUNT_LAUNCH(c);
        k_batch_V<<<wblk((long)b->G * nB), 256, 0, st>>>(a.Vr, nB, cols, b->w, a.dscale, b->G, active, b->xv,
                                                           precision == GS_C64 ? b->xv32 : nullptr);
    }
    GS_COUNT_LAUNCH(c);
    if (precision == GS_C64) {
        k_batch_Bcombine32<<<wblk(b->Ntot), 256, 0, st>>>(b->B32[angle], b->Ntot, nB, b->gid, b->nc, active, b->xv32,
                                                           nB, x, b->T, b->s, y);
    } else {
        k_batch_Bcombine<<<wblk(b->Ntot), 256, 0, st>>>(b->B[angle], b->Ntot, nB, b->gid, b->nc, active, b->xv, nB, x,
                                                         b->T, b->s, y);
    }
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

int batch_rhs(gs_ctx *c, gs_batch *b, int angle, cplx *out) {
    const AngleData &a = c->ang[angle];
    const Layout &ly = c->lay;
    const int nB = ly.nB(), cols = ly.cols;
    cudaStream_t st = c->stream;
    // A^+ f is the same for every geometry: one column (G = 1), then B_g for all rows
    GS_COUNT_LAUNCH(c);
    k_batch_UH<<<wblk(cols), 256, 0, st>>>(a.W, ly.rows, ly.row_g2v, cols, a.f, ly.rows, a.coef, 1, nullptr, b->w);
    GS_COUNT_LAUNCH(c);
    k_batch_V<<<wblk(nB), 256, 0, st>>>(a.Vr, nB, cols, b->w, a.dscale, 1, nullptr, b->xv);
    GS_COUNT_LAUNCH(c);
    k_batch_Bcombine<<<wblk(b->Ntot), 256, 0, st>>>(b->B[angle], b->Ntot, nB, b->gid, b->nc, nullptr, b->xv, 0, nullptr,
                                                     nullptr, b->s, out);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

int seg_norms(gs_ctx *c, gs_batch *b, const cplx *v, const int *active, std::vector<double> &out) {
    GS_COUNT_LAUNCH(c);
    k_seg_norm<<<b->G, 256, 0, c->stream>>>(v, b->geo, b->nc, active, b->nrm, nullptr, 0, 0, nullptr);
    GS_CUDA(c, cudaMemcpyAsync(b->hbuf, b->nrm, sizeof(double) * b->G, cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    out.assign(b->hbuf, b->hbuf + b->G);
    return GS_OK;
}

// one Arnoldi step for every active geometry, j read from b->jdev; captured into a graph
template <typename TB>
int arnoldi_step_t(gs_ctx *c, gs_batch *b, int angle, int precision) {
    cudaStream_t st = c->stream;
    const long N = b->Ntot;
    TB *V = (TB *)b->Vk;
    GS_COUNT_LAUNCH(c);
    k_seg_fetch<TB><<<nblk(N), 256, 0, st>>>(V, N, b->jdev, b->X);
    GS_TRY(batch_apply(c, b, angle, b->X, b->Y, precision, b->active));
    const SegStep ss{b->geo, b->gid, b->active, b->jdev, b->H, b->hp, b->cs, b->sn, b->gg, b->nrm, b->res, b->npart,
                     b->w32, b->cf32, N, b->G, b->kdim, b->nc};
    GS_TRY(seg_cgs2<TB>(c, ss, V, b->Y, st));
    GS_COUNT_LAUNCH(c);
    k_inc<<<1, 32, 0, st>>>(b->jdev);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

int arnoldi_step(gs_ctx *c, gs_batch *b, int angle, int precision) {
    return precision == GS_C64 ? arnoldi_step_t<float2>(c, b, angle, precision)
                               : arnoldi_step_t<cplx>(c, b, angle, precision);
}

int step_graph(gs_ctx *c, gs_batch *b, int angle, int precision) {
    const int q = precision == GS_C64 ? 1 : 0;
    if (b->step_exec[q] && b->step_angle[q] == angle) return GS_OK;
    if (b->step_exec[q]) {
        cudaGraphExecDestroy(b->step_exec[q]);
        b->step_exec[q] = nullptr;
    }
    if (!c->stream) return GS_OK;   // the legacy default stream cannot be captured: run eagerly
    cudaGraph_t gph;
    GS_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int st = arnoldi_step(c, b, angle, precision);
    cudaError_t e = cudaStreamEndCapture(c->stream, &gph);
    if (st != GS_OK) return st;
    if (e != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->step_exec[q], gph, 0);
    cudaGraphDestroy(gph);
    if (e != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    b->step_angle[q] = angle;
    return GS_OK;
}

// lockstep restarted GMRES on all geometries: solves L_prec x_g = rhs_g until
// ||rhs_g - L x_g|| <= tolabs[g]; geometries with tolabs <= 0 ... are skipped when already converged
int batch_gmres(gs_ctx *c, gs_batch *b, int angle, const cplx *rhs, cplx *x, bool x_zero,
                const std::vector<double> &tolabs, std::vector<int> &done, const std::vector<int> &maxit_g,
                int restart, int precision, std::vector<int> &iters, std::vector<double> &resabs) {
    cudaStream_t st = c->stream;
    const long N = b->Ntot;
    const int G = b->G, ld = b->kdim + 1, eb = nblk(N);
    const int kd = std::min(restart, b->kdim);
    if (x_zero) GS_CUDA(c, cudaMemsetAsync(x, 0, sizeof(cplx) * N, st));
    std::vector<int> act(G), kk(G);
    std::vector<double> nr;
    bool first = x_zero;
    std::vector<int> used(G, 0);       // iterations spent in this call, per geometry
    std::vector<int> est_conv(G, 0);   // the last cycle ended on the residual estimate
    for (;;) {
        // r = rhs - L x
        if (first) {
            GS_CUDA(c, cudaMemcpyAsync(b->r, rhs, sizeof(cplx) * N, cudaMemcpyDeviceToDevice, st));
        } else {
            GS_TRY(batch_apply(c, b, angle, x, b->r, precision, nullptr));
            GS_COUNT_LAUNCH(c);
            k_vsub<<<eb, 256, 0, st>>>(rhs, b->r, N, b->r);
        }
        first = false;
        GS_TRY(seg_norms(c, b, b->r, nullptr, nr));
        int nact = 0;
        for (int g = 0; g < G; ++g) {
            resabs[g] = nr[g];
            // as in the single-geometry solve, a cycle that converged on its estimate is accepted when
            // the recomputed residual is within 10x of the target (rounding of the operator)
            const double lim = est_conv[g] ? 10.0 * tolabs[g] : tolabs[g];
            act[g] = (!done[g] && nr[g] > lim && used[g] < maxit_g[g]) ? 1 : 0;
            if (!act[g]) done[g] = 1;
            nact += act[g];
        }
        if (nact == 0) break;
        GS_CUDA(c, cudaMemcpyAsync(b->active, act.data(), sizeof(int) * G, cudaMemcpyHostToDevice, st));
        GS_CUDA(c, cudaMemcpyAsync(b->nrm, nr.data(), sizeof(double) * G, cudaMemcpyHostToDevice, st));
        GS_COUNT_LAUNCH(c);
        if (precision == GS_C64)
            k_seg_start<float2><<<eb, 256, 0, st>>>(b->r, (float2 *)b->Vk, N, b->gid, b->nc, b->nrm, b->active);
        else
            k_seg_start<cplx><<<eb, 256, 0, st>>>(b->r, b->Vk, N, b->gid, b->nc, b->nrm, b->active);
        GS_COUNT_LAUNCH(c);
        k_seg_g0<<<nblk((long)G * ld), 256, 0, st>>>(b->gg, ld, b->nrm, G);
        GS_CUDA(c, cudaMemsetAsync(b->H, 0, sizeof(cplx) * (size_t)G * b->kdim * ld, st));
        GS_CUDA(c, cudaMemsetAsync(b->jdev, 0, sizeof(int), st));
        GS_TRY(step_graph(c, b, angle, precision));
        std::fill(kk.begin(), kk.end(), 0);
        std::vector<int> live = act;
        int j = 0;
        for (; j < kd; ++j) {
            if (b->step_exec[precision == GS_C64 ? 1 : 0]) {
                GS_CUDA(c, cudaGraphLaunch(b->step_exec[precision == GS_C64 ? 1 : 0], st));
            } else {
                GS_TRY(arnoldi_step(c, b, angle, precision));
            }
            GS_CUDA(c, cudaMemcpyAsync(b->hbuf, b->res, sizeof(double) * G, cudaMemcpyDeviceToHost, st));
            GS_CUDA(c, cudaStreamSynchronize(st));
            int nlive = 0;
            bool changed = false;
            for (int g = 0; g < G; ++g) {
                if (!live[g]) continue;
                iters[g] += 1;
                used[g] += 1;
                kk[g] = j + 1;
                if (b->hbuf[g] <= tolabs[g] || used[g] >= maxit_g[g]) {
                    est_conv[g] = b->hbuf[g] <= tolabs[g];
                    live[g] = 0;
                    changed = true;
                } else {
                    ++nlive;
                }
            }
            if (nlive == 0) break;
            if (changed) GS_CUDA(c, cudaMemcpyAsync(b->active, live.data(), sizeof(int) * G, cudaMemcpyHostToDevice, st));
        }
        for (int g = 0; g < G; ++g)
            if (live[g]) est_conv[g] = 0;
        GS_CUDA(c, cudaMemcpyAsync(b->kk, kk.data(), sizeof(int) * G, cudaMemcpyHostToDevice, st));
        GS_COUNT_LAUNCH(c);
        k_seg_backsolve<<<G, 256, 0, st>>>(b->H, ld, b->kdim, b->kk, b->gg, b->yy, G);
        GS_COUNT_LAUNCH(c);
        if (precision == GS_C64)
            k_seg_update<float2><<<eb, 256, 0, st>>>(x, (const float2 *)b->Vk, N, b->gid, b->nc, b->kk, b->yy, ld);
        else
            k_seg_update<cplx><<<eb, 256, 0, st>>>(x, b->Vk, N, b->gid, b->nc, b->kk, b->yy, ld);
        GS_CHECK_LAUNCH(c);
    }
    return GS_OK;
}

// Krylov workspace for a restart length of up to 512 (the Givens kernels stage a column in shared memory)
int ensure_krylov(gs_ctx *c, gs_batch *b, int restart) {
    const int want = std::max(1, std::min(restart, 512));
    if (b->Vk && b->kdim >= want) return GS_OK;
    b->kdim = want;
    const int ld = b->kdim + 1, G = b->G;
    for (int q = 0; q < 2; ++q)
        if (b->step_exec[q]) {
            cudaGraphExecDestroy(b->step_exec[q]);
            b->step_exec[q] = nullptr;
            b->step_angle[q] = -1;
        }
    GS_TRY(dalloc_b(c, &b->Vk, (size_t)ld * b->Ntot));
    GS_TRY(dalloc_b(c, &b->H, (size_t)G * b->kdim * ld));
    GS_TRY(dalloc_b(c, &b->cs, (size_t)G * ld));
    GS_TRY(dalloc_b(c, &b->sn, (size_t)G * ld));
    GS_TRY(dalloc_b(c, &b->gg, (size_t)G * ld));
    GS_TRY(dalloc_b(c, &b->yy, (size_t)G * ld));
    GS_TRY(dalloc_b(c, &b->hp, (size_t)G * ld));
    GS_TRY(dalloc_b(c, &b->cf32, (size_t)G * ld));
    GS_TRY(dalloc_b(c, &b->w32, (size_t)b->Ntot));
    GS_TRY(dalloc_b(c, &b->npart, (size_t)G * SEG_NQ));
    return GS_OK;
}

int autotune(gs_ctx *c, gs_batch *b, int angle) {
    // times the batched complex64 translation for candidate (chunk, blocks per SM) and keeps the best
    const int chunks[3] = {512, 1024, 2048};
    const int bps[3] = {2, 4, 8};
    float best = 1e30f;
    int bc = 1024, bb = 4;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    GS_CUDA(c, cudaMemsetAsync(b->X, 0, sizeof(cplx) * b->Ntot, c->stream));
    for (int ci : chunks) {
        GS_TRY(build_items(c, b, ci));
        for (int bi : bps) {
            b->bpsm = bi;
            GS_TRY(batch_translate(c, b, c->ang[angle], b->X, b->T, GS_C64, nullptr));   // warm
            cudaEventRecord(e0, c->stream);
            GS_TRY(batch_translate(c, b, c->ang[angle], b->X, b->T, GS_C64, nullptr));
            cudaEventRecord(e1, c->stream);
            GS_CUDA(c, cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bc = ci;
                bb = bi;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->bpsm = bb;
    GS_TRY(build_items(c, b, bc));
    b->tuned = true;
    return GS_OK;
}

// runs the batch's work on its own stream, ordered after the context stream's earlier work and
// before its later work (the context stream may be the legacy default stream, which cannot be
// captured into a graph)
struct OnBatchStream {
    gs_ctx *c;
    cudaStream_t saved;
    OnBatchStream(gs_ctx *cc) : c(cc), saved(cc->stream) {
        gs_batch *b = c->batch;
        cudaEventRecord(b->ev_in, saved);
        cudaStreamWaitEvent(b->bst, b->ev_in, 0);
        c->stream = b->bst;
    }
    ~OnBatchStream() {
        gs_batch *b = c->batch;
        cudaEventRecord(b->ev_out, b->bst);
        cudaStreamWaitEvent(saved, b->ev_out, 0);
        c->stream = saved;
    }
};

}  // namespace

void gs_batch_destroy(gs_ctx *c) {
    if (c && c->batch) {
        batch_free(c->batch);
        c->batch = nullptr;
    }
}

extern "C" {

int gs_set_inclusions_batch(gs_ctx *c, int G, const gs_inclusions *geos) {
    if (!c) return GS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, "cudaSetDevice");
    if (G < 1 || G > 4096 || !geos) return gs_fail(c, GS_ERR_ARG, "need 1..4096 geometries");
    if (!c->have_layers) return gs_fail(c, GS_ERR_STATE, "gs_set_layers must come first");
    const int p = geos[0].p;
    for (int g = 0; g < G; ++g)
        if (geos[g].p != p) return gs_fail(c, GS_ERR_ARG, "all geometries of a batch share the multipole order");
    // validate each geometry through the single-geometry path (overlaps, interface band)
    for (int g = 0; g < G; ++g) {
        int stt = gs_set_inclusions(c, &geos[g]);
        if (stt != GS_OK) return gs_fail(c, stt, "geometry " + std::to_string(g) + ": " + c->err);
    }
    gs_batch_destroy(c);
    gs_batch *b = new gs_batch();
    c->batch = b;
    b->G = G;
    b->p = p;
    b->nc = 2 * p + 1;
    b->M.resize(G);
    b->moff.resize(G);
    b->noff.resize(G);
    int mo = 0;
    for (int g = 0; g < G; ++g) {
        b->M[g] = geos[g].M;
        b->moff[g] = mo;
        b->noff[g] = (long)mo * b->nc;
        mo += geos[g].M;
    }
    b->Mtot = mo;
    b->Ntot = (long)mo * b->nc;
    GS_CUDA(c, cudaStreamCreateWithFlags(&b->bst, cudaStreamNonBlocking));
    GS_CUDA(c, cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    GS_CUDA(c, cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    std::vector<double> xy(2 * (size_t)mo), rad(mo), kp(mo);
    std::vector<int> gid(mo);
    std::vector<Geo> geo(G);
    for (int g = 0; g < G; ++g) {
        for (int i = 0; i < geos[g].M; ++i) {
            xy[2 * (size_t)(b->moff[g] + i)] = geos[g].xy[2 * i];
            xy[2 * (size_t)(b->moff[g] + i) + 1] = geos[g].xy[2 * i + 1];
            rad[b->moff[g] + i] = geos[g].radius[i];
            kp[b->moff[g] + i] = geos[g].kp[i];
            gid[b->moff[g] + i] = g;
        }
        geo[g] = Geo{b->M[g], b->moff[g], (int)b->noff[g]};
    }
    GS_TRY(dalloc_b(c, &b->xy, xy.size()));
    GS_TRY(dalloc_b(c, &b->radius, mo));
    GS_TRY(dalloc_b(c, &b->kp, mo));
    GS_TRY(dalloc_b(c, &b->gid, mo));
    GS_TRY(dalloc_b(c, &b->geo, G));
    GS_CUDA(c, cudaMemcpy(b->xy, xy.data(), sizeof(double) * xy.size(), cudaMemcpyHostToDevice));
    GS_CUDA(c, cudaMemcpy(b->radius, rad.data(), sizeof(double) * mo, cudaMemcpyHostToDevice));
    GS_CUDA(c, cudaMemcpy(b->kp, kp.data(), sizeof(double) * mo, cudaMemcpyHostToDevice));
    GS_CUDA(c, cudaMemcpy(b->gid, gid.data(), sizeof(int) * mo, cudaMemcpyHostToDevice));
    GS_CUDA(c, cudaMemcpy(b->geo, geo.data(), sizeof(Geo) * G, cudaMemcpyHostToDevice));
    return GS_OK;
}

int gs_factor_batch(gs_ctx *c) {
    if (!c || !c->batch) return c ? gs_fail(c, GS_ERR_STATE, "gs_set_inclusions_batch has not run") : GS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, "cudaSetDevice");
    if (c->thetas.empty()) return gs_fail(c, GS_ERR_STATE, "gs_set_incidence must come first");
    gs_batch *b = c->batch;
    c->p = b->p;
    c->nc = b->nc;
    GS_TRY(gs_ensure_grating(c));
    OnBatchStream on(c);
    const Layout &ly = c->lay;
    const int G = b->G, nA = (int)c->ang.size();
    const long N = b->Ntot;
    // coupling per geometry and angle
    GS_TRY(dalloc_b(c, &b->s, N));
    for (int g = 0; g < G; ++g)
        GS_TRY(gs_mie_geo(c, b->M[g], b->radius + b->moff[g], b->kp + b->moff[g], nullptr, b->s + b->noff[g]));
    std::vector<size_t> coff(G);
    size_t o = 0;
    for (int g = 0; g < G; ++g) {
        coff[g] = o;
        o += (size_t)ly.nC() * b->M[g] * b->nc;
    }
    b->call_elems = o;
    GS_TRY(dalloc_b(c, &b->coff, G));
    GS_CUDA(c, cudaMemcpy(b->coff, coff.data(), sizeof(size_t) * G, cudaMemcpyHostToDevice));
    b->coffh = coff;
    for (auto &p : b->B) dfree_b(p);
    for (auto &p : b->B32) dfree_b(p);
    for (auto &p : b->C2) dfree_b(p);
    for (auto &p : b->Cm) dfree_b(p);
    for (auto &p : b->beta) dfree_b(p);
    b->B.assign(nA, nullptr);
    b->B32.assign(nA, nullptr);
    b->C2.assign(nA, nullptr);
    b->Cm.assign(nA, nullptr);
    b->beta.assign(nA, nullptr);
    b->iters.assign(nA, std::vector<int>(G, 0));
    b->relres.assign(nA, std::vector<double>(G, -1.0));
    for (int q = 0; q < nA; ++q) {
        GS_TRY(dalloc_b(c, &b->B[q], (size_t)N * ly.nB()));
        GS_TRY(dalloc_b(c, &b->Cm[q], o));
        GS_TRY(dalloc_b(c, &b->beta[q], N));
        GS_CUDA(c, cudaMemsetAsync(b->beta[q], 0, sizeof(cplx) * N, c->stream));
        for (int g = 0; g < G; ++g) {
            GS_TRY(gs_assemble_B_geo(c, c->ang[q], b->M[g], b->xy + 2 * (size_t)b->moff[g],
                                     b->B[q] + (size_t)b->noff[g] * ly.nB()));
            GS_TRY(gs_assemble_C_geo(c, c->ang[q], b->M[g], b->xy + 2 * (size_t)b->moff[g], b->Cm[q] + coff[g]));
        }
        const long nb = (long)N * ly.nB();
        GS_TRY(dalloc_b(c, &b->B32[q], nb));
        GS_COUNT_LAUNCH(c);
        k_to_c64_b<<<nblk(nb), 256, 0, c->stream>>>(b->B[q], nb, b->B32[q]);
        GS_CHECK_LAUNCH(c);
        // double-float copy of C (the mixed inner operator's C x), unless an entry is out of range
        // (no room for the copy, or an entry out of range: the FP64 product stays for this angle)
        if (!b->dflag) GS_TRY(dalloc_b(c, &b->dflag, 1));
        if (cudaMalloc((void **)&b->C2[q], sizeof(float4) * o) != cudaSuccess) {
            cudaGetLastError();
            b->C2[q] = nullptr;
        } else {
            GS_CUDA(c, cudaMemsetAsync(b->dflag, 0, sizeof(int), c->stream));
            GS_COUNT_LAUNCH(c);
            k_b_split_df<<<nblk((long)o), 256, 0, c->stream>>>(b->Cm[q], (long)o, b->C2[q], GS_DF_LIMIT, b->dflag);
            GS_CHECK_LAUNCH(c);
            int big = 0;
            GS_CUDA(c, cudaMemcpyAsync(&big, b->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            GS_CUDA(c, cudaStreamSynchronize(c->stream));
            if (big) dfree_b(b->C2[q]);
        }
        GS_TRY(gs_prepare_apinv_df(c, c->ang[q]));   // the angle's A^+ in double-float, shared by all geometries
    }
    // workspace
    b->kdim = 0;
    dfree_b(b->Vk);
    GS_TRY(dalloc_b(c, &b->X, N));
    GS_TRY(dalloc_b(c, &b->Y, N));
    GS_TRY(dalloc_b(c, &b->T, N));
    GS_TRY(dalloc_b(c, &b->b, N));
    GS_TRY(dalloc_b(c, &b->r, N));
    GS_TRY(dalloc_b(c, &b->dx, N));
    GS_TRY(dalloc_b(c, &b->xr, N));
    GS_TRY(dalloc_b(c, &b->b32, N));
    GS_TRY(dalloc_b(c, &b->img32, 3 * (size_t)b->Mtot));
    GS_TRY(dalloc_b(c, &b->xdf, N));
    GS_TRY(dalloc_b(c, &b->adf, (size_t)G * std::max(ly.nC(), ly.cols)));
    for (int g = 0; g < G; ++g)
        GS_TRY(gs_build_images_c64(c, b->xy + 2 * (size_t)b->moff[g], b->M[g], b->img32 + 3 * (size_t)b->moff[g],
                                   c->stream));
    GS_TRY(dalloc_b(c, &b->gC, (size_t)G * ly.nC()));
    GS_TRY(dalloc_b(c, &b->w, (size_t)G * ly.cols));
    GS_TRY(dalloc_b(c, &b->xv, (size_t)G * ly.cols));
    GS_TRY(dalloc_b(c, &b->xv32, (size_t)G * ly.cols));
    GS_TRY(dalloc_b(c, &b->active, G));
    GS_TRY(ensure_krylov(c, b, 200));
    GS_TRY(dalloc_b(c, &b->nrm, G));
    GS_TRY(dalloc_b(c, &b->res, G));
    GS_TRY(dalloc_b(c, &b->jdev, 1));
    GS_TRY(dalloc_b(c, &b->kk, G));
    GS_TRY(dalloc_b(c, &b->counter, 1));
    GS_TRY(dalloc_b(c, &b->tbase, b->Mtot));
    GS_TRY(dalloc_b(c, &b->tchunks, b->Mtot));
    GS_TRY(dalloc_b(c, &b->tw, b->Mtot));
    if (!b->hbuf) GS_CUDA(c, cudaMallocHost((void **)&b->hbuf, sizeof(double) * G));
    GS_TRY(build_items(c, b, b->chunk));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    GS_TRY(autotune(c, b, 0));
    // complex64 pair tables for the mixed inner translation, when all of them fit the table budget
    for (auto &t : b->tab32) dfree_b(t.h);
    b->tab32.clear();
    dfree_b(b->b3);
    dfree_b(b->tpart);
    {
        size_t need = 0;
        int Mmax = 0;
        for (int g = 0; g < G; ++g) {
            need += gs_tab32_bytes(b->M[g], b->p);
            Mmax = std::max(Mmax, b->M[g]);
        }
        size_t fr = 0, totm = 0;
        GS_CUDA(c, cudaMemGetInfo(&fr, &totm));
        const double budget = c->table_budget_gb >= 0 ? c->table_budget_gb * 1e9 : 0.5 * (double)fr;
        if ((double)need <= budget) {
            b->tab32.assign(G, gs_tab32());
            int r = GS_OK;
            for (int g = 0; g < G && r == GS_OK; ++g)
                r = gs_tab32_build(c, b->xy + 2 * (size_t)b->moff[g], b->M[g], b->p, nullptr, &b->tab32[g], c->stream);
            if (r == GS_OK) {
                b->tpart_elems = (size_t)64 * Mmax * b->nc;
                r = dalloc_b(c, &b->b3, (size_t)((3L * Mmax + 31) / 32) * 32 * b->nc);
                if (r == GS_OK) r = dalloc_b(c, &b->tpart, b->tpart_elems);
            }
            if (r != GS_OK) {
                for (auto &t : b->tab32) dfree_b(t.h);
                b->tab32.clear();
                dfree_b(b->b3);
                dfree_b(b->tpart);
                if (r != GS_ERR_OOM) return r;
                cudaGetLastError();
            }
        }
    }
    for (int q = 0; q < 2; ++q)
        if (b->step_exec[q]) {
            cudaGraphExecDestroy(b->step_exec[q]);
            b->step_exec[q] = nullptr;
            b->step_angle[q] = -1;
        }
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    b->factored = true;
    return GS_OK;
}

int gs_apply_batch(gs_ctx *c, int angle, const gs_c128 *x_dev, gs_c128 *y_dev, int precision) {
    if (!c || !c->batch || !c->batch->factored) return c ? gs_fail(c, GS_ERR_STATE, "gs_factor_batch has not run") : GS_ERR_ARG;
    if (angle < 0 || angle >= (int)c->ang.size() || !x_dev || !y_dev) return gs_fail(c, GS_ERR_ARG, "bad argument");
    if (precision != GS_FP64 && precision != GS_C64) return gs_fail(c, GS_ERR_ARG, "bad precision");
    OnBatchStream on(c);
    return batch_apply(c, c->batch, angle, (const cplx *)x_dev, (cplx *)y_dev, precision, nullptr);
}

int gs_solve_batch(gs_ctx *c, int angle, const gs_solve_opts *o) {
    if (!c || !c->batch || !c->batch->factored) return c ? gs_fail(c, GS_ERR_STATE, "gs_factor_batch has not run") : GS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, "cudaSetDevice");
    if (angle < 0 || angle >= (int)c->ang.size() || !o || !(o->tol > 0) || o->maxit < 1 || o->restart < 1)
        return gs_fail(c, GS_ERR_ARG, "bad argument");
    if (o->precision != GS_FP64 && o->precision != GS_C64) return gs_fail(c, GS_ERR_ARG, "bad precision");
    gs_batch *b = c->batch;
    OnBatchStream on(c);
    const int G = b->G;
    const long N = b->Ntot;
    cudaStream_t st = c->stream;
    cplx *x = b->beta[angle];
    GS_TRY(batch_rhs(c, b, angle, b->b));
    std::vector<double> bn;
    GS_TRY(seg_norms(c, b, b->b, nullptr, bn));
    std::vector<int> iters(G, 0), done(G, 0);
    std::vector<double> resabs(G, 0.0), tolabs(G);
    for (int g = 0; g < G; ++g) tolabs[g] = o->tol * bn[g];
    GS_TRY(ensure_krylov(c, b, o->restart));
    if (o->precision == GS_FP64) {
        std::vector<int> cap(G, o->maxit);
        GS_TRY(batch_gmres(c, b, angle, b->b, x, true, tolabs, done, cap, o->restart, GS_FP64, iters, resabs));
    } else {
        // mixed refinement in lockstep: FP64 residuals, complex64 inner solves
        GS_CUDA(c, cudaMemsetAsync(x, 0, sizeof(cplx) * N, st));
        const double floor_tol = o->inner_tol > 0 ? o->inner_tol : 1e-6;
        const int max_sweeps = o->max_sweeps > 0 ? o->max_sweeps : 30;
        std::vector<double> rn(G);
        for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
            if (sweep == 0) {
                GS_CUDA(c, cudaMemcpyAsync(b->xr, b->b, sizeof(cplx) * N, cudaMemcpyDeviceToDevice, st));
                rn = bn;
            } else {
                GS_TRY(batch_apply(c, b, angle, x, b->xr, GS_FP64, nullptr));
                GS_COUNT_LAUNCH(c);
                k_vsub<<<nblk(N), 256, 0, st>>>(b->b, b->xr, N, b->xr);
                GS_TRY(seg_norms(c, b, b->xr, nullptr, rn));
            }
            int open = 0;
            std::vector<int> idone(G, 0);
            std::vector<double> itol(G);
            for (int g = 0; g < G; ++g) {
                resabs[g] = rn[g];
                if (rn[g] <= tolabs[g] || bn[g] == 0.0) {
                    idone[g] = 1;
                    itol[g] = 0.0;
                } else {
                    ++open;
                    double rel = rn[g] / bn[g];
                    itol[g] = std::max(floor_tol, 0.5 * o->tol / rel) * rn[g];
                }
            }
            if (open == 0 || sweep == max_sweeps) break;
            std::vector<int> cap(G);
            int anyleft = 0;
            for (int g = 0; g < G; ++g) {
                cap[g] = std::max(0, o->maxit - iters[g]);
                if (cap[g] == 0) idone[g] = 1;
                anyleft += !idone[g];
            }
            if (anyleft == 0) break;
            std::vector<double> rtmp(G);
            GS_TRY(batch_gmres(c, b, angle, b->xr, b->dx, true, itol, idone, cap, o->restart, GS_C64, iters, rtmp));
            // x += dx for the geometries that were still open (dx = 0 for the others)
            GS_COUNT_LAUNCH(c);
            k_vadd<<<nblk(N), 256, 0, st>>>(x, b->dx, N);
            GS_CHECK_LAUNCH(c);
        }
    }
    bool ok = true;
    for (int g = 0; g < G; ++g) {
        b->iters[angle][g] = iters[g];
        b->relres[angle][g] = bn[g] > 0 ? resabs[g] / bn[g] : 0.0;
        if (b->relres[angle][g] > 10.0 * o->tol) ok = false;
    }
    return ok ? GS_OK : GS_ERR_NOT_CONVERGED;
}

int gs_batch_stats(gs_ctx *c, int angle, int g, int *iters, double *relres) {
    if (!c || !c->batch || !c->batch->factored) return c ? gs_fail(c, GS_ERR_STATE, "no batch") : GS_ERR_ARG;
    if (angle < 0 || angle >= (int)c->ang.size() || g < 0 || g >= c->batch->G) return gs_fail(c, GS_ERR_ARG, "bad index");
    if (iters) *iters = c->batch->iters[angle][g];
    if (relres) *relres = c->batch->relres[angle][g];
    return GS_OK;
}

int gs_get_beta_batch(gs_ctx *c, int angle, int g, gs_c128 *beta_dev) {
    if (!c || !c->batch || !c->batch->factored) return c ? gs_fail(c, GS_ERR_STATE, "no batch") : GS_ERR_ARG;
    gs_batch *b = c->batch;
    if (angle < 0 || angle >= (int)c->ang.size() || g < 0 || g >= b->G || !beta_dev) return gs_fail(c, GS_ERR_ARG, "bad argument");
    OnBatchStream on(c);
    GS_CUDA(c, cudaMemcpyAsync(beta_dev, b->beta[angle] + b->noff[g], sizeof(cplx) * b->M[g] * b->nc,
                               cudaMemcpyDeviceToDevice, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

int gs_bragg_batch(gs_ctx *c, int angle, int g, int *n_top, int *orders_top, gs_c128 *cc, int *n_bot, int *orders_bot,
                   gs_c128 *dd, double *flux_err) {
    if (!c || !c->batch || !c->batch->factored) return c ? gs_fail(c, GS_ERR_STATE, "no batch") : GS_ERR_ARG;
    gs_batch *b = c->batch;
    if (angle < 0 || angle >= (int)c->ang.size() || g < 0 || g >= b->G) return gs_fail(c, GS_ERR_ARG, "bad index");
    if (!n_top || !orders_top || !cc || !n_bot || !orders_bot || !dd || !flux_err) return gs_fail(c, GS_ERR_ARG, "null output");
    const AngleData &a = c->ang[angle];
    const Layout &ly = c->lay;
    const int n = b->M[g] * b->nc, K = ly.K, K2 = 2 * K + 1, ncd = 2 * K2;
    OnBatchStream on(c);
    cudaStream_t st = c->stream;
    std::vector<cplx> cd(ncd);
    cplx *gbuf = nullptr, *wbuf = nullptr, *xbuf = nullptr;
    double *fl = nullptr;
    GS_TRY(dalloc_b(c, &gbuf, ly.rows));
    GS_TRY(dalloc_b(c, &wbuf, ly.cols));
    GS_TRY(dalloc_b(c, &xbuf, ncd));
    GS_TRY(dalloc_b(c, &fl, 1));
    GS_COUNT_LAUNCH(c);
    k_b_f_minus_Cx<<<wblk(ly.rows), 256, 0, st>>>(b->Cm[angle] + b->coffh[g], ly.nC(), n, b->beta[angle] + b->noff[g],
                                                   a.f, ly.rows, gbuf);
    GS_COUNT_LAUNCH(c);
    k_batch_UH<<<wblk(ly.cols), 256, 0, st>>>(a.W, ly.rows, ly.rows, ly.cols, gbuf, ly.rows, a.coef, 1, nullptr, wbuf);
    GS_COUNT_LAUNCH(c);
    k_batch_V<<<wblk(ncd), 256, 0, st>>>(a.Vr + (size_t)ly.col_c * ly.cols, ncd, ly.cols, wbuf, a.dscale + ly.col_c, 1,
                                         nullptr, xbuf);
    GS_COUNT_LAUNCH(c);
    double w1, w3;
    gs_layer_weights(c, &w1, &w3);
    k_b_flux<<<1, 1, 0, st>>>(K, xbuf, a.k1n, a.k3n, 1.0 / w1, 1.0 / w3, c->L.k1 * fabs(sin(a.theta)) / w1, fl);
    GS_CHECK_LAUNCH(c);
    double flux = 0;
    GS_CUDA(c, cudaMemcpyAsync(cd.data(), xbuf, sizeof(cplx) * ncd, cudaMemcpyDeviceToHost, st));
    GS_CUDA(c, cudaMemcpyAsync(&flux, fl, sizeof(double), cudaMemcpyDeviceToHost, st));
    std::vector<cplx> k1n(K2), k3n(K2);
    GS_CUDA(c, cudaMemcpyAsync(k1n.data(), a.k1n, sizeof(cplx) * K2, cudaMemcpyDeviceToHost, st));
    GS_CUDA(c, cudaMemcpyAsync(k3n.data(), a.k3n, sizeof(cplx) * K2, cudaMemcpyDeviceToHost, st));
    GS_CUDA(c, cudaStreamSynchronize(st));
    dfree_b(gbuf);
    dfree_b(wbuf);
    dfree_b(xbuf);
    dfree_b(fl);
    int nt = 0, nb = 0;
    bool finite = std::isfinite(flux);
    for (int q = 0; q < K2; ++q) {
        if (k1n[q].y == 0.0 && k1n[q].x > 0.0) {
            orders_top[nt] = q - K;
            cc[nt].re = cd[q].x;
            cc[nt].im = cd[q].y;
            finite = finite && std::isfinite(cd[q].x) && std::isfinite(cd[q].y);
            ++nt;
        }
        if (k3n[q].y == 0.0 && k3n[q].x > 0.0) {
            orders_bot[nb] = q - K;
            dd[nb].re = cd[K2 + q].x;
            dd[nb].im = cd[K2 + q].y;
            finite = finite && std::isfinite(cd[K2 + q].x) && std::isfinite(cd[K2 + q].y);
            ++nb;
        }
    }
    *n_top = nt;
    *n_bot = nb;
    *flux_err = flux;
    return finite ? GS_OK : gs_fail(c, GS_ERR_NUMERIC, "non-finite Bragg amplitude");
}

int gs_batch_tuning(gs_ctx *c, int *chunk, int *blocks_per_sm) {
    if (!c || !c->batch || !c->batch->factored) return c ? gs_fail(c, GS_ERR_STATE, "no batch") : GS_ERR_ARG;
    if (chunk) *chunk = c->batch->chunk;
    if (blocks_per_sm) *blocks_per_sm = c->batch->bpsm;
    return GS_OK;
}

}  // extern "C"
