// Factorisation of the empty-grating block on the GPU (FP64, Sec. 5 "We precompute A = U Sigma V^*").
//
// The J-expansion columns of A are rescaled to unit 2-norm (Sec. 3, Fig. 2a remark).  The SVD of
// the scaled matrix A D is then taken by preconditioned one-sided Jacobi (Drmac-Veselic):
//   1. Householder QR with column pivoting, A D P = Q R (one thread block picks the pivot by the
//      trailing column norms and builds the reflector; one block per trailing column applies it and
//      recomputes that column's trailing norm);
//   2. one-sided (Hestenes) Jacobi on X = R^*: column pairs of X are rotated until every pair is
//      orthogonal to relative precision tol, giving X V_x = W_x with orthogonal columns; pairs
//      follow the round-robin (circle) schedule, n/2 disjoint pairs per launch, one block per pair.
//      The sweeps run in two phases: first an FP32 copy of R^* is swept in FP32 (64 times the FP64
//      rate) with its rotations accumulated in FP32; their product is made orthonormal to FP64
//      precision by Newton-Schulz steps V <- V (3I - V^H V)/2 (quadratic convergence from the
//      ~1e-5 defect); then X = R^* V is formed in FP64 and ordinary FP64 sweeps take its nearly
//      orthogonal columns to tol in a few quadratically convergent sweeps, continuing to
//      accumulate into V.  The result is an FP64 one-sided Jacobi SVD; FP32 only does the bulk of
//      the rotating;
//   3. R = V_x W_x^*, hence A D = (Q V_x) Sigma (P W_x Sigma^{-1})^*: U = Q V_x is formed by
//      applying the reflectors to V_x, and V Sigma = P W_x.
// U is orthonormal to working precision by construction (reflectors and rotations), which keeps
// the clipped pseudo-inverse safe in the near-null directions.  A^+ g = D V Sigma^+ U^* g with
// Sigma^+ = min(1/sigma, 1/eps) (Eq. applypA) is applied as D (P W_x) (coef .* (U^* g)) with
// coef_j = 1/(sigma_j max(sigma_j, eps)), sigma_j = ||W_x e_j||.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gs_internal.h"

namespace {

constexpr int JTPB = 256;

// FP64 accumulations written as FMA chains: the FP64 pipe is the bound of the kernels below, and
// a*b + c*d + acc as written costs a multiply, an FMA and an add where two FMAs do
__device__ __forceinline__ double abs2_acc(cplx a, double s) { return fma(a.x, a.x, fma(a.y, a.y, s)); }
__device__ __forceinline__ void cdot_acc(double &re, double &im, cplx a, cplx b) {   // += conj(a) b
    re = fma(a.x, b.x, fma(a.y, b.y, re));
    im = fma(a.x, b.y, fma(-a.y, b.x, im));
}
__device__ __forceinline__ cplx csub_mul(cplx y, cplx f, cplx v) {   // y - f v
    return C(fma(-f.x, v.x, fma(f.y, v.y, y.x)), fma(-f.x, v.y, fma(-f.y, v.x, y.y)));
}

__global__ void k_colnorm_scale(cplx *A, int lda, int rows, int c0, int c1, double *dscale) {
    int col = c0 + blockIdx.x;
    if (col >= c1) return;
    __shared__ double sh[32];
    cplx *a = A + (size_t)col * lda;
    double s = 0.0;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) s = abs2_acc(a[i], s);
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

// Rotation of the column pair (pc, qc), pc < qc, of W (columns of length m) and of V (length n) by
// the whole block, if the pair is further than tol from orthogonal (then *nrot is incremented).
__device__ void jacobi_pair(cplx *W, int m, cplx *V, int n, int pc, int qc, double tol, unsigned long long *nrot) {
    cplx *wp = W + (size_t)pc * m, *wq = W + (size_t)qc * m;
    __shared__ double4 sh4[32];
    __shared__ double rot[5];
    double al = 0, be = 0, gr = 0, gi = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        cplx x = wp[i], y = wq[i];
        al = abs2_acc(x, al);
        be = abs2_acc(y, be);
        cdot_acc(gr, gi, x, y);   // conj(x) y
    }
    // the four sums in one block reduction
    al = warp_sum(al);
    be = warp_sum(be);
    gr = warp_sum(gr);
    gi = warp_sum(gi);
    {
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
        if (l == 0) sh4[w] = make_double4(al, be, gr, gi);
        __syncthreads();
        if (w == 0) {
            double4 t = (l < nw) ? sh4[l] : make_double4(0.0, 0.0, 0.0, 0.0);
            t.x = warp_sum(t.x);
            t.y = warp_sum(t.y);
            t.z = warp_sum(t.z);
            t.w = warp_sum(t.w);
            if (l == 0) sh4[0] = t;
        }
        __syncthreads();
        const double4 r = sh4[0];
        al = r.x;
        be = r.y;
        gr = r.z;
        gi = r.w;
    }
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
            rot[3] = gr / g;   // e^{-i phi} = conj(conj(w_p) w_q) / |.|, phi = arg(conj(w_p) w_q)
            rot[4] = -gi / g;
            atomicAdd(nrot, 1ull);
        }
    }
    __syncthreads();
    if (rot[0] == 0.0) return;
    double cc = rot[1], ss = rot[2];
    const cplx e = C(rot[3], rot[4]);
    cplx *vp = V + (size_t)pc * n, *vq = V + (size_t)qc * n;
    if (cc == 1.0) {
        // |t| below ~1e-8 (most rotations once the sweeps converge): cos rounds to 1, and the
        // rotation is x - s e y, s x + e y, a third fewer FP64 operations
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const cplx x = wp[i], y = cmul(wq[i], e);
            wp[i] = csub(x, cscale(y, ss));
            wq[i] = cadd(cscale(x, ss), y);
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const cplx x = vp[i], y = cmul(vq[i], e);
            vp[i] = csub(x, cscale(y, ss));
            vq[i] = cadd(cscale(x, ss), y);
        }
        return;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        cplx x = wp[i], y = cmul(wq[i], e);
        wp[i] = csub(cscale(x, cc), cscale(y, ss));
        wq[i] = cadd(cscale(x, ss), cscale(y, cc));
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        cplx x = vp[i], y = cmul(vq[i], e);
        vp[i] = csub(cscale(x, cc), cscale(y, ss));
        vq[i] = cadd(cscale(x, ss), cscale(y, cc));
    }
}

// One round of the circle schedule: block k rotates the pair (player(k), player(npad-1-k)).
__global__ void __launch_bounds__(JTPB) k_jacobi_round(cplx *W, int m, cplx *V, int n, int r, int npad,
                                                       double tol, unsigned long long *nrot) {
    const int k = blockIdx.x;
    auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + r) % (npad - 1)) + 1; };
    const int a = player(k), b = player(npad - 1 - k);
    if (a >= n || b >= n) return;
    jacobi_pair(W, m, V, n, a < b ? a : b, a < b ? b : a, tol, nrot);
}

// One round of listed pairs (disjoint columns): block k rotates pairs[k] = (pc, qc), pc < qc
__global__ void __launch_bounds__(JTPB) k_jacobi_pairs(cplx *W, int m, cplx *V, int n, const int2 *pairs,
                                                       double tol, unsigned long long *nrot) {
    const int2 pq = pairs[blockIdx.x];
    jacobi_pair(W, m, V, n, pq.x, pq.y, tol, nrot);
}

// The pairs (i, c) with c one of the nt columns cols[] (inT[] flags them) that lie further than tol
// from orthogonal, by the criterion of jacobi_pair, from the columns themselves (a warp per (c, i));
// appended to pairs[] as (min, max), a pair of two listed columns once
__global__ void k_cols_violators(const cplx *__restrict__ W, int m, int n, const int *__restrict__ cols, int nt,
                                 const int *__restrict__ inT, double tol, int2 *__restrict__ pairs,
                                 unsigned long long *count) {
    const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= (long)nt * n) return;
    const int k = (int)(gw / n), i = (int)(gw % n), cc = cols[k];
    if (i == cc || (inT[i] && i < cc)) return;
    const cplx *wi = W + (size_t)i * m, *wc = W + (size_t)cc * m;
    double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
    for (int e = lane; e < m; e += 32) {
        const cplx x = wi[e], y = wc[e];
        al = abs2_acc(x, al);
        be = abs2_acc(y, be);
        cdot_acc(gr, gi, x, y);
    }
    al = warp_sum(al);
    be = warp_sum(be);
    gr = warp_sum(gr);
    gi = warp_sum(gi);
    if (lane == 0) {
        const double g = hypot(gr, gi);
        if (g != 0.0 && g > tol * sqrt(al * be)) {
            const unsigned long long q = atomicAdd(count, 1ull);
            pairs[q] = make_int2(min(i, cc), max(i, cc));
        }
    }
}

// The pairs (r, c), r < c, whose Gram entry G[r][c] = <w_r, w_c> (G column-major n x n) lies further
// than tol from orthogonal, by the criterion of jacobi_pair; appended to pairs[] through *count
__global__ void k_gram_violators(const cplx *G, int n, double tol, int2 *pairs, unsigned long long *count) {
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)n * n) return;
    const int r = (int)(id % n), c = (int)(id / n);
    if (r >= c) return;
    const cplx g = G[id];
    const double ga = hypot(g.x, g.y);
    if (ga == 0.0 || ga <= tol * sqrt(G[(size_t)r * n + r].x * G[(size_t)c * n + c].x)) return;
    const unsigned long long k = atomicAdd(count, 1ull);
    pairs[k] = make_int2(r, c);
}

// FP32 copy of a complex128 array
__global__ void k_to_c64(const cplx *__restrict__ X, long n, float2 *__restrict__ Y) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) Y[e] = make_float2((float)X[e].x, (float)X[e].y);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// the four sums of a Jacobi pair in one block reduction (one barrier pass instead of four)
__device__ __forceinline__ void block_sum4_f(float &a, float &b, float &c, float &d, float4 *sh) {
    a = warp_sum_f(a);
    b = warp_sum_f(b);
    c = warp_sum_f(c);
    d = warp_sum_f(d);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0) sh[w] = make_float4(a, b, c, d);
    __syncthreads();
    if (w == 0) {
        float4 t = (l < nw) ? sh[l] : make_float4(0.f, 0.f, 0.f, 0.f);
        t.x = warp_sum_f(t.x);
        t.y = warp_sum_f(t.y);
        t.z = warp_sum_f(t.z);
        t.w = warp_sum_f(t.w);
        if (l == 0) sh[0] = t;
    }
    __syncthreads();
    const float4 r = sh[0];
    a = r.x;
    b = r.y;
    c = r.z;
    d = r.w;
}

// FP32 round on the copy W32 with the rotations accumulated in V (FP32), one block per pair: the
// pair's rotation is computed in FP64 from FP32 dot products and applied in FP32.  (One warp per
// pair was measured slower: a round then has too few blocks to hide the memory latency.)
__device__ void rotate_pair_f32(float2 *W32, int m, float2 *V, int n, int pc, int qc, float tol,
                                unsigned long long *nrot) {
    float2 *wp = W32 + (size_t)pc * m, *wq = W32 + (size_t)qc * m;
    __shared__ float4 sh4[32];
    __shared__ double rot[5];
    float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const float2 x = wp[i], y = wq[i];
        al = fmaf(x.x, x.x, fmaf(x.y, x.y, al));
        be = fmaf(y.x, y.x, fmaf(y.y, y.y, be));
        gr = fmaf(x.x, y.x, fmaf(x.y, y.y, gr));   // conj(x) y
        gi = fmaf(x.x, y.y, fmaf(-x.y, y.x, gi));
    }
    block_sum4_f(al, be, gr, gi, sh4);
    if (threadIdx.x == 0) {
        const double g = hypot((double)gr, (double)gi);
        if (g == 0.0 || g <= (double)tol * sqrt((double)al * (double)be)) {
            rot[0] = 0.0;
        } else {
            const double zeta = ((double)be - (double)al) / (2.0 * g);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double cc = 1.0 / sqrt(1.0 + t * t);
            rot[0] = 1.0;
            rot[1] = cc;
            rot[2] = cc * t;
            rot[3] = (double)gr / g;   // e^{-i phi}, phi = arg(conj(w_p) w_q)
            rot[4] = -(double)gi / g;
            atomicAdd(nrot, 1ull);
        }
    }
    __syncthreads();
    if (rot[0] == 0.0) return;
    const double cc = rot[1], ss = rot[2];
    const float cf = (float)cc, sf = (float)ss, er = (float)rot[3], ei = (float)rot[4];   // applied in FP32
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const float2 x = wp[i], y0 = wq[i];
        const float2 y = make_float2(y0.x * er - y0.y * ei, y0.x * ei + y0.y * er);
        wp[i] = make_float2(cf * x.x - sf * y.x, cf * x.y - sf * y.y);
        wq[i] = make_float2(sf * x.x + cf * y.x, sf * x.y + cf * y.y);
    }
    float2 *vp = V + (size_t)pc * n, *vq = V + (size_t)qc * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 x = vp[i], y0 = vq[i];
        const float2 y = make_float2(y0.x * er - y0.y * ei, y0.x * ei + y0.y * er);
        vp[i] = make_float2(cf * x.x - sf * y.x, cf * x.y - sf * y.y);
        vq[i] = make_float2(sf * x.x + cf * y.x, sf * x.y + cf * y.y);
    }
}

__global__ void __launch_bounds__(JTPB) k_jacobi_round_f32(float2 *W32, int m, float2 *V, int n, int r, int npad,
                                                           float tol, unsigned long long *nrot) {
    const int k = blockIdx.x;
    auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + r) % (npad - 1)) + 1; };
    const int a = player(k), b = player(npad - 1 - k);
    if (a >= n || b >= n) return;
    rotate_pair_f32(W32, m, V, n, a < b ? a : b, a < b ? b : a, tol, nrot);
}

// FP32 round of listed pairs (disjoint columns): block k rotates pairs[k] = (pc, qc), pc < qc
__global__ void __launch_bounds__(JTPB) k_jacobi_pairs_f32(float2 *W32, int m, float2 *V, int n, const int2 *pairs,
                                                           float tol, unsigned long long *nrot) {
    const int2 pq = pairs[blockIdx.x];
    rotate_pair_f32(W32, m, V, n, pq.x, pq.y, tol, nrot);
}

// k_gram_violators on an FP32 Gram matrix
__global__ void k_gram_violators_f32(const float2 *G, int n, float tol, int2 *pairs, unsigned long long *count) {
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)n * n) return;
    const int r = (int)(id % n), c = (int)(id / n);
    if (r >= c) return;
    const float2 g = G[id];
    const double ga = hypot((double)g.x, (double)g.y);
    if (ga == 0.0 || ga <= (double)tol * sqrt((double)G[(size_t)r * n + r].x * (double)G[(size_t)c * n + c].x)) return;
    const unsigned long long k = atomicAdd(count, 1ull);
    pairs[k] = make_int2(r, c);
}

// ---- one whole FP32 sweep per launch (cooperative) -------------------------------------------------
// The FP32 rounds are latency-bound (a round of ~845 pair rotations of 1689-long columns is ~1 us of
// FP32 work but a launch, two dependent passes over the columns and a block reduction): one
// cooperative launch runs all rounds of a sweep, the resident blocks taking the round's pairs in
// turn and meeting at a grid barrier between rounds.  Columns written in one round are read by other
// SMs in the next, so they move through L2 only (__ldcg / __stcg); the barrier publishes them with
// __threadfence.  Every barrier wait is bounded (~1 s): a block that gives up sets *err and all
// blocks leave at the next barrier.

// Sense-reversing barrier over the grid on (count, gen); false if the wait gave up or an error is set
__device__ bool grid_barrier(unsigned *count, volatile unsigned *gen, unsigned nblocks, int *err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd((unsigned *)gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (clock64() - t0 > 2000000000LL) {
                    atomicExch(err, 1);
                    break;
                }
            }
        }
        __threadfence();
        if (*(volatile int *)err) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

// rotation of one FP32 pair (pc < qc) of W32 (columns of length m) and of V (length n), as
// k_jacobi_round_f32; all threads of the block take part; loads and stores through L2
__device__ void jacobi_pair_f32(float2 *W32, int m, float2 *V, int n, int pc, int qc, float tol,
                                unsigned long long *nrot, float4 *sh4, float *rot) {
    float2 *wp = W32 + (size_t)pc * m, *wq = W32 + (size_t)qc * m;
    float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const float2 x = __ldcg(&wp[i]), y = __ldcg(&wq[i]);
        al = fmaf(x.x, x.x, fmaf(x.y, x.y, al));
        be = fmaf(y.x, y.x, fmaf(y.y, y.y, be));
        gr = fmaf(x.x, y.x, fmaf(x.y, y.y, gr));   // conj(x) y
        gi = fmaf(x.x, y.y, fmaf(-x.y, y.x, gi));
    }
    block_sum4_f(al, be, gr, gi, sh4);
    if (threadIdx.x == 0) {
        // FP32 throughout: the FP32 sweeps only need FP32-accurate rotations (their product V is made
        // orthonormal to FP64 precision afterwards), and FP64 divisions and square roots here would sit
        // on every round's critical path
        const float g = hypotf(gr, gi);
        if (g == 0.f || g <= tol * sqrtf(al) * sqrtf(be)) {
            rot[0] = 0.f;
        } else {
            const float zeta = (be - al) / (2.f * g);
            const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + hypotf(1.f, zeta));
            const float cc = 1.f / sqrtf(fmaf(t, t, 1.f));   // correctly rounded: V accumulates ~10^4 rotations per column
            rot[0] = 1.f;
            rot[1] = cc;
            rot[2] = cc * t;
            rot[3] = gr / g;   // e^{-i phi} = conj(conj(w_p) w_q) / |.|
            rot[4] = -gi / g;
            atomicAdd(nrot, 1ull);
        }
    }
    __syncthreads();
    if (rot[0] == 0.f) return;   // uniform over the block
    const float cf = rot[1], sf = rot[2], er = rot[3], ei = rot[4];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const float2 x = __ldcg(&wp[i]), y0 = __ldcg(&wq[i]);
        const float2 y = make_float2(y0.x * er - y0.y * ei, y0.x * ei + y0.y * er);
        __stcg(&wp[i], make_float2(cf * x.x - sf * y.x, cf * x.y - sf * y.y));
        __stcg(&wq[i], make_float2(sf * x.x + cf * y.x, sf * x.y + cf * y.y));
    }
    float2 *vp = V + (size_t)pc * n, *vq = V + (size_t)qc * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 x = __ldcg(&vp[i]), y0 = __ldcg(&vq[i]);
        const float2 y = make_float2(y0.x * er - y0.y * ei, y0.x * ei + y0.y * er);
        __stcg(&vp[i], make_float2(cf * x.x - sf * y.x, cf * x.y - sf * y.y));
        __stcg(&vq[i], make_float2(sf * x.x + cf * y.x, sf * x.y + cf * y.y));
    }
}

// all npad - 1 rounds of the circle schedule; launched cooperatively (all blocks resident)
__global__ void __launch_bounds__(JTPB) k_jacobi_sweep_f32(float2 *W32, int m, float2 *V, int n, int npad, float tol,
                                                           unsigned long long *nrot, unsigned *bar, int *err) {
    __shared__ float4 sh4[32];
    __shared__ float rot[5];
    for (int r = 0; r < npad - 1; ++r) {
        for (int k = blockIdx.x; k < npad / 2; k += gridDim.x) {
            const int a = k == 0 ? 0 : ((k - 1 + r) % (npad - 1)) + 1;
            const int pb = npad - 1 - k;
            const int b = pb == 0 ? 0 : ((pb - 1 + r) % (npad - 1)) + 1;
            if (a < n && b < n) jacobi_pair_f32(W32, m, V, n, a < b ? a : b, a < b ? b : a, tol, nrot, sh4, rot);
            __syncthreads();   // rot and sh4 are reused by the block's next pair
        }
        if (!grid_barrier(bar, bar + 1, gridDim.x, err)) return;
    }
}

// ---- blocked FP32 sweep: super-columns of SC columns held in shared memory (cooperative) -----------
// The columns are grouped into super-columns of SC; a round of the circle schedule over the
// super-columns gives each block two of them.  The block copies their 2 SC columns of W32 into shared
// memory, rotates all SC^2 cross pairs there in SC local rounds of SC disjoint pairs (in the first
// round also the pairs inside each super-column), accumulates the local rotations into a 2SC x 2SC
// unitary Q, writes the columns back and applies Q to the same columns of V in one pass.  A sweep is
// then ceil(n / SC) - 1 grid rounds instead of n - 1, each moving the columns through L2 once, and
// every column pair is still rotated once per sweep (a block-cyclic ordering).
constexpr int SC = 6;
constexpr int SCT = SC * 64;   // two warps per pair slot

__device__ __forceinline__ int circle_player(int pos, int r, int np) {
    return pos == 0 ? 0 : ((pos - 1 + r) % (np - 1)) + 1;
}

__global__ void __launch_bounds__(SCT) k_jacobi_sweep_blk_f32(float2 *W32, int m, float2 *V, int n, int nsc, int nscp,
                                                              float tol, unsigned long long *nrot, unsigned *bar,
                                                              int *err) {
    extern __shared__ float2 xs[];   // 2 SC columns of length m
    __shared__ float2 Qc[2 * SC][2 * SC];   // Qc[j][i] = Q[i][j]: column j of Q
    __shared__ float4 red[SC][2];
    __shared__ float rot[SC][5];
    __shared__ int gcol[2 * SC];
    __shared__ unsigned cnt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pr = warp >> 1, half = warp & 1, tp = threadIdx.x & 63;

    // one local round: pair slot pr rotates local columns (lp, lq) if both exist
    auto local_round = [&](int lp, int lq) {
        const int gp = gcol[lp], gq = gcol[lq];
        const bool live = gp >= 0 && gq >= 0;
        if (live && gp > gq) {   // the lower global column plays p, as in the circle sweep
            const int t = lp;
            lp = lq;
            lq = t;
        }
        float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
        if (live) {
            const float2 *xp = xs + (size_t)lp * m, *xq = xs + (size_t)lq * m;
            for (int i = tp; i < m; i += 64) {
                const float2 x = xp[i], y = xq[i];
                al = fmaf(x.x, x.x, fmaf(x.y, x.y, al));
                be = fmaf(y.x, y.x, fmaf(y.y, y.y, be));
                gr = fmaf(x.x, y.x, fmaf(x.y, y.y, gr));   // conj(x) y
                gi = fmaf(x.x, y.y, fmaf(-x.y, y.x, gi));
            }
            al = warp_sum_f(al);
            be = warp_sum_f(be);
            gr = warp_sum_f(gr);
            gi = warp_sum_f(gi);
            if (lane == 0) red[pr][half] = make_float4(al, be, gr, gi);
        }
        __syncthreads();
        if (live && tp == 0) {
            const float4 u = red[pr][0], v = red[pr][1];
            al = u.x + v.x;
            be = u.y + v.y;
            gr = u.z + v.z;
            gi = u.w + v.w;
            const float g = hypotf(gr, gi);
            if (g == 0.f || g <= tol * sqrtf(al) * sqrtf(be)) {
                rot[pr][0] = 0.f;
            } else {
                const float zeta = (be - al) / (2.f * g);
                const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + hypotf(1.f, zeta));
                const float cc = 1.f / sqrtf(fmaf(t, t, 1.f));
                rot[pr][0] = 1.f;
                rot[pr][1] = cc;
                rot[pr][2] = cc * t;
                rot[pr][3] = gr / g;
                rot[pr][4] = -gi / g;
                atomicAdd(&cnt, 1u);
            }
        }
        __syncthreads();
        if (live && rot[pr][0] != 0.f) {
            const float cf = rot[pr][1], sf = rot[pr][2], er = rot[pr][3], ei = rot[pr][4];
            float2 *xp = xs + (size_t)lp * m, *xq = xs + (size_t)lq * m;
            for (int i = tp; i < m; i += 64) {
                const float2 x = xp[i], y0 = xq[i];
                const float2 y = make_float2(y0.x * er - y0.y * ei, y0.x * ei + y0.y * er);
                xp[i] = make_float2(cf * x.x - sf * y.x, cf * x.y - sf * y.y);
                xq[i] = make_float2(sf * x.x + cf * y.x, sf * x.y + cf * y.y);
            }
            if (tp < 2 * SC) {
                const float2 x = Qc[lp][tp], y0 = Qc[lq][tp];
                const float2 y = make_float2(y0.x * er - y0.y * ei, y0.x * ei + y0.y * er);
                Qc[lp][tp] = make_float2(cf * x.x - sf * y.x, cf * x.y - sf * y.y);
                Qc[lq][tp] = make_float2(sf * x.x + cf * y.x, sf * x.y + cf * y.y);
            }
        }
        __syncthreads();
    };

    for (int r = 0; r < nscp - 1; ++r) {
        for (int k = blockIdx.x; k < nscp / 2; k += gridDim.x) {
            const int A = circle_player(k, r, nscp), B = circle_player(nscp - 1 - k, r, nscp);
            if (threadIdx.x < 2 * SC) {
                const int sc = threadIdx.x < SC ? A : B, j = sc * SC + threadIdx.x % SC;
                gcol[threadIdx.x] = (sc < nsc && j < n) ? j : -1;
            }
            if (threadIdx.x < 4 * SC * SC) {
                const int j = threadIdx.x / (2 * SC), i = threadIdx.x % (2 * SC);
                Qc[j][i] = make_float2(i == j ? 1.f : 0.f, 0.f);
            }
            if (threadIdx.x == 0) cnt = 0;
            __syncthreads();
            // the 2 SC columns come in through L2 (written by other SMs in the previous round), the
            // loads of a row index all in flight at once
            for (int i = threadIdx.x; i < m; i += SCT) {
                float2 v[2 * SC];
#pragma unroll
                for (int l = 0; l < 2 * SC; ++l)
                    v[l] = gcol[l] >= 0 ? __ldcg(&W32[(size_t)gcol[l] * m + i]) : make_float2(0.f, 0.f);
#pragma unroll
                for (int l = 0; l < 2 * SC; ++l) xs[(size_t)l * m + i] = v[l];
            }
            __syncthreads();
            if (r == 0) {   // the pairs inside each super-column: a circle over its SC columns
                for (int t = 0; t < SC - 1; ++t) {
                    const int u = pr % (SC / 2), base = pr < SC / 2 ? 0 : SC;
                    local_round(base + circle_player(u, t, SC), base + circle_player(SC - 1 - u, t, SC));
                }
            }
            for (int t = 0; t < SC; ++t) local_round(pr, SC + (pr + t) % SC);
            for (int l = 0; l < 2 * SC; ++l) {
                if (gcol[l] < 0) continue;
                float2 *dst = W32 + (size_t)gcol[l] * m;
                for (int i = threadIdx.x; i < m; i += SCT) __stcg(&dst[i], xs[(size_t)l * m + i]);
            }
#pragma unroll 2
            for (int row = threadIdx.x; row < n; row += SCT) {
                float2 v[2 * SC];
#pragma unroll
                for (int l = 0; l < 2 * SC; ++l)
                    v[l] = gcol[l] >= 0 ? __ldcg(&V[(size_t)gcol[l] * n + row]) : make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < 2 * SC; ++j) {
                    if (gcol[j] < 0) continue;
                    float2 o = make_float2(0.f, 0.f);
#pragma unroll
                    for (int l = 0; l < 2 * SC; ++l) {
                        const float2 q = Qc[j][l];
                        o.x = fmaf(v[l].x, q.x, fmaf(-v[l].y, q.y, o.x));
                        o.y = fmaf(v[l].x, q.y, fmaf(v[l].y, q.x, o.y));
                    }
                    __stcg(&V[(size_t)gcol[j] * n + row], o);
                }
            }
            if (threadIdx.x == 0 && cnt) atomicAdd(nrot, (unsigned long long)cnt);
            __syncthreads();   // shared state is reused by the block's next super-column pair
        }
        if (!grid_barrier(bar, bar + 1, gridDim.x, err)) return;
    }
}

__global__ void k_identity_f32(float2 *V, int n) {
    long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)n * n) return;
    int r = (int)(id % n), c = (int)(id / n);
    V[id] = make_float2(r == c ? 1.f : 0.f, 0.f);
}

__global__ void k_to_c128(const float2 *__restrict__ X, long n, cplx *__restrict__ Y) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) Y[e] = C((double)X[e].x, (double)X[e].y);
}

// G <- 1.5 I - 0.5 G (Newton-Schulz step towards the orthogonal polar factor)
__global__ void k_ns_step(cplx *G, int n) {
    long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)n * n) return;
    int r = (int)(id % n), c = (int)(id / n);
    const cplx g = G[id];
    G[id] = C((r == c ? 1.5 : 0.0) - 0.5 * g.x, -0.5 * g.y);
}

// out[0] = max |G - I| (non-negative doubles order like their bit patterns), out[1] (a double) +=
// ||G - I||_F^2; 256 threads per block
__global__ void __launch_bounds__(256) k_offdiag_max(const cplx *G, int n, unsigned long long *out) {
    __shared__ double ssq[8];
    long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0, q = 0.0;
    if (id < (long)n * n) {
        int r = (int)(id % n), c = (int)(id / n);
        const cplx g = G[id];
        const double re = g.x - (r == c ? 1.0 : 0.0);
        v = hypot(re, g.y);
        q = re * re + g.y * g.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(v));
        ssq[threadIdx.x >> 5] = q;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += ssq[w];
        atomicAdd((double *)(out + 1), t);
    }
}

// C = A^H B, complex128, all n x n column-major
__global__ void __launch_bounds__(256) k_zgemm_hn(const cplx *__restrict__ A, const cplx *__restrict__ B,
                                                  cplx *__restrict__ Cm, int n);

// C = A B, complex128, all n x n column-major (64 x 64 tile per block, 4 x 4 per thread); with
// LOWER_A, A is lower triangular (R^*) and a row tile stops at its last non-zero column
constexpr int ZG = 64, ZK = 8;
template <bool LOWER_A = false>
__global__ void __launch_bounds__(256) k_zgemm_nn(const cplx *__restrict__ A, const cplx *__restrict__ B,
                                                  cplx *__restrict__ Cm, int n) {
    __shared__ cplx As[ZK][ZG + 1], Bs[ZK][ZG + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * ZG, j0 = blockIdx.y * ZG;
    const int kend = LOWER_A ? min(n, i0 + ZG) : n;
    cplx acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = C(0.0, 0.0);
    for (int k0 = 0; k0 < kend; k0 += ZK) {
        __syncthreads();
        for (int e = threadIdx.x; e < ZG * ZK; e += 256) {
            const int i = e % ZG, k = e / ZG;
            As[k][i] = (i0 + i < n && k0 + k < n) ? A[(size_t)(k0 + k) * n + i0 + i] : C(0.0, 0.0);
            const int kk = e % ZK, j = e / ZK;
            Bs[kk][j] = (k0 + kk < n && j0 + j < n) ? B[(size_t)(j0 + j) * n + k0 + kk] : C(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < ZK; ++k) {
            cplx a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = i0 + ty + 16 * i;
        if (row >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = j0 + tx + 16 * j;
            if (col < n) Cm[(size_t)col * n + row] = acc[i][j];
        }
    }
}

__global__ void __launch_bounds__(256) k_zgemm_hn(const cplx *__restrict__ A, const cplx *__restrict__ B,
                                                  cplx *__restrict__ Cm, int n) {
    __shared__ cplx As[ZK][ZG + 1], Bs[ZK][ZG + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * ZG, j0 = blockIdx.y * ZG;
    cplx acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = C(0.0, 0.0);
    for (int k0 = 0; k0 < n; k0 += ZK) {
        __syncthreads();
        for (int e = threadIdx.x; e < ZG * ZK; e += 256) {
            const int kk = e % ZK, idx = e / ZK;
            // (A^H)[i][k] = conj(A[k][i]); column i of A is contiguous in k
            As[kk][idx] = (i0 + idx < n && k0 + kk < n) ? cconj(A[(size_t)(i0 + idx) * n + k0 + kk]) : C(0.0, 0.0);
            Bs[kk][idx] = (k0 + kk < n && j0 + idx < n) ? B[(size_t)(j0 + idx) * n + k0 + kk] : C(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < ZK; ++k) {
            cplx a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = i0 + ty + 16 * i;
        if (row >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = j0 + tx + 16 * j;
            if (col < n) Cm[(size_t)col * n + row] = acc[i][j];
        }
    }
}

// ---- one FP32 Newton-Schulz step on the FP32 rotations (end of the FP32 sweeps) --------------------
// V32 collects ~10^4 FP32 rotations per column and leaves the FP32 sweeps ~1e-4..1e-3 from orthogonal;
// one FP32 step V <- V (3I - V^H V)/2 brings it to the FP32 floor (~1e-6), so that the FP64 steps
// that follow start there.  Complex FP32 GEMMs with the tiling of the FP64 ones below.
__device__ __forceinline__ void cfma_f(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

// C = A^H B (conj_a) or A B, complex64, all n x n column-major (64 x 64 tile per block, 4 x 4 per thread)
template <bool CONJ_A>
__global__ void __launch_bounds__(256) k_cgemm_f32(const float2 *__restrict__ A, const float2 *__restrict__ B,
                                                   float2 *__restrict__ Cm, int n) {
    constexpr int TG = 64, TK = 8;
    __shared__ float2 As[TK][TG + 1], Bs[TK][TG + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * TG, j0 = blockIdx.y * TG;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < n; k0 += TK) {
        __syncthreads();
        for (int e = threadIdx.x; e < TG * TK; e += 256) {
            if (CONJ_A) {   // (A^H)[i][k] = conj(A[k][i]); column i of A is contiguous in k
                const int kk = e % TK, idx = e / TK;
                float2 v = make_float2(0.f, 0.f);
                if (i0 + idx < n && k0 + kk < n) {
                    v = A[(size_t)(i0 + idx) * n + k0 + kk];
                    v.y = -v.y;
                }
                As[kk][idx] = v;
            } else {
                const int i = e % TG, k = e / TG;
                As[k][i] = (i0 + i < n && k0 + k < n) ? A[(size_t)(k0 + k) * n + i0 + i] : make_float2(0.f, 0.f);
            }
            const int kk = e % TK, j = e / TK;
            Bs[kk][j] = (k0 + kk < n && j0 + j < n) ? B[(size_t)(j0 + j) * n + k0 + kk] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; ++k) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma_f(acc[i][j], a[i], b[j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = i0 + ty + 16 * i;
        if (row >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = j0 + tx + 16 * j;
            if (col < n) Cm[(size_t)col * n + row] = acc[i][j];
        }
    }
}

// G <- 1.5 I - 0.5 G in complex64
__global__ void k_ns_step_f32(float2 *G, int n) {
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)n * n) return;
    const int r = (int)(id % n), c = (int)(id / n);
    const float2 g = G[id];
    G[id] = make_float2((r == c ? 1.5f : 0.f) - 0.5f * g.x, -0.5f * g.y);
}

__global__ void k_sigma(const cplx *W, int m, int n, double eps, double *sigma, double *coef) {
    int col = blockIdx.x;
    if (col >= n) return;
    __shared__ double sh[32];
    const cplx *a = W + (size_t)col * m;
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s = abs2_acc(a[i], s);
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


// ---- Householder QR with column pivoting ----------------------------------------------------------

// Pivot + reflector for step j (single block): p = argmax_{k >= j} nrm2[k]; swap columns j and p;
// H = I - tau v v^*, v = [1; x/(x0 - beta)], beta = -sign(Re x0) ||A[j:, j]||, tau = (beta - x0)/beta,
// so that H^* A[j:, j] = beta e_1 (the LAPACK zlarfg convention).
__global__ void __launch_bounds__(1024) k_qr_pivot_house(cplx *A, int m, int n, int j, double *nrm2, int *perm,
                                                        cplx *tau) {
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ double shs[32];
    __shared__ int piv;
    __shared__ cplx hb[2];   // beta (real in .x), scale 1/(x0 - beta)
    double best = -1.0;
    int bi = j;
    for (int k = j + threadIdx.x; k < n; k += blockDim.x) {
        double v = nrm2[k];
        if (v > best) {
            best = v;
            bi = k;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
        }
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0) {
        sv[w] = best;
        si[w] = bi;
    }
    __syncthreads();
    if (w == 0) {
        best = l < nw ? sv[l] : -1.0;
        bi = l < nw ? si[l] : n;
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (l == 0) piv = bi;
    }
    __syncthreads();
    const int p = piv;
    if (p != j) {
        cplx *a = A + (size_t)j * m, *b = A + (size_t)p * m;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            cplx t = a[i];
            a[i] = b[i];
            b[i] = t;
        }
        if (threadIdx.x == 0) {
            double t = nrm2[j];
            nrm2[j] = nrm2[p];
            nrm2[p] = t;
            int ti = perm[j];
            perm[j] = perm[p];
            perm[p] = ti;
        }
    }
    __syncthreads();
    cplx *a = A + (size_t)j * m;
    double s2 = 0.0;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) s2 = abs2_acc(a[i], s2);
    s2 = block_sum(s2, shs);
    if (threadIdx.x == 0) {
        cplx x0 = a[j];
        if (s2 == 0.0 && x0.y == 0.0) {
            tau[j] = C(0.0, 0.0);
            hb[0] = C(x0.x, 0.0);
            hb[1] = C(0.0, 0.0);
        } else {
            double beta = -copysign(sqrt(cabs2(x0) + s2), x0.x);
            tau[j] = C((beta - x0.x) / beta, -x0.y / beta);
            hb[0] = C(beta, 0.0);
            hb[1] = cdiv(C(1.0, 0.0), C(x0.x - beta, x0.y));
        }
    }
    __syncthreads();
    cplx sc = hb[1];
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) a[i] = cmul(a[i], sc);
    if (threadIdx.x == 0) a[j] = hb[0];
}

// Applies H_j^* to trailing column k = j + 1 + blockIdx.x and recomputes its trailing norm.
__global__ void k_qr_apply(cplx *A, int m, int n, int j, const cplx *tau, double *nrm2) {
    int k = j + 1 + blockIdx.x;
    if (k >= n) return;
    __shared__ double sh[32];
    const cplx *v = A + (size_t)j * m;   // v_j = 1 implicit, v_i = A[i, j] for i > j
    cplx *a = A + (size_t)k * m;
    double wr = 0.0, wi = 0.0;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
        cplx vi = (i == j) ? C(1.0, 0.0) : v[i];
        cplx ai = a[i];
        cdot_acc(wr, wi, vi, ai);
    }
    wr = block_sum(wr, sh);
    wi = block_sum(wi, sh);
    cplx f = cmul(cconj(tau[j]), C(wr, wi));   // conj(tau) (v^* a)
    double s2 = 0.0;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
        cplx vi = (i == j) ? C(1.0, 0.0) : v[i];
        cplx ai = csub_mul(a[i], f, vi);
        a[i] = ai;
        if (i > j) s2 = abs2_acc(ai, s2);
    }
    s2 = block_sum(s2, sh);
    if (threadIdx.x == 0) nrm2[k] = s2;
}

__global__ void k_colnorm2(const cplx *A, int m, int n, double *nrm2) {
    int col = blockIdx.x;
    if (col >= n) return;
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s = abs2_acc(A[(size_t)col * m + i], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) nrm2[col] = s;
}

__global__ void k_iota(int *p, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

// X = R^* (n x n, column-major, lower triangular): X[i, j] = conj(R[j, i]) for i >= j
__global__ void k_r_adjoint(const cplx *A, int m, int n, cplx *X) {
    long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)n * n) return;
    int i = (int)(id % n), j = (int)(id / n);
    X[id] = (i >= j) ? cconj(A[(size_t)i * m + j]) : C(0.0, 0.0);
}

// Y (m x n, column-major) = [Vx; 0]
__global__ void k_pad_rows(const cplx *Vx, int n, int m, cplx *Y) {
    long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)m * n) return;
    int i = (int)(id % m), j = (int)(id / m);
    Y[id] = (i < n) ? Vx[(size_t)j * n + i] : C(0.0, 0.0);
}

// Y[j:, col] = H_j Y[j:, col] = Y - tau_j v (v^* Y), block per column col
__global__ void k_apply_reflector(const cplx *Aqr, int m, int j, const cplx *tau, cplx *Y, int ncols) {
    int col = blockIdx.x;
    if (col >= ncols) return;
    __shared__ double sh[32];
    const cplx *v = Aqr + (size_t)j * m;
    cplx *y = Y + (size_t)col * m;
    double wr = 0.0, wi = 0.0;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
        cplx vi = (i == j) ? C(1.0, 0.0) : v[i];
        cplx yi = y[i];
        cdot_acc(wr, wi, vi, yi);
    }
    wr = block_sum(wr, sh);
    wi = block_sum(wi, sh);
    cplx f = cmul(tau[j], C(wr, wi));
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
        cplx vi = (i == j) ? C(1.0, 0.0) : v[i];
        y[i] = csub_mul(y[i], f, vi);
    }
}

// Y[:, col] = H_0 H_1 ... H_{nr-1} Y[:, col] for every column at once, block per column: the column
// stays in shared memory (m complex values) while the reflectors are applied from the last to the
// first, in one launch instead of one launch per reflector (the columns are independent; each
// column's arithmetic is that of k_apply_reflector, in the same order)
__global__ void __launch_bounds__(256) k_apply_reflectors_all(const cplx *__restrict__ Aqr, int m, int nr,
                                                              const cplx *__restrict__ tau, cplx *__restrict__ Y,
                                                              int ncols) {
    extern __shared__ cplx ys[];
    __shared__ double sh[32];
    const int col = blockIdx.x;
    if (col >= ncols) return;
    cplx *y = Y + (size_t)col * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = y[i];
    __syncthreads();
    for (int j = nr - 1; j >= 0; --j) {
        const cplx *v = Aqr + (size_t)j * m;
        double wr = 0.0, wi = 0.0;
        for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
            const cplx vi = (i == j) ? C(1.0, 0.0) : __ldg(&v[i]);
            const cplx yi = ys[i];
            cdot_acc(wr, wi, vi, yi);
        }
        wr = block_sum(wr, sh);
        wi = block_sum(wi, sh);
        const cplx f = cmul(tau[j], C(wr, wi));
        for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
            const cplx vi = (i == j) ? C(1.0, 0.0) : __ldg(&v[i]);
            ys[i] = csub_mul(ys[i], f, vi);
        }
        __syncthreads();   // the next reflector's inner product reads entries other threads updated
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] = ys[i];
}

// Vr (row-major) = P W_x: row perm[i] of Vr is row i of W_x (column-major n x n)
__global__ void k_permute_rows(const cplx *Wx, int n, const int *perm, cplx *Vr) {
    long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)n * n) return;
    int i = (int)(id % n), j = (int)(id / n);
    Vr[(size_t)perm[i] * n + j] = Wx[id];
}

// Rounds of disjoint pairs for the nv pairs listed at dlist (device): taken in column order (so that
// the factorisation does not depend on the order in which the device listed them), each pair goes to
// the round after the later of its two columns' last rounds.  The pairs are written round by round
// to dsched (device) and round r holds dsched[rstart[r] .. rstart[r+1]).
int schedule_pairs(gs_ctx *c, const int2 *dlist, size_t nv, int n, int2 *dsched, std::vector<int> &rstart,
                   std::vector<int2> &hp, std::vector<int2> &hs) {
    hp.resize(nv);
    GS_CUDA(c, cudaMemcpyAsync(hp.data(), dlist, sizeof(int2) * nv, cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    std::sort(hp.begin(), hp.end(), [](int2 u, int2 v) { return u.x != v.x ? u.x < v.x : u.y < v.y; });
    std::vector<int> last(n, -1), rnd(nv);
    int nr = 0;
    for (size_t q = 0; q < nv; ++q) {
        const int r = std::max(last[hp[q].x], last[hp[q].y]) + 1;
        last[hp[q].x] = last[hp[q].y] = r;
        rnd[q] = r;
        nr = std::max(nr, r + 1);
    }
    rstart.assign(nr + 1, 0);
    for (size_t q = 0; q < nv; ++q) ++rstart[rnd[q] + 1];
    for (int r = 0; r < nr; ++r) rstart[r + 1] += rstart[r];
    hs.resize(nv);
    std::vector<int> pos(rstart.begin(), rstart.end() - 1);
    for (size_t q = 0; q < nv; ++q) hs[pos[rnd[q]]++] = hp[q];
    GS_CUDA(c, cudaMemcpyAsync(dsched, hs.data(), sizeof(int2) * nv, cudaMemcpyHostToDevice, c->stream));
    return GS_OK;
}

}  // namespace

int gs_factor_angle(gs_ctx *c, AngleData &a) {
    const Layout &ly = c->lay;
    const int m = ly.rows, n = ly.cols;
    cudaStream_t st = c->stream;
    a.A2_ready = false;   // W, Vr and coef are rewritten: their double-float copies are stale
    a.A2_off = false;
    cplx *Aqr = c->Vtmp;                       // m x n: scaled A, then R and the reflectors
    cplx *X = c->Xtmp;                         // n x n: R^*, rotated into W_x
    cplx *Vx = c->Vxtmp;                       // n x n: accumulated rotations
    double *nrm2 = c->nrm2;
    int *perm = c->perm;
    cplx *tau = c->tau;
    // phase timing: assembly, QR, FP32 sweeps, polar step + R^* V, FP64 sweeps, U and V Sigma
    struct Ev {
        cudaEvent_t e[7] = {};
        ~Ev() {
            for (auto &x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    for (auto &x : ev.e) GS_CUDA(c, cudaEventCreate(&x));
    GS_CUDA(c, cudaEventRecord(ev.e[0], st));
    GS_TRY(gs_assemble_A(c, a, Aqr, m));
    GS_TRY(gs_assemble_f(c, a, a.f));
    GS_COUNT_LAUNCH(c);
    k_fill<<<(n + 255) / 256, 256, 0, st>>>(a.dscale, n, 1.0);
    GS_COUNT_LAUNCH(c);
    k_colnorm_scale<<<ly.col_c - ly.col_a2, 256, 0, st>>>(Aqr, m, m, ly.col_a2, ly.col_c, a.dscale);
    // 1. QR with column pivoting
    GS_CUDA(c, cudaEventRecord(ev.e[1], st));
    GS_COUNT_LAUNCH(c);
    k_colnorm2<<<n, 256, 0, st>>>(Aqr, m, n, nrm2);
    GS_COUNT_LAUNCH(c);
    k_iota<<<(n + 255) / 256, 256, 0, st>>>(perm, n);
    for (int j = 0; j < n; ++j) {
        GS_COUNT_LAUNCH(c);
        k_qr_pivot_house<<<1, 1024, 0, st>>>(Aqr, m, n, j, nrm2, perm, tau);
        if (j + 1 < n) {
            GS_COUNT_LAUNCH(c);
            k_qr_apply<<<n - j - 1, 256, 0, st>>>(Aqr, m, n, j, tau, nrm2);
        }
    }
    GS_CHECK_LAUNCH(c);
    // 2. one-sided Jacobi on X = R^*
    GS_CUDA(c, cudaEventRecord(ev.e[2], st));
    GS_COUNT_LAUNCH(c);
    k_r_adjoint<<<(int)(((long)n * n + 255) / 256), 256, 0, st>>>(Aqr, m, n, X);
    GS_COUNT_LAUNCH(c);
    k_identity<<<(int)(((long)n * n + 255) / 256), 256, 0, st>>>(Vx, n);
    GS_CHECK_LAUNCH(c);
    int npad = n + (n & 1);
    // 2a. FP32 sweeps on a copy of R^*, rotations accumulated in FP32, until no pair is further
    //     than 1e-5 from orthogonal at FP32 resolution
    const long nn = (long)n * n;
    const int eb = (int)((nn + 255) / 256);
    float2 *X32 = c->X32tmp, *V32 = c->X32tmp + nn;
    GS_COUNT_LAUNCH(c);
    k_to_c64<<<eb, 256, 0, st>>>(X, nn, X32);
    GS_COUNT_LAUNCH(c);
    k_identity_f32<<<eb, 256, 0, st>>>(V32, n);
    GS_CHECK_LAUNCH(c);
    a.sweeps32 = 0;
    for (int q = 0; q < 32; ++q) a.rot32[q] = a.rot64[q] = 0;
    // Once a sweep has rotated fewer than half of the pairs, the next ones start from the FP32 Gram
    // matrix X32^H X32 and rotate only the pairs it lists (as the FP64 sweeps below)
    const dim3 zg((n + ZG - 1) / ZG, (n + ZG - 1) / ZG);
    const long npairs = (long)n * (n - 1) / 2;
    int2 *vlist = (int2 *)a.W, *vsched = vlist + npairs;   // a.W (m x n complex128) is free until step 2b
    std::vector<int2> hpairs, hsched;
    std::vector<int> rstart;
    long long prev_rot = npairs;
    // one cooperative launch per sweep when all its blocks can be resident, else one launch per round;
    // the blocked form when two super-columns of W32 fit the shared memory of a block
    int coop = 0, per_sm = 0, dev_coop = 0, blk = 0, smem_optin = 0;
    const int nsc = (n + SC - 1) / SC, nscp = nsc + (nsc & 1);
    const size_t blk_smem = sizeof(float2) * 2 * SC * (size_t)n;
    cudaDeviceGetAttribute(&dev_coop, cudaDevAttrCooperativeLaunch, c->device);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (dev_coop && blk_smem + 4096 <= (size_t)smem_optin &&
        cudaFuncSetAttribute(k_jacobi_sweep_blk_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)blk_smem) ==
            cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_sweep_blk_f32, SCT, blk_smem) == cudaSuccess &&
        per_sm > 0)
        blk = std::min(nscp / 2, per_sm * c->sms);
    if (dev_coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_sweep_f32, JTPB, 0) == cudaSuccess)
        coop = std::min(npad / 2, per_sm * c->sms);
    cudaGetLastError();
    for (int sweep = 0; sweep < 20; ++sweep) {
        GS_CUDA(c, cudaMemsetAsync(c->dcount, 0, 2 * sizeof(unsigned long long), st));
        bool circle = true;
        if (sweep > 0 && npairs > 0 && 2 * prev_rot < npairs) {
            float2 *G32 = (float2 *)a.Vr;
            GS_COUNT_LAUNCH(c);
            k_cgemm_f32<true><<<zg, 256, 0, st>>>(X32, X32, G32, n);
            GS_COUNT_LAUNCH(c);
            k_gram_violators_f32<<<eb, 256, 0, st>>>(G32, n, 1e-5f, vlist, c->dcount + 1);
            GS_CHECK_LAUNCH(c);
            unsigned long long nv = 0;
            GS_CUDA(c, cudaMemcpyAsync(&nv, c->dcount + 1, sizeof(nv), cudaMemcpyDeviceToHost, st));
            GS_CUDA(c, cudaStreamSynchronize(st));
            if (nv == 0) {
                a.sweeps32 = sweep + 1;
                a.rot32[sweep] = 0;
                break;
            }
            // listed rounds unless there are more of them than a circle sweep has
            if ((long)nv <= npairs / 4) GS_TRY(schedule_pairs(c, vlist, nv, n, vsched, rstart, hpairs, hsched));
            if ((long)nv <= npairs / 4 && (int)rstart.size() - 1 <= npad - 1) {
                circle = false;
                const int nr = (int)rstart.size() - 1;
                for (int r = 0; r < nr; ++r) {
                    GS_COUNT_LAUNCH(c);
                    k_jacobi_pairs_f32<<<rstart[r + 1] - rstart[r], JTPB, 0, st>>>(X32, n, V32, n, vsched + rstart[r],
                                                                                1e-5f, c->dcount);
                }
                GS_CHECK_LAUNCH(c);
            }
        }
        if (circle && blk > 0) {
            GS_CUDA(c, cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned), st));
            GS_CUDA(c, cudaMemsetAsync(c->terr, 0, sizeof(int), st));
            float tol32 = 1e-5f;
            int mm = n, nn_ = n, nsc_ = nsc, nscp_ = nscp;
            void *args[] = {&X32, &mm, &V32, &nn_, &nsc_, &nscp_, &tol32, &c->dcount, &c->bar, &c->terr};
            GS_COUNT_LAUNCH(c);
            GS_CUDA(c, cudaLaunchCooperativeKernel((const void *)k_jacobi_sweep_blk_f32, dim3(blk), dim3(SCT), args,
                                                   blk_smem, st));
        } else if (circle && coop > 0) {
            GS_CUDA(c, cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned), st));
            GS_CUDA(c, cudaMemsetAsync(c->terr, 0, sizeof(int), st));
            float tol32 = 1e-5f;
            int mm = n, nn_ = n, np_ = npad;
            void *args[] = {&X32, &mm, &V32, &nn_, &np_, &tol32, &c->dcount, &c->bar, &c->terr};
            GS_COUNT_LAUNCH(c);
            GS_CUDA(c, cudaLaunchCooperativeKernel((const void *)k_jacobi_sweep_f32, dim3(coop), dim3(JTPB), args, 0, st));
        } else if (circle) {
            for (int r = 0; r < npad - 1; ++r) {
                GS_COUNT_LAUNCH(c);
                k_jacobi_round_f32<<<npad / 2, JTPB, 0, st>>>(X32, n, V32, n, r, npad, 1e-5f, c->dcount);
            }
        }
        GS_CHECK_LAUNCH(c);
        if (circle && (blk > 0 || coop > 0)) {
            int herr = 0;
            GS_CUDA(c, cudaMemcpyAsync(&herr, c->terr, sizeof(int), cudaMemcpyDeviceToHost, st));
            GS_CUDA(c, cudaStreamSynchronize(st));
            if (herr) {
                GS_CUDA(c, cudaMemsetAsync(c->terr, 0, sizeof(int), st));
                return gs_fail(c, GS_ERR_TIMEOUT, "grating factorisation: a grid barrier wait gave up");
            }
        }
        unsigned long long h = 0;
        GS_CUDA(c, cudaMemcpyAsync(&h, c->dcount, sizeof(h), cudaMemcpyDeviceToHost, st));
        GS_CUDA(c, cudaStreamSynchronize(st));
        a.sweeps32 = sweep + 1;
        a.rot32[sweep] = (long long)h;
        prev_rot = (long long)h;
        if (h == 0) break;
    }
    GS_CUDA(c, cudaEventRecord(ev.e[3], st));
    // 2b. V_x = the FP64 orthogonal polar factor of V32 (Newton-Schulz, V <- V (3I - V^H V)/2, a defect
    //     e of V^H V - I going to 0.75 e^2 - 0.25 e^3: one step in FP32, then FP64), X = R^* V_x in FP64
    cplx *G = a.Vr, *T = a.W;   // n x n scratch (both are written later)
    {
        // one FP32 step first (its G32 and T32 in the n x n complex128 scratch G, two complex64 halves)
        float2 *G32 = (float2 *)G, *T32 = (float2 *)G + nn;
        GS_COUNT_LAUNCH(c);
        k_cgemm_f32<true><<<zg, 256, 0, st>>>(V32, V32, G32, n);
        GS_COUNT_LAUNCH(c);
        k_ns_step_f32<<<eb, 256, 0, st>>>(G32, n);
        GS_COUNT_LAUNCH(c);
        k_cgemm_f32<false><<<zg, 256, 0, st>>>(V32, G32, T32, n);
        GS_CHECK_LAUNCH(c);
        GS_CUDA(c, cudaMemcpyAsync(V32, T32, sizeof(float2) * nn, cudaMemcpyDeviceToDevice, st));
    }
    GS_COUNT_LAUNCH(c);
    k_to_c128<<<eb, 256, 0, st>>>(V32, nn, Vx);
    double prev_defect = 1.0;
    for (int q = 0; q < 6; ++q) a.ns_defect[q] = 0.0;
    a.ns_iters = 6;
    for (int it = 0; it < 6; ++it) {
        GS_COUNT_LAUNCH(c);
        k_zgemm_hn<<<zg, 256, 0, st>>>(Vx, Vx, G, n);
        GS_CUDA(c, cudaMemsetAsync(c->dcount, 0, 2 * sizeof(unsigned long long), st));
        GS_COUNT_LAUNCH(c);
        k_offdiag_max<<<eb, 256, 0, st>>>(G, n, c->dcount);
        GS_CHECK_LAUNCH(c);
        unsigned long long hb[2] = {0, 0};
        GS_CUDA(c, cudaMemcpyAsync(hb, c->dcount, sizeof(hb), cudaMemcpyDeviceToHost, st));
        GS_CUDA(c, cudaStreamSynchronize(st));
        double defect, fro2;
        std::memcpy(&defect, &hb[0], sizeof(defect));
        std::memcpy(&fro2, &hb[1], sizeof(fro2));
        if (!(defect < 0.5)) return gs_fail(c, GS_ERR_NUMERIC, "grating factorisation: FP32 rotations not orthogonal");
        // Stop when V is as orthogonal as FP64 can show.  A step maps a defect d to about 0.75 d^2, but
        // the FP64 Gram matrix itself carries rounding of sqrt(n) eps to n eps (4.5e-15 to 1.9e-13 at
        // n = 1689): a small measured defect far above the previous one's square is that rounding
        a.ns_defect[it] = defect;
        a.ns_iters = it;
        if (defect < 1e-14) break;
        if (it > 0 && defect < 1e-10 && defect > 100.0 * 0.75 * prev_defect * prev_defect) break;
        prev_defect = defect;
        // ||V^H V - I||_2 <= ||V^H V - I||_F, and a step leaves at most 0.75 x^2 + 0.25 x^3 of a
        // spectral defect x: below x = 1e-7 the step about to be taken ends below 1e-14, where the
        // loop stops anyway, so the Gram matrix need not be formed again to see it
        const double xf = std::sqrt(fro2);
        const bool last = xf < 1e-7;
        GS_COUNT_LAUNCH(c);
        k_ns_step<<<eb, 256, 0, st>>>(G, n);
        GS_COUNT_LAUNCH(c);
        k_zgemm_nn<<<zg, 256, 0, st>>>(Vx, G, T, n);
        GS_CUDA(c, cudaMemcpyAsync(Vx, T, sizeof(cplx) * nn, cudaMemcpyDeviceToDevice, st));
        if (last && it + 1 < 6) {
            a.ns_defect[it + 1] = 0.75 * xf * xf + 0.25 * xf * xf * xf;   // the bound, not a measurement
            a.ns_iters = it + 1;
            break;
        }
    }
    GS_COUNT_LAUNCH(c);
    k_zgemm_nn<true><<<zg, 256, 0, st>>>(X, Vx, T, n);
    GS_CHECK_LAUNCH(c);
    GS_CUDA(c, cudaMemcpyAsync(X, T, sizeof(cplx) * nn, cudaMemcpyDeviceToDevice, st));
    GS_CUDA(c, cudaEventRecord(ev.e[4], st));
    const double tol = 1e-14;
    a.sweeps = 0;
    // From the third sweep on the pairs still to rotate are few (~1% of them, then a handful): the
    // Gram matrix X^H X (one FP64 GEMM, at several times the FP64 rate of a dots-only circle sweep)
    // finds them, and only they are rotated, in rounds of disjoint pairs.  A sweep ends the phase
    // when the Gram matrix shows no pair further than tol from orthogonal or when none of the
    // listed pairs, re-tested from its columns, needs a rotation.
    // After a listed pass that touched few columns, only the pairs involving those columns can have
    // moved since the last check (every other pair was below tol then and is unchanged), so the next
    // check computes just their inner products from the columns instead of the whole Gram matrix.
    constexpr int TMAX = 128;
    int *dcols = (int *)(vsched + npairs), *dinT = dcols + TMAX;   // after both pair lists in a.W
    std::vector<int> tcols, tflag;
    bool partial = false;
    const bool room_t = (size_t)m * n * sizeof(cplx) >= sizeof(int2) * 2 * (size_t)npairs + sizeof(int) * (TMAX + n);
    for (int sweep = 0; sweep < 30; ++sweep) {
        GS_CUDA(c, cudaMemsetAsync(c->dcount, 0, 2 * sizeof(unsigned long long), st));
        bool circle = true;
        if (sweep >= 2 && npairs > 0) {
            if (partial) {
                tflag.assign(n, 0);
                for (int q : tcols) tflag[q] = 1;
                GS_CUDA(c, cudaMemcpyAsync(dcols, tcols.data(), sizeof(int) * tcols.size(), cudaMemcpyHostToDevice, st));
                GS_CUDA(c, cudaMemcpyAsync(dinT, tflag.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
                const long warps = (long)tcols.size() * n;
                GS_COUNT_LAUNCH(c);
                k_cols_violators<<<(int)((warps * 32 + 255) / 256), 256, 0, st>>>(X, n, n, dcols, (int)tcols.size(),
                                                                                 dinT, tol, vlist, c->dcount + 1);
            } else {
                GS_COUNT_LAUNCH(c);
                k_zgemm_hn<<<zg, 256, 0, st>>>(X, X, G, n);
                GS_COUNT_LAUNCH(c);
                k_gram_violators<<<eb, 256, 0, st>>>(G, n, tol, vlist, c->dcount + 1);
            }
            GS_CHECK_LAUNCH(c);
            unsigned long long nv = 0;
            GS_CUDA(c, cudaMemcpyAsync(&nv, c->dcount + 1, sizeof(nv), cudaMemcpyDeviceToHost, st));
            GS_CUDA(c, cudaStreamSynchronize(st));
            if (nv == 0) {
                a.sweeps = sweep + 1;
                if (sweep < 32) a.rot64[sweep] = 0;
                break;
            }
            if ((long)nv <= npairs / 4) GS_TRY(schedule_pairs(c, vlist, nv, n, vsched, rstart, hpairs, hsched));
            if ((long)nv <= npairs / 4 && (int)rstart.size() - 1 <= npad - 1) {
                circle = false;
                const int nr = (int)rstart.size() - 1;
                for (int r = 0; r < nr; ++r) {
                    GS_COUNT_LAUNCH(c);
                    k_jacobi_pairs<<<rstart[r + 1] - rstart[r], JTPB, 0, st>>>(X, n, Vx, n, vsched + rstart[r], tol,
                                                                            c->dcount);
                }
                GS_CHECK_LAUNCH(c);
                // the columns this pass touched (hpairs holds its listed pairs)
                tcols.clear();
                tflag.assign(n, 0);
                for (const int2 &pq : hpairs) {
                    for (int q : {pq.x, pq.y})
                        if (!tflag[q]) {
                            tflag[q] = 1;
                            tcols.push_back(q);
                        }
                    if ((int)tcols.size() > TMAX) break;
                }
            }
        }
        partial = !circle && (int)tcols.size() <= TMAX && room_t;
        if (circle) {
            for (int r = 0; r < npad - 1; ++r) {
                GS_COUNT_LAUNCH(c);
                k_jacobi_round<<<npad / 2, JTPB, 0, st>>>(X, n, Vx, n, r, npad, tol, c->dcount);
            }
        }
        GS_CHECK_LAUNCH(c);
        unsigned long long h = 0;
        GS_CUDA(c, cudaMemcpyAsync(&h, c->dcount, sizeof(h), cudaMemcpyDeviceToHost, st));
        GS_CUDA(c, cudaStreamSynchronize(st));
        a.sweeps = sweep + 1;
        if (sweep < 32) a.rot64[sweep] = (long long)h;
        if (h == 0) break;
    }
    GS_CUDA(c, cudaEventRecord(ev.e[5], st));
    GS_COUNT_LAUNCH(c);
    k_sigma<<<n, 256, 0, st>>>(X, n, n, c->L.eps_pinv, a.sigma, a.coef);
    // 3. U = Q V_x (reflectors applied to [V_x; 0] in reverse order), V Sigma = P W_x
    GS_COUNT_LAUNCH(c);
    k_pad_rows<<<(int)(((long)m * n + 255) / 256), 256, 0, st>>>(Vx, n, m, a.W);
    if ((size_t)m * sizeof(cplx) <= 48 * 1024) {   // the column fits the default shared memory
        GS_COUNT_LAUNCH(c);
        k_apply_reflectors_all<<<n, 256, (size_t)m * sizeof(cplx), st>>>(Aqr, m, n, tau, a.W, n);
    } else {
        for (int j = n - 1; j >= 0; --j) {
            GS_COUNT_LAUNCH(c);
            k_apply_reflector<<<n, 256, 0, st>>>(Aqr, m, j, tau, a.W, n);
        }
    }
    GS_COUNT_LAUNCH(c);
    k_permute_rows<<<(int)(((long)n * n + 255) / 256), 256, 0, st>>>(X, n, perm, a.Vr);
    GS_CHECK_LAUNCH(c);
    GS_CUDA(c, cudaEventRecord(ev.e[6], st));
    GS_CUDA(c, cudaEventSynchronize(ev.e[6]));
    for (int q = 0; q < 6; ++q) {
        float ms = 0.f;
        GS_CUDA(c, cudaEventElapsedTime(&ms, ev.e[q], ev.e[q + 1]));
        a.phase_ms[q] = ms;
    }
    return GS_OK;
}

int gs_factor_stats(gs_ctx *c, int angle, int *sweeps32, int *sweeps64, double *phase_ms, long long *rot32,
                    long long *rot64, int *ns_steps, double *ns_defect) {
    if (!c) return GS_ERR_ARG;
    if (!c->grating_ready) return gs_fail(c, GS_ERR_STATE, "the grating has not been factored");
    if (angle < 0 || angle >= (int)c->ang.size()) return gs_fail(c, GS_ERR_ARG, "angle index out of range");
    const AngleData &a = c->ang[angle];
    if (sweeps32) *sweeps32 = a.sweeps32;
    if (sweeps64) *sweeps64 = a.sweeps;
    if (phase_ms)
        for (int q = 0; q < 6; ++q) phase_ms[q] = a.phase_ms[q];
    for (int q = 0; q < 32; ++q) {
        if (rot32) rot32[q] = a.rot32[q];
        if (rot64) rot64[q] = a.rot64[q];
    }
    if (ns_steps) *ns_steps = a.ns_iters;
    if (ns_defect)
        for (int q = 0; q < 6; ++q) ns_defect[q] = a.ns_defect[q];
    return GS_OK;
}
