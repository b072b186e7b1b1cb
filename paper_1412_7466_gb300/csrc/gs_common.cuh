// Shared device helpers: complex arithmetic on double2/float2, cylinder-function seeds, window.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define GS_PI 3.14159265358979323846
#define GS_EULER 0.57721566490153286061

typedef double2 cplx;

__host__ __device__ __forceinline__ cplx C(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return C(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return C(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
    return C(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return C(a.x, -a.y); }
__host__ __device__ __forceinline__ cplx cscale(cplx a, double s) { return C(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ cplx cmuli(cplx a) { return C(-a.y, a.x); }   // i * a
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
__device__ __forceinline__ void cfma(cplx &acc, cplx a, cplx b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    double den = b.x * b.x + b.y * b.y;
    return C((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ cplx cexpi(double t) {
    double s, c;
    sincos(t, &s, &c);
    return C(c, s);
}
// integer power of a unit-modulus complex number (small |n|)
__device__ __forceinline__ cplx cpowi(cplx a, int n) {
    cplx r = C(1.0, 0.0);
    cplx b = n < 0 ? cconj(a) : a;     // valid for |a| == 1
    int e = n < 0 ? -n : n;
    for (int i = 0; i < e; ++i) r = cmul(r, b);
    return r;
}

// H0(x), H1(x) of the first kind at real x > 0 from the CUDA math library's Bessel functions.
__device__ __forceinline__ void hankel01(double x, cplx &h0, cplx &h1) {
    h0 = C(j0(x), y0(x));
    h1 = C(j1(x), y1(x));
}

// J_n(x) for any integer n and x >= 0 (J_{-n} = (-1)^n J_n) by Miller's backward recurrence
// J_{k-1} = (2k/x) J_k - J_{k+1}, started at an order well above max(|n|, x) and normalised with
// J_0 + 2 sum_k J_{2k} = 1 (Miller 1952; Abramowitz & Stegun 9.12): stable for every order /
// argument ratio, including orders far above the argument, where the library's jn returned NaN
// (orders ~44 at x ~ 8 in the L2L expansion of an inclusion that crosses a period wall).
__device__ inline double besselj_int(int n, double x) {
    const int an = n < 0 ? -n : n;
    if (x == 0.0) return an == 0 ? 1.0 : 0.0;
    const double big = fmax((double)an, x);
    const int m = 2 * (((int)big + 16 + (int)sqrt(40.0 * big)) / 2);
    double jp = 0.0, jc = 1e-200, norm = 0.0, val = 0.0;
    for (int k = m; k >= 0; --k) {
        if (k == an) val = jc;
        norm += (k == 0) ? jc : ((k & 1) ? 0.0 : 2.0 * jc);
        if (k > 0) {
            const double jm = (2.0 * k / x) * jc - jp;
            jp = jc;
            jc = jm;
        }
        if (fabs(jc) > 1e200) {   // rescale the recurrence and what it has accumulated
            jc *= 1e-200;
            jp *= 1e-200;
            norm *= 1e-200;
            val *= 1e-200;
        }
    }
    const double r = val / norm;
    return (n < 0 && (an & 1)) ? -r : r;
}
// Y_n(x) for any integer n (Y_{-n} = (-1)^n Y_n).
// J_n(z) of complex argument by its power series sum_k (-z^2/4)^k (z/2)^|n| / (k! (|n|+k)!)
// (DLMF 10.2.2), for the disk coefficients of lossy inclusions: terms peak near k ~ |z|/2, so for
// |z| <= 12 the cancellation costs at most ~1e3 units of the last place; callers keep |z| there.
__device__ inline cplx besselj_cplx(int n, cplx z) {
    const int an = n < 0 ? -n : n;
    const cplx h = cscale(z, 0.5);
    cplx lead = C(1.0, 0.0);                    // (z/2)^|n| / |n|!
    for (int q = 1; q <= an; ++q) lead = cscale(cmul(lead, h), 1.0 / q);
    const cplx w = cscale(cmul(h, h), -1.0);    // -z^2/4
    cplx term = lead, sum = lead;
    for (int k = 1; k < 200; ++k) {
        term = cscale(cmul(term, w), 1.0 / ((double)k * (double)(an + k)));
        sum = cadd(sum, term);
        if (cabs2(term) < 1e-36 * cabs2(sum)) break;
    }
    return (n < 0 && (an & 1)) ? cscale(sum, -1.0) : sum;
}

__device__ __forceinline__ double bessely_int(int n, double x) {
    if (n >= 0) return yn(n, x);
    double v = yn(-n, x);
    return ((-n) & 1) ? -v : v;
}

// C-infinity flat-top window of the singular-quadrature log coefficient (fraction of a period).
#define GS_WIN_A 0.05
#define GS_WIN_B 0.45
__device__ __forceinline__ double gs_window(double u) {
    u = fabs(u);
    if (u <= GS_WIN_A) return 1.0;
    if (u >= GS_WIN_B) return 0.0;
    double v = (u - GS_WIN_A) / (GS_WIN_B - GS_WIN_A);
    double f1 = exp(-1.0 / v), f2 = exp(-1.0 / (1.0 - v));
    return f2 / (f1 + f2);
}

// block-wide sum of a double (blockDim.x multiple of 32, <= 1024); result valid in all threads
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = (threadIdx.x < (unsigned)nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    double r = sh[0];
    __syncthreads();
    return r;
}

// ---- double-float arithmetic: a value held as an unevaluated sum hi + lo of two floats (Dekker
// 1971), sums by Knuth's TwoSum, products by the FMA form of Dekker's exact product.  A complex
// double-float number is a float4 (hi.re, hi.im, lo.re, lo.im): 48-bit significands on the FP32
// pipe, for products whose FP64 form would be bound by the FP64 pipe.

// s + e = a + b exactly
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// (hi, lo) += a * b, lo not folded back: the exact product error and the TwoSum error go to lo
__device__ __forceinline__ void df_mac_nr(float &hi, float &lo, float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    float s, e;
    df_two_sum(hi, p, s, e);
    hi = s;
    lo += e + pe;
}
// fold lo back into hi so that |lo| is at most half an ulp of hi
__device__ __forceinline__ void df_renorm(float &hi, float &lo) {
    const float s = hi + lo;
    lo -= s - hi;
    hi = s;
}
struct dfc {
    float rh, rl, ih, il;   // real (hi, lo), imaginary (hi, lo)
};
// s += c * x for complex double-float c, x, without the final renormalisation; the lo * lo terms
// (2^-48 of the product) are dropped
__device__ __forceinline__ void dfc_mac_nr(dfc &s, float4 c, float4 x) {
    s.rl = fmaf(c.x, x.z, fmaf(c.z, x.x, fmaf(-c.y, x.w, fmaf(-c.w, x.y, s.rl))));
    s.il = fmaf(c.x, x.w, fmaf(c.z, x.y, fmaf(c.y, x.z, fmaf(c.w, x.x, s.il))));
    df_mac_nr(s.rh, s.rl, c.x, x.x);
    df_mac_nr(s.rh, s.rl, -c.y, x.y);
    df_mac_nr(s.ih, s.il, c.x, x.y);
    df_mac_nr(s.ih, s.il, c.y, x.x);
}
__device__ __forceinline__ void dfc_renorm(dfc &s) {
    df_renorm(s.rh, s.rl);
    df_renorm(s.ih, s.il);
}
__device__ __forceinline__ void dfc_add(dfc &a, const dfc &b) {
    float s, e;
    df_two_sum(a.rh, b.rh, s, e);
    a.rl += e + b.rl;
    a.rh = s + a.rl;
    a.rl -= a.rh - s;
    df_two_sum(a.ih, b.ih, s, e);
    a.il += e + b.il;
    a.ih = s + a.il;
    a.il -= a.ih - s;
}
// warp-wide double-float sum (all lanes get it)
__device__ __forceinline__ void dfc_warp_sum(dfc &a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dfc b;
        b.rh = __shfl_xor_sync(0xffffffffu, a.rh, o);
        b.rl = __shfl_xor_sync(0xffffffffu, a.rl, o);
        b.ih = __shfl_xor_sync(0xffffffffu, a.ih, o);
        b.il = __shfl_xor_sync(0xffffffffu, a.il, o);
        dfc_add(a, b);
    }
}
// s += sum_c a[c] x[c] over c = t, t + T, t + 2T, ... < n (T threads, t this thread).  Batches of
// U = 4 entries per thread, software-pipelined: the next batch's eight 16-byte loads (C streamed,
// evict-first; x from L2) are issued before the current batch's arithmetic; one renormalisation
// per batch (lo then holds at most ~8 half-ulps of hi before it is folded back).
template <int T>
__device__ __forceinline__ void dfc_row_dot(dfc &s, const float4 *__restrict__ a, const float4 *__restrict__ x, long n,
                                            int t) {
    constexpr int U = 4;
    long c = t;
    float4 an[U], xn[U];
    bool have = c + (long)(U - 1) * T < n;
    if (have) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            an[u] = __ldcs(&a[c + u * T]);
            xn[u] = __ldg(&x[c + u * T]);
        }
    }
    while (have) {
        float4 ac[U], xc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ac[u] = an[u];
            xc[u] = xn[u];
        }
        c += (long)U * T;
        have = c + (long)(U - 1) * T < n;
        if (have) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                an[u] = __ldcs(&a[c + u * T]);
                xn[u] = __ldg(&x[c + u * T]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) dfc_mac_nr(s, ac[u], xc[u]);
        dfc_renorm(s);
    }
    for (; c < n; c += T) {
        dfc_mac_nr(s, __ldcs(&a[c]), __ldg(&x[c]));
        dfc_renorm(s);
    }
}

// (hi, lo) complex64 split of a complex128 value: hi the nearest complex64, lo the nearest
// complex64 to the (exact) remainder
__device__ __forceinline__ float4 df_split(double re, double im) {
    const float hr = (float)re, hi = (float)im;
    return make_float4(hr, hi, (float)(re - (double)hr), (float)(im - (double)hi));
}

// H0(z), H1(z) in single precision from the polynomial approximations of Abramowitz & Stegun
// 9.4.1-9.4.6 (Allen 1956): for z <= 3 power series in (z/3)^2 with the logarithmic terms of Y0, Y1;
// for z > 3 modulus and phase, H_n = z^{-1/2} f_n e^{i theta_n}, as polynomials in 3/z.  Absolute
// error below ~1e-7 (relative error of H0, H1 below 1.2e-7 for z > 0.05), all in FP32.
__device__ __forceinline__ void hankel01_f32(float z, float2 &h0, float2 &h1) {
    if (z <= 3.0f) {
        const float t = (z * (1.0f / 3.0f)) * (z * (1.0f / 3.0f));
        const float j0 = 1.0f + t * (-2.2499997f + t * (1.2656208f + t * (-0.3163866f + t * (0.0444479f +
                         t * (-0.0039444f + t * 0.0002100f)))));
        const float j1 = z * (0.5f + t * (-0.56249985f + t * (0.21093573f + t * (-0.03954289f + t * (0.00443319f +
                         t * (-0.00031761f + t * 0.00001109f))))));
        const float lg = (2.0f / 3.14159265f) * logf(0.5f * z);
        const float y0 = lg * j0 + (0.36746691f + t * (0.60559366f + t * (-0.74350384f + t * (0.25300117f +
                         t * (-0.04261214f + t * (0.00427916f + t * -0.00024846f))))));
        const float y1 = lg * j1 + (-0.6366198f + t * (0.2212091f + t * (2.1682709f + t * (-1.3164827f +
                         t * (0.3123951f + t * (-0.0400976f + t * 0.0027873f)))))) / z;
        h0 = make_float2(j0, y0);
        h1 = make_float2(j1, y1);
    } else {
        const float u = 3.0f / z;
        const float f0 = 0.79788456f + u * (-0.00000077f + u * (-0.00552740f + u * (-0.00009512f + u * (0.00137237f +
                         u * (-0.00072805f + u * 0.00014476f)))));
        const float p0 = -0.78539816f + u * (-0.04166397f + u * (-0.00003954f + u * (0.00262573f + u * (-0.00054125f +
                         u * (-0.00029333f + u * 0.00013558f)))));
        const float f1 = 0.79788456f + u * (0.00000156f + u * (0.01659667f + u * (0.00017105f + u * (-0.00249511f +
                         u * (0.00113653f + u * -0.00020033f)))));
        const float p1 = -2.35619449f + u * (0.12499612f + u * (0.00005650f + u * (-0.00637879f + u * (0.00074348f +
                         u * (0.00079824f + u * -0.00029166f)))));
        const float r = rsqrtf(z);
        float s0, c0, s1, c1;
        sincosf(z + p0, &s0, &c0);
        sincosf(z + p1, &s1, &c1);
        h0 = make_float2(r * f0 * c0, r * f0 * s0);
        h1 = make_float2(r * f1 * c1, r * f1 * s1);
    }
}
