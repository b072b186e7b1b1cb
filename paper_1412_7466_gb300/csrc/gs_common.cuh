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

// J_n(x) for any integer n (J_{-n} = (-1)^n J_n).
__device__ __forceinline__ double besselj_int(int n, double x) {
    if (n >= 0) return jn(n, x);
    double v = jn(-n, x);
    return ((-n) & 1) ? -v : v;
}
// Y_n(x) for any integer n (Y_{-n} = (-1)^n Y_n).
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
