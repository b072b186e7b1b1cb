// Pair contribution of the Graf translation (Sec. 4.2 Eq. trans): for one target and one source
// image at offset (dx, dy) = c_i - c_j - l d, adds sum_n H_{n-m}(k R) e^{i(n-m) Th} b[n] to acc[m],
// with H_0, H_1 seeded once and the order recurrence in registers.  Shared by the batched kernels.
#pragma once
#include "gs_common.cuh"

typedef float2 cplxf_t;
__device__ __forceinline__ cplxf_t gs_cf(float r, float i) { return make_float2(r, i); }
__device__ __forceinline__ cplxf_t gs_cmulf(cplxf_t a, cplxf_t b) {
    return gs_cf(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void gs_cfmaf(cplxf_t &acc, cplxf_t a, cplxf_t b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// FP64: b[] already carries the image phase
template <int P>
__device__ __forceinline__ void gs_pair_f64(double dx, double dy, double k, const cplx (&b)[2 * P + 1],
                                            cplx (&acc)[2 * P + 1]) {
    constexpr int NC = 2 * P + 1;
    const double R = hypot(dx, dy), z = k * R, twoz = 2.0 / z;
    cplx Hm1, Hc;
    hankel01(z, Hm1, Hc);
    const cplx u1 = C(dx / R, dy / R);
    cplx up = u1;
#pragma unroll
    for (int m = 0; m < NC; ++m) cfma(acc[m], Hm1, b[m]);
#pragma unroll
    for (int q = 1; q <= 2 * P; ++q) {
        const cplx hq = cmul(Hc, up);
        cplx hmq = cmul(Hc, cconj(up));
        if (q & 1) hmq = C(-hmq.x, -hmq.y);
#pragma unroll
        for (int m = 0; m + q < NC; ++m) cfma(acc[m], hq, b[m + q]);
#pragma unroll
        for (int m = q; m < NC; ++m) cfma(acc[m], hmq, b[m - q]);
        if (q < 2 * P) {
            const cplx Hn = csub(cscale(Hc, q * twoz), Hm1);
            Hm1 = Hc;
            Hc = Hn;
            up = cmul(up, u1);
        }
    }
}

// complex64: offsets already reduced to float (two-float differences by the caller)
template <int P>
__device__ __forceinline__ void gs_pair_c64(float dx, float dy, float k, const cplxf_t (&b)[2 * P + 1],
                                            cplxf_t (&acc)[2 * P + 1]) {
    constexpr int NC = 2 * P + 1;
    const float R = hypotf(dx, dy), z = k * R, twoz = 2.0f / z;
    cplxf_t Hm1 = gs_cf(j0f(z), y0f(z)), Hc = gs_cf(j1f(z), y1f(z));
    const float iR = 1.0f / R;
    const cplxf_t u1 = gs_cf(dx * iR, dy * iR);
    cplxf_t up = u1;
#pragma unroll
    for (int m = 0; m < NC; ++m) gs_cfmaf(acc[m], Hm1, b[m]);
#pragma unroll
    for (int q = 1; q <= 2 * P; ++q) {
        const cplxf_t hq = gs_cmulf(Hc, up);
        cplxf_t hmq = gs_cmulf(Hc, gs_cf(up.x, -up.y));
        if (q & 1) hmq = gs_cf(-hmq.x, -hmq.y);
#pragma unroll
        for (int m = 0; m + q < NC; ++m) gs_cfmaf(acc[m], hq, b[m + q]);
#pragma unroll
        for (int m = q; m < NC; ++m) gs_cfmaf(acc[m], hmq, b[m - q]);
        if (q < 2 * P) {
            const float f = q * twoz;
            const cplxf_t Hn = gs_cf(fmaf(f, Hc.x, -Hm1.x), fmaf(f, Hc.y, -Hm1.y));
            Hm1 = Hc;
            Hc = Hn;
            up = gs_cmulf(up, u1);
        }
    }
}
