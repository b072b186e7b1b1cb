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

// complex64 (offsets already reduced to float by the caller) with packed two-wide FP32
// multiply-adds (__ffma2_rn, one instruction for both halves of a float2): h b = Re(h) (b.x, b.y) + Im(h) (-b.y, b.x), so the pair keeps two packed
// accumulators per order, Pa[m] += (Re h, Re h) b and Qa[m] += (Im h, Im h) b, and the product is
// (Pa.x - Qa.y, Pa.y + Qa.x) at the end (gs_pq_combine).  Half the instructions of four scalar
// FMAs per complex product, so the unrolled Toeplitz block also takes half the instruction cache.
template <int P>
__device__ __forceinline__ void gs_pair_c64x2(float dx, float dy, float k, const cplxf_t (&b)[2 * P + 1],
                                              cplxf_t (&Pa)[2 * P + 1], cplxf_t (&Qa)[2 * P + 1]) {
    constexpr int NC = 2 * P + 1;
    const float R = hypotf(dx, dy), z = k * R, twoz = 2.0f / z;
    cplxf_t Hm1, Hc;
    hankel01_f32(z, Hm1, Hc);
    const float iR = 1.0f / R;
    const cplxf_t u1 = gs_cf(dx * iR, dy * iR);
    cplxf_t up = u1;
    {
        const cplxf_t hr = gs_cf(Hm1.x, Hm1.x), hi = gs_cf(Hm1.y, Hm1.y);
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            Pa[m] = __ffma2_rn(hr, b[m], Pa[m]);
            Qa[m] = __ffma2_rn(hi, b[m], Qa[m]);
        }
    }
#pragma unroll
    for (int q = 1; q <= 2 * P; ++q) {
        const cplxf_t hq = gs_cmulf(Hc, up);
        cplxf_t hmq = gs_cmulf(Hc, gs_cf(up.x, -up.y));
        if (q & 1) hmq = gs_cf(-hmq.x, -hmq.y);
        const cplxf_t pr = gs_cf(hq.x, hq.x), pi = gs_cf(hq.y, hq.y);
        const cplxf_t mr = gs_cf(hmq.x, hmq.x), mi = gs_cf(hmq.y, hmq.y);
#pragma unroll
        for (int m = 0; m + q < NC; ++m) {
            Pa[m] = __ffma2_rn(pr, b[m + q], Pa[m]);
            Qa[m] = __ffma2_rn(pi, b[m + q], Qa[m]);
        }
#pragma unroll
        for (int m = q; m < NC; ++m) {
            Pa[m] = __ffma2_rn(mr, b[m - q], Pa[m]);
            Qa[m] = __ffma2_rn(mi, b[m - q], Qa[m]);
        }
        if (q < 2 * P) {
            const float f = q * twoz;
            const cplxf_t Hn = gs_cf(fmaf(f, Hc.x, -Hm1.x), fmaf(f, Hc.y, -Hm1.y));
            Hm1 = Hc;
            Hc = Hn;
            up = gs_cmulf(up, u1);
        }
    }
}

template <int NC>
__device__ __forceinline__ void gs_pq_combine(const cplxf_t (&Pa)[NC], const cplxf_t (&Qa)[NC], cplxf_t (&acc)[NC]) {
#pragma unroll
    for (int m = 0; m < NC; ++m) acc[m] = gs_cf(Pa[m].x - Qa[m].y, Pa[m].y + Qa[m].x);
}

// Sum over the 32 lanes of a warp of its per-lane complex64 accumulators, through a warp-private
// shared buffer red[2 NC][33] (row v = real or imaginary part of order m = v / 2, one column per
// lane; the 33rd column staggers the banks so that the row writes and the column reads are both
// conflict-free).  Lane v (and v + 32, ...) adds column v by a pairwise tree in FP32 and writes the
// sum as a double to o[v] when `store`; o holds NC interleaved complex128 values.
template <int NC>
__device__ __forceinline__ void gs_warp_sum_c64(const cplxf_t (&acc)[NC], float *red, int lane, double *o,
                                                bool store) {
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        red[(2 * m) * 33 + lane] = acc[m].x;
        red[(2 * m + 1) * 33 + lane] = acc[m].y;
    }
    __syncwarp();
    for (int v = lane; v < 2 * NC; v += 32) {
        float t[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) t[u] = red[v * 33 + u];
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1) {
#pragma unroll
            for (int u = 0; u < h; ++u) t[u] += t[u + h];
        }
        if (store) o[v] = (double)t[0];
    }
    __syncwarp();
}
