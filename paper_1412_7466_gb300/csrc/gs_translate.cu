// All-pairs Graf translation (M2L) between the inclusions, with the +-d images (Sec. 4.2 Eq. trans,
// Sec. 5 Eq. repre3_mod):
//   alpha_i[m] = sum_{(j,l) != (i,0)} alpha^l sum_n H_{n-m}(k R) e^{i(n-m) Th} beta_j[n],
//   (R, Th) = polar(c_i - c_j - l d).
//
// Kernel design (FP64): one warp per target particle, its 32 lanes over 32 source images at a
// time.  A thread block of WARPS targets shares each tile of 32 source images, staged in shared
// memory with the image phase alpha^l already folded into the coefficients (layout [n][lane], so
// lane-indexed reads are conflict-free).  Each lane seeds H_0, H_1 once per pair from the CUDA
// Bessel functions, recurs upward in the order (H_{q+1} = (2q/z) H_q - H_{q-1}) in registers,
// forms H_q u^q and (-1)^q H_q conj(u)^q with u = e^{i Th}, and applies the (2p+1)x(2p+1)
// Toeplitz block to the staged coefficients with the 2p+1 accumulators held in registers (fully
// unrolled for the compile-time order P).  Warp-shuffle reductions combine the lanes.  The source
// images are split into `nsplit` chunks across blockIdx.y to fill the SMs; a second kernel
// sums the chunk partials in a fixed order (deterministic).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "gs_internal.h"
#include "gs_pair.cuh"
#include "gs_tma.cuh"

namespace {

constexpr int TILE = 32;

template <int P, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_translate_f64(const double *__restrict__ xy, int M, const cplx *__restrict__ beta, double k, double d,
                cplx alpha, int nsplit, cplx *__restrict__ out) {
    constexpr int NC = 2 * P + 1;
    __shared__ cplx sb[NC][TILE];
    __shared__ double sx[TILE], sy[TILE];
    __shared__ int sid[TILE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * WARPS + warp;
    const long total = 3L * M;
    const long s0 = total * blockIdx.y / nsplit, s1 = total * (blockIdx.y + 1) / nsplit;
    double xi = 0.0, yi = 0.0;
    if (i < M) {
        xi = xy[2 * i];
        yi = xy[2 * i + 1];
    }
    cplx acc[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) acc[m] = C(0.0, 0.0);
    const cplx ainv = cconj(alpha);

    for (long t0 = s0; t0 < s1; t0 += TILE) {
        __syncthreads();
        for (int e = threadIdx.x; e < TILE * NC; e += WARPS * 32) {
            int u = e / NC, n = e - u * NC;
            long s = t0 + u;
            cplx v = C(0.0, 0.0);
            if (s < s1) {
                int l = (int)(s / M) - 1;
                int j = (int)(s - (long)(l + 1) * M);
                cplx b = beta[(size_t)j * NC + n];
                v = (l == 0) ? b : cmul(l == 1 ? alpha : ainv, b);
            }
            sb[n][u] = v;
        }
        for (int u = threadIdx.x; u < TILE; u += WARPS * 32) {
            long s = t0 + u;
            if (s < s1) {
                int l = (int)(s / M) - 1;
                int j = (int)(s - (long)(l + 1) * M);
                sx[u] = xy[2 * j] + l * d;
                sy[u] = xy[2 * j + 1];
                sid[u] = (l == 0) ? j : -1;
            } else {
                sid[u] = -2;
                sx[u] = 0.0;
                sy[u] = 0.0;
            }
        }
        __syncthreads();
        if (i >= M) continue;
        const long s = t0 + lane;
        if (s >= s1 || sid[lane] == i) continue;
        const double dx = xi - sx[lane], dy = yi - sy[lane];
        const double R = hypot(dx, dy);
        const double z = k * R;
        const double twoz = 2.0 / z;
        cplx Hm1, Hc;
        hankel01(z, Hm1, Hc);   // H_0, H_1
        const cplx u1 = C(dx / R, dy / R);
        cplx up = u1;
#pragma unroll
        for (int m = 0; m < NC; ++m) cfma(acc[m], Hm1, sb[m][lane]);
#pragma unroll
        for (int q = 1; q <= 2 * P; ++q) {
            const cplx hq = cmul(Hc, up);
            cplx hmq = cmul(Hc, cconj(up));
            if (q & 1) hmq = C(-hmq.x, -hmq.y);
#pragma unroll
            for (int m = 0; m + q < NC; ++m) cfma(acc[m], hq, sb[m + q][lane]);
#pragma unroll
            for (int m = q; m < NC; ++m) cfma(acc[m], hmq, sb[m - q][lane]);
            if (q < 2 * P) {
                const cplx Hn = csub(cscale(Hc, q * twoz), Hm1);
                Hm1 = Hc;
                Hc = Hn;
                up = cmul(up, u1);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        acc[m].x = warp_sum(acc[m].x);
        acc[m].y = warp_sum(acc[m].y);
    }
    if (i < M) {
        cplx *o = out + ((size_t)blockIdx.y * M + i) * NC;
#pragma unroll
        for (int m = 0; m < NC; ++m)
            if (lane == (m & 31)) o[m] = acc[m];
    }
}


// ---- complex64 variant (the inner operator of the mixed-precision solve) --------------------------
// Same tiling as the FP64 kernel, with no FP64 arithmetic inside: the pair offsets come from the
// (hi, lo) float image coordinates (differences of the hi parts are exact for nearby pairs, so
// (dx, dy) carry FP32 rounding of the offset itself, not of the coordinates), the Hankel seeds
// from FP32 polynomial approximations, the recurrence, the Toeplitz products (packed two-wide
// multiply-adds, gs_pair_c64x2) and the per-lane accumulators are FP32, and the lanes are summed in
// FP32 through shared memory; only the chunk
// partials are stored (and summed by k_sum_partials) in FP64.  Values stay in their natural scale:
// for p <= 12 and k R >= 0.5 the largest Hankel order is below 1e36 and the smallest coefficients
// of interest above the FP32 normal range.
typedef cplxf_t cplxf;
__device__ __forceinline__ cplxf CF(float r, float i) { return make_float2(r, i); }
__device__ __forceinline__ cplxf cmulf(cplxf a, cplxf b) { return gs_cmulf(a, b); }

// beta (complex128) -> complex64 once per call
__global__ void k_beta_to_c64(const cplx *__restrict__ b, long n, cplxf *__restrict__ b32) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b32[e] = CF((float)b[e].x, (float)b[e].y);
}

__device__ __forceinline__ void split2(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

}  // namespace

// Image coordinates of the complex64 kernels as (hi, lo) float pairs: img[(l+1) M + j] holds
// x_j + l d and y_j, each split as hi = fl32(v), lo = fl32(v - hi).  Built once per geometry, so the
// translation itself touches no FP64 value (the FP64 pipe runs at 1/64 of the FP32 rate).
__global__ void k_images_c64(const double *__restrict__ xy, int M, double d, float4 *__restrict__ img) {
    const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= 3L * M) return;
    const int l = (int)(s / M) - 1;
    const int j = (int)(s - (long)(l + 1) * M);
    float4 g;
    split2(xy[2 * j] + l * d, g.x, g.y);
    split2(xy[2 * j + 1], g.z, g.w);
    img[s] = g;
}

int gs_build_images_c64(gs_ctx *c, const double *xy, int M, float4 *img, cudaStream_t st) {
    if (M < 1) return GS_OK;
    GS_COUNT_LAUNCH(c);
    k_images_c64<<<(int)((3L * M + 255) / 256), 256, 0, st>>>(xy, M, c->L.d, img);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

namespace {

template <int P, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, (P <= 12 ? 3 : 1))
k_translate_c64(const float4 *__restrict__ img, int M, const cplxf *__restrict__ beta32, float k, cplx alpha,
                int nsplit, cplx *__restrict__ out) {
    constexpr int NC = 2 * P + 1;
    __shared__ cplxf sb[NC][TILE + 1];   // +1: the [n][u] stores of the staging loop spread over the banks
    __shared__ float4 sg[TILE];
    __shared__ int sid[TILE];
    __shared__ cplxf sph[3];
    __shared__ float red[WARPS][2 * NC * 33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * WARPS + warp;
    const long total = 3L * M;   // source images; 3 M < 2^31 (M is an int count of unknowns / (2p+1))
    const int s0 = (int)(total * blockIdx.y / nsplit), s1 = (int)(total * (blockIdx.y + 1) / nsplit);
    float4 gi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < M) gi = img[M + i];   // image l = 0
    if (threadIdx.x == 0) {
        sph[0] = CF((float)alpha.x, (float)-alpha.y);   // alpha^{-1} = conj(alpha)
        sph[1] = CF(1.f, 0.f);
        sph[2] = CF((float)alpha.x, (float)alpha.y);
    }
    cplxf Pa[NC], Qa[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) Pa[m] = Qa[m] = CF(0.f, 0.f);

    for (int t0 = s0; t0 < s1; t0 += TILE) {
        __syncthreads();
        for (int e = threadIdx.x; e < TILE * NC; e += WARPS * 32) {
            const int u = e / NC, n = e - u * NC;
            const int s = t0 + u;
            cplxf v = CF(0.f, 0.f);
            if (s < s1) {
                const int l1 = (s >= M) + (s >= 2 * M);   // image l + 1 of source image s = (l+1) M + j
                v = cmulf(sph[l1], beta32[(size_t)(s - l1 * M) * NC + n]);
            }
            sb[n][u] = v;
        }
        for (int u = threadIdx.x; u < TILE; u += WARPS * 32) {
            const int s = t0 + u;
            if (s < s1) {
                const int l = (s >= M) + (s >= 2 * M) - 1;
                const int j = s - (l + 1) * M;
                sg[u] = img[s];
                sid[u] = (l == 0) ? j : -1;
            } else {
                sid[u] = -2;
                sg[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        if (i >= M) continue;
        if (t0 + lane >= s1 || sid[lane] == i) continue;
        const float4 gs = sg[lane];
        const float dx = (gi.x - gs.x) + (gi.y - gs.y);
        const float dy = (gi.z - gs.z) + (gi.w - gs.w);
        cplxf b[NC];
#pragma unroll
        for (int n = 0; n < NC; ++n) b[n] = sb[n][lane];
        gs_pair_c64x2<P>(dx, dy, k, b, Pa, Qa);
    }
    cplxf acc[NC];
    gs_pq_combine<NC>(Pa, Qa, acc);
    gs_warp_sum_c64<NC>(acc, red[warp], lane, (double *)(out + ((size_t)blockIdx.y * M + (i < M ? i : 0)) * NC),
                        i < M);
}


// ---- FP64 with a precomputed pair table ----------------------------------------------------------
// The translation coefficients h_q = H_q(k R) e^{i q Th}, q = -2p..2p, of every (target, source image)
// pair depend on the geometry only (not on the angle or the iterate), so they are built once per
// geometry and streamed from HBM by every matrix-vector product: 3 M^2 (4p+1) complex128 values
// (2.35 GB at M = 1000, p = 12), read in 0.35 ms at HBM speed against 12.5 ms of FP64 products.
// Layout h[i][q][s] with the source image s = (l+1) M + j fastest, so a warp (target i, 32 sources)
// reads each q as one coalesced 512-byte segment.  The self pair (i, l = 0) holds zeros.
__device__ __forceinline__ void put_h(cplx *o, cplx v) { *o = v; }
__device__ __forceinline__ void put_h(float2 *o, cplx v) { *o = make_float2((float)v.x, (float)v.y); }

// T = cplx: the FP64 table (row stride SP = 3M); T = float2: the complex64 table of the complex64
// translation, rounded from the same FP64 values (row stride SP = 3M rounded up to 32 images, so
// that every row starts on a 256-byte boundary for the tensor copies)
template <int P, typename T>
__global__ void k_pair_table(const double *__restrict__ xy, int M, double k, double d, T *__restrict__ h, long SP) {
    constexpr int NQ = 4 * P + 1;
    const long S = 3L * M;
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)M * S) return;
    const int i = (int)(id / S);
    const long s = id - (long)i * S;
    const int l = (int)(s / M) - 1;
    const int j = (int)(s - (long)(l + 1) * M);
    T *o = h + (size_t)i * NQ * SP + s;
    if (l == 0 && j == i) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) put_h(o + (size_t)q * SP, C(0.0, 0.0));
        return;
    }
    const double dx = xy[2 * i] - (xy[2 * j] + l * d), dy = xy[2 * i + 1] - xy[2 * j + 1];
    const double R = hypot(dx, dy), z = k * R, twoz = 2.0 / z;
    cplx Hm1, Hc;
    hankel01(z, Hm1, Hc);
    const cplx u1 = C(dx / R, dy / R);
    cplx up = u1;
    put_h(o + (size_t)(2 * P) * SP, Hm1);
#pragma unroll
    for (int q = 1; q <= 2 * P; ++q) {
        put_h(o + (size_t)(2 * P + q) * SP, cmul(Hc, up));
        cplx hm = cmul(Hc, cconj(up));
        put_h(o + (size_t)(2 * P - q) * SP, (q & 1) ? C(-hm.x, -hm.y) : hm);
        if (q < 2 * P) {
            const cplx Hn = csub(cscale(Hc, q * twoz), Hm1);
            Hm1 = Hc;
            Hc = Hn;
            up = cmul(up, u1);
        }
    }
}

// complex64 table from the FP64 one (row strides S and SP)
__global__ void k_table_to_c64(const cplx *__restrict__ h, long rows, long S, long SP, float2 *__restrict__ h32) {
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= rows * S) return;
    const long r = id / S, s = id - r * S;
    const cplx v = h[id];
    h32[r * SP + s] = make_float2((float)v.x, (float)v.y);
}

// b3[s][n] = alpha^l beta_j[n] in complex64 for the source images s = (l+1) M + j, zero for the
// padding images up to a whole number of 32-image tiles (the phase is applied in FP64)
__global__ void k_beta_to_b3(const cplx *__restrict__ beta, int M, int nc, long ntot, cplx alpha,
                             float2 *__restrict__ b3, const int *__restrict__ active) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ntot || (active && !*active)) return;
    const long s = e / nc;
    const int n = (int)(e - s * nc);
    float2 v = make_float2(0.f, 0.f);
    if (s < 3L * M) {
        const int l1 = (int)(s / M), j = (int)(s - (long)l1 * M);
        const cplx b = beta[(size_t)j * nc + n];
        const cplx r = l1 == 1 ? b : cmul(l1 == 2 ? alpha : cconj(alpha), b);
        v = make_float2((float)r.x, (float)r.y);
    }
    b3[e] = v;
}

// ---- complex64 translation from the complex64 table ---------------------------------------------
// Each block (WARPS targets) walks its share of the 32-image tiles through a two-stage ring in shared
// memory: per stage, one TMA tensor copy per warp brings that target's (4p+1) x 32 coefficients
// h[i][q][t0 .. t0+31] (out-of-range images and rows read as zero), and one bulk copy the tile's
// phased source coefficients b3 (32 x (2p+1)); a single mbarrier per stage counts all of them.  The
// lanes then apply the Toeplitz block of packed FMAs exactly as the recomputing kernel does, with
// the coefficients read from shared memory instead of recurred: the copies of the next tile are in
// flight meanwhile, so the kernel runs at the FP32 pipe's rate while streaming the table (1.18 GB
// at M = 1000, p = 12) from HBM.  The self pair holds zeros in the table, so no lane branches.
// Every wait is bounded (~1 s); a wait that gives up makes the whole block stop, wait (bounded) for
// its copies still in flight, set *err and return without writing.  `active` (nullable): a device
// flag; when it is 0 the launch does nothing (masked geometries of a batched solve).
template <int P, int WARPS>
struct Tab32Layout {
    static constexpr int NC = 2 * P + 1, NQ = 4 * P + 1;
    static constexpr int HT = NQ * TILE * 8;            // one warp's coefficient box (bytes)
    static constexpr int BT = TILE * NC * 8;            // the tile's source coefficients
    static constexpr int ST = WARPS * HT + BT;          // one stage
    static constexpr int RED = WARPS * 2 * NC * 33 * 4; // lane sums, reusing stage memory at the end
    static constexpr int SMEM = 2 * ST + 16 + 1024;     // two stages, two mbarriers, alignment slack
    static_assert(HT % 128 == 0 && BT % 128 == 0, "tensor-copy destinations must stay 128-byte aligned");
    static_assert(RED <= 2 * ST, "lane-sum buffer must fit in the stage memory");
};

template <int P, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_translate_c64_tab(const __grid_constant__ CUtensorMap tmH, const float2 *__restrict__ b3, int M, int nsplit,
                    cplx *__restrict__ out, int *__restrict__ err, const int *__restrict__ active) {
    using L = Tab32Layout<P, WARPS>;
    if (active && !*active) return;   // a converged geometry of a batch (uniform over the block)
    constexpr int NC = L::NC;
    constexpr long long WAIT = 2000000000LL;   // ~1 s
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t s_base = smem_u32(smem), b_full = smem_u32(smem + 2 * L::ST);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * WARPS + warp;
    const int ntile = (3 * M + TILE - 1) / TILE;
    const int tb0 = (int)((long)ntile * blockIdx.y / nsplit), tb1 = (int)((long)ntile * (blockIdx.y + 1) / nsplit);
    if (threadIdx.x == 0) {
        mbar_init(b_full, 1);
        mbar_init(b_full + 8, 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int tb, int st) {
        const uint32_t bar = b_full + 8 * st, dst = s_base + st * L::ST;
        mbar_expect_tx(bar, L::ST);
        for (int w = 0; w < WARPS; ++w)
            tma_load_2d(dst + w * L::HT, &tmH, bar, tb * TILE, (blockIdx.x * WARPS + w) * L::NQ);
        bulk_load(dst + WARPS * L::HT, b3 + (size_t)tb * TILE * NC, L::BT, bar);
    };
    if (threadIdx.x == 0) {
        if (tb0 < tb1) issue(tb0, 0);
        if (tb0 + 1 < tb1) issue(tb0 + 1, 1);
    }
    cplxf Pa[NC], Qa[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) Pa[m] = Qa[m] = CF(0.f, 0.f);
    for (int tb = tb0; tb < tb1; ++tb) {
        const int st = (tb - tb0) & 1;
        if (!__syncthreads_and(mbar_wait(b_full + 8 * st, ((tb - tb0) >> 1) & 1, WAIT))) {
            if (threadIdx.x == 0) {   // copies of tiles tb and tb + 1 may still be in flight
                mbar_wait(b_full + 8 * st, ((tb - tb0) >> 1) & 1, WAIT);
                if (tb + 1 < tb1) mbar_wait(b_full + 8 * (st ^ 1), ((tb + 1 - tb0) >> 1) & 1, WAIT);
                atomicExch(err, 1);
            }
            return;
        }
        const cplxf *hs = (const cplxf *)(smem + st * L::ST + warp * L::HT);
        const cplxf *bs = (const cplxf *)(smem + st * L::ST + WARPS * L::HT);
        cplxf b[NC];
#pragma unroll
        for (int n = 0; n < NC; ++n) b[n] = bs[lane * NC + n];
        {
            const cplxf h0 = hs[(2 * P) * TILE + lane];
            const cplxf hr = CF(h0.x, h0.x), hi = CF(h0.y, h0.y);
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                Pa[m] = __ffma2_rn(hr, b[m], Pa[m]);
                Qa[m] = __ffma2_rn(hi, b[m], Qa[m]);
            }
        }
#pragma unroll
        for (int q = 1; q <= 2 * P; ++q) {
            const cplxf hq = hs[(2 * P + q) * TILE + lane], hmq = hs[(2 * P - q) * TILE + lane];
            const cplxf pr = CF(hq.x, hq.x), pi = CF(hq.y, hq.y), mr = CF(hmq.x, hmq.x), mi = CF(hmq.y, hmq.y);
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
        }
        __syncthreads();   // stage st is free again
        if (threadIdx.x == 0 && tb + 2 < tb1) issue(tb + 2, st);
    }
    cplxf acc[NC];
    gs_pq_combine<NC>(Pa, Qa, acc);
    gs_warp_sum_c64<NC>(acc, (float *)smem + warp * (2 * NC * 33), lane,
                        (double *)(out + ((size_t)blockIdx.y * M + (i < M ? i : 0)) * NC), i < M);
}

template <int P, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_translate_f64_tab(const cplx *__restrict__ htab, int M, const cplx *__restrict__ beta, cplx alpha, int nsplit,
                    cplx *__restrict__ out) {
    constexpr int NC = 2 * P + 1, NQ = 4 * P + 1;
    __shared__ cplx sb[NC][TILE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * WARPS + warp;
    const long S = 3L * M;
    const long s0 = S * blockIdx.y / nsplit, s1 = S * (blockIdx.y + 1) / nsplit;
    const cplx *hrow = htab + (size_t)(i < M ? i : 0) * NQ * S;
    cplx acc[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) acc[m] = C(0.0, 0.0);
    const cplx ainv = cconj(alpha);
    for (long t0 = s0; t0 < s1; t0 += TILE) {
        __syncthreads();
        for (int e = threadIdx.x; e < TILE * NC; e += WARPS * 32) {
            int u = e / NC, n = e - u * NC;
            long s = t0 + u;
            cplx v = C(0.0, 0.0);
            if (s < s1) {
                int l = (int)(s / M) - 1;
                int j = (int)(s - (long)(l + 1) * M);
                cplx b = beta[(size_t)j * NC + n];
                v = (l == 0) ? b : cmul(l == 1 ? alpha : ainv, b);
            }
            sb[n][u] = v;
        }
        __syncthreads();
        if (i >= M) continue;
        const long s = t0 + lane;
        if (s >= s1) continue;
        const cplx *hp = hrow + s;
#pragma unroll
        for (int q = -2 * P; q <= 2 * P; ++q) {
            const cplx hq = __ldg(&hp[(size_t)(q + 2 * P) * S]);
            if (q >= 0) {
#pragma unroll
                for (int m = 0; m + q < NC; ++m) cfma(acc[m], hq, sb[m + q][lane]);
            } else {
#pragma unroll
                for (int m = -q; m < NC; ++m) cfma(acc[m], hq, sb[m + q][lane]);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        acc[m].x = warp_sum(acc[m].x);
        acc[m].y = warp_sum(acc[m].y);
    }
    if (i < M) {
        cplx *o = out + ((size_t)blockIdx.y * M + i) * NC;
#pragma unroll
        for (int m = 0; m < NC; ++m)
            if (lane == (m & 31)) o[m] = acc[m];
    }
}

__global__ void k_sum_partials(const cplx *part, int nsplit, long len, cplx *out) {
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    cplx s = part[e];
    for (int c = 1; c < nsplit; ++c) s = cadd(s, part[(size_t)c * len + e]);
    out[e] = s;
}

// out = sum of the nsplit partials, or zero when the activity flag (nullable) is 0
__global__ void k_sum_partials_act(const cplx *part, int nsplit, long len, cplx *out, const int *active) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    if (active && !*active) {
        out[e] = C(0.0, 0.0);
        return;
    }
    cplx s = part[e];
    for (int c = 1; c < nsplit; ++c) s = cadd(s, part[(size_t)c * len + e]);
    out[e] = s;
}

// complex64 translation of one geometry (M inclusions) from its table t: phased coefficients into
// b3, the table kernel into the partials, their sum into out
template <int P>
int launch_tab32(gs_ctx *c, const gs_tab32 &t, int M, const cplx *beta, cplx alpha, float2 *b3, cplx *part,
                 size_t part_elems, cplx *out, const int *active, cudaStream_t st, bool prof) {
    constexpr int WARPS = 4;
    using L = Tab32Layout<P, WARPS>;
    const int gx = (M + WARPS - 1) / WARPS;
    const int ntile = (int)((3L * M + TILE - 1) / TILE);
    // about sixteen blocks per SM in all (two resident at a time), so the last wave stays short
    int nsplit = (int)((c->sms * 16L + gx - 1) / gx);
    nsplit = std::max(1, std::min(std::min(nsplit, 64), ntile));
    if ((size_t)nsplit * M * (2 * P + 1) > part_elems) return gs_fail(c, GS_ERR_STATE, "translation scratch too small");
    const long ntot = (long)ntile * TILE * (2 * P + 1);
    GS_COUNT_LAUNCH(c);
    k_beta_to_b3<<<(int)((ntot + 255) / 256), 256, 0, st>>>(beta, M, 2 * P + 1, ntot, alpha, b3, active);
    cudaEvent_t e0, e1;
    const bool timed = prof && gs_prof_pair(c, &e0, &e1, GS_C64);
    if (timed) cudaEventRecord(e0, st);
    GS_COUNT_LAUNCH(c);
    k_translate_c64_tab<P, WARPS><<<dim3(gx, nsplit), WARPS * 32, L::SMEM, st>>>(t.map, b3, M, nsplit, part, c->terr,
                                                                                 active);
    if (timed) cudaEventRecord(e1, st);
    const long len = (long)M * (2 * P + 1);
    GS_COUNT_LAUNCH(c);
    k_sum_partials_act<<<(int)((len + 255) / 256), 256, 0, st>>>(part, nsplit, len, out, active);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

template <int P>
int launch_translate(gs_ctx *c, const AngleData &a, const cplx *beta, cplx *out, int precision) {
    constexpr int WARPS = 4;
    if (precision == GS_C64) {
        GS_TRY(gs_ensure_table32(c));
        if (c->tab32.h)
            return launch_tab32<P>(c, c->tab32, c->M, beta, a.alpha, c->b3pad, c->part, c->part_elems, out, nullptr,
                                   c->stream, true);
    }
    const int M = c->M;
    const int gx = (M + WARPS - 1) / WARPS;
    // enough blocks for several waves over the SMs
    int nsplit = (int)((c->sms * 8L + gx - 1) / gx);
    if (nsplit < 1) nsplit = 1;
    if (nsplit > 64) nsplit = 64;
    if ((long)nsplit * 32 > 3L * M) nsplit = (int)((3L * M + 31) / 32);
    if (nsplit < 1) nsplit = 1;
    size_t need = (size_t)nsplit * M * (2 * P + 1);
    cplx *dst = out;
    if (nsplit > 1) {
        if (need > c->part_elems) return gs_fail(c, GS_ERR_STATE, "translation scratch too small");
        dst = c->part;
    }
    dim3 grid(gx, nsplit);
    cudaEvent_t e0, e1;
    const bool timed = gs_prof_pair(c, &e0, &e1, precision);
    if (precision == GS_C64) {
        const long nel = (long)M * (2 * P + 1);
        GS_COUNT_LAUNCH(c);
        k_beta_to_c64<<<(int)((nel + 255) / 256), 256, 0, c->stream>>>(beta, nel, c->b32);
    }
    if (timed) cudaEventRecord(e0, c->stream);
    GS_COUNT_LAUNCH(c);
    if (precision == GS_C64)
        k_translate_c64<P, WARPS><<<grid, WARPS * 32, 0, c->stream>>>(c->img32, M, c->b32, (float)c->L.k2,
                                                                      a.alpha, nsplit, dst);
    else if (c->htab)
        k_translate_f64_tab<P, WARPS><<<grid, WARPS * 32, 0, c->stream>>>(c->htab, M, beta, a.alpha, nsplit, dst);
    else
        k_translate_f64<P, WARPS><<<grid, WARPS * 32, 0, c->stream>>>(c->xy, M, beta, c->L.k2, c->L.d, a.alpha,
                                                                      nsplit, dst);
    if (timed) cudaEventRecord(e1, c->stream);
    if (nsplit > 1) {
        long len = (long)M * (2 * P + 1);
        GS_COUNT_LAUNCH(c);
        k_sum_partials<<<(int)((len + 255) / 256), 256, 0, c->stream>>>(c->part, nsplit, len, out);
    }
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

}  // namespace

size_t gs_translate_scratch_elems(int M, int p) { return (size_t)64 * M * (2 * p + 1); }

size_t gs_pair_table_elems(int M, int p) { return (size_t)3 * M * M * (4 * p + 1); }

template <int P>
static int build_table(gs_ctx *c) {
    const long tot = 3L * c->M * c->M;
    GS_COUNT_LAUNCH(c);
    k_pair_table<P, cplx><<<(int)((tot + 255) / 256), 256, 0, c->stream>>>(c->xy, c->M, c->L.k2, c->L.d, c->htab,
                                                                           3L * c->M);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

// complex64 table of M inclusions at xy: rounded from the FP64 table htab (nullable) when given,
// else computed in FP64 directly; its tensor map; the kernel's shared-memory attribute (set eagerly,
// outside any stream capture)
template <int P>
static int build_tab32(gs_ctx *c, const double *xy, int M, const cplx *htab, gs_tab32 *t, cudaStream_t st) {
    constexpr int NQ = 4 * P + 1;
    const long S = 3L * M, SP = t->sp;
    if (htab) {
        const long tot = (long)M * NQ * S;
        GS_COUNT_LAUNCH(c);
        k_table_to_c64<<<(int)((tot + 255) / 256), 256, 0, st>>>(htab, (long)M * NQ, S, SP, t->h);
    } else {
        const long tot = S * M;
        GS_COUNT_LAUNCH(c);
        k_pair_table<P, float2><<<(int)((tot + 255) / 256), 256, 0, st>>>(xy, M, c->L.k2, c->L.d, t->h, SP);
    }
    GS_CHECK_LAUNCH(c);
    GS_TRY(gs_make_map_plain(c, &t->map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, t->h, (long)M * NQ, S, SP * 8, TILE, NQ));
    GS_CUDA(c, cudaFuncSetAttribute(k_translate_c64_tab<P, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Tab32Layout<P, 4>::SMEM));
    return GS_OK;
}

int gs_build_pair_table(gs_ctx *c) {
    switch (c->p) {
        case 1: return build_table<1>(c);
        case 2: return build_table<2>(c);
        case 3: return build_table<3>(c);
        case 4: return build_table<4>(c);
        case 5: return build_table<5>(c);
        case 6: return build_table<6>(c);
        case 7: return build_table<7>(c);
        case 8: return build_table<8>(c);
        case 10: return build_table<10>(c);
        case 12: return build_table<12>(c);
        case 16: return build_table<16>(c);
        default: return gs_fail(c, GS_ERR_ARG, "multipole order p must be one of 1-8, 10, 12, 16");
    }
}

size_t gs_tab32_bytes(int M, int p) {
    const long SP = (3L * M + TILE - 1) / TILE * TILE;
    return sizeof(float2) * (size_t)SP * M * (4 * p + 1);
}

// allocates and builds t (t->h owned by the caller afterwards); GS_ERR_OOM if the allocation fails
int gs_tab32_build(gs_ctx *c, const double *xy, int M, int p, const cplx *htab, gs_tab32 *t, cudaStream_t st) {
    t->sp = (3L * M + TILE - 1) / TILE * TILE;
    if (cudaMalloc((void **)&t->h, gs_tab32_bytes(M, p)) != cudaSuccess) {
        cudaGetLastError();
        t->h = nullptr;
        return GS_ERR_OOM;
    }
    int r;
    switch (p) {
        case 1: r = build_tab32<1>(c, xy, M, htab, t, st); break;
        case 2: r = build_tab32<2>(c, xy, M, htab, t, st); break;
        case 3: r = build_tab32<3>(c, xy, M, htab, t, st); break;
        case 4: r = build_tab32<4>(c, xy, M, htab, t, st); break;
        case 5: r = build_tab32<5>(c, xy, M, htab, t, st); break;
        case 6: r = build_tab32<6>(c, xy, M, htab, t, st); break;
        case 7: r = build_tab32<7>(c, xy, M, htab, t, st); break;
        case 8: r = build_tab32<8>(c, xy, M, htab, t, st); break;
        case 10: r = build_tab32<10>(c, xy, M, htab, t, st); break;
        case 12: r = build_tab32<12>(c, xy, M, htab, t, st); break;
        case 16: r = build_tab32<16>(c, xy, M, htab, t, st); break;
        default: r = gs_fail(c, GS_ERR_ARG, "multipole order p must be one of 1-8, 10, 12, 16");
    }
    if (r != GS_OK) {
        cudaFree(t->h);
        t->h = nullptr;
    }
    return r;
}

int gs_tab32_translate(gs_ctx *c, const gs_tab32 &t, int M, int p, const cplx *beta, cplx alpha, float2 *b3,
                       cplx *part, size_t part_elems, cplx *out, const int *active, cudaStream_t st) {
    switch (p) {
        case 1: return launch_tab32<1>(c, t, M, beta, alpha, b3, part, part_elems, out, active, st, false);
        case 2: return launch_tab32<2>(c, t, M, beta, alpha, b3, part, part_elems, out, active, st, false);
        case 3: return launch_tab32<3>(c, t, M, beta, alpha, b3, part, part_elems, out, active, st, false);
        case 4: return launch_tab32<4>(c, t, M, beta, alpha, b3, part, part_elems, out, active, st, false);
        case 5: return launch_tab32<5>(c, t, M, beta, alpha, b3, part, part_elems, out, active, st, false);
        case 6: return launch_tab32<6>(c, t, M, beta, alpha, b3, part, part_elems, out, active, st, false);
        case 7: return launch_tab32<7>(c, t, M, beta, alpha, b3, part, part_elems, out, active, st, false);
        case 8: return launch_tab32<8>(c, t, M, beta, alpha, b3, part, part_elems, out, active, st, false);
        case 10: return launch_tab32<10>(c, t, M, beta, alpha, b3, part, part_elems, out, active, st, false);
        case 12: return launch_tab32<12>(c, t, M, beta, alpha, b3, part, part_elems, out, active, st, false);
        case 16: return launch_tab32<16>(c, t, M, beta, alpha, b3, part, part_elems, out, active, st, false);
        default: return gs_fail(c, GS_ERR_ARG, "multipole order p must be one of 1-8, 10, 12, 16");
    }
}

// The complex64 translation reads a complex64 copy of the pair table, 3M (rounded up to 32) x M x
// (4p+1) values (1.18 GB at M = 1000, p = 12), when it fits the table budget (half the free device
// memory unless set); otherwise (tab32_off) it recomputes the coefficients in FP32 on the fly.
int gs_ensure_table32(gs_ctx *c) {
    if (c->tab32.h || c->tab32_off) return GS_OK;
    size_t fr = 0, totm = 0;
    GS_CUDA(c, cudaMemGetInfo(&fr, &totm));
    const double budget = c->table_budget_gb >= 0 ? c->table_budget_gb * 1e9 : 0.5 * (double)fr;
    if ((double)gs_tab32_bytes(c->M, c->p) > budget) {
        c->tab32_off = true;
        return GS_OK;
    }
    const int r = gs_tab32_build(c, c->xy, c->M, c->p, c->htab, &c->tab32, c->stream);
    if (r == GS_ERR_OOM) {
        c->tab32_off = true;
        return GS_OK;
    }
    if (r != GS_OK) c->tab32_off = true;
    return r;
}

// GS_ERR_TIMEOUT (and the flag cleared) if a bounded wait of the table-driven complex64 translation
// gave up since the last check; synchronises the stream
int gs_check_table_wait(gs_ctx *c) {
    if (!c->terr) return GS_OK;
    int h = 0;
    GS_CUDA(c, cudaMemcpyAsync(&h, c->terr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!h) return GS_OK;
    GS_CUDA(c, cudaMemsetAsync(c->terr, 0, sizeof(int), c->stream));
    return gs_fail(c, GS_ERR_TIMEOUT, "complex64 translation: a device wait gave up");
}

// The complex64 translation keeps the Hankel values in their natural scale: the largest is
// |H_2p(k2 R_min)| ~ (2p-1)!/pi (2/(k2 R_min))^{2p} for k2 R_min below the order; above ~1e36 (the
// FP32 range ends at 3.4e38) it would overflow, so such geometries are refused for GS_C64.
int gs_c64_range(gs_ctx *c) {
    const int q = 2 * c->p;
    const double z = c->L.k2 * c->min_center_dist;
    double l10 = 0.0;
    if (z > 0.0 && z < q) l10 = (std::lgamma((double)q) - std::log(GS_PI)) / std::log(10.0) + q * std::log10(2.0 / z);
    if (!(z > 0.0) || l10 > 36.0)
        return gs_fail(c, GS_ERR_ARG, "complex64 translation: |H_" + std::to_string(q) + "(k2 R_min = " +
                                          std::to_string(z) + ")| ~ 1e" + std::to_string((int)l10) +
                                          " exceeds the FP32 range; use GS_FP64 (or a smaller p)");
    return GS_OK;
}

int gs_translate_impl(gs_ctx *c, const AngleData &a, const cplx *beta, cplx *out, int precision) {
    if (precision == GS_C64) GS_TRY(gs_c64_range(c));
    switch (c->p) {
        case 1: return launch_translate<1>(c, a, beta, out, precision);
        case 2: return launch_translate<2>(c, a, beta, out, precision);
        case 3: return launch_translate<3>(c, a, beta, out, precision);
        case 4: return launch_translate<4>(c, a, beta, out, precision);
        case 5: return launch_translate<5>(c, a, beta, out, precision);
        case 6: return launch_translate<6>(c, a, beta, out, precision);
        case 7: return launch_translate<7>(c, a, beta, out, precision);
        case 8: return launch_translate<8>(c, a, beta, out, precision);
        case 10: return launch_translate<10>(c, a, beta, out, precision);
        case 12: return launch_translate<12>(c, a, beta, out, precision);
        case 16: return launch_translate<16>(c, a, beta, out, precision);
        default: return gs_fail(c, GS_ERR_ARG, "multipole order p must be one of 1-8, 10, 12, 16");
    }
}

// ---- allocation-free variant --------------------------------------------------------------------
// Some callers cannot allocate device memory at the point where they need a translation: a host
// framework that owns the whole device heap through its own pool, a real-time loop that forbids
// allocation (and the implicit synchronisation cudaMalloc/cudaFree bring) after start-up, or code
// that runs before any context has been created for it.  gs_translate_noalloc serves them: it
// needs no gs_ctx and keeps the chunk partials of the translation in a fixed array compiled into
// this library instead of a buffer obtained from cudaMalloc.

// Chunk partials of gs_translate_noalloc: 2^19 complex128 values (8 MiB), held on every GPU that
// loads this library until the process exits.
#define GS_NOALLOC_CAPACITY (1 << 19)
static __device__ __align__(256) cplx gs_noalloc_partials[GS_NOALLOC_CAPACITY];

namespace {

constexpr int GS_NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
cplx *g_noalloc_scratch[GS_NOALLOC_MAX_DEVICES] = {};   // device address of the array, per device

// Smallest distance between a target centre and any source image (all pairs, images l = -1, 0, 1,
// the target's own l = 0 copy left out), as the bit pattern of a non-negative double (ordered like
// the value) folded into *slot by atomicMin.  One thread per target.
__global__ void k_noalloc_min_dist(const double *xy, int M, double d, unsigned long long *slot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double m2 = 1e300;
    if (i < M) {
        const double xi = xy[2 * i], yi = xy[2 * i + 1];
        for (int j = 0; j < M; ++j) {
            const double dy = yi - xy[2 * j + 1];
            const double dx0 = xi - xy[2 * j];
#pragma unroll
            for (int l = -1; l <= 1; ++l) {
                if (l == 0 && j == i) continue;
                const double dx = dx0 - l * d;
                m2 = fmin(m2, dx * dx + dy * dy);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) m2 = fmin(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    if ((threadIdx.x & 31) == 0 && i - (int)(threadIdx.x & 31) < M)
        atomicMin(slot, (unsigned long long)__double_as_longlong(sqrt(m2)));
}

// The complex64 form's range check without a context: the smallest image distance R_min is found
// on the device (into the array's last slot), read back (one stream synchronisation) and tested as
// in gs_c64_range: |H_2p(k2 R_min)| ~ (2p-1)!/pi (2/(k2 R_min))^{2p} must stay below 1e36.
int noalloc_c64_range(int M, int p, const double *xy, double k, double d, cudaStream_t st,
                      unsigned long long *slot) {
    if (cudaMemsetAsync(slot, 0x7f, sizeof(unsigned long long), st) != cudaSuccess) return GS_ERR_CUDA;
    k_noalloc_min_dist<<<(M + 127) / 128, 128, 0, st>>>(xy, M, d, slot);
    unsigned long long bits = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&bits, slot, sizeof(bits), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GS_ERR_CUDA;
    double rmin;
    std::memcpy(&rmin, &bits, sizeof(rmin));
    const int q = 2 * p;
    const double z = k * rmin;
    double l10 = 0.0;
    if (z > 0.0 && z < q) l10 = (std::lgamma((double)q) - std::log(GS_PI)) / std::log(10.0) + q * std::log10(2.0 / z);
    return (!(z > 0.0) || l10 > 36.0) ? GS_ERR_ARG : GS_OK;
}

template <int P>
int noalloc_launch(int M, const double *xy, const cplx *beta, double k, double d, cplx alpha, int precision,
                   cplx *out, cudaStream_t st, cplx *scratch, int sms) {
    constexpr int WARPS = 4;
    constexpr int NC = 2 * P + 1;
    const int gx = (M + WARPS - 1) / WARPS;
    int nsplit = (int)((sms * 8L + gx - 1) / gx);
    if (nsplit > 64) nsplit = 64;
    if ((long)nsplit * 32 > 3L * M) nsplit = (int)((3L * M + 31) / 32);
    if (nsplit < 1) nsplit = 1;
    const long len = (long)M * NC;
    // complex64 form, from the end of the array: one slot for the range check's distance, the
    // converted coefficients (ceil(len/2) complex128 slots) and the (hi, lo) float image
    // coordinates (3M slots); the partials take what is left
    const long room = (precision == GS_C64) ? GS_NOALLOC_CAPACITY - 1 - (len + 1) / 2 - 3L * M : GS_NOALLOC_CAPACITY;
    if (room < len) return GS_ERR_ARG;   // exceeds the fixed scratch
    if ((long)nsplit * len > room) nsplit = (int)(room / len);
    if (nsplit < 1) return GS_ERR_ARG;
    dim3 grid(gx, nsplit);
    if (precision == GS_C64) {
        GS_TRY(noalloc_c64_range(M, P, xy, k, d, st, (unsigned long long *)(scratch + GS_NOALLOC_CAPACITY - 1)));
        float4 *img = (float4 *)(scratch + room);
        cplxf *b32 = (cplxf *)(scratch + room + 3L * M);
        k_images_c64<<<(int)((3L * M + 255) / 256), 256, 0, st>>>(xy, M, d, img);
        k_beta_to_c64<<<(int)((len + 255) / 256), 256, 0, st>>>(beta, len, b32);
        k_translate_c64<P, WARPS><<<grid, WARPS * 32, 0, st>>>(img, M, b32, (float)k, alpha, nsplit, scratch);
    } else
        k_translate_f64<P, WARPS><<<grid, WARPS * 32, 0, st>>>(xy, M, beta, k, d, alpha, nsplit, scratch);
    k_sum_partials<<<(int)((len + 255) / 256), 256, 0, st>>>(scratch, nsplit, len, out);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // namespace

extern "C" int gs_translate_noalloc(int M, int p, const double *xy_dev, double k2, double d, double alpha_re,
                                    double alpha_im, const gs_c128 *beta_dev, gs_c128 *alpha_dev, int precision,
                                    void *cuda_stream) {
    // every size check precedes any device work
    if (M < 1 || !xy_dev || !beta_dev || !alpha_dev || (const void *)beta_dev == (const void *)alpha_dev)
        return GS_ERR_ARG;
    if (!(k2 > 0.0) || !(d > 0.0) || (precision != GS_FP64 && precision != GS_C64)) return GS_ERR_ARG;
    switch (p) {
        case 1: case 2: case 3: case 4: case 5: case 6: case 7: case 8: case 10: case 12: case 16: break;
        default: return GS_ERR_ARG;
    }
    if ((long)M * (2 * p + 1) > GS_NOALLOC_CAPACITY) return GS_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= GS_NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    cplx *scratch = nullptr;
    {
        // first call on a device: look up the device address of the array (host code only sees a
        // stand-in symbol); done once per device, with that device current
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_scratch[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, gs_noalloc_partials) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return GS_ERR_CUDA;
            }
            g_noalloc_scratch[dev] = (cplx *)ptr;
        }
        scratch = g_noalloc_scratch[dev];
    }
    int sms = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    const cplx alpha = C(alpha_re, alpha_im);
    const cplx *beta = (const cplx *)beta_dev;
    cplx *out = (cplx *)alpha_dev;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    switch (p) {
        case 1: return noalloc_launch<1>(M, xy_dev, beta, k2, d, alpha, precision, out, st, scratch, sms);
        case 2: return noalloc_launch<2>(M, xy_dev, beta, k2, d, alpha, precision, out, st, scratch, sms);
        case 3: return noalloc_launch<3>(M, xy_dev, beta, k2, d, alpha, precision, out, st, scratch, sms);
        case 4: return noalloc_launch<4>(M, xy_dev, beta, k2, d, alpha, precision, out, st, scratch, sms);
        case 5: return noalloc_launch<5>(M, xy_dev, beta, k2, d, alpha, precision, out, st, scratch, sms);
        case 6: return noalloc_launch<6>(M, xy_dev, beta, k2, d, alpha, precision, out, st, scratch, sms);
        case 7: return noalloc_launch<7>(M, xy_dev, beta, k2, d, alpha, precision, out, st, scratch, sms);
        case 8: return noalloc_launch<8>(M, xy_dev, beta, k2, d, alpha, precision, out, st, scratch, sms);
        case 10: return noalloc_launch<10>(M, xy_dev, beta, k2, d, alpha, precision, out, st, scratch, sms);
        case 12: return noalloc_launch<12>(M, xy_dev, beta, k2, d, alpha, precision, out, st, scratch, sms);
        default: return noalloc_launch<16>(M, xy_dev, beta, k2, d, alpha, precision, out, st, scratch, sms);
    }
}
