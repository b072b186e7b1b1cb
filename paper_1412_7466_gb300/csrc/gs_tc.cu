// Tensor-core (tcgen05) matrix product for the multi-right-hand-side translation.
//
// The translation of R coefficient vectors at once (R incidence angles of one geometry, Sec. 4.2
// Eq. trans with the image phases of each angle) is a dense contraction: with the image-separated
// blocks T_l (l = -1, 0, 1; T_l[(i,m),(j,n)] = H_{n-m}(k R) e^{i(n-m) Th} of the pair (i, j, l)),
//   alpha_r = [T_-1  T_0  T_1] [a_r^-1 beta_r; beta_r; a_r beta_r]     (a_r = e^{i k1 cos(theta_r) d}),
// and in real arithmetic [Re; Im] rows against [Re; Im] columns of 2x2 blocks [[Re, -Im], [Im, Re]].
// That product, C[M][N] = A[M][K] B[N][K]^T with A (the operator, bfloat16), B (the stacked
// right-hand sides, bfloat16) and C in FP32, runs here on the 5th-generation tensor cores:
//
//   * one CTA per 128 x 256 tile of C, four warps; thread 0 of warp 0 streams the K dimension in
//     64-wide slices through a 4-stage ring of shared-memory buffers with TMA (128-byte swizzle),
//     thread 0 of warp 1 issues tcgen05.mma (M 128, N 256, K 16, BF16 in, FP32 accumulate) into a
//     256-column tensor-memory accumulator and releases each stage with tcgen05.commit; after the
//     last slice all four warps read their 32 TMEM lanes with tcgen05.ld and write C.
//   * every wait on an mbarrier is bounded (about 2 s); a wait that gives up sets *err, the kernel
//     still waits (bounded) for its own tensor-core work, frees its tensor memory and returns.
//   * split K (gridDim.z slices): CTA z accumulates only its share of the K slices and writes its
//     tile to the z-th copy of C; the caller adds the copies in FP64.  The tensor memory accumulates
//     in FP32 along K, so shorter chains keep sums with large cancelling terms accurate.
#include <cuda.h>

#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "gs_internal.h"
#include "gs_tma.cuh"

namespace {

constexpr int TBM = 128, TBN = 256, TBK = 64, TST = 4;
constexpr int TA_BYTES = TBM * TBK * 2;               // 16 KB
constexpr int TB_BYTES = TBN * TBK * 2;               // 32 KB
constexpr int TSTAGE = TA_BYTES + TB_BYTES;           // 48 KB
constexpr int TSMEM = TST * TSTAGE + 1024 + 256;      // stages (1024-aligned) + barriers
constexpr int TMEM_COLS = 256;

// instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1), A and B bfloat16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                           ((uint32_t)(TBM >> 4) << 24);

// shared-memory matrix descriptor of a K-major tile written by TMA with the 128-byte swizzle:
// start address >> 4 (bits 0-13), leading byte offset (unused for this layout; 16 B), stride byte
// offset 1024 B between 8-row groups (bits 32-45), descriptor version 1 (bits 46-47), layout
// SWIZZLE_128B = 2 (bits 61-63)
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(128, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, float *__restrict__ C,
          int M, int N, int K, int *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + TST * TSTAGE);   // full[TST], empty[TST], accum
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * TST + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TBM, n0 = blockIdx.y * TBN;
    const int nk = K / TBK;
    const int kb0 = (int)((long)blockIdx.z * nk / gridDim.z), kb1 = (int)((long)(blockIdx.z + 1) * nk / gridDim.z);
    C += (size_t)blockIdx.z * M * N;
    const uint32_t s_base = smem_u32(smem);
    const uint32_t b_full = smem_u32(bars), b_empty = smem_u32(bars + TST), b_acc = smem_u32(bars + 2 * TST);

    if (threadIdx.x == 0) {
        for (int s = 0; s < TST; ++s) {
            mbar_init(b_full + 8 * s, 1);
            mbar_init(b_empty + 8 * s, 1);
        }
        mbar_init(b_acc, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0 && lane == 0) {
        // producer: K slices of A (128 x 64) and B (256 x 64) into the stage ring
        int stage = 0;
        uint32_t phase = 0;
        for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(b_empty + 8 * stage, phase ^ 1)) {
                ok = false;
                break;
            }
            const uint32_t sa = s_base + stage * TSTAGE;
            mbar_expect_tx(b_full + 8 * stage, TSTAGE);
            tma_load_2d(sa, &tmA, b_full + 8 * stage, kb * TBK, m0);
            tma_load_2d(sa + TA_BYTES, &tmB, b_full + 8 * stage, kb * TBK, n0);
            if (++stage == TST) {
                stage = 0;
                phase ^= 1;
            }
        }
    } else if (warp == 1 && lane == 0) {
        // tensor-core issue: four K = 16 steps per slice (32 bytes along the swizzled rows)
        int stage = 0;
        uint32_t phase = 0;
        for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(b_full + 8 * stage, phase)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sa = s_base + stage * TSTAGE, sb = sa + TA_BYTES;
#pragma unroll
            for (int kk = 0; kk < TBK / 16; ++kk)
                umma_bf16(tmem, desc_sw128(sa + 32 * kk), desc_sw128(sb + 32 * kk), kb != kb0 || kk != 0);
            umma_commit(b_empty + 8 * stage);
            if (++stage == TST) {
                stage = 0;
                phase ^= 1;
            }
        }
        umma_commit(b_acc);   // arrives once every MMA issued above has completed
    }
    __syncwarp();

    // epilogue: warp w owns TMEM lanes 32w..32w+31 = rows m0 + 32w + lane
    const bool acc_ok = mbar_wait(b_acc, 0);
    tc_fence_after();
    if (acc_ok) {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < TBN; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row < M) {
                float4 *dst = (float4 *)(C + (size_t)row * N + n0 + c0);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    dst[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                         __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
            }
        }
    }
    if (!ok || !acc_ok) atomicExch(err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    });
    return fn;
}

// 2-D bfloat16 tensor map of a row-major rows x cols matrix, box 64 (cols) x box_rows, 128-byte swizzle
int make_map(gs_ctx *c, CUtensorMap *m, const void *base, long rows, long cols, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return gs_fail(c, GS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)TBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return gs_fail(c, GS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
    return GS_OK;
}

}  // namespace

// 2-D tensor map over a row-major rows x cols array (row stride row_bytes, a multiple of 16), box
// box_cols x box_rows elements, no swizzle (a box lands in shared memory row after row);
// out-of-range elements of a box read as zero
int gs_make_map_plain(gs_ctx *c, CUtensorMap *m, CUtensorMapDataType dt, const void *base, long rows, long cols,
                      long row_bytes, int box_cols, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return gs_fail(c, GS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return gs_fail(c, GS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
    return GS_OK;
}

// C[M][N] = A[M][K] B[N][K]^T (bfloat16 in, FP32 out) on stream st; M % 128, N % 256, K % 64 == 0,
// 16-byte aligned rows.  err_dev: device int, set to 1 if a wait gave up.  kslices > 1 splits K:
// C then holds kslices consecutive M x N partial products (kslices <= K / 64), to be summed.
int gs_tc_gemm_impl(gs_ctx *c, const void *A, const void *B, float *C, long M, long N, long K, int *err_dev,
                    cudaStream_t st, int kslices) {
    if (M <= 0 || N <= 0 || K <= 0 || M % TBM || N % TBN || K % TBK)
        return gs_fail(c, GS_ERR_ARG, "tensor-core product needs M % 128 == 0, N % 256 == 0, K % 64 == 0");
    if (kslices < 1 || kslices > K / TBK || kslices > 65535) return gs_fail(c, GS_ERR_ARG, "bad K split");
    if (M / TBM > 2147483647L || N / TBN > 65535 || K > 2147483647L) return gs_fail(c, GS_ERR_ARG, "size out of range");
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) & 15) return gs_fail(c, GS_ERR_ARG, "pointers must be 16-byte aligned");
    CUtensorMap ma, mb;
    GS_TRY(make_map(c, &ma, A, M, K, TBM));
    GS_TRY(make_map(c, &mb, B, N, K, TBN));
    // the function attribute is per device: set once per device, outside any stream capture (the
    // first product on a device is never inside one: gs_tc_split_prepare and the eager calls come first)
    {
        static std::mutex mu;
        static bool done[64] = {};
        std::lock_guard<std::mutex> lock(mu);
        const int d = (c->device >= 0 && c->device < 64) ? c->device : 0;
        if (!done[d]) {
            GS_CUDA(c, cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, TSMEM));
            done[d] = true;
        }
    }
    GS_COUNT_LAUNCH(c);
    k_tc_gemm<<<dim3((unsigned)(M / TBM), (unsigned)(N / TBN), (unsigned)kslices), 128, TSMEM, st>>>(
        ma, mb, C, (int)M, (int)N, (int)K, err_dev);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

namespace {

// A[2(i nc + m) + a][2(s nc + n) + b] for the source image s = (l+1) M + j of target i: the real
// 2x2 form [[Re h, -Im h], [Im h, Re h]] of h = H_{n-m}(k R) e^{i(n-m) Th}, (R, Th) = polar(c_i -
// c_j - l d) (zero for the particle itself, l = 0, j = i).  One thread per (target, source image):
// H_0, H_1 seeded in FP64, orders by upward recurrence, rounded to bfloat16 on the way out.
// Entries are stored rescaled, h gamma^(|m| + |n|) (orders m, n in -p..p): with gamma = min(1, k r_min)
// and R >= 2 r_min (disks do not overlap), |H_q(k R)| (2 gamma / (k R))^q <= (q - 1)!/pi keeps every
// entry inside the bfloat16 range (23!/pi = 8e21 at p = 12); the coefficients are divided by
// gamma^|n| on the way in and the results by gamma^|m| on the way out.
//
// With A1 and A2 given, each entry is split into three bfloat16 parts: A holds its rounding, A1 the
// rounding of the remainder and A2 the rounding of what is then left (A + A1 + A2 carries ~24
// significant bits, the precision of FP32, instead of 8).
template <int P>
__global__ void k_tc_build_A(const double *__restrict__ xy, int M, double k, double d, double gamma, long lda,
                             __nv_bfloat16 *__restrict__ A, __nv_bfloat16 *__restrict__ A1,
                             __nv_bfloat16 *__restrict__ A2) {
    constexpr int NC = 2 * P + 1, NQ = 4 * P + 1;
    const long S = 3L * M;
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long)M * S) return;
    const int i = (int)(id / S);
    const long s = id - (long)i * S;
    const int l = (int)(s / M) - 1;
    const int j = (int)(s - (long)(l + 1) * M);
    if (l == 0 && j == i) return;   // stays zero
    const double dx = xy[2 * i] - (xy[2 * j] + l * d), dy = xy[2 * i + 1] - xy[2 * j + 1];
    const double R = hypot(dx, dy), z = k * R, twoz = 2.0 / z;
    cplx h[NQ];                       // h[q + 2P] = H_q(z) e^{i q Th}
    cplx Hm1, Hc;
    hankel01(z, Hm1, Hc);
    const cplx u1 = C(dx / R, dy / R);
    cplx up = u1;
    h[2 * P] = Hm1;
#pragma unroll
    for (int q = 1; q <= 2 * P; ++q) {
        h[2 * P + q] = cmul(Hc, up);
        const cplx hm = cmul(Hc, cconj(up));
        h[2 * P - q] = (q & 1) ? C(-hm.x, -hm.y) : hm;
        if (q < 2 * P) {
            const cplx Hn = csub(cscale(Hc, q * twoz), Hm1);
            Hm1 = Hc;
            Hc = Hn;
            up = cmul(up, u1);
        }
    }
    double gp[P + 1];   // gamma^e
    gp[0] = 1.0;
#pragma unroll
    for (int e = 1; e <= P; ++e) gp[e] = gp[e - 1] * gamma;
    const long col0 = 2 * s * NC;
#pragma unroll 1
    for (int m = 0; m < NC; ++m) {
        const double gm = gp[m < P ? P - m : m - P];
        const long r_re = (2 * ((long)i * NC + m)) * lda + col0, r_im = (2 * ((long)i * NC + m) + 1) * lda + col0;
        __nv_bfloat162 *re_row = (__nv_bfloat162 *)(A + r_re);
        __nv_bfloat162 *im_row = (__nv_bfloat162 *)(A + r_im);
#pragma unroll
        for (int n = 0; n < NC; ++n) {
            const cplx v = cscale(h[n - m + 2 * P], gm * gp[n < P ? P - n : n - P]);
            double vr = v.x, vi = v.y;
            __nv_bfloat16 *parts[3] = {A, A1, A2};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (!parts[q]) break;
                const __nv_bfloat16 pr = __float2bfloat16_rn((float)vr), pi = __float2bfloat16_rn((float)vi);
                ((__nv_bfloat162 *)(parts[q] + r_re))[n] = __halves2bfloat162(pr, __hneg(pi));
                ((__nv_bfloat162 *)(parts[q] + r_im))[n] = __halves2bfloat162(pi, pr);
                vr -= (double)__bfloat162float(pr);
                vi -= (double)__bfloat162float(pi);
            }
        }
    }
}

// Bt[r][2(s nc + n) + b] = part b of a_r^l beta_r[j nc + n], s = (l+1) M + j (a_r^-1 = conj(a_r))
struct GammaPow {
    double inv[17];   // gamma^-e, e = 0..p (p <= 16)
};

__global__ void k_tc_pack_B(const cplx *__restrict__ beta, const cplx *__restrict__ alpha, int R, int M, int nc,
                            GammaPow gpw, long ldb, __nv_bfloat16 *__restrict__ Bt) {
    const long n = (long)M * nc;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;   // over R x 3n complex entries
    if (e >= (long)R * 3 * n) return;
    const int r = (int)(e / (3 * n));
    const long q = e - (long)r * 3 * n;      // = s nc + n_order
    const int l = (int)(q / n) - 1;
    const cplx b = beta[(long)r * n + (q - (long)(l + 1) * n)];
    const cplx a = alpha[r];
    const int p = nc / 2, o = (int)(q % nc) - p;
    const cplx v = cscale(l == 0 ? b : (l == 1 ? cmul(a, b) : cmul(cconj(a), b)), gpw.inv[abs(o)]);
    ((__nv_bfloat162 *)(Bt + (long)r * ldb))[q] = __floats2bfloat162_rn((float)v.x, (float)v.y);
}

// out_r[e] = (C[2e][r] + i C[2e+1][r]) / gamma^|m|, e = i nc + m
__global__ void k_tc_unpack(const float *__restrict__ Cm, long ldc, int R, long n, int nc, GammaPow gpw,
                            cplx *__restrict__ out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)R * n) return;
    const int r = (int)(e / n);
    const long q = e - (long)r * n;
    const int o = (int)(q % nc) - nc / 2;
    const double sc = gpw.inv[abs(o)];
    out[e] = C(sc * (double)Cm[(2 * q) * ldc + r], sc * (double)Cm[(2 * q + 1) * ldc + r]);
}

// three-part split of the stacked right-hand sides: row b R + r of Bt (b = 0, 1, 2) holds part b of
// a_r^l beta_r[j nc + n] / gamma^|n| (layout of k_tc_pack_B): its bfloat16 rounding, then the
// rounding of the remainder, then the rounding of what is left
__global__ void k_tc_pack_B_split(const cplx *__restrict__ beta, const cplx *__restrict__ alpha, int R, int M, int nc,
                                  GammaPow gpw, long ldb, __nv_bfloat16 *__restrict__ Bt) {
    const long n = (long)M * nc;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)R * 3 * n) return;
    const int r = (int)(e / (3 * n));
    const long q = e - (long)r * 3 * n;
    const int l = (int)(q / n) - 1;
    const cplx b = beta[(long)r * n + (q - (long)(l + 1) * n)];
    const cplx a = alpha[r];
    const int p = nc / 2, o = (int)(q % nc) - p;
    const cplx v = cscale(l == 0 ? b : (l == 1 ? cmul(a, b) : cmul(cconj(a), b)), gpw.inv[abs(o)]);
    double vr = v.x, vi = v.y;
#pragma unroll
    for (int part = 0; part < 3; ++part) {
        const __nv_bfloat16 pr = __float2bfloat16_rn((float)vr), pi = __float2bfloat16_rn((float)vi);
        ((__nv_bfloat162 *)(Bt + (long)(part * R + r) * ldb))[q] = __halves2bfloat162(pr, pi);
        vr -= (double)__bfloat162float(pr);
        vi -= (double)__bfloat162float(pi);
    }
}

// out_r[e] = sum over operator part a and coefficient part b with a + b <= 2 of A_a B_b, / gamma^|m|:
// Ca = A_a [B_0; ...; B_{2-a}]^T holds column b R + r for each b <= 2 - a, in S K-slice copies of
// Mr x ld_a each (summed here in FP64); rows 2e and 2e + 1 are the real and imaginary parts
__global__ void k_tc_unpack_split(const float *__restrict__ C0, long ld0, const float *__restrict__ C1, long ld1,
                                  const float *__restrict__ C2, long ld2, long Mr, int S, int R, long n, int nc,
                                  GammaPow gpw, cplx *__restrict__ out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)R * n) return;
    const int r = (int)(e / n);
    const long q = e - (long)r * n;
    const int o = (int)(q % nc) - nc / 2;
    const double sc = gpw.inv[abs(o)];
    double re = 0.0, im = 0.0;
    for (int z = 0; z < S; ++z) {
        const float *c0 = C0 + (size_t)z * Mr * ld0, *c1 = C1 + (size_t)z * Mr * ld1, *c2 = C2 + (size_t)z * Mr * ld2;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            re += (double)c0[(2 * q) * ld0 + b * R + r];
            im += (double)c0[(2 * q + 1) * ld0 + b * R + r];
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            re += (double)c1[(2 * q) * ld1 + b * R + r];
            im += (double)c1[(2 * q + 1) * ld1 + b * R + r];
        }
        re += (double)c2[(2 * q) * ld2 + r];
        im += (double)c2[(2 * q + 1) * ld2 + r];
    }
    out[e] = C(sc * re, sc * im);
}

// out[0] = min over the inclusions of the radius (one block)
__global__ void k_min_radius(const double *__restrict__ radius, int M, double *__restrict__ out) {
    __shared__ double sh[32];
    double v = 1e300;
    for (int i = threadIdx.x; i < M; i += blockDim.x) v = fmin(v, radius[i]);
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 1e300;
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) out[0] = v;
    }
}

template <int P>
int build_A(gs_ctx *c, long lda) {
    const long tot = 3L * c->M * c->M;
    GS_COUNT_LAUNCH(c);
    k_tc_build_A<P><<<(int)((tot + 127) / 128), 128, 0, c->stream>>>(c->xy, c->M, c->L.k2, c->L.d, c->tc_gamma, lda,
                                                                     (__nv_bfloat16 *)c->tcA,
                                                                     (__nv_bfloat16 *)c->tcA_sp[0],
                                                                     (__nv_bfloat16 *)c->tcA_sp[1]);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

inline long round_up(long v, long m) { return (v + m - 1) / m * m; }

}  // namespace

// the bfloat16 operator [T_-1 T_0 T_1] of the current geometry in real 2x2 form (built on first use);
// with_split: also the second and third bfloat16 parts of every entry (the three-part split)
int gs_tc_operator(gs_ctx *c, bool with_split = false) {
    const long n = c->n();
    const long rows = round_up(2 * n, TBM), cols = round_up(6 * n, TBK);
    if (c->tcA && c->tcA_rows == rows && c->tcA_cols == cols && (!with_split || (c->tcA_sp[0] && c->tcA_sp[1])))
        return GS_OK;
    void **bufs[3] = {&c->tcA, &c->tcA_sp[0], &c->tcA_sp[1]};
    for (void **b : bufs) {
        if (*b) cudaFree(*b);
        *b = nullptr;
    }
    const size_t bytes = sizeof(__nv_bfloat16) * (size_t)rows * cols;
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < (with_split ? 3 : 1) && e == cudaSuccess; ++q) e = cudaMalloc(bufs[q], bytes);
    if (e != cudaSuccess) {
        for (void **b : bufs) {
            if (*b) cudaFree(*b);
            *b = nullptr;
        }
        cudaGetLastError();
        return gs_fail(c, GS_ERR_OOM, std::string("cudaMalloc (tensor-core operator): ") + cudaGetErrorString(e));
    }
    c->tcA_rows = rows;
    c->tcA_cols = cols;
    for (void **b : bufs)
        if (*b) GS_CUDA(c, cudaMemsetAsync(*b, 0, bytes, c->stream));
    GS_COUNT_LAUNCH(c);
    k_min_radius<<<1, 1024, 0, c->stream>>>(c->radius, c->M, c->dscal + 10);
    GS_CHECK_LAUNCH(c);
    GS_CUDA(c, cudaMemcpyAsync(c->hscal + 10, c->dscal + 10, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    c->tc_gamma = std::min(1.0, c->L.k2 * c->hscal[10]);
    switch (c->p) {
        case 1: return build_A<1>(c, cols);
        case 2: return build_A<2>(c, cols);
        case 3: return build_A<3>(c, cols);
        case 4: return build_A<4>(c, cols);
        case 5: return build_A<5>(c, cols);
        case 6: return build_A<6>(c, cols);
        case 7: return build_A<7>(c, cols);
        case 8: return build_A<8>(c, cols);
        case 10: return build_A<10>(c, cols);
        case 12: return build_A<12>(c, cols);
        case 16: return build_A<16>(c, cols);
        default: return gs_fail(c, GS_ERR_ARG, "multipole order p must be one of 1-8, 10, 12, 16");
    }
}

extern "C" int gs_translate_multi(gs_ctx *c, int R, const gs_c128 *alpha_host, const gs_c128 *beta_dev,
                                  gs_c128 *out_dev) {
    if (!c) return GS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, "cudaSetDevice");
    if (!c->factored) return gs_fail(c, GS_ERR_STATE, "gs_factor has not run");
    if (R < 1 || R > 65536 || !alpha_host || !beta_dev || !out_dev)
        return gs_fail(c, GS_ERR_ARG, "need 1..65536 right-hand sides and non-null pointers");
    cudaStream_t st = c->stream;
    const long n = c->n();
    GS_TRY(gs_tc_operator(c));
    const long K = c->tcA_cols, Mr = c->tcA_rows, Rp = round_up(R, TBN);
    // scratch: alphas, stacked right-hand sides (bfloat16), product (FP32), wait flag
    const size_t need = sizeof(cplx) * R + sizeof(__nv_bfloat16) * (size_t)Rp * K + 256 + sizeof(float) * (size_t)Mr * Rp +
                        256 + 256;
    if (need > c->tc_scratch_bytes) {
        if (c->tc_scratch) cudaFree(c->tc_scratch);
        c->tc_scratch = nullptr;
        c->tc_scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&c->tc_scratch, need);
        if (e != cudaSuccess) {
            c->tc_scratch = nullptr;
            cudaGetLastError();
            return gs_fail(c, GS_ERR_OOM, std::string("cudaMalloc (tensor-core scratch): ") + cudaGetErrorString(e));
        }
        c->tc_scratch_bytes = need;
        c->tc_zeroed_rp = c->tc_zeroed_k = c->tc_zeroed_R = -1;
    }
    uint8_t *p = (uint8_t *)c->tc_scratch;
    cplx *al = (cplx *)p;
    p += round_up(sizeof(cplx) * R, 256);
    __nv_bfloat16 *Bt = (__nv_bfloat16 *)p;
    p += round_up(sizeof(__nv_bfloat16) * (size_t)Rp * K, 256);
    float *Cm = (float *)p;
    p += round_up(sizeof(float) * (size_t)Mr * Rp, 256);
    int *err = (int *)p;
    GS_CUDA(c, cudaMemcpyAsync(al, alpha_host, sizeof(cplx) * R, cudaMemcpyHostToDevice, st));
    if (c->tc_zeroed_rp != Rp || c->tc_zeroed_k != K || c->tc_zeroed_R != R) {
        // padding rows (r >= R) and columns (>= 6n) stay zero; the packing overwrites the rest
        GS_CUDA(c, cudaMemsetAsync(Bt, 0, sizeof(__nv_bfloat16) * (size_t)Rp * K, st));
        c->tc_zeroed_rp = Rp;
        c->tc_zeroed_k = K;
        c->tc_zeroed_R = R;
    }
    GS_CUDA(c, cudaMemsetAsync(err, 0, sizeof(int), st));
    GammaPow gpw;
    gpw.inv[0] = 1.0;
    for (int e = 1; e <= 16; ++e) gpw.inv[e] = gpw.inv[e - 1] / c->tc_gamma;
    GS_COUNT_LAUNCH(c);
    k_tc_pack_B<<<(int)((3L * n * R + 255) / 256), 256, 0, st>>>((const cplx *)beta_dev, al, R, c->M, c->nc, gpw, K,
                                                                 Bt);
    GS_CHECK_LAUNCH(c);
    cudaEvent_t e0, e1;
    const bool timed = gs_prof_pair(c, &e0, &e1, GS_TC_BF16);
    if (timed) cudaEventRecord(e0, st);
    GS_TRY(gs_tc_gemm_impl(c, c->tcA, Bt, Cm, Mr, Rp, K, err, st));
    if (timed) cudaEventRecord(e1, st);
    GS_COUNT_LAUNCH(c);
    k_tc_unpack<<<(int)((n * R + 255) / 256), 256, 0, st>>>(Cm, Rp, R, n, c->nc, gpw, (cplx *)out_dev);
    GS_CHECK_LAUNCH(c);
    int herr = 0;
    GS_CUDA(c, cudaMemcpyAsync(c->hscal + 8, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GS_CUDA(c, cudaStreamSynchronize(st));
    std::memcpy(&herr, c->hscal + 8, sizeof(int));
    if (herr) return gs_fail(c, GS_ERR_TIMEOUT, "tensor-core product: a device wait gave up");
    return GS_OK;
}

namespace {
// K slices of the three-part product: each CTA's FP32 accumulation runs over 1/16 of the operator's
// 6n columns (the slices are added in FP64), which keeps the sums' cancellation errors near those of
// the CUDA-core complex64 translation, whose FP32 chains are similarly short
constexpr int SPLIT_KSLICES = 16;

// scratch of the three-part product for R right-hand sides: the stacked coefficient parts Bt
// (3R rows, padded to 256) and the products C_a = A_a [B_0 .. B_{2-a}]^T of the operator parts
// (SPLIT_KSLICES copies each)
struct SplitLayout {
    long K, Mr, Np[3];
    int S;
    __nv_bfloat16 *Bt;
    float *Cp[3];
    size_t bytes;
};
SplitLayout split_layout(gs_ctx *c, int R, void *base) {
    SplitLayout L;
    L.K = c->tcA_cols;
    L.Mr = c->tcA_rows;
    L.S = (int)std::min<long>(SPLIT_KSLICES, L.K / TBK);
    size_t off[4];
    off[0] = 0;
    for (int a = 0; a < 3; ++a) L.Np[a] = round_up((3L - a) * R, TBN);
    size_t o = (size_t)round_up(sizeof(__nv_bfloat16) * L.Np[0] * L.K, 256);
    for (int a = 0; a < 3; ++a) {
        off[a + 1] = o;
        o += (size_t)round_up(sizeof(float) * L.S * L.Mr * L.Np[a], 256);
    }
    L.bytes = o;
    uint8_t *p = (uint8_t *)base;
    L.Bt = (__nv_bfloat16 *)p;
    for (int a = 0; a < 3; ++a) L.Cp[a] = p ? (float *)(p + off[a + 1]) : nullptr;
    return L;
}
GammaPow gamma_pows(double gamma) {
    GammaPow g;
    g.inv[0] = 1.0;
    for (int e = 1; e <= 16; ++e) g.inv[e] = g.inv[e - 1] / gamma;
    return g;
}
}  // namespace

int gs_tc_split_prepare(gs_ctx *c, int R) {
    if (R < 1 || R > 65536) return gs_fail(c, GS_ERR_ARG, "need 1..65536 right-hand sides");
    GS_CUDA(c, cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, TSMEM));
    GS_TRY(gs_tc_operator(c, true));
    const SplitLayout L = split_layout(c, R, nullptr);
    if (L.bytes > c->sp_scratch_bytes) {
        if (c->sp_scratch) cudaFree(c->sp_scratch);
        c->sp_scratch = nullptr;
        c->sp_scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&c->sp_scratch, L.bytes);
        if (e != cudaSuccess) {
            c->sp_scratch = nullptr;
            cudaGetLastError();
            return gs_fail(c, GS_ERR_OOM, std::string("cudaMalloc (tensor-core split scratch): ") + cudaGetErrorString(e));
        }
        c->sp_scratch_bytes = L.bytes;
        c->sp_zeroed_R = -1;
    }
    if (c->sp_zeroed_R != R) {
        // padding rows (>= 3R) and columns (>= 6n) of the stacked coefficient parts stay zero
        const SplitLayout Lb = split_layout(c, R, c->sp_scratch);
        GS_CUDA(c, cudaMemsetAsync(Lb.Bt, 0, sizeof(__nv_bfloat16) * (size_t)Lb.Np[0] * Lb.K, c->stream));
        c->sp_zeroed_R = R;
    }
    return GS_OK;
}

int gs_tc_split_translate(gs_ctx *c, int R, const cplx *alpha_dev, const cplx *x, cplx *out, int *err_dev,
                          cudaStream_t st) {
    if (!c->tcA || !c->tcA_sp[0] || !c->tcA_sp[1] || c->sp_zeroed_R != R)
        return gs_fail(c, GS_ERR_STATE, "gs_tc_split_prepare has not run");
    const long n = c->n();
    const SplitLayout L = split_layout(c, R, c->sp_scratch);
    const GammaPow gpw = gamma_pows(c->tc_gamma);
    const void *Ap[3] = {c->tcA, c->tcA_sp[0], c->tcA_sp[1]};
    GS_COUNT_LAUNCH(c);
    k_tc_pack_B_split<<<(int)((3L * n * R + 255) / 256), 256, 0, st>>>(x, alpha_dev, R, c->M, c->nc, gpw, L.K, L.Bt);
    GS_CHECK_LAUNCH(c);
    for (int a = 0; a < 3; ++a)
        GS_TRY(gs_tc_gemm_impl(c, Ap[a], L.Bt, L.Cp[a], L.Mr, L.Np[a], L.K, err_dev, st, L.S));
    GS_COUNT_LAUNCH(c);
    k_tc_unpack_split<<<(int)((n * R + 255) / 256), 256, 0, st>>>(L.Cp[0], L.Np[0], L.Cp[1], L.Np[1], L.Cp[2], L.Np[2],
                                                                   L.Mr, L.S, R, n, c->nc, gpw, out);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

extern "C" int gs_translate_multi_split(gs_ctx *c, int R, const gs_c128 *alpha_host, const gs_c128 *beta_dev,
                                        gs_c128 *out_dev) {
    if (!c) return GS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, "cudaSetDevice");
    if (!c->factored) return gs_fail(c, GS_ERR_STATE, "gs_factor has not run");
    if (R < 1 || R > 65536 || !alpha_host || !beta_dev || !out_dev)
        return gs_fail(c, GS_ERR_ARG, "need 1..65536 right-hand sides and non-null pointers");
    GS_TRY(gs_tc_split_prepare(c, R));
    cplx *al = nullptr;
    GS_CUDA(c, cudaMalloc((void **)&al, sizeof(cplx) * R + 256));
    int *err = (int *)((uint8_t *)al + round_up(sizeof(cplx) * R, 16));
    int st = GS_OK;
    cudaError_t e = cudaMemcpyAsync(al, alpha_host, sizeof(cplx) * R, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) st = gs_fail(c, GS_ERR_CUDA, cudaGetErrorString(e));
    cudaEvent_t e0, e1;
    const bool timed = st == GS_OK && gs_prof_pair(c, &e0, &e1, GS_TC_BF16);
    if (timed) cudaEventRecord(e0, c->stream);
    if (st == GS_OK) st = gs_tc_split_translate(c, R, al, (const cplx *)beta_dev, (cplx *)out_dev, err, c->stream);
    if (timed) cudaEventRecord(e1, c->stream);
    int herr = 0;
    if (st == GS_OK) {
        e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = gs_fail(c, GS_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(al);
    if (st == GS_OK && herr) st = gs_fail(c, GS_ERR_TIMEOUT, "tensor-core product: a device wait gave up");
    return st;
}

extern "C" int gs_tc_gemm_bf16(gs_ctx *c, const void *A_dev, const void *B_dev, float *C_dev, long M, long N,
                               long K) {
    if (!c) return GS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, "cudaSetDevice");
    if (!A_dev || !B_dev || !C_dev) return gs_fail(c, GS_ERR_ARG, "null pointer");
    int *err = nullptr;
    GS_CUDA(c, cudaMalloc((void **)&err, sizeof(int)));
    cudaMemsetAsync(err, 0, sizeof(int), c->stream);
    int st = gs_tc_gemm_impl(c, A_dev, B_dev, C_dev, M, N, K, err, c->stream);
    int herr = 0;
    if (st == GS_OK) {
        cudaError_t e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = gs_fail(c, GS_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaFree(err);
    if (st == GS_OK && herr) st = gs_fail(c, GS_ERR_TIMEOUT, "tensor-core product: a device wait gave up");
    return st;
}
