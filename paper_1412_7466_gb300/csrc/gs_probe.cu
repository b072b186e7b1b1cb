// FMA-throughput probe: the denominator of the ALU roofline of the translation kernels.  Each
// thread runs 8 independent multiply-add chains so that the FMA pipe, not latency, is the limit.
// The packed form issues fma.rn.f32x2 (two FP32 multiply-adds per instruction and lane).
#include <type_traits>

#include "gs_internal.h"

namespace {

template <typename T>
__global__ void k_fma_chains(T *out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = x[i] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_fma2_chains(float2 *out, int iters, float a, float b) {
    unsigned long long x[8], av, bv;
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    av = *reinterpret_cast<const unsigned long long *>(&a2);
    bv = *reinterpret_cast<const unsigned long long *>(&b2);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float2 v = make_float2((float)(threadIdx.x + i), (float)(threadIdx.x + 2 * i));
        x[i] = *reinterpret_cast<const unsigned long long *>(&v);
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[i]) : "l"(av), "l"(bv));
    }
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float2 v = *reinterpret_cast<const float2 *>(&x[i]);
        s.x += v.x;
        s.y += v.y;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
void launch_chains(T *buf, int blocks, int threads, int iters, cudaStream_t st) {
    k_fma_chains<T><<<blocks, threads, 0, st>>>(buf, iters, (T)0.999999, (T)1e-7);
}
template <>
void launch_chains<float2>(float2 *buf, int blocks, int threads, int iters, cudaStream_t st) {
    k_fma2_chains<<<blocks, threads, 0, st>>>(buf, iters, 0.999999f, 1e-7f);
}

template <typename T>
int run(gs_ctx *c, int iters, double *tflops) {
    int dev = c->device, sms = 0;
    GS_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;
    T *buf = nullptr;
    GS_CUDA(c, cudaMalloc((void **)&buf, sizeof(T) * blocks * threads));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    GS_COUNT_LAUNCH(c);
    launch_chains<T>(buf, blocks, threads, iters, c->stream);   // warm-up
    cudaEventRecord(e0, c->stream);
    GS_COUNT_LAUNCH(c);
    launch_chains<T>(buf, blocks, threads, iters, c->stream);
    cudaEventRecord(e1, c->stream);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (err != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, cudaGetErrorString(err));
    const double lanes = std::is_same<T, float2>::value ? 2.0 : 1.0;   // FMAs per instruction and lane
    *tflops = 2.0 * lanes * 8.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
    return GS_OK;
}

}  // namespace

extern "C" int gs_probe_fma(gs_ctx *c, int precision, double *tflops) {
    if (!c || !tflops) return GS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, "cudaSetDevice");
    if (precision == GS_FP64) return run<double>(c, 20000, tflops);
    if (precision == GS_C64) return run<float>(c, 400000, tflops);
    if (precision == GS_PROBE_F32X2) return run<float2>(c, 200000, tflops);
    return gs_fail(c, GS_ERR_ARG, "bad precision");
}
