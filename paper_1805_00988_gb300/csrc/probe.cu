// probe.cu -- arithmetic peak microbenchmarks used as roofline denominators.
//
// The complex128 per-gate path does 8 FP64 FMAs per amplitude and can be
// bound by FP64 issue rather than HBM; the complex64 tile passes by FP32 FMA
// issue.  These kernels measure the FMA rates of this GPU: every thread runs
// eight independent FMA chains (enough to cover the pipeline latency), the
// grid fills every SM, and the device time of the launch is taken with CUDA
// events.  Results feed the "alu" roofline of the bench.
#include <algorithm>

#include "internal.cuh"

namespace qsim {

namespace {

constexpr int kProbeIters = 4096;

__global__ void __launch_bounds__(256) k_fma_f32(float *out, float a, float b)
{
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 1234.5f) out[blockIdx.x] = s;     // never true; keeps the chains live
}

__device__ __forceinline__ void fma2(float &x0, float &x1, float a0, float a1, float b0, float b1)
{
    asm("{.reg .b64 rx, ra, rb;\n"
        " mov.b64 rx, {%0,%1};\n mov.b64 ra, {%2,%3};\n mov.b64 rb, {%4,%5};\n"
        " fma.rn.f32x2 rx, rx, ra, rb;\n mov.b64 {%0,%1}, rx;}\n"
        : "+f"(x0), "+f"(x1) : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

__global__ void __launch_bounds__(256) k_fma_f32x2(float *out, float a, float b)
{
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) fma2(x[2 * i], x[2 * i + 1], a, a, b, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += x[i];
    if (s == 1234.5f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_fma_f64(double *out, double a, double b)
{
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < kProbeIters / 8; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 1234.5) out[blockIdx.x] = s;
}

}  // namespace

}  // namespace qsim

using namespace qsim;

extern "C" int sim_measure_fma_peak(int which, double *tflops)
{
    set_error("");
    if (!tflops || which < 0 || which > 2) return fail(SIM_EINVAL, "sim_measure_fma_peak: which must be 0..2");
    int dev = 0, sms = 0;
    QSIM_CUDA(cudaGetDevice(&dev));
    QSIM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;
    void *buf = nullptr;
    QSIM_CUDA(cudaMalloc(&buf, blocks * sizeof(double)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0);
        double flops;
        if (which == 0) {
            k_fma_f32<<<blocks, threads>>>((float *)buf, 0.999f, 1e-3f);
            flops = 2.0 * 8 * kProbeIters * (double)blocks * threads;
        } else if (which == 1) {
            k_fma_f32x2<<<blocks, threads>>>((float *)buf, 0.999f, 1e-3f);
            flops = 2.0 * 16 * kProbeIters * (double)blocks * threads;
        } else {
            k_fma_f64<<<blocks, threads>>>((double *)buf, 0.999, 1e-3);
            flops = 2.0 * 8 * (kProbeIters / 8) * (double)blocks * threads;
        }
        cudaEventRecord(e1);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaFree(buf);
            return cuda_fail(e, "fma probe");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    QSIM_CUDA(cudaGetLastError());
    *tflops = best;
    return SIM_OK;
}
