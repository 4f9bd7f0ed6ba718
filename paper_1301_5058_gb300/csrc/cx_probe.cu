// cx_probe.cu -- cx_alu_peak: the multiply-add rate of one precision,
// measured with a register-only kernel.  The paper has no counterpart; the
// figure is the denominator of the arithmetic roofline of the step kernels
// (GB300's FP64 rate is a small fraction of its FP32 rate, so the FP64
// stepper is judged against the FP64 pipe, measured rather than assumed).
#include <stdio.h>

#include "cx_internal.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;  // independent multiply-add chains per thread

// Each thread advances kProbeChains independent chains x <- x a + c for
// `iters` rounds and writes their sum, so that nothing is optimised away.
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) alu_probe_kernel(T *out, int iters, T a, T c)
{
    T x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = fma(x[k], a, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += x[k];
    out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

int probe_fail(int code, const char *what, cudaError_t e)
{
    char buf[300];
    snprintf(buf, sizeof buf, "cx_alu_peak: %s%s%s", what, e != cudaSuccess ? ": " : "",
             e != cudaSuccess ? cudaGetErrorString(e) : "");
    return cx::record_error(code, buf);
}

}  // namespace

extern "C" int cx_alu_peak(int32_t precision, int32_t repeats, double *flops_per_s)
{
    if (!flops_per_s) return probe_fail(CX_ERR_INVALID_ARG, "flops_per_s must not be NULL", cudaSuccess);
    if (precision != CX_PREC_F64 && precision != CX_PREC_F32)
        return probe_fail(CX_ERR_INVALID_ARG, "precision must be CX_PREC_F64 or CX_PREC_F32", cudaSuccess);
    if (repeats < 1 || repeats > 100)
        return probe_fail(CX_ERR_INVALID_ARG, "repeats must lie in 1..100", cudaSuccess);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms < 1) return probe_fail(CX_ERR_CUDA, "device query", e);
    // enough resident warps to keep either pipe busy; a few milliseconds per
    // launch (FP64 on GB300 runs about 1/64 of the FP32 rate)
    const int blocks = 4 * sms;
    const int iters = precision == CX_PREC_F64 ? 2048 : 65536;
    const size_t elem = precision == CX_PREC_F64 ? sizeof(double) : sizeof(float);
    void *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaMalloc(&out, (size_t)blocks * kProbeThreads * elem);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    double best = 0.0;
    for (int r = -1; r < repeats && e == cudaSuccess; ++r) {  // r = -1: warm-up
        e = cudaEventRecord(t0, st);
        if (precision == CX_PREC_F64)
            alu_probe_kernel<double><<<blocks, kProbeThreads, 0, st>>>((double *)out, iters,
                                                                       0.9999999, 1e-7);
        else
            alu_probe_kernel<float><<<blocks, kProbeThreads, 0, st>>>((float *)out, iters,
                                                                      0.9999999f, 1e-7f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(t1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && r >= 0 && ms > 0.f) {
            const double flops = 2.0 * kProbeChains * (double)iters * blocks * kProbeThreads;
            const double rate = flops / (ms * 1e-3);
            if (rate > best) best = rate;
        }
    }
    const cudaError_t first = e;
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (first != cudaSuccess) return probe_fail(CX_ERR_CUDA, "probe launch", first);
    *flops_per_s = best;
    return CX_OK;
}
