// lbm_peak.cu -- the measured FP64 instruction rate of the device, against which the FP64
// step's roofline is reported (the step is bound by the FP64 pipe, not by HBM).
#include <cuda_runtime.h>

#include "../../include/lbm.h"

namespace {

constexpr int PEAK_NT = 256;
constexpr int PEAK_CHAINS = 8;

// Eight independent chains of FP64 fused multiply-adds per thread (a = a b + c, with
// b < 1 so that the values converge to c / (1 - b) and stay normal).  The result is
// stored only under a condition that the values never meet, so the loop is kept but
// nothing is written.
__global__ void __launch_bounds__(PEAK_NT) dfma_loop(double* out, int iters, double b, double c)
{
    double a[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
    if (s == -1.0) out[blockIdx.x * PEAK_NT + threadIdx.x] = s;
}

}  // namespace

extern "C" int lbm_measure_fp64_rate(double* ginst_per_s, double* ms_out)
{
    if (!ginst_per_s) return LBM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    const int blocks = 8 * sms, iters = 4096;
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * PEAK_NT * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = -1.0f;
    for (int rep = 0; rep < 8 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0);
        dfma_loop<<<blocks, PEAK_NT>>>(out, iters, 0.9999, 1e-3);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep >= 3 && (best < 0.0f || ms < best)) best = ms;  // 3 untimed launches
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || best <= 0.0f) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    const double inst = (double)blocks * PEAK_NT * PEAK_CHAINS * iters;
    *ginst_per_s = inst / (best * 1e-3) / 1e9;
    if (ms_out) *ms_out = best;
    return LBM_OK;
}
