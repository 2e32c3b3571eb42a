// Measured arithmetic peaks (FMA throughput) for the roofline denominators of ALU-bound
// kernels.  Each thread runs 8 independent FMA chains so the pipes stay full; the grid
// covers every SM several times.  Timed with CUDA events on the given stream.
#include "common.cuh"

namespace nlp {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T *out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = x[i] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == (T)12345.678) out[0] = s;   // keeps the chains live
}

}  // namespace nlp

extern "C" nlp_status nlp_measure_alu_peak(int precision, void *stream, double *flops_per_s) {
    using namespace nlp;
    if (!flops_per_s || (precision != NLP_FP64 && precision != NLP_FP32)) return NLP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void *buf = nullptr;
    NLP_CUDA_TRY(cudaMalloc(&buf, 64));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 8, threads = 256;
    const int iters = precision == NLP_FP64 ? 2048 : 65536;
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        if (precision == NLP_FP64)
            k_fma_peak<double><<<blocks, threads, 0, st>>>((double *)buf, iters, 0.999999, 1e-7);
        else
            k_fma_peak<float><<<blocks, threads, 0, st>>>((float *)buf, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double fl = 2.0 * 8.0 * (double)iters * blocks * threads;
        if (rep > 0 && ms > 0) best = fl / (ms * 1e-3) > best ? fl / (ms * 1e-3) : best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (cudaGetLastError() != cudaSuccess) return NLP_ERR_CUDA;
    *flops_per_s = best;
    return NLP_OK;
}
