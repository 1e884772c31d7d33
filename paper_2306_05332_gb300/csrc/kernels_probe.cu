// FP64 throughput probe: the FP64 pipe's rate on this device, the ceiling of
// the kernels that issue FP64 arithmetic (the FP64 solve's stages, the
// acceleration).  Eight independent FMA chains per thread keep the pipe busy.
#include "sg_internal.cuh"

namespace sg {

namespace {

__global__ void k_fp64_fma_chains(double* out, int iters, double a, double b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = 1e-3 * (t & 1023) + c;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    out[t] = s;                       // keeps the chains live
}

}  // namespace

cudaError_t probe_fp64_rate(double* tflops, double* ms_out) {
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int threads = 256, blocks = sms * 16, iters = 4096;
    double* out = nullptr;
    if ((e = cudaMalloc(&out, size_t(blocks) * threads * sizeof(double))) != cudaSuccess) return e;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_fp64_fma_chains<<<blocks, threads>>>(out, iters / 8, 0.9999999, 1e-7);      // warm-up
    cudaEventRecord(a);
    k_fp64_fma_chains<<<blocks, threads>>>(out, iters, 0.9999999, 1e-7);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return e;
    // one FMA = 2 flops; 8 chains x iters per thread
    *tflops = 2.0 * 8.0 * iters * double(blocks) * threads / (double(ms) * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return cudaGetLastError();
}

}  // namespace sg
