// Measured FP32 FMA throughput of the current device (sph_fp32_peak, declared in
// include/sph.h): the denominator of the pair sweeps' arithmetic roofline.  The paper has
// no counterpart; this is a measurement aid of the library.
//
// Every thread runs kChains independent FMA chains (x = x * a + b with |a| < 1, so the
// values stay finite), enough independent work per warp to cover the FMA latency on every
// scheduler; the grid is a multiple of the SM count.  The result is written only under a
// condition that never holds for these inputs, so the compiler keeps every FMA.
#include <cuda_runtime.h>

#include "../../include/sph.h"

namespace sph {
void set_error(const char* fmt, ...);
}

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

__global__ void __launch_bounds__(kThreads) k_fma_peak(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = (float)(threadIdx.x + c);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < kUnroll; u++)
#pragma unroll
      for (int c = 0; c < kChains; c++) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  if (s == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true: keeps the work
}

}  // namespace

extern "C" sph_status sph_fp32_peak(int32_t iters, double* tflops, int32_t* sm_count, double* ms) {
  if (iters < 1 || !tflops) { sph::set_error("iters must be >= 1 and tflops non-null"); return SPH_ERR_INVALID; }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) { sph::set_error("%s", cudaGetErrorString(e)); return SPH_ERR_CUDA; }
  int blocks = sms * kBlocksPerSM;
  float* out = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaStream_t s = nullptr;
  e = cudaMalloc(&out, sizeof(float) * (size_t)blocks * kThreads);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {  // the first launch warms up
    k_fma_peak<<<blocks, kThreads, 0, s>>>(out, iters, 0.999f, 0.5f);
    cudaEventRecord(t0, s);
    k_fma_peak<<<blocks, kThreads, 0, s>>>(out, iters, 0.999f, 0.5f);
    cudaEventRecord(t1, s);
    e = cudaEventSynchronize(t1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, t0, t1);
    if (e == cudaSuccess && (best == 0.f || t < best)) best = t;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  if (e != cudaSuccess) { sph::set_error("%s", cudaGetErrorString(e)); return SPH_ERR_CUDA; }
  double flop = 2.0 * (double)kChains * kUnroll * (double)iters * (double)blocks * kThreads;
  *tflops = flop / (best * 1e-3) / 1e12;
  if (sm_count) *sm_count = sms;
  if (ms) *ms = best;
  return SPH_OK;
}
