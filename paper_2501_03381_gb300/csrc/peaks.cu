// Arithmetic peaks of the CUDA cores, measured: the FP32 (FFMA) and FP64
// (DFMA) rates that bound the nplet kernels and the FP64 re-factor.  Every
// thread runs CH independent multiply-add chains (enough in flight to cover
// the pipe latency at any occupancy), the grid fills every SM several times
// over, and the rate is counted as 2 FLOP per multiply-add over the CUDA-
// event time of the launch.  Not part of the method; it gives the roofline
// denominators of the measurement.
#include "internal.cuh"

namespace thoi {

constexpr int PK_NT = 256;
constexpr int PK_CH = 8;

template <typename T>
__global__ void __launch_bounds__(PK_NT) k_fma_peak(int iters, T b, T c, T* __restrict__ sink) {
  T x[PK_CH];
#pragma unroll
  for (int j = 0; j < PK_CH; j++) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 16; u++)
#pragma unroll
      for (int j = 0; j < PK_CH; j++) x[j] = fma(x[j], b, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < PK_CH; j++) s += x[j];
  // never true for the arguments the host passes; keeps the chains alive
  if (s == (T)-1.2345e30) sink[blockIdx.x] = s;
}

}  // namespace thoi

using namespace thoi;

extern "C" thoi_status thoi_fma_peak(int32_t fp64, int32_t iters, double* tflops, double* ms,
                                     void* stream) {
  if (!tflops || iters < 1) return THOI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return THOI_ERR_CUDA;
  const int grid = sms * 8;
  void* sink = nullptr;
  if (cudaMalloc(&sink, (size_t)grid * 8) != cudaSuccess) return THOI_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float t = 0.f;
  for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {  // the first launch warms up
    e = cudaEventRecord(e0, s);
    if (fp64)
      k_fma_peak<double><<<grid, PK_NT, 0, s>>>(iters, 0.999999, 1e-7, (double*)sink);
    else
      k_fma_peak<float><<<grid, PK_NT, 0, s>>>(iters, 0.999999f, 1e-7f, (float*)sink);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? THOI_ERR_OOM : THOI_ERR_CUDA;
  }
  const double flop = 2.0 * (double)grid * PK_NT * PK_CH * 16.0 * (double)iters;
  *tflops = flop / ((double)t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return THOI_OK;
}
