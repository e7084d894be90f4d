// peak.cu -- measured FMA throughput of the CUDA cores (FP64 and FP32): the
// denominators of the solve kernels' arithmetic rooflines.
//
// Every thread of a grid that fills all SMs runs CHAINS independent chains
// x <- x * a + b (no chain depends on another, so the pipe, not the FMA
// latency, bounds the rate); the time of one launch under CUDA events gives
// flops = 2 * chains * iterations * threads per second.  The chains' final
// values feed a store (to a device variable) that never happens at run time
// but that the compiler cannot prove dead.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace chemgpu {
namespace {

constexpr int PEAK_THREADS = 256;

// the never-taken store's target (a valid address, whatever the element type)
__device__ double g_peak_sink;
constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_UNROLL = 8;

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) fma_peak_kernel(T a, T b, long long iters) {
  T x[PEAK_CHAINS];
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (long long i = 0; i < iters; i += PEAK_UNROLL) {
#pragma unroll
    for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
      for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) s += x[c];
  if (s == (T)-1.25) g_peak_sink = (double)s;   // never: every x stays positive
}

template <typename T>
cudaError_t time_peak(int blocks, long long iters, cudaStream_t s, float *ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  // a = 1 - 2^-20, b = 2^-20: every chain converges to 1 and stays finite
  const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1048576.0);
  if ((e = cudaEventRecord(e0, s)) == cudaSuccess) {
    fma_peak_kernel<T><<<blocks, PEAK_THREADS, 0, s>>>(a, b, iters);
    if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaEventRecord(e1, s)) == cudaSuccess &&
        (e = cudaEventSynchronize(e1)) == cudaSuccess)
      e = cudaEventElapsedTime(ms, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

template <typename T>
cudaError_t measure(cudaStream_t s, double *tflops, double *ms_out) {
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<T>, PEAK_THREADS, 0)) != cudaSuccess)
    return e;
  const int blocks = n_sm * (per_sm > 0 ? per_sm : 1);
  // calibrate to about 50 ms per launch, then take the best of three
  long long iters = 4096;
  float ms = 0.0f;
  for (int k = 0; k < 12; ++k) {
    if ((e = time_peak<T>(blocks, iters, s, &ms)) != cudaSuccess) return e;
    if (ms >= 10.0f) break;
    iters *= 4;
  }
  iters = (long long)((double)iters * 50.0 / (ms > 0.0f ? ms : 1.0f)) / PEAK_UNROLL * PEAK_UNROLL;
  if (iters < PEAK_UNROLL) iters = PEAK_UNROLL;
  float best = 0.0f;
  for (int k = 0; k < 3; ++k) {
    if ((e = time_peak<T>(blocks, iters, s, &ms)) != cudaSuccess) return e;
    if (k == 0 || ms < best) best = ms;
  }
  const double flops = 2.0 * PEAK_CHAINS * (double)iters * (double)blocks * PEAK_THREADS;
  *tflops = flops / (best * 1e-3) / 1e12;
  *ms_out = best;
  return cudaSuccess;
}

}  // namespace
}  // namespace chemgpu

using namespace chemgpu;

extern "C" int chem_measure_fma_peak(int32_t precision, double *tflops, double *ms, void *stream) {
  set_last_error("");
  if (!tflops || !ms) {
    set_last_error("NULL argument");
    return CHEM_EINVAL;
  }
  if (precision != 64 && precision != 32) {
    set_last_error("precision must be 64 or 32");
    return CHEM_EINVAL;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e = precision == 64 ? measure<double>(s, tflops, ms) : measure<float>(s, tflops, ms);
  if (e != cudaSuccess) {
    set_last_error(std::string("FMA peak kernel: ") + cudaGetErrorString(e));
    return CHEM_ECUDA;
  }
  return 0;
}
