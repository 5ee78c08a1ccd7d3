// Arithmetic-pipe ceilings of the CUDA cores, measured: FP32 FFMA and FP64
// DFMA throughput of the current GPU.  The roofline fractions of the FP32
// and FP64 forms of chi divide by these.
//
// Each thread runs 8 independent FMA chains (x <- x a + b, converging to a
// fixed point so that no value overflows or becomes subnormal), enough
// independent work per warp to keep the pipes issuing; the grid holds 8 CTAs
// of 256 threads per SM.  Timed with CUDA events after a warm-up launch.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* __restrict__ sink, long long iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = static_cast<T>(threadIdx.x + c) * static_cast<T>(1e-3);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // a store no value can skip (x is never exactly -1), so the chains stay live
  if (s == static_cast<T>(-1)) sink[blockIdx.x] = s;
}

template <typename T>
int run(long long iters, double* tflops, double* ms_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -6;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -6;
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T) * sms * 8) != cudaSuccess) return -5;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256;
  const T a = static_cast<T>(0.9999), b = static_cast<T>(1e-4);
  k_fma_chains<T><<<blocks, threads>>>(sink, iters / 8 + 1, a, b);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, threads>>>(sink, iters, a, b);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) return -6;
  const double flops = 2.0 * kChains * kUnroll * static_cast<double>(iters) * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return 0;
}

}  // namespace

extern "C" {

// FMA throughput of the current device in TFLOP/s (2 flops per FMA), best of
// three timed launches: fp64 = 0 for FFMA (FP32), 1 for DFMA (FP64).  iters
// sets the work (iterations of 8 x 16 FMAs per thread); ms_out (may be NULL)
// receives the best launch time.  Returns 0, -5 (allocation failed) or -6
// (a CUDA call failed).
int gw_fma_peak(int fp64, long long iters, double* tflops, double* ms_out) {
  if (!tflops || iters <= 0) return -1;
  return fp64 ? run<double>(iters, tflops, ms_out) : run<float>(iters, tflops, ms_out);
}

}  // extern "C"
