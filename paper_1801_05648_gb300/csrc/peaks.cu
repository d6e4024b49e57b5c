// FMA-throughput probes behind include/fsi_peaks.h: every thread runs eight
// independent multiply-add chains a <- a * b + c (b slightly below 1, so the
// values stay normal and bounded), enough warps per SM to cover the pipe's
// latency; FMAs per second = threads x 8 x trips / kernel time.
#include "../../include/fsi_peaks.h"

#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T b, T c, T* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  T a0 = T(t & 255) * T(1e-3), a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
  T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
    a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
  }
  out[t] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}

template <class T>
int probe(int iters, int reps, double* rate, double* best) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -3;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -3;
  const int grid = sms * kCtasPerSm;
  T* out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = 0;
  float best_ms = -1.0f;
  if (cudaMalloc(&out, sizeof(T) * (size_t)grid * kThreads) != cudaSuccess) return -3;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = -3;
  }
  for (int r = -1; rc == 0 && r < reps; ++r) {
    cudaEventRecord(e0, s);
    k_fma_chains<T><<<grid, kThreads, 0, s>>>(iters, T(0.9999999), T(1e-7), out);
    cudaEventRecord(e1, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) { rc = -3; break; }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r >= 0 && (best_ms < 0.0f || ms < best_ms)) best_ms = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  if (rc != 0) return rc;
  *rate = (double)grid * kThreads * 8.0 * (double)iters / (best_ms * 1e-3);
  if (best) *best = best_ms;
  return 0;
}

}  // namespace

extern "C" int fsi_probe_fma_rate(int bits, int iters, int reps, double* fma_per_s, double* best_ms) {
  if (!fma_per_s || iters < 1 || reps < 1) return -1;
  if (bits == 64) return probe<double>(iters, reps, fma_per_s, best_ms);
  if (bits == 32) return probe<float>(iters, reps, fma_per_s, best_ms);
  return -1;
}
