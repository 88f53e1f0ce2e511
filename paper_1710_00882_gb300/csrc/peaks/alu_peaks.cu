// Throughput of the FP32 and FP64 fused multiply-add pipes of the device, measured
// with independent FMA chains: the measured peak beside which the benchmark reports
// the force kernels' achieved flop rates (the force evaluation is bound by these
// pipes, not by memory).  Built into its own library (libalu_peaks.so), separate from
// libtersoff.so: it is a measurement aid, not part of the Tersoff C ABI.
//
// Each thread runs CHAINS independent chains x <- fma(x, a, b) for `iters` rounds,
// enough independent work per warp to cover the FMA latency.  a = 1 - 2^-12 and a
// small b keep every x near 1 (no overflow, no subnormals).  The chains' sum is
// stored only under a condition that never holds, so the work stays live.
// Flops = 2 per FMA.  Timed with CUDA events on a stream of the library's own; no
// clock or power setting of the device is touched.
#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;

template <class T, int CHAINS>
__global__ void __launch_bounds__(kThreads) k_fma_chains(const T *__restrict__ seed, T *__restrict__ sink, int iters)
{
  const T a = seed[0], b = seed[1];
  T x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = seed[2] + T(c) * T(1e-3) + T(threadIdx.x) * T(1e-6);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  if (s == T(-1)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T, int CHAINS>
int measure(int blocks, int iters, int reps, double *tflops, double *ms_best)
{
  T *seed = nullptr, *sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = 0;
  const T h_seed[3] = {T(1) - T(1.0 / 4096.0), T(1.0 / 8192.0), T(0.5)};
  if (cudaMalloc(&seed, 3 * sizeof(T)) != cudaSuccess ||
      cudaMalloc(&sink, (size_t)blocks * kThreads * sizeof(T)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = -2;
  }
  if (rc == 0 && cudaMemcpyAsync(seed, h_seed, sizeof(h_seed), cudaMemcpyHostToDevice, st) != cudaSuccess) rc = -3;
  float best = 0.0f;
  for (int r = 0; rc == 0 && r < reps + 1; ++r) {   // the first run is a warm-up
    cudaEventRecord(e0, st);
    k_fma_chains<T, CHAINS><<<blocks, kThreads, 0, st>>>(seed, sink, iters);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      rc = -3;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (rc == 0) {
    const double flops = 2.0 * CHAINS * (double)iters * blocks * kThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    *ms_best = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (seed) cudaFree(seed);
  if (sink) cudaFree(sink);
  return rc;
}

}  // namespace

// out[0] FP32 FMA TFLOP/s, out[1] its best launch time (ms), out[2] FP64 FMA TFLOP/s,
// out[3] its best launch time (ms), out[4] the number of SMs.  Runs on the device
// current at the call.  Returns 0, or a negative value when a CUDA call failed.
extern "C" int alu_peaks_measure(double *out)
{
  if (!out) return -1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -3;
  // 8 blocks of 256 threads per SM: every scheduler holds several warps of 8 chains
  int rc = measure<float, 8>(8 * sms, 4096, 5, &out[0], &out[1]);
  if (rc == 0) rc = measure<double, 4>(8 * sms, 128, 3, &out[2], &out[3]);
  out[4] = sms;
  return rc;
}
