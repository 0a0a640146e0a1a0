// fc_probe.cu -- arithmetic throughput probe of the current GPU.
//
// The FP64-row smoother kernels (patch apply, residual) are bound by the
// FP64 pipe on this part, not by HBM, so their roofline needs the pipe's
// throughput.  The probe runs independent FMA chains on every SM (no memory
// traffic inside the timed loop) and times one launch with CUDA events after
// a warm-up launch.  It reads nothing but the clocks the GPU runs at and
// changes no setting.
#include <math.h>

#include "fc_internal.cuh"

namespace {

constexpr int kChains = 8;    // independent FMA chains per thread (hide the pipe latency)
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains_kernel(int iters, T a, T c, T* sink) {
  T v[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) v[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) v[k] = v[k] * a + c;  // one FMA each
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += v[k];
  // the store keeps the chains alive; the condition is never true for the
  // bounded values the chains take (a < 1, |c| small)
  if (s == (T)-12345.0) sink[blockIdx.x] = s;
}

template <typename T>
cudaError_t run_probe(double* flops, double* ms_out) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chains_kernel<T>, kThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int blocks = nsm * per_sm;
  T* sink = nullptr;
  e = cudaMalloc((void**)&sink, sizeof(T) * blocks);
  if (e != cudaSuccess) return e;
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  // FP64 runs at a small fraction of the FP32 rate: fewer iterations keep
  // both launches near 20-50 ms
  const int iters = sizeof(T) == 8 ? 4096 : 262144;
  float ms = 0.f;
  if (e == cudaSuccess) {
    fma_chains_kernel<T><<<blocks, kThreads, 0, s>>>(iters / 4, (T)0.999999, (T)1e-7, sink);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) {
    fma_chains_kernel<T><<<blocks, kThreads, 0, s>>>(iters, (T)0.999999, (T)1e-7, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  fc::note_launches(2);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (s) cudaStreamDestroy(s);
  cudaFree(sink);
  if (e != cudaSuccess) return e;
  const double fmas = (double)blocks * kThreads * kChains * (double)iters;
  *flops = ms > 0.f ? 2.0 * fmas / (ms * 1e-3) : 0.0;
  if (ms_out) *ms_out = ms;
  return cudaSuccess;
}

}  // namespace

extern "C" fc_status fc_probe_fma_rate(int precision, double* flop_per_s, double* launch_ms) {
  if (!flop_per_s || (precision != 0 && precision != 1)) return FC_ERR_INVALID;
  cudaError_t e = precision == 0 ? run_probe<double>(flop_per_s, launch_ms) : run_probe<float>(flop_per_s, launch_ms);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FC_ERR_CUDA;
  }
  return FC_OK;
}
