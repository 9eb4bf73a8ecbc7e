// msf_peak.cu -- FMA throughput of the CUDA cores in FP32 and FP64, the
// denominator of the arithmetic roofline of the flux kernels (the FP64 path
// is bound by the FP64 pipes, not by HBM). A measurement service of the
// library; the method itself does not use it.
//
// Every thread runs kChains independent fused multiply-add chains x <- x a + b
// (|a| < 1, so the values stay bounded and normal) for `iters` iterations;
// the grid fills every SM several times over. Flops = 2 per FMA.
#include <cuda_runtime.h>

#include "../../include/msf.h"

extern "C" void msf_internal_set_error(const char* msg);  // defined with the other entry points

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* sink, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; k++) s += x[k];
  if (s == T(-1)) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

template <typename T>
msf_status run(int iters, double* flops, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, kThreads, 0) != cudaSuccess) {
    msf_internal_set_error("msf_fma_peak: device query failed");
    return MSF_ECUDA;
  }
  const int blocks = sms * (per_sm > 0 ? per_sm : 1) * 4;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    msf_internal_set_error("msf_fma_peak: event creation failed");
    return MSF_ECUDA;
  }
  const T a = T(0.999999), b = T(1e-7);
  float best = 0.0f;
  k_fma_chains<T><<<blocks, kThreads, 0, s>>>(nullptr, iters, a, b);  // warm-up
  for (int rep = 0; rep < 5; rep++) {
    cudaEventRecord(e0, s);
    k_fma_chains<T><<<blocks, kThreads, 0, s>>>(nullptr, iters, a, b);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep == 0 || ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !(best > 0.0f)) {
    msf_internal_set_error("msf_fma_peak: kernel failed");
    return MSF_ECUDA;
  }
  *flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads / (1e-3 * (double)best);
  return MSF_OK;
}

}  // namespace

extern "C" msf_status msf_fma_peak(int32_t precision, double* flops_per_s, void* stream) {
  if (!flops_per_s || (precision != MSF_FP64 && precision != MSF_FP32_BULK)) {
    msf_internal_set_error("msf_fma_peak: precision must be MSF_FP64 or MSF_FP32_BULK, output non-NULL");
    return MSF_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return precision == MSF_FP64 ? run<double>(1 << 12, flops_per_s, s) : run<float>(1 << 17, flops_per_s, s);
}
