// Measured issue rates of the units the near-field gather is bound by: the
// SFU's ex2 and the FP32 FMA pipe (scalar FFMA and packed FFMA2), in results
// per SM per clock.  They confirm the per-clock figures the roofline's ALU
// peak is built from.
//
// One 1024-thread block per SM (its shared-memory request keeps a second block
// off the SM) runs 8 independent dependency chains per thread; the block
// times itself with the SM's own clock, so the result does not depend on the
// clock frequency.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "api_internal.h"
#include "common.cuh"

namespace gmi {

namespace {

constexpr int kRateThreads = 1024;
constexpr int kRateIters = 2048;
constexpr int kRateChains = 8;
constexpr size_t kRateSmem = 160 * 1024;   // more than half an SM's shared memory

template <int OP>   // 0: ex2, 1: FFMA, 2: FFMA2
__global__ void __launch_bounds__(kRateThreads) unit_rate_kernel(float* sink, long long* cycles) {
  extern __shared__ float pad[];
  float x[kRateChains];
  float2 y[kRateChains];
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) {
    x[c] = 0.5f + 0.001f * (float)(threadIdx.x + c);
    y[c] = make_float2(x[c], 1.0f - x[c]);
  }
  const float2 b2 = make_float2(0.9999f, 0.9998f), c2 = make_float2(1e-4f, 2e-4f);
  __syncthreads();
  long long t0 = clock64();
  for (int it = 0; it < kRateIters; ++it) {
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) {
      if (OP == 0) x[c] = ex2(-x[c]);                        // stays in (0.5, 0.71)
      else if (OP == 1) x[c] = fmaf(x[c], 0.9999f, 1e-4f);   // stays near 1
      else y[c] = __ffma2_rn(y[c], b2, c2);
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) s += x[c] + y[c].x + y[c].y;
  if (s == 12345.0f) pad[threadIdx.x] = s;   // keeps the chains live
  sink[blockIdx.x * kRateThreads + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int OP>
bool measure(int sms, float* sink, long long* dcyc, double* rate) {
  auto k = unit_rate_kernel<OP>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRateSmem) != cudaSuccess)
    return false;
  std::vector<long long> cyc(sms);
  for (int rep = 0; rep < 2; ++rep) {   // the first run warms the clocks up
    k<<<sms, kRateThreads, kRateSmem>>>(sink, dcyc);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return false;
  }
  if (cudaMemcpy(cyc.data(), dcyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
  std::sort(cyc.begin(), cyc.end());
  const double results = (double)kRateThreads * kRateIters * kRateChains * (OP == 2 ? 2.0 : 1.0);
  *rate = results / (double)cyc[sms / 2];   // median block
  return true;
}

}  // namespace

}  // namespace gmi

extern "C" gmi_status gmi_measure_unit_rates(double* rates) {
  using namespace gmi;
  if (!rates) return GMI_ERR_INVALID_ARG;
  const int sms = device_sm_count();
  float* sink = nullptr;
  long long* dcyc = nullptr;
  if (cudaMalloc(&sink, sizeof(float) * (size_t)sms * kRateThreads) != cudaSuccess) return GMI_ERR_CUDA;
  if (cudaMalloc(&dcyc, sizeof(long long) * (size_t)sms) != cudaSuccess) {
    cudaFree(sink);
    return GMI_ERR_CUDA;
  }
  const bool ok = measure<0>(sms, sink, dcyc, &rates[0]) && measure<1>(sms, sink, dcyc, &rates[1]) &&
                  measure<2>(sms, sink, dcyc, &rates[2]);
  cudaFree(sink);
  cudaFree(dcyc);
  return ok ? GMI_OK : GMI_ERR_CUDA;
}
