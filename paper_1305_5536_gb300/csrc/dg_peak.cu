// dg_peak.cu -- measured fused multiply-add throughput of the device, the
// denominator of the roofline of kernels bound by an arithmetic pipe (the FP64
// stage kernels: GB300 runs FP64 at a small fraction of its FP32 rate).
//
// Every thread of a grid that fills all SMs runs 8 independent FMA chains
// x <- x * a + b (|a| < 1, so the values stay bounded); the flop count is 2 per
// FMA.  Timed with CUDA events on a private stream; the best of several runs is
// reported.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/dg.h"
#include "dg_internal.h"

namespace dgk {
namespace {

constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(256) fma_chains_kernel(T* sink, T a, T b, int iters) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == T(-1.25)) sink[blockIdx.x] = s;  // never true: keeps the chains live
}

template <class T>
dg_status measure(double* flops, std::string& msg) {
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chains_kernel<T>, 256, 0) !=
          cudaSuccess) {
    cudaGetLastError();
    msg = "device query failed";
    return DG_ECUDA;
  }
  const int grid = nsm * (per_sm > 0 ? per_sm : 1);
  T* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&sink, grid * sizeof(T)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(sink);
    if (st) cudaStreamDestroy(st);
    msg = "allocation of the measurement buffers failed";
    return DG_ENOMEM;
  }
  double best = 0.0;
  int iters = 256;
  dg_status s = DG_OK;
  for (int rep = 0; rep < 8 && s == DG_OK; ++rep) {
    cudaEventRecord(e0, st);
    fma_chains_kernel<T><<<grid, 256, 0, st>>>(sink, T(0.999999), T(1e-6), iters);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      msg = "measurement kernel failed";
      s = DG_ECUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double f = 2.0 * kChains * (double)iters * grid * 256.0 / (ms * 1e-3);
    if (f > best && ms > 5.0f) best = f;
    // aim at ~20 ms per run
    if (ms < 20.0f) iters = (int)std::min(1e8, iters * (ms > 0.05f ? 20.0 / ms : 64.0));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  cudaFree(sink);
  *flops = best;
  return s;
}

}  // namespace
}  // namespace dgk

extern "C" dg_status dg_peak_fma(int precision, double* flops_per_s) {
  if (!flops_per_s || (precision != DG_FP64 && precision != DG_FP32)) {
    dgk::set_global_error("dg_peak_fma: precision must be DG_FP64 or DG_FP32, output non-null");
    return DG_EINVAL;
  }
  std::string msg;
  dg_status s = precision == DG_FP64 ? dgk::measure<double>(flops_per_s, msg)
                                     : dgk::measure<float>(flops_per_s, msg);
  if (s != DG_OK) dgk::set_global_error("dg_peak_fma: " + msg);
  return s;
}
