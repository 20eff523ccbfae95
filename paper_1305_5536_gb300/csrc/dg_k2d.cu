// dg_k2d.cu -- instantiations and launchers of the 2D stage kernels.
#include <cuda_runtime.h>

#include "dg_internal.h"
#include "dg_stage2d.cuh"

namespace dgk {

template <int EQ, class TC, class TS, int TX, int TY>
static cudaError_t launch2d(int stage, const Stage2DArgs<TS>& a, cudaStream_t st) {
  constexpr size_t smem = stage2d_smem_bytes<EQ, TX, TY, TC>();
  static_assert(smem <= 227 * 1024, "tile too large for shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e1 = cudaFuncSetAttribute(stage2d_kernel<EQ, TC, TS, TX, TY, 1>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaError_t e2 = cudaFuncSetAttribute(stage2d_kernel<EQ, TC, TS, TX, TY, 2>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e1 != cudaSuccess) return e1;
    if (e2 != cudaSuccess) return e2;
    attr_set = true;
  }
  dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
  if (stage == 1) stage2d_kernel<EQ, TC, TS, TX, TY, 1><<<grid, TX * TY, smem, st>>>(a);
  else stage2d_kernel<EQ, TC, TS, TX, TY, 2><<<grid, TX * TY, smem, st>>>(a);
  return cudaGetLastError();
}

// Tile shapes per precision (variant 0 is the default before tuning).
int stage2d_variants(int, int) { return 3; }

const char* stage2d_variant_name(int, int fp32, int v) {
  static const char* n64[] = {"16x8", "8x8", "32x4"};
  static const char* n32[] = {"16x16", "32x8", "16x8"};
  if (v < 0 || v > 2) return "?";
  return fp32 ? n32[v] : n64[v];
}

cudaError_t launch_stage2d(int eq, int variant, int stage, const Stage2DArgs<double>& a,
                           cudaStream_t st) {
  if (eq == 0) {
    switch (variant) {
      case 1: return launch2d<0, double, double, 8, 8>(stage, a, st);
      case 2: return launch2d<0, double, double, 32, 4>(stage, a, st);
      default: return launch2d<0, double, double, 16, 8>(stage, a, st);
    }
  }
  switch (variant) {
    case 1: return launch2d<1, double, double, 8, 8>(stage, a, st);
    case 2: return launch2d<1, double, double, 32, 4>(stage, a, st);
    default: return launch2d<1, double, double, 16, 8>(stage, a, st);
  }
}

cudaError_t launch_stage2d(int eq, int variant, int stage, const Stage2DArgs<float>& a,
                           cudaStream_t st) {
  if (eq == 0) {
    switch (variant) {
      case 1: return launch2d<0, float, float, 32, 8>(stage, a, st);
      case 2: return launch2d<0, float, float, 16, 8>(stage, a, st);
      default: return launch2d<0, float, float, 16, 16>(stage, a, st);
    }
  }
  switch (variant) {
    case 1: return launch2d<1, float, float, 32, 8>(stage, a, st);
    case 2: return launch2d<1, float, float, 16, 8>(stage, a, st);
    default: return launch2d<1, float, float, 16, 16>(stage, a, st);
  }
}

}  // namespace dgk
