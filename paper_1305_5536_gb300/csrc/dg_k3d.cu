// dg_k3d.cu -- instantiations and launchers of the 3D stage kernels.
#include <cuda_runtime.h>

#include "dg_internal.h"
#include "dg_stage3d.cuh"

namespace dgk {

template <class TC, class TS, int TX, int TY, int TZ, bool WENO>
static cudaError_t launch3d_w(int stage, const Stage3DArgs<TS>& a, cudaStream_t st) {
  constexpr size_t smem = stage3d_smem_bytes<TX, TY, TZ, TC>();
  static_assert(smem <= 227 * 1024, "tile too large for shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e1 = cudaFuncSetAttribute(stage3d_kernel<TC, TS, TX, TY, TZ, 1, WENO>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaError_t e2 = cudaFuncSetAttribute(stage3d_kernel<TC, TS, TX, TY, TZ, 2, WENO>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e1 != cudaSuccess) return e1;
    if (e2 != cudaSuccess) return e2;
    attr_set = true;
  }
  dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + TZ - 1) / TZ);
  if (stage == 1) return launch_pdl(stage3d_kernel<TC, TS, TX, TY, TZ, 1, WENO>, grid, TX * TY * TZ, smem, st, a);
  return launch_pdl(stage3d_kernel<TC, TS, TX, TY, TZ, 2, WENO>, grid, TX * TY * TZ, smem, st, a);
}

// The WENO-type limiter only in the instantiation that needs it.
template <class TC, class TS, int TX, int TY, int TZ>
static cudaError_t launch3d(int stage, const Stage3DArgs<TS>& a, cudaStream_t st) {
  if (a.limiter == 2) return launch3d_w<TC, TS, TX, TY, TZ, true>(stage, a, st);
  return launch3d_w<TC, TS, TX, TY, TZ, false>(stage, a, st);
}

int stage3d_variants(int) { return 2; }

const char* stage3d_variant_name(int fp32, int v) {
  static const char* n64[] = {"4x4x4", "8x4x2"};
  static const char* n32[] = {"8x8x4", "8x4x4"};
  if (v < 0 || v > 1) return "?";
  return fp32 ? n32[v] : n64[v];
}

cudaError_t launch_stage3d(int variant, int stage, const Stage3DArgs<double>& a, cudaStream_t st) {
  if (variant == 1) return launch3d<double, double, 8, 4, 2>(stage, a, st);
  return launch3d<double, double, 4, 4, 4>(stage, a, st);
}

cudaError_t launch_stage3d(int variant, int stage, const Stage3DArgs<float>& a, cudaStream_t st) {
  if (variant == 1) return launch3d<float, float, 8, 4, 4>(stage, a, st);
  return launch3d<float, float, 8, 8, 4>(stage, a, st);
}

}  // namespace dgk
