// dg_k3m.cu -- instantiations and launchers of the 3D MHD stage kernels.
#include <cuda_runtime.h>

#include "dg_internal.h"
#include "dg_stage3m.cuh"

namespace dgk {

template <class TC, class TS, int TX, int TY, int TZ, bool WENO>
static cudaError_t launch3m_t(int stage, const Stage3DArgs<TS>& a, cudaStream_t st) {
  constexpr size_t smem = stage3m_smem_bytes<TX, TY, TZ, TC>();
  static_assert(smem <= 227 * 1024, "tile too large for shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e1 = cudaFuncSetAttribute(stage3m_kernel<TC, TS, TX, TY, TZ, 1, WENO>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaError_t e2 = cudaFuncSetAttribute(stage3m_kernel<TC, TS, TX, TY, TZ, 2, WENO>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e1 != cudaSuccess) return e1;
    if (e2 != cudaSuccess) return e2;
    attr_set = true;
  }
  dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + TZ - 1) / TZ);
  if (stage == 1) return launch_pdl(stage3m_kernel<TC, TS, TX, TY, TZ, 1, WENO>, grid, TX * TY * TZ, smem, st, a);
  return launch_pdl(stage3m_kernel<TC, TS, TX, TY, TZ, 2, WENO>, grid, TX * TY * TZ, smem, st, a);
}

template <class TC, class TS, int TX, int TY, int TZ>
static cudaError_t launch3m(int stage, const Stage3DArgs<TS>& a, cudaStream_t st) {
  if (a.limiter == 2) return launch3m_t<TC, TS, TX, TY, TZ, true>(stage, a, st);
  return launch3m_t<TC, TS, TX, TY, TZ, false>(stage, a, st);
}

int stage3m_variants(int fp32) { return fp32 ? 2 : 1; }

const char* stage3m_variant_name(int fp32, int v) {
  static const char* n64[] = {"4x4x4"};
  static const char* n32[] = {"8x4x4", "8x8x4"};
  if (v < 0 || v > (fp32 ? 1 : 0)) return "?";
  return fp32 ? n32[v] : n64[v];
}

cudaError_t launch_stage3m(int variant, int stage, const Stage3DArgs<double>& a, cudaStream_t st) {
  if (variant != 0) return cudaErrorInvalidValue;
  return launch3m<double, double, 4, 4, 4>(stage, a, st);
}

cudaError_t launch_stage3m(int variant, int stage, const Stage3DArgs<float>& a, cudaStream_t st) {
  if (variant == 1) return launch3m<float, float, 8, 8, 4>(stage, a, st);
  if (variant != 0) return cudaErrorInvalidValue;
  return launch3m<float, float, 8, 4, 4>(stage, a, st);
}

}  // namespace dgk
