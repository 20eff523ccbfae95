// dg_kmh3m.cu -- instantiations and launchers of the 3D MHD MUSCL-Hancock step kernels.
#include <cuda_runtime.h>

#include "dg_internal.h"
#include "dg_mh3m.cuh"

namespace dgk {

template <class TC, class TS, int TX, int TY, int TZ, int NGF, bool WENO>
static cudaError_t launch_mh3m_t(const Stage3DArgs<TS>& a, cudaStream_t st) {
  constexpr size_t smem = mh3m_smem_bytes<TX, TY, TZ, NGF, TC>();
  static_assert(smem <= 227 * 1024, "tile too large for shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(mh3m_kernel<TC, TS, TX, TY, TZ, NGF, WENO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + TZ - 1) / TZ);
  return launch_pdl(mh3m_kernel<TC, TS, TX, TY, TZ, NGF, WENO>, grid, TX * TY * TZ, smem, st, a);
}

template <class TC, class TS, int TX, int TY, int TZ>
static cudaError_t launch_mh3m_ngf(int face_points, const Stage3DArgs<TS>& a, cudaStream_t st) {
  if (a.limiter == 2) {
    if (face_points == 2) return launch_mh3m_t<TC, TS, TX, TY, TZ, 2, true>(a, st);
    return launch_mh3m_t<TC, TS, TX, TY, TZ, 1, true>(a, st);
  }
  if (face_points == 2) return launch_mh3m_t<TC, TS, TX, TY, TZ, 2, false>(a, st);
  return launch_mh3m_t<TC, TS, TX, TY, TZ, 1, false>(a, st);
}

int mh3m_variants(int fp32) { return fp32 ? 2 : 1; }

const char* mh3m_variant_name(int fp32, int v) {
  static const char* n64[] = {"4x4x4"};
  static const char* n32[] = {"8x4x4", "8x8x4"};
  if (v < 0 || v > (fp32 ? 1 : 0)) return "?";
  return fp32 ? n32[v] : n64[v];
}

cudaError_t launch_mh3m(int variant, int face_points, const Stage3DArgs<double>& a,
                        cudaStream_t st) {
  if (variant != 0) return cudaErrorInvalidValue;
  return launch_mh3m_ngf<double, double, 4, 4, 4>(face_points, a, st);
}

cudaError_t launch_mh3m(int variant, int face_points, const Stage3DArgs<float>& a,
                        cudaStream_t st) {
  if (variant == 1) return launch_mh3m_ngf<float, float, 8, 8, 4>(face_points, a, st);
  if (variant != 0) return cudaErrorInvalidValue;
  return launch_mh3m_ngf<float, float, 8, 4, 4>(face_points, a, st);
}

}  // namespace dgk
