// dg_kmh3d.cu -- instantiations and launchers of the 3D MUSCL-Hancock step kernels.
#include <cuda_runtime.h>

#include "dg_internal.h"
#include "dg_mh3d.cuh"

namespace dgk {

template <class TC, class TS, int TX, int TY, int TZ, int NGF, bool WENO>
static cudaError_t launch_mh3d_t(const Stage3DArgs<TS>& a, cudaStream_t st) {
  constexpr size_t smem = mh3d_smem_bytes<TX, TY, TZ, NGF, TC>();
  static_assert(smem <= 227 * 1024, "tile too large for shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(mh3d_kernel<TC, TS, TX, TY, TZ, NGF, WENO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + TZ - 1) / TZ);
  return launch_pdl(mh3d_kernel<TC, TS, TX, TY, TZ, NGF, WENO>, grid, TX * TY * TZ, smem, st, a);
}

template <class TC, class TS, int TX, int TY, int TZ>
static cudaError_t launch_mh3d_ngf(int face_points, const Stage3DArgs<TS>& a, cudaStream_t st) {
  if (a.limiter == 2) {
    if (face_points == 2) return launch_mh3d_t<TC, TS, TX, TY, TZ, 2, true>(a, st);
    return launch_mh3d_t<TC, TS, TX, TY, TZ, 1, true>(a, st);
  }
  if (face_points == 2) return launch_mh3d_t<TC, TS, TX, TY, TZ, 2, false>(a, st);
  return launch_mh3d_t<TC, TS, TX, TY, TZ, 1, false>(a, st);
}

int mh3d_variants(int) { return 2; }

const char* mh3d_variant_name(int fp32, int v) {
  static const char* n64[] = {"4x4x4", "8x4x2"};
  static const char* n32[] = {"8x8x4", "8x4x4"};
  if (v < 0 || v > 1) return "?";
  return fp32 ? n32[v] : n64[v];
}

cudaError_t launch_mh3d(int variant, int face_points, const Stage3DArgs<double>& a,
                        cudaStream_t st) {
  switch (variant) {
    case 0: return launch_mh3d_ngf<double, double, 4, 4, 4>(face_points, a, st);
    case 1: return launch_mh3d_ngf<double, double, 8, 4, 2>(face_points, a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mh3d(int variant, int face_points, const Stage3DArgs<float>& a,
                        cudaStream_t st) {
  switch (variant) {
    case 0: return launch_mh3d_ngf<float, float, 8, 8, 4>(face_points, a, st);
    case 1: return launch_mh3d_ngf<float, float, 8, 4, 4>(face_points, a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dgk
