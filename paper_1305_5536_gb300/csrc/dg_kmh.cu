// dg_kmh.cu -- instantiations and launchers of the MUSCL-Hancock step kernels.
#include <cuda_runtime.h>

#include "dg_internal.h"
#include "dg_mh2d.cuh"

namespace dgk {

template <int EQ, class TC, class TS, int TX, int TY, int NGF, bool WENO>
static cudaError_t launch_mh2d_t(const Stage2DArgs<TS>& a, cudaStream_t st) {
  constexpr size_t smem = mh2d_smem_bytes<EQ, TX, TY, NGF, TC>();
  static_assert(smem <= 227 * 1024, "tile too large for shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(mh2d_kernel<EQ, TC, TS, TX, TY, NGF, WENO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
  return launch_pdl(mh2d_kernel<EQ, TC, TS, TX, TY, NGF, WENO>, grid, TX * TY, smem, st, a);
}

template <int EQ, class TC, class TS, int TX, int TY>
static cudaError_t launch_mh2d_ngf(int face_points, const Stage2DArgs<TS>& a, cudaStream_t st) {
  if (a.limiter == 2) {
    if (face_points == 2) return launch_mh2d_t<EQ, TC, TS, TX, TY, 2, true>(a, st);
    return launch_mh2d_t<EQ, TC, TS, TX, TY, 1, true>(a, st);
  }
  if (face_points == 2) return launch_mh2d_t<EQ, TC, TS, TX, TY, 2, false>(a, st);
  return launch_mh2d_t<EQ, TC, TS, TX, TY, 1, false>(a, st);
}

int mh2d_variants(int, int) { return 3; }

const char* mh2d_variant_name(int, int fp32, int v) {
  static const char* n64[] = {"16x8", "8x8", "32x4"};
  static const char* n32[] = {"16x8", "16x16", "32x8"};
  if (v < 0 || v > 2) return "?";
  return fp32 ? n32[v] : n64[v];
}

template <int EQ>
static cudaError_t launch_mh2d_eq(int variant, int fp, const Stage2DArgs<double>& a,
                                  cudaStream_t st) {
  switch (variant) {
    case 0: return launch_mh2d_ngf<EQ, double, double, 16, 8>(fp, a, st);
    case 1: return launch_mh2d_ngf<EQ, double, double, 8, 8>(fp, a, st);
    case 2: return launch_mh2d_ngf<EQ, double, double, 32, 4>(fp, a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int EQ>
static cudaError_t launch_mh2d_eq(int variant, int fp, const Stage2DArgs<float>& a,
                                  cudaStream_t st) {
  switch (variant) {
    case 0: return launch_mh2d_ngf<EQ, float, float, 16, 8>(fp, a, st);
    case 1: return launch_mh2d_ngf<EQ, float, float, 16, 16>(fp, a, st);
    case 2: return launch_mh2d_ngf<EQ, float, float, 32, 8>(fp, a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mh2d(int eq, int variant, int face_points, const Stage2DArgs<double>& a,
                        cudaStream_t st) {
  return eq == 0 ? launch_mh2d_eq<0>(variant, face_points, a, st)
                 : launch_mh2d_eq<1>(variant, face_points, a, st);
}

cudaError_t launch_mh2d(int eq, int variant, int face_points, const Stage2DArgs<float>& a,
                        cudaStream_t st) {
  return eq == 0 ? launch_mh2d_eq<0>(variant, face_points, a, st)
                 : launch_mh2d_eq<1>(variant, face_points, a, st);
}

}  // namespace dgk
