// dg_k2d.cu -- instantiations and launchers of the 2D stage kernels.
#include <cuda_runtime.h>

#include <cuda.h>

#include <map>
#include <tuple>

#include "dg_internal.h"
#include "dg_stage2d.cuh"
#include "dg_stage2d_tma.cuh"

namespace dgk {

template <int EQ, class TC, class TS, int TX, int TY, bool WENO>
static cudaError_t launch2d_w(int stage, const Stage2DArgs<TS>& a, cudaStream_t st) {
  constexpr size_t smem = stage2d_smem_bytes<EQ, TX, TY, TC>();
  static_assert(smem <= 227 * 1024, "tile too large for shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e1 = cudaFuncSetAttribute(stage2d_kernel<EQ, TC, TS, TX, TY, 1, WENO>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaError_t e2 = cudaFuncSetAttribute(stage2d_kernel<EQ, TC, TS, TX, TY, 2, WENO>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e1 != cudaSuccess) return e1;
    if (e2 != cudaSuccess) return e2;
    attr_set = true;
  }
  dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
  if (stage == 1) return launch_pdl(stage2d_kernel<EQ, TC, TS, TX, TY, 1, WENO>, grid, TX * TY, smem, st, a);
  return launch_pdl(stage2d_kernel<EQ, TC, TS, TX, TY, 2, WENO>, grid, TX * TY, smem, st, a);
}

// The WENO-type limiter only in the instantiation that needs it.
template <int EQ, class TC, class TS, int TX, int TY>
static cudaError_t launch2d(int stage, const Stage2DArgs<TS>& a, cudaStream_t st) {
  if (a.limiter == 2) return launch2d_w<EQ, TC, TS, TX, TY, true>(stage, a, st);
  return launch2d_w<EQ, TC, TS, TX, TY, false>(stage, a, st);
}

// ---------------------------------------------------------------------------
// TMA variants: tensor maps of the stage input (averages and derivative
// coefficients as 3D tensors x, y, plane), encoded through the driver entry point
// and cached by address and shape.
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  }
  return fn;
}

static bool tensor_map(CUtensorMap* out, const void* ptr, bool f64, int nx, int ny, int planes,
                       int bx, int by, int bz) {
  typedef std::tuple<const void*, bool, int, int, int, int, int, int> Key;
  static std::map<Key, CUtensorMap> cache;
  Key key(ptr, f64, nx, ny, planes, bx, by, bz);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *out = it->second;
    return true;
  }
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t es = f64 ? 8 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)nx * es, (cuuint64_t)nx * ny * es};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
  cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMap m;
  CUresult r = enc(&m, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                   const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  cache[key] = m;
  *out = m;
  return true;
}

template <int EQ, class TC, class TS, int TX, int TY>
static cudaError_t launch2d_tma(int stage, const Stage2DArgs<TS>& a, cudaStream_t st) {
  using T = Tile2D<EQ, TX, TY>;
  using B = TmaBox2D<EQ, TS, TX, TY>;
  // 16-byte aligned rows and planes for both tensors
  if ((a.nx * (int)sizeof(TS)) % 16 != 0 || (a.nx * 8) % 16 != 0) return cudaErrorNotSupported;
  constexpr size_t smem = stage2d_tma_smem_bytes<EQ, TS, TX, TY, TC>();
  static_assert(smem <= 227 * 1024, "tile too large for shared memory");
  auto k1 = stage2d_tma_kernel<EQ, TC, TS, TX, TY, 1>;
  auto k2 = stage2d_tma_kernel<EQ, TC, TS, TX, TY, 2>;
  static int per_sm[2] = {-1, -1}, nsm = 0;
  if (per_sm[0] < 0) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k1, T::NT, smem)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k2, T::NT, smem)) != cudaSuccess) return e;
    if (per_sm[0] < 1 || per_sm[1] < 1) return cudaErrorInvalidConfiguration;
  }
  CUtensorMap mc0, msl;
  if (!tensor_map(&mc0, a.in.c0, true, a.nx, a.ny, T::NV, T::R2X, T::R2Y, T::NV) ||
      !tensor_map(&msl, a.in.sl, sizeof(TS) == 8, a.nx, a.ny, T::NS, B::SXW, T::R1Y, T::NS))
    return cudaErrorNotSupported;
  const int tiles_x = (a.nx + TX - 1) / TX;
  const int ntiles = tiles_x * ((a.ny + TY - 1) / TY);
  int grid = per_sm[stage == 1 ? 0 : 1] * nsm;
  if (a.max_ctas > 0 && grid > a.max_ctas) grid = a.max_ctas;
  if (grid > ntiles) grid = ntiles;
  const long long spin = 1LL << 26;
  if (stage == 1) k1<<<grid, T::NT, smem, st>>>(a, mc0, msl, tiles_x, ntiles, spin);
  else k2<<<grid, T::NT, smem, st>>>(a, mc0, msl, tiles_x, ntiles, spin);
  return cudaGetLastError();
}

// Tile shapes per precision (variant 0 is the default before tuning); variants 3
// and 4 are the persistent TMA kernels (grids whose rows are 16-byte aligned).
int stage2d_variants(int, int) { return 5; }

const char* stage2d_variant_name(int, int fp32, int v) {
  static const char* n64[] = {"16x8", "8x8", "32x4", "tma16x8", "tma32x4"};
  static const char* n32[] = {"16x16", "32x8", "16x8", "tma16x8", "tma16x16"};
  if (v < 0 || v > 4) return "?";
  return fp32 ? n32[v] : n64[v];
}

cudaError_t launch_stage2d(int eq, int variant, int stage, const Stage2DArgs<double>& a,
                           cudaStream_t st) {
  if (eq == 0) {
    switch (variant) {
      case 1: return launch2d<0, double, double, 8, 8>(stage, a, st);
      case 2: return launch2d<0, double, double, 32, 4>(stage, a, st);
      case 3: return launch2d_tma<0, double, double, 16, 8>(stage, a, st);
      case 4: return launch2d_tma<0, double, double, 32, 4>(stage, a, st);
      default: return launch2d<0, double, double, 16, 8>(stage, a, st);
    }
  }
  switch (variant) {
    case 1: return launch2d<1, double, double, 8, 8>(stage, a, st);
    case 2: return launch2d<1, double, double, 32, 4>(stage, a, st);
    case 3: return launch2d_tma<1, double, double, 16, 8>(stage, a, st);
    case 4: return launch2d_tma<1, double, double, 32, 4>(stage, a, st);
    default: return launch2d<1, double, double, 16, 8>(stage, a, st);
  }
}

cudaError_t launch_stage2d(int eq, int variant, int stage, const Stage2DArgs<float>& a,
                           cudaStream_t st) {
  if (eq == 0) {
    switch (variant) {
      case 1: return launch2d<0, float, float, 32, 8>(stage, a, st);
      case 2: return launch2d<0, float, float, 16, 8>(stage, a, st);
      case 3: return launch2d_tma<0, float, float, 16, 8>(stage, a, st);
      case 4: return launch2d_tma<0, float, float, 16, 16>(stage, a, st);
      default: return launch2d<0, float, float, 16, 16>(stage, a, st);
    }
  }
  switch (variant) {
    case 1: return launch2d<1, float, float, 32, 8>(stage, a, st);
    case 2: return launch2d<1, float, float, 16, 8>(stage, a, st);
    case 3: return launch2d_tma<1, float, float, 16, 8>(stage, a, st);
    case 4: return launch2d_tma<1, float, float, 16, 16>(stage, a, st);
    default: return launch2d<1, float, float, 16, 16>(stage, a, st);
  }
}

}  // namespace dgk
