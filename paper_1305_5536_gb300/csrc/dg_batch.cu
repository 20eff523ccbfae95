// dg_batch.cu -- one persistent launch per SSP-RK2 step for many independent 2D
// problems of different grid sizes.
//
// The tiles of all problems form one flat work list (problem p owns tiles
// [tile_begin, tile_begin + ntiles)).  A cooperative launch of as many CTAs as
// fit on the GPU at once walks the list for stage 1, meets at a grid barrier,
// walks it again for stage 2.  Each problem has its own control block: its own
// Courant time step, and the last of its tiles to finish stage 2 publishes the
// signal speed of its new state.  The barrier wait is bounded: after the limit
// the kernel records ERR_TIMEOUT and carries on, so it never hangs.
#include <cuda_runtime.h>

#include "dg_batch.h"
#include "dg_internal.h"
#include "dg_stage2d.cuh"

namespace dgk {

namespace {

__device__ __forceinline__ int find_problem(const BatchProb* P, int nprob, int t) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (P[mid].tile_begin <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Grid-wide barrier of a cooperative launch: bar[0] counts arrivals, bar[1] is
// the generation.  Returns false if the wait ran past `limit` polls.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, long long limit) {
  __shared__ bool ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    ok = true;
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g) {
        if (++it > limit) {
          ok = false;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok;
}

template <class TS>
__device__ __forceinline__ Stage2DArgs<TS> problem_args(const BatchArgs<TS>& B, const BatchProb& p,
                                                        int ip, int stage) {
  Stage2DArgs<TS> a;
  a.nx = p.nx;
  a.ny = p.ny;
  a.ncell = p.ncell;
  a.dx = p.dx;
  a.dy = p.dy;
  a.gamma = B.gamma;
  a.gas = B.gas;
  a.cfl = B.cfl;
  a.dt_override = B.dt_override;
  a.limiter = B.limiter;
  const int in = stage == 1 ? 0 : 1, out = stage == 1 ? 1 : 2;
  a.in.c0 = B.c0[in] + p.c0_off;
  a.in.sl = B.sl[in] + p.sl_off;
  a.base.c0 = B.c0[0] + p.c0_off;
  a.base.sl = B.sl[0] + p.sl_off;
  a.out.c0 = B.c0[out] + p.c0_off;
  a.out.sl = B.sl[out] + p.sl_off;
  a.lim_sl = B.sl[2] + p.sl_off;  // the step's output buffer
  a.ctl = B.ctl + ip;
  return a;
}

template <int EQ, class TC, class TS, int TX, int TY, int STAGE, bool WENO>
__device__ __forceinline__ void sweep(const BatchArgs<TS>& B, unsigned char* smem) {
  for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const int ip = find_problem(B.probs, B.nprob, t);
    const BatchProb p = B.probs[ip];
    const int lt = t - p.tile_begin;
    const int ty = lt / p.tiles_x, tx = lt - ty * p.tiles_x;
    const Stage2DArgs<TS> a = problem_args(B, p, ip, STAGE);
    __syncthreads();  // the previous tile is done with shared memory
    stage2d_tile<EQ, TC, TS, TX, TY, STAGE, WENO>(a, tx * TX, ty * TY, (unsigned)p.ntiles, smem);
  }
}

// WENO = false compiles the WENO-type limiter out (launches with limiter 0 or 1),
// as in the single-problem stage kernels: the tile code is then the same.
template <int EQ, class TC, class TS, int TX, int TY, bool WENO>
__global__ void __launch_bounds__(TX * TY, (StageMinBlocks<TX * TY, TC>::v))
    batch2d_kernel(const BatchArgs<TS> B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  sweep<EQ, TC, TS, TX, TY, 1, WENO>(B, smem_raw);
  if (!grid_barrier(B.bar, gridDim.x + B.barrier_extra, B.spin_limit)) {
    if (threadIdx.x == 0) atomicOr(&B.ctl[0].err, ERR_TIMEOUT);
  }
  sweep<EQ, TC, TS, TX, TY, 2, WENO>(B, smem_raw);
}

template <int EQ, class TC, class TS, int TX, int TY, bool WENO>
cudaError_t launch_batch_w(const BatchArgs<TS>& B, cudaStream_t st, int* grid_out) {
  constexpr size_t smem = stage2d_smem_bytes<EQ, TX, TY, TC>();
  auto kern = batch2d_kernel<EQ, TC, TS, TX, TY, WENO>;
  static int per_sm = -1, nsm = 0;
  if (per_sm < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, smem)) != cudaSuccess)
      return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
  }
  int grid = per_sm * nsm;
  if (B.max_ctas > 0 && grid > B.max_ctas) grid = B.max_ctas;
  if (grid > B.ntiles) grid = B.ntiles;
  if (grid_out) *grid_out = grid;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(TX * TY);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, B);
}

template <int EQ, class TC, class TS, int TX, int TY>
cudaError_t launch_batch_t(const BatchArgs<TS>& B, cudaStream_t st, int* grid_out) {
  if (B.limiter == 2) return launch_batch_w<EQ, TC, TS, TX, TY, true>(B, st, grid_out);
  return launch_batch_w<EQ, TC, TS, TX, TY, false>(B, st, grid_out);
}

}  // namespace

cudaError_t launch_batch2d(int eq, int variant, const BatchArgs<double>& B, cudaStream_t st,
                           int* grid) {
  if (eq == 0) {
    switch (variant) {
      case 1: return launch_batch_t<0, double, double, 8, 8>(B, st, grid);
      case 2: return launch_batch_t<0, double, double, 32, 4>(B, st, grid);
      default: return launch_batch_t<0, double, double, 16, 8>(B, st, grid);
    }
  }
  switch (variant) {
    case 1: return launch_batch_t<1, double, double, 8, 8>(B, st, grid);
    case 2: return launch_batch_t<1, double, double, 32, 4>(B, st, grid);
    default: return launch_batch_t<1, double, double, 16, 8>(B, st, grid);
  }
}

cudaError_t launch_batch2d(int eq, int variant, const BatchArgs<float>& B, cudaStream_t st,
                           int* grid) {
  if (eq == 0) {
    switch (variant) {
      case 1: return launch_batch_t<0, float, float, 32, 8>(B, st, grid);
      case 2: return launch_batch_t<0, float, float, 16, 8>(B, st, grid);
      default: return launch_batch_t<0, float, float, 16, 16>(B, st, grid);
    }
  }
  switch (variant) {
    case 1: return launch_batch_t<1, float, float, 32, 8>(B, st, grid);
    case 2: return launch_batch_t<1, float, float, 16, 8>(B, st, grid);
    default: return launch_batch_t<1, float, float, 16, 16>(B, st, grid);
  }
}

int batch2d_tile_x(int fp32, int variant) {
  static const int x64[] = {16, 8, 32}, x32[] = {16, 32, 16};
  return fp32 ? x32[variant < 0 || variant > 2 ? 0 : variant] : x64[variant < 0 || variant > 2 ? 0 : variant];
}
int batch2d_tile_y(int fp32, int variant) {
  static const int y64[] = {8, 8, 4}, y32[] = {16, 8, 8};
  return fp32 ? y32[variant < 0 || variant > 2 ? 0 : variant] : y64[variant < 0 || variant > 2 ? 0 : variant];
}

}  // namespace dgk
