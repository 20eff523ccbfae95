// dg_stage2d_tma.cuh -- persistent 2D stage kernel whose halo tiles arrive by TMA.
//
// Each CTA walks tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...  For a tile whose
// halo lies inside the grid (no periodic wrap), one thread issues two 3D tensor
// loads (all average planes of the halo-2 box, all derivative planes of the halo-1
// box) that complete on an mbarrier; the CTA unpacks them into its working arrays
// and immediately starts the next tile's loads, which then overlap this tile's
// limiter, Riemann fluxes and right-hand side.  Tiles at the periodic seams load
// element by element (stage2d_load).  The compute is the one of stage2d_kernel.
#pragma once

#include "dg_stage2d.cuh"
#include "dg_tma.cuh"

namespace dgk {

// Raw TMA boxes of one tile in shared memory.
template <int EQ, class TS, int TX, int TY>
struct TmaBox2D {
  using T = Tile2D<EQ, TX, TY>;
  // averages (FP64): box (R2X, R2Y, NV) at (i0 - 2, j0 - 2, 0)
  static constexpr int C0_BYTES = T::R2X * T::R2Y * T::NV * 8;
  // derivative coefficients: box (SXW, R1Y, NS) at (i0 - SX0, j0 - 1, 0); the first
  // column is moved down to a 16-byte boundary, so the halo-1 column 0 sits at SOFF
  static constexpr int SX0 = sizeof(TS) == 4 ? 4 : 2;
  static constexpr int SXW = TX + 2 * SX0;
  static constexpr int SOFF = SX0 - 1;
  static constexpr int SL_BYTES = SXW * T::R1Y * T::NS * (int)sizeof(TS);
  static constexpr int SL_OFF = (C0_BYTES + 127) / 128 * 128;
  static constexpr int RAW_BYTES = (SL_OFF + SL_BYTES + 127) / 128 * 128;
  static_assert(TX % 4 == 0, "TMA tiles need 16-byte aligned columns");
  static_assert((T::R2X * 8) % 16 == 0 && (SXW * (int)sizeof(TS)) % 16 == 0, "box rows");
  static_assert(T::R2X <= 256 && T::R2Y <= 256 && SXW <= 256, "box extent");
};

template <int EQ, class TS, int TX, int TY, class TC>
__host__ __device__ constexpr size_t stage2d_tma_smem_bytes() {
  return (size_t)TmaBox2D<EQ, TS, TX, TY>::RAW_BYTES + stage2d_smem_bytes<EQ, TX, TY, TC>();
}

template <int EQ, class TC, class TS, int TX, int TY, int STAGE>
__global__ void __launch_bounds__(TX * TY)
    stage2d_tma_kernel(const Stage2DArgs<TS> A, const __grid_constant__ CUtensorMap mc0,
                       const __grid_constant__ CUtensorMap msl, int tiles_x, int ntiles,
                       long long spin_limit) {
  using T = Tile2D<EQ, TX, TY>;
  using B = TmaBox2D<EQ, TS, TX, TY>;
  extern __shared__ __align__(128) unsigned char smem[];
  double* raw_c0 = reinterpret_cast<double*>(smem);
  TS* raw_sl = reinterpret_cast<TS*>(smem + B::SL_OFF);
  const TileMem<TC> M = tile_mem<EQ, TX, TY, TC>(smem + B::RAW_BYTES);
  __shared__ TileScalars<TX * TY> S;
  __shared__ __align__(8) uint64_t bar;
  const int tid = threadIdx.x;
  const int nx = A.nx, ny = A.ny;
  auto interior = [&](int i0, int j0) {
    return i0 >= B::SX0 && i0 + TX + B::SX0 <= nx && j0 >= 2 && j0 + TY + 2 <= ny;
  };
  auto issue = [&](int i0, int j0) {
    mbar_arrive_expect_tx(&bar, B::C0_BYTES + B::SL_BYTES);
    tma_load_3d(raw_c0, &mc0, i0 - 2, j0 - 2, 0, &bar);
    tma_load_3d(raw_sl, &msl, i0 - B::SX0, j0 - 1, 0, &bar);
  };
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  unsigned phase = 0;
  // `pending`: a TMA load of this CTA's current tile is in flight (the same value
  // in every thread).  After a wait has run out the CTA stops using TMA: it records
  // ERR_TIMEOUT (the launch's results are then invalid), waits once more, bounded,
  // for the copy in flight, and stages the rest of its tiles element by element.
  bool tma_ok = true;
  int t = blockIdx.x;
  bool pending = t < ntiles && interior((t % tiles_x) * TX, (t / tiles_x) * TY);
  if (tid == 0 && pending) issue((t % tiles_x) * TX, (t / tiles_x) * TY);
  for (; t < ntiles; t += gridDim.x) {
    const int ty = t / tiles_x, tx = t - ty * tiles_x;
    const int i0 = tx * TX, j0 = ty * TY;
    __syncthreads();  // the previous tile is done with shared memory
    stage2d_setup<EQ, TC, TS, TX, TY>(A, i0, j0, M, S);
    __syncthreads();
    bool use_raw = false;
    if (pending) {
      const bool late = !mbar_wait_bounded(&bar, phase, spin_limit);
      if (__syncthreads_or(late)) {
        if (tid == 0) atomicOr(&S.err, ERR_TIMEOUT);
        (void)mbar_wait_bounded(&bar, phase, spin_limit);  // drain the copy in flight
        tma_ok = false;
      } else {
        use_raw = true;
      }
      phase ^= 1u;
    }
    if (use_raw) {
      for (int e = tid; e < T::NV * T::R2; e += T::NT) M.c0[e] = Cvt<TC>::to_tc(raw_c0[e]);
      for (int e = tid; e < T::NS * T::R1; e += T::NT) {
        const int v = e / T::R1, r = e - v * T::R1;
        const int ry = r / T::R1X, rx = r - ry * T::R1X;
        M.sl[e] = (TC)raw_sl[(v * T::R1Y + ry) * B::SXW + rx + B::SOFF];
      }
    } else {
      stage2d_load<EQ, TC, TS, TX, TY>(A, M);
    }
    fence_proxy_async_smem();
    __syncthreads();
    // the raw boxes are free: start loading the next tile of this CTA
    const int tn = t + gridDim.x;
    pending = tma_ok && tn < ntiles && interior((tn % tiles_x) * TX, (tn / tiles_x) * TY);
    if (tid == 0 && pending) issue((tn % tiles_x) * TX, (tn / tiles_x) * TY);
    stage2d_compute<EQ, TC, TS, TX, TY, STAGE>(A, i0, j0, (unsigned)ntiles, M, S);
  }
}

}  // namespace dgk
