// dg_batch.h -- work list of the persistent batched 2D step (dg_batch.cu).
#pragma once

#include <cuda_runtime.h>

#include "dg_common.cuh"

namespace dgk {

// One problem of a batch: grid, its tiles in the flat work list, and the
// element offsets of its arrays inside the batch's state buffers.
struct BatchProb {
  int nx, ny;
  int tiles_x, ntiles;
  int tile_begin;
  int pad;
  long ncell;
  double dx, dy;
  long c0_off, sl_off;
};

// Arguments of one batched step: state buffers 0 = V^n, 1 = V^1, 2 = V^{n+1}.
template <class TS>
struct BatchArgs {
  const BatchProb* probs;
  int nprob;
  int ntiles;
  double gamma, cfl, dt_override;
  GasPair gas;
  int limiter;
  double* c0[3];
  TS* sl[3];
  Ctl* ctl;
  unsigned* bar;          // grid barrier: arrivals, generation
  long long spin_limit;   // polls before a barrier wait gives up
  int barrier_extra;      // expected arrivals beyond the grid (0; 1 in a timeout test)
  int max_ctas = 0;       // largest grid (0: every resident CTA; a test hook sets it so
                          // that each CTA walks many tiles)
};

cudaError_t launch_batch2d(int eq, int variant, const BatchArgs<double>& B, cudaStream_t st,
                           int* grid);
cudaError_t launch_batch2d(int eq, int variant, const BatchArgs<float>& B, cudaStream_t st,
                           int* grid);
int batch2d_tile_x(int fp32, int variant);
int batch2d_tile_y(int fp32, int variant);

}  // namespace dgk
