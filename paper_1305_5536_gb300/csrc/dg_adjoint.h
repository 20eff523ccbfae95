// dg_adjoint.h -- reverse-mode (vector-Jacobian) products of the SSP-RK2 step of
// the 2D DG scheme, and the checkpoint store used to run them backwards
// over a recorded trajectory.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/dg.h"

struct AdjointStore {
  // recording: interchange-layout checkpoints every k steps and the time steps
  double* ckpt = nullptr;
  double* dt_hist = nullptr;
  long long cap_steps = 0;
  long long nrec = 0;
  // changes whenever the recorded trajectory does (a recording extended, ended or
  // restarted), so that a caller holding a recording can tell that it is gone
  long long generation = 0;
  size_t ckpt_elems = 0;
  long ncell = 0;
  int nplanes = 0;
  // work buffers of the reverse sweep (allocated on first use)
  void* work = nullptr;
  size_t work_bytes = 0;
  long work_ncell = 0;
  int work_fp32 = -1;
};

struct AdjointCall {
  int eq;  // DG_EULER or DG_MHD
  int nx, ny;
  double dx, dy, gamma;
  int limiter, fp32;
  cudaStream_t stream;
};

void adjoint_free(AdjointStore& s);
void adjoint_reset(AdjointStore& s);
dg_status adjoint_reserve(AdjointStore& s, int nplanes, long ncell, int k, long long nsteps,
                          std::string& msg);
dg_status adjoint_step(AdjointStore& s, const AdjointCall& c, const double* u_n,
                       const double* lam_next, double* lam_prev, double dt, std::string& msg);
dg_status adjoint_run(AdjointStore& s, const AdjointCall& c, int nplanes, int k,
                      const double* lam_N, double* lam_0, std::string& msg);
