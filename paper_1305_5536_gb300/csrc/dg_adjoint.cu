// dg_adjoint.cu -- placeholder until the reverse-mode kernels land.
#include "dg_adjoint.h"

void adjoint_free(AdjointStore& s) {
  cudaFree(s.ckpt);
  cudaFree(s.dt_hist);
  cudaFree(s.work);
  s = AdjointStore();
}
void adjoint_reset(AdjointStore& s) { s.nrec = 0; }
dg_status adjoint_reserve(AdjointStore&, int, long, int, long long, std::string& msg) {
  msg = "adjoint not available in this build";
  return DG_ESTATE;
}
dg_status adjoint_step(AdjointStore&, const AdjointCall&, const double*, const double*, double*,
                       double, std::string& msg) {
  msg = "adjoint not available in this build";
  return DG_ESTATE;
}
dg_status adjoint_run(AdjointStore&, const AdjointCall&, int, int, const double*, double*,
                      std::string& msg) {
  msg = "adjoint not available in this build";
  return DG_ESTATE;
}
