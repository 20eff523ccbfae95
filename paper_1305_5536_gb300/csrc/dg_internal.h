// dg_internal.h -- declarations shared by the translation units of libdg.so.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "dg_common.cuh"

namespace dgk {

// Mapping of the interchange planes onto the internal state: plane p is average
// number idx[p] (kind 0) or derivative coefficient number idx[p] (kind 1).
struct PlaneMap {
  int nplanes;
  int kind[32];
  int idx[32];
};

// Number of tile shapes compiled for each (equations, dimension, precision).
int stage2d_variants(int eq, int fp32);
int stage3d_variants(int fp32);
const char* stage2d_variant_name(int eq, int fp32, int v);
const char* stage3d_variant_name(int fp32, int v);

cudaError_t launch_stage2d(int eq, int variant, int stage, const Stage2DArgs<double>& a,
                           cudaStream_t st);
cudaError_t launch_stage2d(int eq, int variant, int stage, const Stage2DArgs<float>& a,
                           cudaStream_t st);
cudaError_t launch_stage3d(int variant, int stage, const Stage3DArgs<double>& a, cudaStream_t st);
cudaError_t launch_stage3d(int variant, int stage, const Stage3DArgs<float>& a, cudaStream_t st);
// 3D MHD (11-function field basis).
int stage3m_variants(int fp32);
const char* stage3m_variant_name(int fp32, int v);
cudaError_t launch_stage3m(int variant, int stage, const Stage3DArgs<double>& a, cudaStream_t st);
cudaError_t launch_stage3m(int variant, int stage, const Stage3DArgs<float>& a, cudaStream_t st);

// MUSCL-Hancock step kernels (one launch per step; face_points 1 or 2).
int mh2d_variants(int eq, int fp32);
const char* mh2d_variant_name(int eq, int fp32, int v);
cudaError_t launch_mh2d(int eq, int variant, int face_points, const Stage2DArgs<double>& a,
                        cudaStream_t st);
cudaError_t launch_mh2d(int eq, int variant, int face_points, const Stage2DArgs<float>& a,
                        cudaStream_t st);
int mh3d_variants(int fp32);
const char* mh3d_variant_name(int fp32, int v);
cudaError_t launch_mh3d(int variant, int face_points, const Stage3DArgs<double>& a,
                        cudaStream_t st);
cudaError_t launch_mh3d(int variant, int face_points, const Stage3DArgs<float>& a,
                        cudaStream_t st);
int mh3m_variants(int fp32);
const char* mh3m_variant_name(int fp32, int v);
cudaError_t launch_mh3m(int variant, int face_points, const Stage3DArgs<double>& a,
                        cudaStream_t st);
cudaError_t launch_mh3m(int variant, int face_points, const Stage3DArgs<float>& a,
                        cudaStream_t st);

// Layout conversion of all interchange planes of one problem (device or
// page-locked host memory) to/from the state, in one launch.
template <class TS>
cudaError_t launch_state_in(const double* src, StateBuf<TS> dst, const PlaneMap& map, long ncell,
                            cudaStream_t st);
template <class TS>
cudaError_t launch_state_out(StateBuf<TS> src, double* dst, const PlaneMap& map, long ncell,
                             cudaStream_t st);

// Layout conversion of one interchange plane (ncell doubles) to/from the state.
template <class TS>
cudaError_t launch_plane_in(const double* src, StateBuf<TS> dst, int kind, int idx, long ncell,
                            cudaStream_t st);
template <class TS>
cudaError_t launch_plane_out(StateBuf<TS> src, double* dst, int kind, int idx, long ncell,
                             cudaStream_t st);

// Courant signal speed of a state: max over cells of sum_d (|v_d| + c_d)/dx_d into
// ctl->vmax_next (atomic max); then commit moves it to vmax_cur.
template <class TS>
cudaError_t launch_cfl(int eq, int dim, StateBuf<TS> s, int nx, int ny, int nz, double dx,
                       double dy, double dz, double gamma, Ctl* ctl, cudaStream_t st);
cudaError_t launch_ctl_reset(Ctl* ctl, int nprob, cudaStream_t st);
cudaError_t launch_ctl_commit(Ctl* ctl, int nprob, double cfl, cudaStream_t st);

// Neumaier-compensated FP64 sums of the average planes: out[v] = sum_cells c0[v].
cudaError_t launch_totals(const double* c0, int nv, long ncell, double* partial, double* out,
                          cudaStream_t st);

// Stokes div-B estimate per cell (2D MHD).
template <class TS>
cudaError_t launch_divb(StateBuf<TS> s, int nx, int ny, double dx, double dy, double* out,
                        cudaStream_t st);

// Message returned by dg_last_error(NULL) (failures without a context).
void set_global_error(const std::string& msg);

}  // namespace dgk
