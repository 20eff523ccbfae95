// dg_misc.cu -- layout conversion, Courant reduction and diagnostics kernels.
#include <cuda_runtime.h>

#include "dg_internal.h"
#include "dg_physics.cuh"

namespace dgk {

// ---------------------------------------------------------------------------
// Layout conversion (one plane at a time, grid-stride, coalesced)
// ---------------------------------------------------------------------------
template <class TS>
__global__ void plane_in_kernel(const double* __restrict__ src, StateBuf<TS> dst, int kind, int idx,
                                long ncell) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < ncell;
       i += (long)gridDim.x * blockDim.x) {
    double v = src[i];
    if (kind == 0) dst.c0[(size_t)idx * ncell + i] = v;
    else dst.sl[(size_t)idx * ncell + i] = (TS)v;
  }
}

template <class TS>
__global__ void plane_out_kernel(StateBuf<TS> src, double* __restrict__ dst, int kind, int idx,
                                 long ncell) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < ncell;
       i += (long)gridDim.x * blockDim.x) {
    dst[i] = kind == 0 ? src.c0[(size_t)idx * ncell + i] : (double)src.sl[(size_t)idx * ncell + i];
  }
}

static inline unsigned grid_for(long n, int threads) {
  long b = (n + threads - 1) / threads;
  if (b > 152L * 16) b = 152L * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

template <class TS>
cudaError_t launch_plane_in(const double* src, StateBuf<TS> dst, int kind, int idx, long ncell,
                            cudaStream_t st) {
  plane_in_kernel<TS><<<grid_for(ncell, 256), 256, 0, st>>>(src, dst, kind, idx, ncell);
  return cudaGetLastError();
}
template <class TS>
cudaError_t launch_plane_out(StateBuf<TS> src, double* dst, int kind, int idx, long ncell,
                             cudaStream_t st) {
  plane_out_kernel<TS><<<grid_for(ncell, 256), 256, 0, st>>>(src, dst, kind, idx, ncell);
  return cudaGetLastError();
}
// All planes of one problem in one launch (blockIdx.y = plane): the interchange
// planes at src (device or page-locked host memory) into the state, or back.
template <class TS>
__global__ void state_in_kernel(const double* __restrict__ src, StateBuf<TS> dst, PlaneMap map,
                                long ncell) {
  const int k = blockIdx.y, kind = map.kind[k];
  const size_t o = (size_t)map.idx[k] * ncell;
  const double* s = src + (size_t)k * ncell;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < ncell;
       i += (long)gridDim.x * blockDim.x) {
    const double v = s[i];
    if (kind == 0) dst.c0[o + i] = v;
    else dst.sl[o + i] = (TS)v;
  }
}

template <class TS>
__global__ void state_out_kernel(StateBuf<TS> src, double* __restrict__ dst, PlaneMap map,
                                 long ncell) {
  const int k = blockIdx.y, kind = map.kind[k];
  const size_t o = (size_t)map.idx[k] * ncell;
  double* d = dst + (size_t)k * ncell;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < ncell;
       i += (long)gridDim.x * blockDim.x)
    d[i] = kind == 0 ? src.c0[o + i] : (double)src.sl[o + i];
}

static inline dim3 state_grid(long ncell, int nplanes) {
  long b = (ncell + 255) / 256, cap = 152L * 16 / (nplanes > 0 ? nplanes : 1);
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return dim3((unsigned)b, (unsigned)nplanes);
}

template <class TS>
cudaError_t launch_state_in(const double* src, StateBuf<TS> dst, const PlaneMap& map, long ncell,
                            cudaStream_t st) {
  state_in_kernel<TS><<<state_grid(ncell, map.nplanes), 256, 0, st>>>(src, dst, map, ncell);
  return cudaGetLastError();
}
template <class TS>
cudaError_t launch_state_out(StateBuf<TS> src, double* dst, const PlaneMap& map, long ncell,
                             cudaStream_t st) {
  state_out_kernel<TS><<<state_grid(ncell, map.nplanes), 256, 0, st>>>(src, dst, map, ncell);
  return cudaGetLastError();
}
template cudaError_t launch_state_in<double>(const double*, StateBuf<double>, const PlaneMap&,
                                             long, cudaStream_t);
template cudaError_t launch_state_in<float>(const double*, StateBuf<float>, const PlaneMap&, long,
                                            cudaStream_t);
template cudaError_t launch_state_out<double>(StateBuf<double>, double*, const PlaneMap&, long,
                                              cudaStream_t);
template cudaError_t launch_state_out<float>(StateBuf<float>, double*, const PlaneMap&, long,
                                             cudaStream_t);

template cudaError_t launch_plane_in<double>(const double*, StateBuf<double>, int, int, long,
                                             cudaStream_t);
template cudaError_t launch_plane_in<float>(const double*, StateBuf<float>, int, int, long,
                                            cudaStream_t);
template cudaError_t launch_plane_out<double>(StateBuf<double>, double*, int, int, long,
                                              cudaStream_t);
template cudaError_t launch_plane_out<float>(StateBuf<float>, double*, int, int, long,
                                             cudaStream_t);

// ---------------------------------------------------------------------------
// Courant signal speed of a state (used when a state is set; during stepping
// the same reduction is fused into stage 2).  Arithmetic in TC = TS, as in the
// fused reduction of the stage kernels.
// ---------------------------------------------------------------------------
template <class TS>
__global__ void cfl_kernel(int eq, int dim, StateBuf<TS> s, int nx, int ny, int nz, double dx,
                           double dy, double dz, double gamma, Ctl* ctl) {
  using TC = TS;
  Gas<TC> G;
  G.set(gamma);
  const long ncell = (long)nx * ny * nz;
  double m = 0.0;
  unsigned err = 0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < ncell;
       i += (long)gridDim.x * blockDim.x) {
    TC rho = (TC)s.c0[i];
    TC inv = TC(1) / rho;
    TC vx = (TC)s.c0[ncell + i] * inv, vy = (TC)s.c0[2 * ncell + i] * inv, vz = TC(0);
    TC kin = TC(0.5) * ((TC)s.c0[ncell + i] * vx + (TC)s.c0[2 * ncell + i] * vy);
    int ie = 3;
    if (dim == 3) {
      vz = (TC)s.c0[3 * ncell + i] * inv;
      kin = TC(0.5) * ((TC)s.c0[ncell + i] * vx + (TC)s.c0[2 * ncell + i] * vy +
                       (TC)s.c0[3 * ncell + i] * vz);
      ie = 4;
    }
    TC bx = TC(0), by = TC(0), bz = TC(0), mag = TC(0);
    if (eq == 1) {
      const int ib = ie + 1;  // the field averages follow the energy
      bx = (TC)s.c0[ib * ncell + i];
      by = (TC)s.c0[(ib + 1) * ncell + i];
      if (dim == 3) bz = (TC)s.c0[(ib + 2) * ncell + i];
      mag = TC(0.5) * (bx * bx + by * by + bz * bz);
    }
    TC p = G.gm1 * ((TC)s.c0[ie * ncell + i] - kin - mag);
    // a non-finite density or pressure is as non-physical as a negative one (an
    // infinite density would give a zero signal speed)
    if (!(rho > TC(0) && p > TC(0) && rho < TC(INFINITY) && p < TC(INFINITY))) {
      err |= ERR_NONPHYS;
      continue;
    }
    TC sp;
    if (eq == 1) {
      TC b2 = bx * bx + by * by + bz * bz;
      sp = (fabs(vx) + fast_speed(G, rho, p, b2, bx)) / (TC)dx +
           (fabs(vy) + fast_speed(G, rho, p, b2, by)) / (TC)dy;
      if (dim == 3) sp += (fabs(vz) + fast_speed(G, rho, p, b2, bz)) / (TC)dz;
    } else {
      TC c = sqrt(G.g * p / rho);
      sp = (fabs(vx) + c) / (TC)dx + (fabs(vy) + c) / (TC)dy;
      if (dim == 3) sp += (fabs(vz) + c) / (TC)dz;
    }
    m = (double)sp > m ? (double)sp : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    double t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(&ctl->vmax_next, (unsigned long long)__double_as_longlong(m));
  if (err) atomicOr(&ctl->err, err);
}

template <class TS>
cudaError_t launch_cfl(int eq, int dim, StateBuf<TS> s, int nx, int ny, int nz, double dx,
                       double dy, double dz, double gamma, Ctl* ctl, cudaStream_t st) {
  long n = (long)nx * ny * nz;
  cfl_kernel<TS><<<grid_for(n, 256), 256, 0, st>>>(eq, dim, s, nx, ny, nz, dx, dy, dz, gamma, ctl);
  return cudaGetLastError();
}
template cudaError_t launch_cfl<double>(int, int, StateBuf<double>, int, int, int, double, double,
                                        double, double, Ctl*, cudaStream_t);
template cudaError_t launch_cfl<float>(int, int, StateBuf<float>, int, int, int, double, double,
                                       double, double, Ctl*, cudaStream_t);

__global__ void ctl_reset_kernel(Ctl* ctl, int nprob) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nprob) {
    ctl[p].vmax_cur = 0.0;
    ctl[p].dt_cur = 0.0;
    ctl[p].vmax_next = 0ull;
    ctl[p].t = 0.0;
    ctl[p].dt_last = 0.0;
    ctl[p].step = 0;
    ctl[p].ticket = 0u;
    ctl[p].err = 0u;
    ctl[p].err_step = -1;
  }
}
__global__ void ctl_commit_kernel(Ctl* ctl, int nprob, double cfl) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nprob) {
    double vm = __longlong_as_double((long long)ctl[p].vmax_next);
    ctl[p].vmax_cur = vm;
    ctl[p].dt_cur = cfl / vm;
    ctl[p].vmax_next = 0ull;
    if (!(vm > 0.0)) ctl[p].err |= ERR_NONPHYS;
    if (ctl[p].err && ctl[p].err_step < 0) ctl[p].err_step = ctl[p].step;
  }
}
cudaError_t launch_ctl_reset(Ctl* ctl, int nprob, cudaStream_t st) {
  ctl_reset_kernel<<<(nprob + 127) / 128, 128, 0, st>>>(ctl, nprob);
  return cudaGetLastError();
}
cudaError_t launch_ctl_commit(Ctl* ctl, int nprob, double cfl, cudaStream_t st) {
  ctl_commit_kernel<<<(nprob + 127) / 128, 128, 0, st>>>(ctl, nprob, cfl);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Neumaier-compensated totals: per block (sum, compensation) pairs, then one
// block combines the partials in a fixed order (deterministic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
  double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x;
  else c += (x - t) + s;
  s = t;
}

__global__ void totals_partial_kernel(const double* __restrict__ c0, long ncell,
                                      double* __restrict__ partial) {
  const int v = blockIdx.y;
  double s = 0.0, c = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < ncell;
       i += (long)gridDim.x * blockDim.x)
    neumaier_add(s, c, c0[(size_t)v * ncell + i]);
  __shared__ double ss[256], cc[256];
  ss[threadIdx.x] = s;
  cc[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, C = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) {
      neumaier_add(S, C, ss[k]);
      C += cc[k];
    }
    partial[((size_t)v * gridDim.x + blockIdx.x) * 2] = S;
    partial[((size_t)v * gridDim.x + blockIdx.x) * 2 + 1] = C;
  }
}

__global__ void totals_final_kernel(const double* __restrict__ partial, int nblk, int nv,
                                    double* __restrict__ out) {
  int v = threadIdx.x;
  if (v >= nv) return;
  double S = 0.0, C = 0.0;
  for (int b = 0; b < nblk; ++b) {
    neumaier_add(S, C, partial[((size_t)v * nblk + b) * 2]);
    C += partial[((size_t)v * nblk + b) * 2 + 1];
  }
  out[v] = S + C;
}

cudaError_t launch_totals(const double* c0, int nv, long ncell, double* partial, double* out,
                          cudaStream_t st) {
  const int nblk = 256;
  totals_partial_kernel<<<dim3(nblk, nv), 256, 0, st>>>(c0, ncell, partial);
  totals_final_kernel<<<1, 32, 0, st>>>(partial, nblk, nv, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sec. 2.6 Stokes div-B estimate per cell (2D MHD): the face-normal field at
// each face Gauss point is the average of both one-sided polynomial values.
// Internal indices: averages b1 = 4, b2 = 5; coefficients a1 = 8, a2 = 9, a3 = 10.
// ---------------------------------------------------------------------------
template <class TS>
__global__ void divb_kernel(StateBuf<TS> s, int nx, int ny, double dx, double dy,
                            double* __restrict__ out) {
  const long ncell = (long)nx * ny;
  const double o = 0.28867513459481288225;  // 1/(2 sqrt 3)
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    int i = (int)(c % nx), j = (int)(c / nx);
    auto BX = [&](long cell, double x, double y) {
      return s.c0[4 * ncell + cell] + (double)s.sl[10 * ncell + cell] * x +
             (double)s.sl[8 * ncell + cell] * y;
    };
    auto BY = [&](long cell, double x, double y) {
      return s.c0[5 * ncell + cell] + (double)s.sl[9 * ncell + cell] * x -
             (double)s.sl[10 * ncell + cell] * y;
    };
    long xp = (long)j * nx + (i + 1) % nx, xm = (long)j * nx + (i + nx - 1) % nx;
    long yp = (long)((j + 1) % ny) * nx + i, ym = (long)((j + ny - 1) % ny) * nx + i;
    double acc = 0.0;
    for (int g = 0; g < 2; ++g) {
      double ty = (g ? 1.0 : -1.0) * o * dy, tx = (g ? 1.0 : -1.0) * o * dx;
      acc += 0.5 * dy * 0.5 * (BX(c, 0.5 * dx, ty) + BX(xp, -0.5 * dx, ty));
      acc -= 0.5 * dy * 0.5 * (BX(c, -0.5 * dx, ty) + BX(xm, 0.5 * dx, ty));
      acc += 0.5 * dx * 0.5 * (BY(c, tx, 0.5 * dy) + BY(yp, tx, -0.5 * dy));
      acc -= 0.5 * dx * 0.5 * (BY(c, tx, -0.5 * dy) + BY(ym, tx, 0.5 * dy));
    }
    out[c] = acc / (dx * dy);
  }
}

template <class TS>
cudaError_t launch_divb(StateBuf<TS> s, int nx, int ny, double dx, double dy, double* out,
                        cudaStream_t st) {
  long n = (long)nx * ny;
  divb_kernel<TS><<<grid_for(n, 256), 256, 0, st>>>(s, nx, ny, dx, dy, out);
  return cudaGetLastError();
}
template cudaError_t launch_divb<double>(StateBuf<double>, int, int, double, double, double*,
                                         cudaStream_t);
template cudaError_t launch_divb<float>(StateBuf<float>, int, int, double, double, double*,
                                        cudaStream_t);

}  // namespace dgk
