// dg_adjoint.cu -- reverse mode of the SSP-RK2 step of the 2D DG scheme (Euler
// and planar MHD, with the min/max limiter or without).
//
// Forward step with the time step dt held fixed (Lambda = limiter, L = DG
// right-hand side):
//   U^n = Lambda(V^n),  V^1 = U^n + dt L(U^n),  U^1 = Lambda(V^1),
//   V^{n+1} = 1/2 U^n + 1/2 U^1 + 1/2 dt L(U^1).
// Given lam = dJ/dV^{n+1}, its transpose is
//   mu1 = 1/2 lam + 1/2 dt J_L(U^1)^T lam          (dJ/dU^1)
//   lam1 = J_Lambda(V^1)^T mu1                      (dJ/dV^1)
//   mu0 = 1/2 lam + lam1 + dt J_L(U^n)^T lam1        (dJ/dU^n)
//   lam^n = J_Lambda(V^n)^T mu0                     (dJ/dV^n)
// J_L^T is applied by a tiled kernel that mirrors the forward one: every face
// Gauss point gets the adjoint of its flux from the two cells' adjoints, one
// reverse sweep through the exact solver gives the adjoints of both one-sided
// states (dg_vjp.cuh), and each cell gathers the contributions of its faces and of
// its 2x2 volume points (reverse sweeps through the physical fluxes).  J_Lambda^T gathers, for each cell, the derivatives of its
// own limited slopes and of its four neighbours' (whose limiter reads this
// cell's averages).  Adjoint arrays use the interchange layout (float64).
#include <cuda_runtime.h>

#include <cstdio>
#include <string>
#include <vector>

#include "dg_adjoint.h"
#include "dg_dual.cuh"
#include "dg_internal.h"
#include "dg_stage2d.cuh"
#include "dg_vjp.cuh"

using namespace dgk;

namespace {

// tile of the transposed right-hand-side kernel (static shared memory < 48 KB)
template <class TC> struct VjpTile;
template <> struct VjpTile<double> { static constexpr int X = 8, Y = 8; };
template <> struct VjpTile<float> { static constexpr int X = 16, Y = 8; };

// ---------------------------------------------------------------------------
// U = Lambda(V): the limited state as its own array (internal layout)
// ---------------------------------------------------------------------------
template <class TC, class TS>
__global__ void limit2d_kernel(StateBuf<TS> V, StateBuf<TS> U, int nx, int ny, double dx,
                               double dy, double gamma) {
  const long ncell = (long)nx * ny;
  Gas<TC> G;
  G.set(gamma);
  const TC hh[2] = {TC(0.5 * dx), TC(0.5 * dy)};
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)(c / nx);
    const long nb[4] = {(long)j * nx + wrap_index(i - 1, nx), (long)j * nx + wrap_index(i + 1, nx),
                        (long)wrap_index(j - 1, ny) * nx + i, (long)wrap_index(j + 1, ny) * nx + i};
    TC cc[4], W[4], Wn[4][4], s[8];
    unsigned err = 0;
#pragma unroll
    for (int v = 0; v < 4; ++v) cc[v] = Cvt<TC>::to_tc(V.c0[v * ncell + c]);
    prims2d<0, TC>(G, cc, W, err);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      TC cn[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) cn[v] = Cvt<TC>::to_tc(V.c0[v * ncell + nb[k]]);
      prims2d<0, TC>(G, cn, Wn[k], err);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] = (TC)V.sl[k * ncell + c];
    limit_cell2d<0, TC>(G, hh, W, Wn, s);
#pragma unroll
    for (int v = 0; v < 4; ++v) U.c0[v * ncell + c] = V.c0[v * ncell + c];
#pragma unroll
    for (int k = 0; k < 8; ++k) U.sl[k * ncell + c] = (TS)s[k];
  }
}

// ---------------------------------------------------------------------------
// out = a1 x1 + a2 x2 + beta J_L(U)^T y   (interchange layout; x2 may be null)
// ---------------------------------------------------------------------------
struct VjpArgs {
  int nx, ny;
  long ncell;
  double dx, dy, gamma;
  const double* y;
  const double* x1;
  double a1;
  const double* x2;
  double a2;
  double beta;
  double* out;
  unsigned* err;
};

template <class TC, class TS>
__global__ void __launch_bounds__(VjpTile<TC>::X * VjpTile<TC>::Y) rhs_vjp2d_kernel(StateBuf<TS> U, VjpArgs A) {
  constexpr int AX = VjpTile<TC>::X, AY = VjpTile<TC>::Y, ANT = AX * AY;
  constexpr int R1X = AX + 2, R1Y = AY + 2, R1 = R1X * R1Y;
  constexpr int NFX = (AX + 1) * AY, NFY = AX * (AY + 1);
  __shared__ TC s_c0[4 * R1], s_sl[8 * R1], s_y[12 * R1];
  __shared__ TC s_lx[8 * 2 * NFX], s_ly[8 * 2 * NFY];
  __shared__ int s_gx[R1X], s_gy[R1Y];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * AX, j0 = blockIdx.y * AY;
  const int nx = A.nx, ny = A.ny;
  const size_t ncell = (size_t)A.ncell;
  Gas<TC> G;
  G.set(A.gamma);
  unsigned err = 0;
  if (tid < R1X) s_gx[tid] = wrap_index(i0 - 1 + tid, nx);
  else if (tid < R1X + R1Y) s_gy[tid - R1X] = wrap_index(j0 - 1 + (tid - R1X), ny) * nx;
  __syncthreads();
  for (int r = tid; r < R1; r += ANT) {
    int ry = r / R1X, rx = r - ry * R1X;
    size_t g = (size_t)s_gy[ry] + s_gx[rx];
#pragma unroll
    for (int v = 0; v < 4; ++v) s_c0[v * R1 + r] = Cvt<TC>::to_tc(U.c0[v * ncell + g]);
#pragma unroll
    for (int k = 0; k < 8; ++k) s_sl[k * R1 + r] = (TC)U.sl[k * ncell + g];
#pragma unroll
    for (int p = 0; p < 12; ++p) s_y[p * R1 + r] = Cvt<TC>::to_tc(A.y[p * ncell + g]);
  }
  __syncthreads();

  const TC dx = (TC)A.dx, dy = (TC)A.dy;
  const TC hx = TC(0.5) * dx, hy = TC(0.5) * dy;
  const TC ox = dx * TC(0.28867513459481288225), oy = dy * TC(0.28867513459481288225);
  const TC c3x = TC(3) / (dx * dx), c3y = TC(3) / (dy * dy);
  const TC r3 = TC(1.7320508075688772935) / (dx * dy);
  const TC i2x = TC(0.5) / dx, i2y = TC(0.5) / dy;

  // ---- faces: adjoint of every Gauss-point flux -> adjoints of both states
  for (int e = tid; e < 2 * (NFX + NFY); e += ANT) {
    const bool xf = e < 2 * NFX;
    const int ee = xf ? e : e - 2 * NFX;
    const int f = ee >> 1, g = ee & 1;
    const TC sg = g ? TC(1) : TC(-1);
    int rl, rr;
    TC xl, yl, xr, yr;
    if (xf) {
      int fy = f / (AX + 1), fx = f - fy * (AX + 1);
      rl = (fy + 1) * R1X + fx;
      rr = rl + 1;
      xl = hx; xr = -hx; yl = yr = sg * oy;
    } else {
      int fy = f / AX, fx = f - fy * AX;
      rl = fy * R1X + fx + 1;
      rr = rl + R1X;
      yl = hy; yr = -hy; xl = xr = sg * ox;
    }
    TC mu[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      TC yl0 = s_y[(3 * q) * R1 + rl], ylx = s_y[(3 * q + 1) * R1 + rl], yly = s_y[(3 * q + 2) * R1 + rl];
      TC yr0 = s_y[(3 * q) * R1 + rr], yrx = s_y[(3 * q + 1) * R1 + rr], yry = s_y[(3 * q + 2) * R1 + rr];
      if (xf)
        mu[q] = (yr0 - yl0) * i2x - c3x * (ylx + yrx) + r3 * sg * (yry - yly);
      else
        mu[q] = (yr0 - yl0) * i2y - c3y * (yly + yry) + r3 * sg * (yrx - ylx);
    }
    TC cl[4], cr[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      cl[v] = s_c0[v * R1 + rl] + s_sl[(2 * v) * R1 + rl] * xl + s_sl[(2 * v + 1) * R1 + rl] * yl;
      cr[v] = s_c0[v * R1 + rr] + s_sl[(2 * v) * R1 + rr] * xr + s_sl[(2 * v + 1) * R1 + rr] * yr;
    }
    // adjoints of both one-sided states, one reverse sweep through the flux
    TC lam[8];
    face_flux2d_vjp<TC>(G, xf ? 0 : 1, cl, cr, mu, lam, lam + 4, err);
    if (xf) {
#pragma unroll
      for (int k = 0; k < 8; ++k) s_lx[(k * 2 + g) * NFX + f] = lam[k];
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) s_ly[(k * 2 + g) * NFY + f] = lam[k];
    }
  }
  __syncthreads();

  // ---- per cell: gather faces and volume points
  const int lx = tid % AX, ly = tid / AX;
  const int gi = i0 + lx, gj = j0 + ly;
  if (gi < nx && gj < ny) {
    const int r = (ly + 1) * R1X + lx + 1;
    TC acc[12];
#pragma unroll
    for (int p = 0; p < 12; ++p) acc[p] = TC(0);
    const int fxm = ly * (AX + 1) + lx, fym = ly * AX + lx;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const TC sg = g ? TC(1) : TC(-1);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        // x faces: this cell is the right state of face fxm, the left of fxm+1
        TC aR = s_lx[((4 + v) * 2 + g) * NFX + fxm];
        TC aL = s_lx[(v * 2 + g) * NFX + fxm + 1];
        acc[3 * v] += aR + aL;
        acc[3 * v + 1] += (aL - aR) * hx;
        acc[3 * v + 2] += (aR + aL) * sg * oy;
        // y faces: upper state of fym, lower state of fym+AX
        TC bU = s_ly[((4 + v) * 2 + g) * NFY + fym];
        TC bL = s_ly[(v * 2 + g) * NFY + fym + AX];
        acc[3 * v] += bU + bL;
        acc[3 * v + 1] += (bU + bL) * sg * ox;
        acc[3 * v + 2] += (bL - bU) * hy;
      }
    }
    // volume points: d(rhs_x)/dF_x = c3x, d(rhs_y)/dF_y = c3y
    TC yx[4], yy[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      yx[q] = c3x * s_y[(3 * q + 1) * R1 + r];
      yy[q] = c3y * s_y[(3 * q + 2) * R1 + r];
    }
#pragma unroll
    for (int qp = 0; qp < 4; ++qp) {
      const TC xq = (qp & 1) ? ox : -ox, yq = (qp & 2) ? oy : -oy;
      TC c[4], a[4];
#pragma unroll
      for (int v = 0; v < 4; ++v)
        c[v] = s_c0[v * R1 + r] + s_sl[(2 * v) * R1 + r] * xq + s_sl[(2 * v + 1) * R1 + r] * yq;
      phys_flux2d_vjp<TC>(G, c, yx, yy, a);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        acc[3 * i] += a[i];
        acc[3 * i + 1] += a[i] * xq;
        acc[3 * i + 2] += a[i] * yq;
      }
    }
    const size_t gc = (size_t)gj * nx + gi;
#pragma unroll
    for (int p = 0; p < 12; ++p) {
      double o = A.a1 * A.x1[p * ncell + gc] + A.beta * Cvt<TC>::to_f64(acc[p]);
      if (A.x2) o += A.a2 * A.x2[p * ncell + gc];
      A.out[p * ncell + gc] = o;
    }
  }
  if (err) atomicOr(A.err, err);
}

// ---------------------------------------------------------------------------
// out = J_Lambda(V)^T nu   (interchange layout)
// ---------------------------------------------------------------------------
template <class TC, class TS>
__global__ void limit_vjp2d_kernel(StateBuf<TS> V, const double* __restrict__ nu, double* out,
                                   int nx, int ny, double dx, double dy, double gamma) {
  const long ncell = (long)nx * ny;
  Gas<TC> G;
  G.set(gamma);
  const TC hh[2] = {TC(0.5 * dx), TC(0.5 * dy)};
  typedef Dn<TC, 4> D;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)(c / nx);
    auto at = [&](int di, int dj) {
      return (long)wrap_index(j + dj, ny) * nx + wrap_index(i + di, nx);
    };
    auto load_c0 = [&](long cell, TC* o) {
#pragma unroll
      for (int v = 0; v < 4; ++v) o[v] = Cvt<TC>::to_tc(V.c0[v * ncell + cell]);
    };
    TC acc[12];
#pragma unroll
    for (int p = 0; p < 12; ++p) acc[p] = TC(0);
    // averages pass through the limiter unchanged
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[3 * v] = Cvt<TC>::to_tc(nu[(3 * v) * ncell + c]);
    const int ofs[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    // (a) this cell's own limiter: derivatives with respect to its averages and
    //     its derivative coefficients (three passes of four directions)
    {
      TC c0v[4], sv[8], cnv[4][4], nus[8];
      load_c0(c, c0v);
#pragma unroll
      for (int k = 0; k < 8; ++k) sv[k] = (TC)V.sl[k * ncell + c];
#pragma unroll
      for (int k = 0; k < 4; ++k) load_c0(at(ofs[k][0], ofs[k][1]), cnv[k]);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        nus[2 * v] = Cvt<TC>::to_tc(nu[(3 * v + 1) * ncell + c]);
        nus[2 * v + 1] = Cvt<TC>::to_tc(nu[(3 * v + 2) * ncell + c]);
      }
#pragma unroll
      for (int pass = 0; pass < 3; ++pass) {
        D c0[4], cn[4][4], s[8];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          c0[v] = dconst<TC, 4>(c0v[v]);
#pragma unroll
          for (int k = 0; k < 4; ++k) cn[k][v] = dconst<TC, 4>(cnv[k][v]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] = dconst<TC, 4>(sv[k]);
        if (pass == 0) {
#pragma unroll
          for (int v = 0; v < 4; ++v) c0[v].d[v] = TC(1);
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t) s[(pass - 1) * 4 + t].d[t] = TC(1);
        }
        dlimit_cell2d<TC, 4>(G, hh, c0, cn, s);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          TC a = TC(0);
#pragma unroll
          for (int k = 0; k < 8; ++k) a += nus[k] * s[k].d[t];
          if (pass == 0) acc[3 * t] += a;
          else {
            int k = (pass - 1) * 4 + t;  // slope index v*2 + d
            acc[3 * (k >> 1) + 1 + (k & 1)] += a;
          }
        }
      }
    }
    // (b) each neighbour e's limiter reads this cell's averages
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      const int ei = ofs[k][0], ej = ofs[k][1];
      const long e = at(ei, ej);
      TC c0v[4], sv[8], nus[8];
      load_c0(e, c0v);
#pragma unroll
      for (int q = 0; q < 8; ++q) sv[q] = (TC)V.sl[q * ncell + e];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        nus[2 * v] = Cvt<TC>::to_tc(nu[(3 * v + 1) * ncell + e]);
        nus[2 * v + 1] = Cvt<TC>::to_tc(nu[(3 * v + 2) * ncell + e]);
      }
      D c0[4], cn[4][4], s[8];
#pragma unroll
      for (int v = 0; v < 4; ++v) c0[v] = dconst<TC, 4>(c0v[v]);
#pragma unroll
      for (int q = 0; q < 8; ++q) s[q] = dconst<TC, 4>(sv[q]);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        TC tmp[4];
        load_c0(at(ei + ofs[m][0], ej + ofs[m][1]), tmp);
#pragma unroll
        for (int v = 0; v < 4; ++v) cn[m][v] = dconst<TC, 4>(tmp[v]);
      }
      // this cell is neighbour number (k ^ 1) of e (left <-> right, down <-> up)
      const int me = k ^ 1;
#pragma unroll
      for (int v = 0; v < 4; ++v) cn[me][v].d[v] = TC(1);
      dlimit_cell2d<TC, 4>(G, hh, c0, cn, s);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        TC a = TC(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) a += nus[q] * s[q].d[t];
        acc[3 * t] += a;
      }
    }
#pragma unroll
    for (int p = 0; p < 12; ++p) out[p * ncell + c] = Cvt<TC>::to_f64(acc[p]);
  }
}

// ---------------------------------------------------------------------------
// Planar MHD (limiter off): out = a1 x1 + a2 x2 + beta J_L(U)^T y.  The face and
// volume flux Jacobians are taken in forward mode: the scalar HLLD solver and
// physical flux instantiated on dual numbers, one pass of six tangents per side
// (the conserved point values rho, mx, my, E, Bx, By), contracted with the flux
// adjoints.  Adjoint arrays in the interchange layout: planes v*3 + k of
// (rho, mx, my, E), then b1, b2, a1, a2, a3 (12 .. 16).
// ---------------------------------------------------------------------------
template <class TC> struct VjpTileM;
template <> struct VjpTileM<double> { static constexpr int X = 8, Y = 4; };
template <> struct VjpTileM<float> { static constexpr int X = 8, Y = 8; };

// The MHD branch of face_flux2d on dual conserved states.
template <class TC, int N>
__device__ void dface_flux2d_mhd(const Gas<Dn<TC, N>>& G, int dir, const Dn<TC, N>* cl,
                                 const Dn<TC, N>* cr, Dn<TC, N>* F, unsigned& err) {
  typedef Dn<TC, N> D;
  const D rl = cl[0], rr = cr[0];
  const D il = TC(1) / rl, ir = TC(1) / rr;
  const D vxl = cl[1] * il, vyl = cl[2] * il, vxr = cr[1] * ir, vyr = cr[2] * ir;
  const D magl = TC(0.5) * (cl[4] * cl[4] + cl[5] * cl[5]);
  const D magr = TC(0.5) * (cr[4] * cr[4] + cr[5] * cr[5]);
  const D pl = G.gm1 * (cl[3] - TC(0.5) * (cl[1] * vxl + cl[2] * vyl) - magl);
  const D pr = G.gm1 * (cr[3] - TC(0.5) * (cr[1] * vxr + cr[2] * vyr) - magr);
  const bool xd = dir == 0;
  const D bn = TC(0.5) * (xd ? cl[4] + cr[4] : cl[5] + cr[5]);
  D Ff[5];
  hlld_flux<D>(G, rl, xd ? vxl : vyl, xd ? vyl : vxl, pl, xd ? cl[5] : cl[4], rr, xd ? vxr : vyr,
               xd ? vyr : vxr, pr, xd ? cr[5] : cr[4], bn, Ff, err);
  F[0] = Ff[0];
  F[3] = Ff[3];
  F[4] = Ff[4];
  if (xd) { F[1] = Ff[1]; F[2] = Ff[2]; }
  else { F[1] = Ff[2]; F[2] = Ff[1]; }
}

template <class TC>
__device__ __forceinline__ void dual_gas(double gamma, Gas<Dn<TC, 6>>& G) {
  G.set(gamma);
}

// Adjoints of both one-sided point states of one face Gauss point: lamL[i] =
// sum_q mu[q] dF_q / dcl[i], lamR likewise.
template <class TC>
__device__ void face_flux2d_mhd_vjp(const Gas<Dn<TC, 6>>& GD, int dir, const TC* cl, const TC* cr,
                                    const TC* mu, TC* lamL, TC* lamR, unsigned& err) {
  typedef Dn<TC, 6> D;
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    D a[6], b[6], F[5];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      a[i] = D(cl[i]);
      b[i] = D(cr[i]);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) (side == 0 ? a : b)[i].d[i] = TC(1);
    dface_flux2d_mhd<TC, 6>(GD, dir, a, b, F, err);
    TC* lam = side == 0 ? lamL : lamR;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      TC t = TC(0);
#pragma unroll
      for (int q = 0; q < 5; ++q) t += mu[q] * F[q].d[i];
      lam[i] = t;
    }
  }
}

// Adjoint of the conserved point state of one volume Gauss point: a[i] =
// sum_v (yx[v] dFx_v/dc_i + yy[v] dFy_v/dc_i).
template <class TC>
__device__ void phys_flux2d_mhd_vjp(const Gas<Dn<TC, 6>>& GD, const TC* c, const TC* yx,
                                    const TC* yy, TC* a, unsigned& err) {
  typedef Dn<TC, 6> D;
  D cd[6], Fx[5], Fy[5];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    cd[i] = D(c[i]);
    cd[i].d[i] = TC(1);
  }
  phys_flux2d<1, D>(GD, cd, Fx, Fy, err);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    TC t = TC(0);
#pragma unroll
    for (int v = 0; v < 5; ++v) t += yx[v] * Fx[v].d[i] + yy[v] * Fy[v].d[i];
    a[i] = t;
  }
}

// Adjoint of the point values (rho, mx, my, E, Bx, By) at local point (x, y) of a
// cell, added to the adjoints of its interchange coefficients (the transpose of
// eval2d<1>: Bx = b1 + a3 x + a1 y, By = b2 + a2 x - a3 y).
template <class TC>
__device__ __forceinline__ void add_point_mhd(TC* acc, const TC* lam, TC x, TC y) {
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    acc[3 * v] += lam[v];
    acc[3 * v + 1] += lam[v] * x;
    acc[3 * v + 2] += lam[v] * y;
  }
  acc[12] += lam[4];
  acc[13] += lam[5];
  acc[14] += lam[4] * y;
  acc[15] += lam[5] * x;
  acc[16] += lam[4] * x - lam[5] * y;
}

template <class TC, class TS>
__global__ void __launch_bounds__(VjpTileM<TC>::X * VjpTileM<TC>::Y)
    rhs_vjp2d_mhd_kernel(StateBuf<TS> U, VjpArgs A) {
  constexpr int AX = VjpTileM<TC>::X, AY = VjpTileM<TC>::Y, ANT = AX * AY;
  constexpr int R1X = AX + 2, R1Y = AY + 2, R1 = R1X * R1Y;
  constexpr int NFX = (AX + 1) * AY, NFY = AX * (AY + 1);
  __shared__ TC s_c0[6 * R1], s_sl[11 * R1], s_y[17 * R1];
  __shared__ TC s_lx[12 * 2 * NFX], s_ly[12 * 2 * NFY];
  __shared__ int s_gx[R1X], s_gy[R1Y];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * AX, j0 = blockIdx.y * AY;
  const int nx = A.nx, ny = A.ny;
  const size_t ncell = (size_t)A.ncell;
  Gas<TC> G;
  G.set(A.gamma);
  Gas<Dn<TC, 6>> GD;
  dual_gas<TC>(A.gamma, GD);
  unsigned err = 0;
  if (tid < R1X) s_gx[tid] = wrap_index(i0 - 1 + tid, nx);
  else if (tid < R1X + R1Y) s_gy[tid - R1X] = wrap_index(j0 - 1 + (tid - R1X), ny) * nx;
  __syncthreads();
  for (int r = tid; r < R1; r += ANT) {
    int ry = r / R1X, rx = r - ry * R1X;
    size_t g = (size_t)s_gy[ry] + s_gx[rx];
#pragma unroll
    for (int v = 0; v < 6; ++v) s_c0[v * R1 + r] = Cvt<TC>::to_tc(U.c0[v * ncell + g]);
#pragma unroll
    for (int k = 0; k < 11; ++k) s_sl[k * R1 + r] = (TC)U.sl[k * ncell + g];
#pragma unroll
    for (int p = 0; p < 17; ++p) s_y[p * R1 + r] = Cvt<TC>::to_tc(A.y[p * ncell + g]);
  }
  __syncthreads();

  const TC dx = (TC)A.dx, dy = (TC)A.dy;
  const TC hx = TC(0.5) * dx, hy = TC(0.5) * dy;
  const TC ox = dx * TC(0.28867513459481288225), oy = dy * TC(0.28867513459481288225);
  const TC c3x = TC(3) / (dx * dx), c3y = TC(3) / (dy * dy);
  const TC r3 = TC(1.7320508075688772935) / (dx * dy);
  const TC ca3 = TC(1.7320508075688772935) / (dx * dx + dy * dy);
  const TC i2x = TC(0.5) / dx, i2y = TC(0.5) / dy;
  auto point = [&](int r, TC x, TC y, TC* c) {
    TC c0[6], sl[11];
#pragma unroll
    for (int v = 0; v < 6; ++v) c0[v] = s_c0[v * R1 + r];
#pragma unroll
    for (int k = 0; k < 11; ++k) sl[k] = s_sl[k * R1 + r];
    eval2d<1, TC>(c0, sl, x, y, c);
  };

  // ---- faces: adjoint of every Gauss-point flux -> adjoints of both states
  for (int e = tid; e < 2 * (NFX + NFY); e += ANT) {
    const bool xf = e < 2 * NFX;
    const int ee = xf ? e : e - 2 * NFX;
    const int f = ee >> 1, g = ee & 1;
    const TC sg = g ? TC(1) : TC(-1);
    int rl, rr;
    TC xl, yl, xr, yr;
    if (xf) {
      int fy = f / (AX + 1), fx = f - fy * (AX + 1);
      rl = (fy + 1) * R1X + fx;
      rr = rl + 1;
      xl = hx; xr = -hx; yl = yr = sg * oy;
    } else {
      int fy = f / AX, fx = f - fy * AX;
      rl = fy * R1X + fx + 1;
      rr = rl + R1X;
      yl = hy; yr = -hy; xl = xr = sg * ox;
    }
    auto yL = [&](int p) { return s_y[p * R1 + rl]; };
    auto yR = [&](int p) { return s_y[p * R1 + rr]; };
    TC mu[5];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (xf)
        mu[q] = (yR(3 * q) - yL(3 * q)) * i2x - c3x * (yL(3 * q + 1) + yR(3 * q + 1)) +
                r3 * sg * (yR(3 * q + 2) - yL(3 * q + 2));
      else
        mu[q] = (yR(3 * q) - yL(3 * q)) * i2y - c3y * (yL(3 * q + 2) + yR(3 * q + 2)) +
                r3 * sg * (yR(3 * q + 1) - yL(3 * q + 1));
    }
    // the transverse-field flux: b2, a2, a3 across x faces; b1, a1, a3 across y faces
    if (xf)
      mu[4] = (yR(13) - yL(13)) * i2x - c3x * (yL(15) + yR(15)) +
              ca3 * (dy / dx) * sg * (yL(16) - yR(16));
    else
      mu[4] = (yR(12) - yL(12)) * i2y - c3y * (yL(14) + yR(14)) -
              ca3 * (dx / dy) * sg * (yL(16) - yR(16));
    TC cl[6], cr[6], lam[12];
    point(rl, xl, yl, cl);
    point(rr, xr, yr, cr);
    face_flux2d_mhd_vjp<TC>(GD, xf ? 0 : 1, cl, cr, mu, lam, lam + 6, err);
    if (xf) {
#pragma unroll
      for (int k = 0; k < 12; ++k) s_lx[(k * 2 + g) * NFX + f] = lam[k];
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) s_ly[(k * 2 + g) * NFY + f] = lam[k];
    }
  }
  __syncthreads();

  // ---- per cell: gather faces and volume points
  const int lx = tid % AX, ly = tid / AX;
  const int gi = i0 + lx, gj = j0 + ly;
  if (gi < nx && gj < ny) {
    const int r = (ly + 1) * R1X + lx + 1;
    TC acc[17];
#pragma unroll
    for (int p = 0; p < 17; ++p) acc[p] = TC(0);
    const int fxm = ly * (AX + 1) + lx, fym = ly * AX + lx;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const TC sg = g ? TC(1) : TC(-1);
      TC l[6];
      // x faces: this cell is the right state of face fxm, the left of fxm+1
#pragma unroll
      for (int v = 0; v < 6; ++v) l[v] = s_lx[((6 + v) * 2 + g) * NFX + fxm];
      add_point_mhd<TC>(acc, l, -hx, sg * oy);
#pragma unroll
      for (int v = 0; v < 6; ++v) l[v] = s_lx[(v * 2 + g) * NFX + fxm + 1];
      add_point_mhd<TC>(acc, l, hx, sg * oy);
      // y faces: the upper state of fym, the lower state of fym+AX
#pragma unroll
      for (int v = 0; v < 6; ++v) l[v] = s_ly[((6 + v) * 2 + g) * NFY + fym];
      add_point_mhd<TC>(acc, l, sg * ox, -hy);
#pragma unroll
      for (int v = 0; v < 6; ++v) l[v] = s_ly[(v * 2 + g) * NFY + fym + AX];
      add_point_mhd<TC>(acc, l, sg * ox, hy);
    }
    // volume points: the x-flux sums enter the x slopes (and a2), the y-flux sums
    // the y slopes (and a1), times 3/dx^2 and 3/dy^2
    TC yx[5], yy[5];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      yx[q] = c3x * s_y[(3 * q + 1) * R1 + r];
      yy[q] = c3y * s_y[(3 * q + 2) * R1 + r];
    }
    yx[4] = c3x * s_y[15 * R1 + r];
    yy[4] = c3y * s_y[14 * R1 + r];
#pragma unroll 1
    for (int qp = 0; qp < 4; ++qp) {
      const TC xq = (qp & 1) ? ox : -ox, yq = (qp & 2) ? oy : -oy;
      TC c[6], a[6];
      point(r, xq, yq, c);
      phys_flux2d_mhd_vjp<TC>(GD, c, yx, yy, a, err);
      add_point_mhd<TC>(acc, a, xq, yq);
    }
    const size_t gc = (size_t)gj * nx + gi;
#pragma unroll
    for (int p = 0; p < 17; ++p) {
      double o = A.a1 * A.x1[p * ncell + gc] + A.beta * Cvt<TC>::to_f64(acc[p]);
      if (A.x2) o += A.a2 * A.x2[p * ncell + gc];
      A.out[p * ncell + gc] = o;
    }
  }
  if (err) atomicOr(A.err, err);
}

// Interchange planes of the internal averages (rho, mx, my, E, b1, b2) and
// derivative coefficients (x and y slopes of the four Taylor variables, a1, a2,
// a3) of a planar MHD state.
__device__ __forceinline__ int mhd_avg_plane(int v) { return v < 4 ? 3 * v : 8 + v; }
__device__ __forceinline__ int mhd_slope_plane(int k) { return k < 8 ? 3 * (k >> 1) + 1 + (k & 1) : 6 + k; }

// U = Lambda(V) for planar MHD (internal layout): the forward limiter of the
// stage kernels, cell by cell from global memory.
template <class TC, class TS>
__global__ void limit2d_mhd_kernel(StateBuf<TS> V, StateBuf<TS> U, int nx, int ny, double dx,
                                   double dy, double gamma) {
  const long ncell = (long)nx * ny;
  Gas<TC> G;
  G.set(gamma);
  const TC hh[2] = {TC(0.5 * dx), TC(0.5 * dy)};
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)(c / nx);
    const long nb[4] = {(long)j * nx + wrap_index(i - 1, nx), (long)j * nx + wrap_index(i + 1, nx),
                        (long)wrap_index(j - 1, ny) * nx + i, (long)wrap_index(j + 1, ny) * nx + i};
    TC cc[6], W[6], Wn[4][6], s[11];
    unsigned err = 0;
#pragma unroll
    for (int v = 0; v < 6; ++v) cc[v] = Cvt<TC>::to_tc(V.c0[v * ncell + c]);
    prims2d<1, TC>(G, cc, W, err);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      TC cn[6];
#pragma unroll
      for (int v = 0; v < 6; ++v) cn[v] = Cvt<TC>::to_tc(V.c0[v * ncell + nb[k]]);
      prims2d<1, TC>(G, cn, Wn[k], err);
    }
#pragma unroll
    for (int k = 0; k < 11; ++k) s[k] = (TC)V.sl[k * ncell + c];
    limit_cell2d<1, TC>(G, hh, W, Wn, s);
#pragma unroll
    for (int v = 0; v < 6; ++v) U.c0[v * ncell + c] = V.c0[v * ncell + c];
#pragma unroll
    for (int k = 0; k < 11; ++k) U.sl[k * ncell + c] = (TS)s[k];
  }
}

// out = J_Lambda(V)^T nu for planar MHD (interchange layout): the forward limiter
// instantiated on dual numbers, six tangents a pass.  A cell's limited slopes
// depend on its own averages and slopes (three passes) and on its four
// neighbours' averages; its averages also enter its neighbours' limiters (one pass
// each).  Branches follow the values (the active branch's derivative).
template <class TC, class TS>
__global__ void limit_vjp2d_mhd_kernel(StateBuf<TS> V, const double* __restrict__ nu, double* out,
                                       int nx, int ny, double dx, double dy, double gamma) {
  typedef Dn<TC, 6> D;
  const long ncell = (long)nx * ny;
  Gas<D> GD;
  GD.set(gamma);
  const D hh[2] = {D(TC(0.5 * dx)), D(TC(0.5 * dy))};
  const int ofs[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncell;
       c += (long)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)(c / nx);
    auto at = [&](int di, int dj) {
      return (long)wrap_index(j + dj, ny) * nx + wrap_index(i + di, nx);
    };
    unsigned err = 0;
    // the limiter of cell e with tangents seeded by `seed` (which inputs, in
    // which order), contracted with e's slope adjoints: a[t] for t < nt
    auto pass = [&](long e, int ei, int ej, int kind, int first, int nt, TC* a) {
      D c0[6], s[11], cn[4][6], W[6], Wn[4][6];
#pragma unroll
      for (int v = 0; v < 6; ++v) c0[v] = D(Cvt<TC>::to_tc(V.c0[v * ncell + e]));
#pragma unroll
      for (int k = 0; k < 11; ++k) s[k] = D((TC)V.sl[k * ncell + e]);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const long q = at(ei + ofs[m][0], ej + ofs[m][1]);
#pragma unroll
        for (int v = 0; v < 6; ++v) cn[m][v] = D(Cvt<TC>::to_tc(V.c0[v * ncell + q]));
      }
      for (int t = 0; t < nt; ++t) {
        if (kind == 0) c0[first + t].d[t] = TC(1);       // own averages
        else if (kind == 1) s[first + t].d[t] = TC(1);   // own slopes
        else cn[kind - 2][first + t].d[t] = TC(1);       // neighbour kind-2's averages
      }
      prims2d<1, D>(GD, c0, W, err);
#pragma unroll
      for (int m = 0; m < 4; ++m) prims2d<1, D>(GD, cn[m], Wn[m], err);
      limit_cell2d<1, D>(GD, hh, W, Wn, s);
      for (int t = 0; t < nt; ++t) {
        TC x = TC(0);
#pragma unroll
        for (int k = 0; k < 11; ++k)
          x += Cvt<TC>::to_tc(nu[mhd_slope_plane(k) * ncell + e]) * s[k].d[t];
        a[t] = x;
      }
    };
    TC acc[17];
#pragma unroll
    for (int p = 0; p < 17; ++p) acc[p] = TC(0);
    // the averages pass through the limiter unchanged
#pragma unroll
    for (int v = 0; v < 6; ++v) acc[mhd_avg_plane(v)] = Cvt<TC>::to_tc(nu[mhd_avg_plane(v) * ncell + c]);
    TC a[6];
    // (a) this cell's own limiter: its averages, then its slopes in two passes
    pass(c, 0, 0, 0, 0, 6, a);
    for (int t = 0; t < 6; ++t) acc[mhd_avg_plane(t)] += a[t];
    pass(c, 0, 0, 1, 0, 6, a);
    for (int t = 0; t < 6; ++t) acc[mhd_slope_plane(t)] += a[t];
    pass(c, 0, 0, 1, 6, 5, a);
    for (int t = 0; t < 5; ++t) acc[mhd_slope_plane(6 + t)] += a[t];
    // (b) each neighbour e's limiter reads this cell's averages as its
    //     neighbour number k ^ 1 (left <-> right, down <-> up)
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      pass(at(ofs[k][0], ofs[k][1]), ofs[k][0], ofs[k][1], 2 + (k ^ 1), 0, 6, a);
      for (int t = 0; t < 6; ++t) acc[mhd_avg_plane(t)] += a[t];
    }
#pragma unroll
    for (int p = 0; p < 17; ++p) out[p * ncell + c] = Cvt<TC>::to_f64(acc[p]);
  }
}

__global__ void axpby_kernel(const double* __restrict__ a, double sa, const double* __restrict__ b,
                             double sb, double* __restrict__ o, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    o[i] = sa * a[i] + (b ? sb * b[i] : 0.0);
}

unsigned grid1d(long n) {
  long b = (n + 255) / 256;
  return (unsigned)(b > 152L * 32 ? 152L * 32 : (b < 1 ? 1 : b));
}

// ---------------------------------------------------------------------------
// work buffers: four internal states, three adjoint arrays, a control block and
// an error word; for the reverse sweep also the states of one segment and two
// adjoint arrays
// ---------------------------------------------------------------------------
struct Work {
  size_t ncell = 0;
  int fp32 = -1;
  int seg = 0;
  double* c0[4];
  void* sl[4];
  double* lam[3];
  double* segbuf;
  double* lamrun[2];
  Ctl* ctl;
  unsigned* err;
};

template <class TS>
StateBuf<TS> sb(const Work& w, int k) {
  StateBuf<TS> s;
  s.c0 = w.c0[k];
  s.sl = reinterpret_cast<TS*>(w.sl[k]);
  return s;
}

// Carve the work block starting at `base` (nullptr: only measure); returns the
// number of bytes the carved buffers span.
size_t carve_into(char* base, const AdjointCall& c, int seg, Work* w) {
  const size_t n = (size_t)c.nx * c.ny;
  const size_t ts = c.fp32 ? 4 : 8;
  const size_t nv = c.eq ? 6 : 4, ns = c.eq ? 11 : 8, np = c.eq ? 17 : 12;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* r = base ? base + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return r;
  };
  Work t;
  t.ncell = n;
  t.fp32 = c.fp32;
  t.seg = seg;
  for (int k = 0; k < 4; ++k) {
    t.c0[k] = (double*)take(n * nv * 8);
    t.sl[k] = take(n * ns * ts);
  }
  for (int k = 0; k < 3; ++k) t.lam[k] = (double*)take(n * np * 8);
  t.lamrun[0] = (double*)take(n * np * 8);
  t.lamrun[1] = (double*)take(n * np * 8);
  t.ctl = (Ctl*)take(sizeof(Ctl));
  t.err = (unsigned*)take(sizeof(unsigned));
  t.segbuf = (double*)take((size_t)seg * n * np * 8);
  if (w) *w = t;
  return off;
}

dg_status ensure_work(AdjointStore& S, const AdjointCall& c, int seg, std::string& msg) {
  const size_t need = carve_into(nullptr, c, seg, nullptr);
  if (S.work && S.work_bytes >= need && S.work_ncell == (long)c.nx * c.ny && S.work_fp32 == c.fp32)
    return DG_OK;
  cudaFree(S.work);
  S.work = nullptr;
  S.work_bytes = 0;
  if (cudaMalloc(&S.work, need) != cudaSuccess) {
    cudaGetLastError();
    msg = "adjoint work buffers: device allocation failed";
    return DG_ENOMEM;
  }
  S.work_bytes = need;
  S.work_ncell = (long)c.nx * c.ny;
  S.work_fp32 = c.fp32;
  return DG_OK;
}

// The carved buffers always lie inside the allocation made by ensure_work.
bool carve(const AdjointStore& S, const AdjointCall& c, int seg, Work* w) {
  return carve_into((char*)S.work, c, seg, w) <= S.work_bytes;
}

// The interchange planes of a 2D state: plane v*3 + k is average v (k = 0) or
// derivative coefficient v*2 + k - 1 of (rho, mx, my, E); planar MHD adds b1, b2
// (averages 4, 5) and a1, a2, a3 (coefficients 8, 9, 10).  Converted in one
// launch per state.
PlaneMap planes2d(int eq) {
  PlaneMap m{};
  m.nplanes = eq ? 17 : 12;
  for (int p = 0; p < 12; ++p) {
    const int v = p / 3, k = p % 3;
    m.kind[p] = k == 0 ? 0 : 1;
    m.idx[p] = k == 0 ? v : v * 2 + (k - 1);
  }
  if (eq) {
    const int kind[5] = {0, 0, 1, 1, 1}, idx[5] = {4, 5, 8, 9, 10};
    for (int q = 0; q < 5; ++q) {
      m.kind[12 + q] = kind[q];
      m.idx[12 + q] = idx[q];
    }
  }
  return m;
}

template <class TS>
cudaError_t to_internal(int eq, const double* src, StateBuf<TS> dst, long n, cudaStream_t st) {
  return launch_state_in<TS>(src, dst, planes2d(eq), n, st);
}

template <class TS>
cudaError_t to_interchange(int eq, StateBuf<TS> src, double* dst, long n, cudaStream_t st) {
  return launch_state_out<TS>(src, dst, planes2d(eq), n, st);
}

template <class TS>
Stage2DArgs<TS> stage_args(const AdjointCall& c, const Work& w, StateBuf<TS> in, StateBuf<TS> base,
                           StateBuf<TS> out, double dt) {
  Stage2DArgs<TS> a;
  a.nx = c.nx; a.ny = c.ny; a.ncell = (long)c.nx * c.ny;
  a.dx = c.dx; a.dy = c.dy;
  a.gamma = c.gamma; a.cfl = 0.3; a.dt_override = dt; a.limiter = c.limiter;
  a.gas.set(c.gamma);
  a.in = in; a.base = base; a.out = out;
  a.lim_sl = nullptr;
  a.ctl = w.ctl;
  return a;
}

template <class TC, class TS>
cudaError_t apply_rhs_vjp(const AdjointCall& c, const Work& w, StateBuf<TS> U, const double* y,
                          const double* x1, double a1, const double* x2, double a2, double beta,
                          double* out) {
  VjpArgs A;
  A.nx = c.nx; A.ny = c.ny; A.ncell = (long)c.nx * c.ny;
  A.dx = c.dx; A.dy = c.dy; A.gamma = c.gamma;
  A.y = y; A.x1 = x1; A.a1 = a1; A.x2 = x2; A.a2 = a2; A.beta = beta; A.out = out;
  A.err = w.err;
  if (c.eq) {
    constexpr int AX = VjpTileM<TC>::X, AY = VjpTileM<TC>::Y;
    dim3 grid((c.nx + AX - 1) / AX, (c.ny + AY - 1) / AY);
    rhs_vjp2d_mhd_kernel<TC, TS><<<grid, AX * AY, 0, c.stream>>>(U, A);
    return cudaGetLastError();
  }
  constexpr int AX = VjpTile<TC>::X, AY = VjpTile<TC>::Y;
  dim3 grid((c.nx + AX - 1) / AX, (c.ny + AY - 1) / AY);
  rhs_vjp2d_kernel<TC, TS><<<grid, AX * AY, 0, c.stream>>>(U, A);
  return cudaGetLastError();
}

// One reverse step given V^n (internal, buffer 0).  lam_next -> lam_prev.
template <class TC, class TS>
cudaError_t reverse_step(const AdjointCall& c, const Work& w, const double* lam_next,
                         double* lam_prev, double dt) {
  const long n = (long)c.nx * c.ny;
  StateBuf<TS> Vn = sb<TS>(w, 0), Un = sb<TS>(w, 1), V1 = sb<TS>(w, 2), U1 = sb<TS>(w, 3);
  cudaError_t e;
  // forward recompute of the stage states
  e = launch_stage2d(c.eq, 0, 1, stage_args<TS>(c, w, Vn, Vn, V1, dt), c.stream);
  if (e != cudaSuccess) return e;
  if (c.limiter && c.eq) {
    limit2d_mhd_kernel<TC, TS><<<grid1d(n), 256, 0, c.stream>>>(Vn, Un, c.nx, c.ny, c.dx, c.dy, c.gamma);
    limit2d_mhd_kernel<TC, TS><<<grid1d(n), 256, 0, c.stream>>>(V1, U1, c.nx, c.ny, c.dx, c.dy, c.gamma);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else if (c.limiter) {
    limit2d_kernel<TC, TS><<<grid1d(n), 256, 0, c.stream>>>(Vn, Un, c.nx, c.ny, c.dx, c.dy, c.gamma);
    limit2d_kernel<TC, TS><<<grid1d(n), 256, 0, c.stream>>>(V1, U1, c.nx, c.ny, c.dx, c.dy, c.gamma);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    Un = Vn;
    U1 = V1;
  }
  double* mu1 = w.lam[0];
  double* lam1 = w.lam[1];
  double* mu0 = w.lam[2];
  // mu1 = 1/2 lam + 1/2 dt J_L(U1)^T lam
  if ((e = apply_rhs_vjp<TC, TS>(c, w, U1, lam_next, lam_next, 0.5, nullptr, 0.0, 0.5 * dt,
                                 mu1)) != cudaSuccess)
    return e;
  // lam1 = J_Lambda(V1)^T mu1
  if (c.limiter && c.eq) {
    limit_vjp2d_mhd_kernel<TC, TS><<<grid1d(n), 128, 0, c.stream>>>(V1, mu1, lam1, c.nx, c.ny,
                                                                    c.dx, c.dy, c.gamma);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else if (c.limiter) {
    limit_vjp2d_kernel<TC, TS><<<grid1d(n), 128, 0, c.stream>>>(V1, mu1, lam1, c.nx, c.ny, c.dx,
                                                                c.dy, c.gamma);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    lam1 = mu1;
  }
  // mu0 = 1/2 lam + lam1 + dt J_L(Un)^T lam1
  double* dst = c.limiter ? mu0 : lam_prev;
  if ((e = apply_rhs_vjp<TC, TS>(c, w, Un, lam1, lam_next, 0.5, lam1, 1.0, dt, dst)) != cudaSuccess)
    return e;
  // lam^n = J_Lambda(V^n)^T mu0
  if (c.limiter && c.eq) {
    limit_vjp2d_mhd_kernel<TC, TS><<<grid1d(n), 128, 0, c.stream>>>(Vn, mu0, lam_prev, c.nx,
                                                                    c.ny, c.dx, c.dy, c.gamma);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else if (c.limiter) {
    limit_vjp2d_kernel<TC, TS><<<grid1d(n), 128, 0, c.stream>>>(Vn, mu0, lam_prev, c.nx, c.ny,
                                                                c.dx, c.dy, c.gamma);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

dg_status finish(const AdjointCall& c, const Work& w, std::string& msg) {
  unsigned h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, w.err, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    msg = std::string("adjoint: ") + cudaGetErrorString(e);
    return DG_ECUDA;
  }
  if (h) {
    char b[96];
    snprintf(b, sizeof(b), "adjoint: device error word 0x%x", h);
    msg = b;
    return DG_ENONPHYS;
  }
  return DG_OK;
}

template <class TC, class TS>
dg_status step_t(AdjointStore& S, const AdjointCall& c, const double* u_n, const double* lam_next,
                 double* lam_prev, double dt, std::string& msg) {
  dg_status s = ensure_work(S, c, 0, msg);
  if (s != DG_OK) return s;
  Work w;
  if (!carve(S, c, 0, &w)) {
    msg = "adjoint work buffers: size mismatch";
    return DG_ESTATE;
  }
  const long n = (long)c.nx * c.ny;
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.err, 0, sizeof(unsigned), c.stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), c.stream)) != cudaSuccess ||
      (e = to_internal<TS>(c.eq, u_n, sb<TS>(w, 0), n, c.stream)) != cudaSuccess ||
      (e = reverse_step<TC, TS>(c, w, lam_next, lam_prev, dt)) != cudaSuccess) {
    msg = std::string("adjoint step: ") + cudaGetErrorString(e);
    return DG_ECUDA;
  }
  return finish(c, w, msg);
}

template <class TC, class TS>
dg_status run_t(AdjointStore& S, const AdjointCall& c, int k, const double* lam_N, double* lam_0,
                std::string& msg) {
  dg_status s = ensure_work(S, c, k, msg);
  if (s != DG_OK) return s;
  Work w;
  if (!carve(S, c, k, &w)) {
    msg = "adjoint work buffers: size mismatch";
    return DG_ESTATE;
  }
  const long n = (long)c.nx * c.ny;
  const size_t plane = (size_t)n * (c.eq ? 17 : 12);
  std::vector<double> dts((size_t)S.nrec);
  cudaError_t e = cudaMemcpyAsync(dts.data(), S.dt_hist, S.nrec * sizeof(double),
                                  cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    msg = std::string("adjoint: ") + cudaGetErrorString(e);
    return DG_ECUDA;
  }
  if ((e = cudaMemsetAsync(w.err, 0, sizeof(unsigned), c.stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), c.stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(w.lamrun[0], lam_N, plane * 8, cudaMemcpyDeviceToDevice, c.stream)) !=
          cudaSuccess) {
    msg = std::string("adjoint: ") + cudaGetErrorString(e);
    return DG_ECUDA;
  }
  int cur = 0;
  const long long nseg = (S.nrec + k - 1) / k;
  for (long long sgi = nseg - 1; sgi >= 0; --sgi) {
    const long long n0 = sgi * k, n1 = std::min<long long>(S.nrec, n0 + k);
    // recompute V^{n0} .. V^{n1-1} from the checkpoint
    const double* ck = S.ckpt + (size_t)sgi * plane;
    if ((e = cudaMemcpyAsync(w.segbuf, ck, plane * 8, cudaMemcpyDeviceToDevice, c.stream)) !=
        cudaSuccess)
      break;
    if ((e = to_internal<TS>(c.eq, ck, sb<TS>(w, 0), n, c.stream)) != cudaSuccess) break;
    int a = 0;  // buffers 0 and 1 take turns as the step's input and output
    for (long long m = n0; m + 1 < n1; ++m) {
      const double dt = dts[(size_t)m];
      if ((e = launch_stage2d(c.eq, 0, 1, stage_args<TS>(c, w, sb<TS>(w, a), sb<TS>(w, a), sb<TS>(w, 2), dt),
                              c.stream)) != cudaSuccess)
        break;
      if ((e = launch_stage2d(c.eq, 0, 2, stage_args<TS>(c, w, sb<TS>(w, 2), sb<TS>(w, a), sb<TS>(w, 1 - a), dt),
                              c.stream)) != cudaSuccess)
        break;
      if ((e = to_interchange<TS>(c.eq, sb<TS>(w, 1 - a), w.segbuf + (size_t)(m + 1 - n0) * plane, n,
                                  c.stream)) != cudaSuccess)
        break;
      a = 1 - a;
    }
    if (e != cudaSuccess) break;
    // reverse through the segment
    for (long long m = n1 - 1; m >= n0; --m) {
      if ((e = to_internal<TS>(c.eq, w.segbuf + (size_t)(m - n0) * plane, sb<TS>(w, 0), n, c.stream)) !=
          cudaSuccess)
        break;
      double* dst = (m == 0) ? lam_0 : w.lamrun[cur ^ 1];
      if ((e = reverse_step<TC, TS>(c, w, w.lamrun[cur], dst, dts[(size_t)m])) != cudaSuccess) break;
      cur ^= 1;
    }
    if (e != cudaSuccess) break;
  }
  if (e != cudaSuccess) {
    msg = std::string("adjoint: ") + cudaGetErrorString(e);
    return DG_ECUDA;
  }
  return finish(c, w, msg);
}

}  // namespace

void adjoint_free(AdjointStore& s) {
  cudaFree(s.ckpt);
  cudaFree(s.dt_hist);
  cudaFree(s.work);
  const long long gen = s.generation;
  s = AdjointStore();
  s.generation = gen + 1;
}

void adjoint_reset(AdjointStore& s) {
  s.nrec = 0;
  s.generation++;
}

dg_status adjoint_reserve(AdjointStore& s, int nplanes, long ncell, int k, long long nsteps,
                          std::string& msg) {
  if (nsteps <= s.cap_steps && s.ncell == ncell && s.nplanes == nplanes) return DG_OK;
  long long cap = std::max<long long>(nsteps, 2 * s.cap_steps);
  const size_t plane = (size_t)nplanes * ncell;
  const size_t nck = (size_t)((cap + k - 1) / k + 1);
  double* ck = nullptr;
  double* dh = nullptr;
  if (cudaMalloc(&ck, nck * plane * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dh, (size_t)cap * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ck);
    msg = "adjoint checkpoint store: device allocation failed";
    return DG_ENOMEM;
  }
  if (s.nrec > 0 && s.ckpt && s.ncell == ncell && s.nplanes == nplanes) {
    const size_t old = (size_t)((s.nrec + k - 1) / k + 1);
    cudaMemcpy(ck, s.ckpt, std::min(old, nck) * plane * sizeof(double), cudaMemcpyDeviceToDevice);
    cudaMemcpy(dh, s.dt_hist, (size_t)s.nrec * sizeof(double), cudaMemcpyDeviceToDevice);
  } else {
    s.nrec = 0;
  }
  cudaFree(s.ckpt);
  cudaFree(s.dt_hist);
  s.ckpt = ck;
  s.dt_hist = dh;
  s.cap_steps = cap;
  s.ncell = ncell;
  s.nplanes = nplanes;
  return DG_OK;
}

dg_status adjoint_step(AdjointStore& s, const AdjointCall& c, const double* u_n,
                       const double* lam_next, double* lam_prev, double dt, std::string& msg) {
  return c.fp32 ? step_t<float, float>(s, c, u_n, lam_next, lam_prev, dt, msg)
                : step_t<double, double>(s, c, u_n, lam_next, lam_prev, dt, msg);
}

dg_status adjoint_run(AdjointStore& s, const AdjointCall& c, int nplanes, int k,
                      const double* lam_N, double* lam_0, std::string& msg) {
  (void)nplanes;
  return c.fp32 ? run_t<float, float>(s, c, k, lam_N, lam_0, msg)
                : run_t<double, double>(s, c, k, lam_N, lam_0, msg);
}
