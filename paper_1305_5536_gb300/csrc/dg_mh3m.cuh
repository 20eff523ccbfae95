// dg_mh3m.cuh -- one MUSCL-Hancock step (Sec. 2.4) of the 3D P1 DG scheme for ideal
// MHD with the 11-function divergence-free field basis of Sec. 2.2 (update of eq.
// `GalerkUpdate`), as one fused kernel: the step structure of dg_mh3d.cuh with
// the limiter, face solver and field right-hand side of dg_stage3m.cuh.
//
// One CTA owns a TX x TY x TZ tile.  Shared memory holds the centroid primitives
// (rho, v, p, B) of the tile plus a halo of 2 cells (the limiter's neighbour
// extrema; the space then takes the face fluxes), the predicted centroid values
// of the tile plus a halo of 1 cell, and the 23 derivative coefficients of the
// same box, replaced in place by the limited primitive gradients of (rho, v, p)
// (slots 0..14, g[v*3+d]) and the limited field coefficients a4..a11 (slots
// 15..22, as in dg_stage3m.cuh).  Steps:
//   1. primitives of the halo-2 box; coefficients of the halo-1 box;
//   2. on the halo-1 box: the limiter (Sec. 2.5: min/max with one factor for
//      the whole field, or the WENO-type one), the primitive gradients of the
//      limited polynomial by the product rule, and the predicted centroid
//      values W_c + dt/2 dW/dt from the primitive form of the equations
//        drho/dt = -v.grad rho - rho div v,
//        dv/dt   = -(v.grad) v - (grad p + grad(B^2/2) - (B.grad) B) / rho,
//        dp/dt   = -v.grad p - gamma p div v,
//        dB/dt   = (B.grad) v - (v.grad) B - B div v
//      (the terms in div B are left out: every cell's field is divergence free);
//   3. per cell: fluxes of the predicted state at the 8 volume Gauss points;
//   4. faces of one orientation at a time: HLLD with the averaged normal field
//      (Sec. 2.6) between the predicted states of both sides at NGF^2 points (1:
//      the face centroid; 4: the 2x2 Gauss points), gathered by both cells;
//   5. the update U^{n+1} = U^n + dt L of the limited coefficients (rebuilt from
//      the limited gradients by the product rule) and the Courant reduction of
//      U^{n+1} for the next step.
#pragma once

#include "dg_mh3d.cuh"
#include "dg_stage3m.cuh"

namespace dgk {

template <int TX, int TY, int TZ, int NGF, class TC>
__host__ __device__ constexpr size_t mh3m_smem_bytes() {
  constexpr size_t R2 = size_t(TX + 4) * (TY + 4) * (TZ + 4);
  constexpr size_t R1 = size_t(TX + 2) * (TY + 2) * (TZ + 2);
  constexpr size_t FS = size_t(8) * NGF * NGF * stage3d_face_max<TX, TY, TZ, TC>();
  return ((8 * R2 > FS ? 8 * R2 : FS) + 8 * R1 + 23 * R1) * sizeof(TC) +
         sizeof(int) * ((TX + 4) + (TY + 4) + (TZ + 4));
}

// Primitive gradients g[v*3+d] of (rho, v, p) from the conserved derivative
// coefficients s[0..14] at centroid primitives W, gB[i][d] = dB_i/dx_d:
//   dv = (dm - v drho)/rho,  dp = (gamma-1)(dE - v^2/2 drho - rho v.dv - B.dB).
template <class TC>
__device__ __forceinline__ void prim_grads3m(const Gas<TC>& G, const TC* W, const TC* s,
                                             const TC (*gB)[3], TC* g) {
  const TC rho = W[0], inv = TC(1) / rho;
  const TC v[3] = {W[1], W[2], W[3]};
  const TC v2h = TC(0.5) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    g[d] = s[d];
    TC vdv = TC(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      g[3 * (1 + i) + d] = (s[3 * (1 + i) + d] - v[i] * g[d]) * inv;
      vdv += v[i] * g[3 * (1 + i) + d];
    }
    const TC BdB = W[5] * gB[0][d] + W[6] * gB[1][d] + W[7] * gB[2][d];
    g[12 + d] = G.gm1 * (s[12 + d] - v2h * g[d] - rho * vdv - BdB);
  }
}

// The product rule back: conserved derivative coefficients s[0..14] from the
// primitive gradients g[] and the field gradients gB at centroid primitives W.
template <class TC>
__device__ __forceinline__ void mh_cons3m(const Gas<TC>& G, const TC* W, const TC* g,
                                          const TC (*gB)[3], TC* s) {
  const TC rho = W[0];
  const TC v[3] = {W[1], W[2], W[3]};
  const TC v2h = TC(0.5) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const TC r = g[d];
    TC vdv = TC(0);
    s[d] = r;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const TC u = g[3 * (1 + i) + d];
      s[3 * (1 + i) + d] = rho * u + v[i] * r;
      vdv += v[i] * u;
    }
    const TC BdB = W[5] * gB[0][d] + W[6] * gB[1][d] + W[7] * gB[2][d];
    s[12 + d] = g[12 + d] * G.inv_gm1 + v2h * r + rho * vdv + BdB;
  }
}

// dW/dt at the centroid from the primitive form above: W (rho, v, p, B), g[]
// the primitive gradients of (rho, v, p), gB[i][d] = dB_i/dx_d.
template <class TC>
__device__ __forceinline__ void mh_rates3m(const Gas<TC>& G, const TC* W, const TC* g,
                                           const TC (*gB)[3], TC* Wt) {
  const TC rho = W[0], inv = TC(1) / rho, p = W[4];
  const TC v[3] = {W[1], W[2], W[3]};
  const TC B[3] = {W[5], W[6], W[7]};
  const TC divv = g[3] + g[7] + g[11];
  Wt[0] = -(v[0] * g[0] + v[1] * g[1] + v[2] * g[2]) - rho * divv;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const TC* gv = g + 3 * (1 + i);
    // d/dx_i (B^2/2) - (B.grad) B_i
    const TC lor = B[0] * gB[0][i] + B[1] * gB[1][i] + B[2] * gB[2][i] -
                   (B[0] * gB[i][0] + B[1] * gB[i][1] + B[2] * gB[i][2]);
    Wt[1 + i] = -(v[0] * gv[0] + v[1] * gv[1] + v[2] * gv[2]) - (g[12 + i] + lor) * inv;
    Wt[5 + i] = (B[0] * gv[0] + B[1] * gv[1] + B[2] * gv[2]) -
                (v[0] * gB[i][0] + v[1] * gB[i][1] + v[2] * gB[i][2]) - B[i] * divv;
  }
  Wt[4] = -(v[0] * g[12] + v[1] * g[13] + v[2] * g[14]) - G.g * p * divv;
}

// Predicted primitive state of a cell at local point (x, y, z): wp[] its predicted
// centroid values, g[] its limited primitive gradients and field coefficients
// (both strided by `st`).
template <class TC>
__device__ __forceinline__ void mh_eval3m(const TC* wp, const TC* g, int st, TC x, TC y, TC z,
                                          TC* W) {
#pragma unroll
  for (int q = 0; q < 5; ++q)
    W[q] = wp[q * st] + g[(3 * q) * st] * x + g[(3 * q + 1) * st] * y + g[(3 * q + 2) * st] * z;
  const TC a4 = g[15 * st], a5 = g[16 * st], a6 = g[17 * st], a7 = g[18 * st];
  const TC a8 = g[19 * st], a9 = g[20 * st], a10 = g[21 * st], a11 = g[22 * st];
  W[5] = wp[5 * st] + (a10 + a11) * x + a4 * y + a5 * z;
  W[6] = wp[6 * st] + a6 * x - a10 * y + a7 * z;
  W[7] = wp[7 * st] + a8 * x + a9 * y - a11 * z;
}

// Physical flux along axis d of a primitive state (rho, v, p, B), in the
// component order of phys_flux3m.
template <class TC>
__device__ __forceinline__ void prim_flux3m(const Gas<TC>& G, const TC* W, int d, TC* F,
                                            unsigned& err) {
  const TC rho = W[0], p = W[4];
  if (!(rho > TC(0) && p > TC(0))) err |= ERR_NONPHYS;
  const TC v[3] = {W[1], W[2], W[3]};
  const TC B[3] = {W[5], W[6], W[7]};
  const TC b2h = TC(0.5) * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  const TC pT = p + b2h;
  const TC vd = d == 0 ? v[0] : (d == 1 ? v[1] : v[2]);
  const TC Bd = d == 0 ? B[0] : (d == 1 ? B[1] : B[2]);
  const TC vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
  const TC E = p * G.inv_gm1 + TC(0.5) * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) + b2h;
  F[0] = rho * vd;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    F[1 + i] = rho * v[i] * vd - B[i] * Bd + (i == d ? pT : TC(0));
    F[5 + i] = B[i] * vd - v[i] * Bd;
  }
  F[4] = (E + pT) * vd - Bd * vB;
}

template <class TC, class TS, int TX, int TY, int TZ, int NGF, bool WENO>
__global__ void __launch_bounds__(TX * TY * TZ) mh3m_kernel(const Stage3DArgs<TS> A) {
  griddep_launch_dependents();  // programmatic dependent launch: see griddep_wait()
  griddep_wait();
  constexpr int R2X = TX + 4, R2Y = TY + 4, R2Z = TZ + 4, R2 = R2X * R2Y * R2Z;
  constexpr int R1X = TX + 2, R1Y = TY + 2, R1Z = TZ + 2, R1 = R1X * R1Y * R1Z;
  constexpr int NT = TX * TY * TZ;
  constexpr int FMAX = stage3d_face_max<TX, TY, TZ, TC>();
  constexpr int NPT = NGF * NGF;
  constexpr int WS = 8 * R2 > 8 * NPT * FMAX ? 8 * R2 : 8 * NPT * FMAX;
  static_assert(NT % 32 == 0, "tile must be whole warps");
  static_assert(NGF == 1 || NGF == 2, "face rule: 1 or 2 points per face dimension");
  (void)R1Z;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* s_w = reinterpret_cast<TC*>(smem_raw);  // 8 x R2 primitives, then face fluxes
  TC* s_f = s_w;
  TC* s_wp = s_w + WS;                        // 8 x R1 predicted centroid values
  TC* s_g = s_wp + 8 * R1;                    // 23 x R1 coefficients -> limited gradients
  int* s_gx = reinterpret_cast<int*>(s_g + 23 * R1);
  int* s_gy = s_gx + R2X;
  int* s_gz = s_gy + R2Y;
  __shared__ double s_dt;
  __shared__ unsigned s_err;
  __shared__ double s_red[NT / 32];

  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * TZ;
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const size_t ncell = (size_t)A.ncell;
  const Gas<TC> G = gas_of<TC>(A.gas);
  unsigned err = 0;
  if (tid == 0) {
    s_err = 0;
    double dt = A.dt_override > 0.0 ? A.dt_override : A.ctl->dt_cur;
    if (!(dt > 0.0) || !(dt < 1e300)) err |= ERR_NONPHYS;
    s_dt = dt;
  }
  if (tid < R2X) s_gx[tid] = wrap_index(i0 - 2 + tid, nx);
  else if (tid < R2X + R2Y) s_gy[tid - R2X] = wrap_index(j0 - 2 + (tid - R2X), ny) * nx;
  else if (tid < R2X + R2Y + R2Z)
    s_gz[tid - R2X - R2Y] = wrap_index(k0 - 2 + (tid - R2X - R2Y), nz) * nx * ny;
  __syncthreads();
  const double dt = s_dt;
  const TC dtc = Cvt<TC>::to_tc(dt);
  const TC hdt = TC(0.5) * dtc;

  // ---- 1. primitives of the halo-2 box; coefficients of the halo-1 box
  stage3d_issue<8, 23, TX, TY, TZ>(A.in, ncell, s_gx, s_gy, s_gz, s_g);
  for (int r = tid; r < R2; r += NT) {
    int rz = r / (R2X * R2Y), rr = r - rz * (R2X * R2Y);
    int ry = rr / R2X, rx = rr - ry * R2X;
    size_t g = (size_t)s_gz[rz] + s_gy[ry] + s_gx[rx];
    TC c[8], W[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) c[v] = Cvt<TC>::to_tc(__ldg(&A.in.c0[v * ncell + g]));
    prims3m<TC>(G, c, W, err);
#pragma unroll
    for (int q = 0; q < 8; ++q) s_w[q * R2 + r] = W[q];
  }
  cp_async_wait_all();
  __syncthreads();

  const TC dx = Cvt<TC>::to_tc(A.dx), dy = Cvt<TC>::to_tc(A.dy), dz = Cvt<TC>::to_tc(A.dz);
  const TC hh[3] = {TC(0.5) * dx, TC(0.5) * dy, TC(0.5) * dz};
  const TC oo[3] = {dx * TC(0.28867513459481288225), dy * TC(0.28867513459481288225),
                    dz * TC(0.28867513459481288225)};
  const TC hd[3] = {dx, dy, dz};

  // ---- 2. limiter, primitive gradients, half-step prediction on the halo-1 box
  for (int r1 = tid; r1 < R1; r1 += NT) {
    int rz = r1 / (R1X * R1Y), rr = r1 - rz * (R1X * R1Y);
    int ry = rr / R1X, rx = rr - ry * R1X;
    int r2 = ((rz + 1) * R2Y + (ry + 1)) * R2X + (rx + 1);
    TC W[8], s[23];
#pragma unroll
    for (int q = 0; q < 8; ++q) W[q] = s_w[q * R2 + r2];
#pragma unroll
    for (int k = 0; k < 23; ++k) s[k] = s_g[k * R1 + r1];
    if (A.limiter) {
      TC Wn[6][8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        Wn[0][q] = s_w[q * R2 + r2 - 1];
        Wn[1][q] = s_w[q * R2 + r2 + 1];
        Wn[2][q] = s_w[q * R2 + r2 - R2X];
        Wn[3][q] = s_w[q * R2 + r2 + R2X];
        Wn[4][q] = s_w[q * R2 + r2 - R2X * R2Y];
        Wn[5][q] = s_w[q * R2 + r2 + R2X * R2Y];
      }
      limit3m<TC, WENO>(G, hh, W, Wn, s);
    }
    TC gB[3][3], g[15], Wt[8];
    field_grad3m<TC>(s, gB);
    prim_grads3m<TC>(G, W, s, gB, g);
    mh_rates3m<TC>(G, W, g, gB, Wt);
#pragma unroll
    for (int k = 0; k < 15; ++k) s_g[k * R1 + r1] = g[k];
#pragma unroll
    for (int k = 15; k < 23; ++k) s_g[k * R1 + r1] = s[k];
#pragma unroll
    for (int q = 0; q < 8; ++q) s_wp[q * R1 + r1] = W[q] + hdt * Wt[q];
  }
  __syncthreads();  // the primitives are dead from here: their space takes the fluxes

  // ---- 3. per cell: volume integral of the predicted state's fluxes
  const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
  const int r1c = ((lz + 1) * R1Y + (ly + 1)) * R1X + (lx + 1);
  TC rc0[8], rs[24];
#pragma unroll
  for (int v = 0; v < 8; ++v) rc0[v] = TC(0);
#pragma unroll
  for (int k = 0; k < 24; ++k) rs[k] = TC(0);
#pragma unroll 1
  for (int qp = 0; qp < 8; ++qp) {
    TC W[8];
    mh_eval3m<TC>(s_wp + r1c, s_g + r1c, R1, (qp & 1) ? oo[0] : -oo[0], (qp & 2) ? oo[1] : -oo[1],
                  (qp & 4) ? oo[2] : -oo[2], W);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      TC F[8];
      prim_flux3m<TC>(G, W, d, F, err);
      const TC w = TC(1.5) / (hd[d] * hd[d]);
#pragma unroll
      for (int v = 0; v < 8; ++v) rs[3 * v + d] += w * F[v];
    }
  }

  // ---- 4. faces, one orientation at a time (rolled loop: one copy of the solver)
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    const int FX = TX + (d == 0), FY = TY + (d == 1), FZ = TZ + (d == 2);
    const int NFACE = FX * FY * FZ;
    static_assert((TX + 1) * (TY + 1) * (TZ + 1) < 16384 && (TX + 1) * (TY + 1) <= 1024,
                  "face indices within the exact range of div_by_magic");
    const unsigned mXY = div_magic(FX * FY), mX = div_magic(FX);
    const int step = d == 0 ? 1 : (d == 1 ? R1X : R1X * R1Y);
    const TC hn = d == 0 ? hh[0] : (d == 1 ? hh[1] : hh[2]);
    const TC o1 = d == 0 ? oo[1] : oo[0], o2 = d == 2 ? oo[1] : oo[2];
    for (int e = tid; e < NPT * NFACE; e += NT) {
      const int f = NPT == 4 ? (e >> 2) : e, g = NPT == 4 ? (e & 3) : 0;
      const int fz = div_by_magic(f, mXY), fr = f - fz * (FX * FY);
      const int fy = div_by_magic(fr, mX), fx = fr - fy * FX;
      // + side cell: halo-1 coordinates (fx+1, fy+1, fz+1); - side one step back
      const int r1r = ((fz + 1) * R1Y + (fy + 1)) * R1X + (fx + 1);
      const int r1l = r1r - step;
      const TC a = NPT == 4 ? ((g & 2) ? o1 : -o1) : TC(0);
      const TC b = NPT == 4 ? ((g & 1) ? o2 : -o2) : TC(0);
      const TC xl = d == 0 ? hn : a, xr = d == 0 ? -hn : a;
      const TC yl = d == 1 ? hn : (d == 0 ? a : b), yr = d == 1 ? -hn : (d == 0 ? a : b);
      const TC zl = d == 2 ? hn : b, zr = d == 2 ? -hn : b;
      TC WL[8], WR[8], F[8];
      mh_eval3m<TC>(s_wp + r1l, s_g + r1l, R1, xl, yl, zl, WL);
      mh_eval3m<TC>(s_wp + r1r, s_g + r1r, R1, xr, yr, zr, WR);
      face_flux_prim3m<TC>(G, d, WL, WR, F, err);
#pragma unroll
      for (int v = 0; v < 8; ++v) s_f[(v * FMAX + f) * NPT + g] = F[v];
    }
    __syncthreads();
    {
      const int fm = (lz * FY + ly) * FX + lx;
      const int fp = fm + (d == 0 ? 1 : (d == 1 ? FX : FX * FY));
      const TC* s_fb = s_f + 5 * FMAX * NPT;  // the three field components
      if (NPT == 4) {
        if (d == 0) {
          gather3d<0, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
          gather3d<0, TC, 3>(s_fb, FMAX, fm, fp, hd, rc0 + 5, rs + 15);
        } else if (d == 1) {
          gather3d<1, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
          gather3d<1, TC, 3>(s_fb, FMAX, fm, fp, hd, rc0 + 5, rs + 15);
        } else {
          gather3d<2, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
          gather3d<2, TC, 3>(s_fb, FMAX, fm, fp, hd, rc0 + 5, rs + 15);
        }
      } else {
        if (d == 0) {
          gather3d_centroid<0, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
          gather3d_centroid<0, TC, 3>(s_fb, FMAX, fm, fp, hd, rc0 + 5, rs + 15);
        } else if (d == 1) {
          gather3d_centroid<1, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
          gather3d_centroid<1, TC, 3>(s_fb, FMAX, fm, fp, hd, rc0 + 5, rs + 15);
        } else {
          gather3d_centroid<2, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
          gather3d_centroid<2, TC, 3>(s_fb, FMAX, fm, fp, hd, rc0 + 5, rs + 15);
        }
      }
    }
    __syncthreads();
  }
  TC rsl[23];
#pragma unroll
  for (int k = 0; k < 15; ++k) rsl[k] = rs[k];
  field_rhs3m<TC>(rs, hd, rsl + 15);

  // ---- 5. update of the limited coefficients, Courant speed of the new state
  const int gi = i0 + lx, gj = j0 + ly, gk = k0 + lz;
  const bool owner = gi < nx && gj < ny && gk < nz;
  const size_t gc = (size_t)s_gz[lz + 2] + s_gy[ly + 2] + s_gx[lx + 2];
  TC sn[23];
  if (A.limiter) {
    TC c[8], W[8], g[15], gB[3][3];
#pragma unroll
    for (int v = 0; v < 8; ++v) c[v] = Cvt<TC>::to_tc(A.in.c0[v * ncell + gc]);
    prims3m<TC>(G, c, W, err);
#pragma unroll
    for (int k = 0; k < 15; ++k) g[k] = s_g[k * R1 + r1c];
#pragma unroll
    for (int k = 15; k < 23; ++k) sn[k] = s_g[k * R1 + r1c];
    field_grad3m<TC>(sn, gB);
    mh_cons3m<TC>(G, W, g, gB, sn);
  } else {
#pragma unroll
    for (int k = 0; k < 23; ++k) sn[k] = (TC)A.in.sl[k * ncell + gc];
  }
  double o0[8];
  TC os[23];
#pragma unroll
  for (int v = 0; v < 8; ++v) o0[v] = fma(dt, Cvt<TC>::to_f64(rc0[v]), A.in.c0[v * ncell + gc]);
#pragma unroll
  for (int k = 0; k < 23; ++k) os[k] = sn[k] + dtc * rsl[k];
  if (owner) {
#pragma unroll
    for (int v = 0; v < 8; ++v) A.out.c0[v * ncell + gc] = o0[v];
#pragma unroll
    for (int k = 0; k < 23; ++k) A.out.sl[k * ncell + gc] = (TS)os[k];
  }

  TC sp = TC(0);
  if (owner) {
    TC c[8], W[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) c[v] = Cvt<TC>::to_tc(o0[v]);
    prims3m<TC>(G, c, W, err);
    const TC b2 = W[5] * W[5] + W[6] * W[6] + W[7] * W[7];
    sp = (fabs(W[1]) + fast_speed(G, W[0], W[4], b2, W[5])) / dx +
         (fabs(W[2]) + fast_speed(G, W[0], W[4], b2, W[6])) / dy +
         (fabs(W[3]) + fast_speed(G, W[0], W[4], b2, W[7])) / dz;
    if (!courant_ok(sp, W[0], W[4])) { err |= ERR_NONPHYS; sp = TC(0); }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    TC t = __shfl_xor_sync(0xffffffffu, sp, o);
    sp = t > sp ? t : sp;
  }
  if ((tid & 31) == 0) s_red[tid >> 5] = Cvt<TC>::to_f64(sp);
  if (err) atomicOr(&s_err, err);
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < NT / 32; ++w) m = s_red[w] > m ? s_red[w] : m;
    Ctl* ctl = A.ctl;
    atomicMax(&ctl->vmax_next, (unsigned long long)__double_as_longlong(m));
    if (s_err) atomicOr(&ctl->err, s_err);
    __threadfence();
    unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    unsigned tk = atomicAdd(&ctl->ticket, 1u);
    if (tk == nblk - 1) {
      __threadfence();
      double vm = __longlong_as_double((long long)atomicAdd(&ctl->vmax_next, 0ull));
      ctl->vmax_cur = vm;
      ctl->dt_cur = A.cfl / vm;
      ctl->vmax_next = 0ull;
      ctl->t += dt;
      ctl->dt_last = dt;
      if (ctl->dt_hist && ctl->step < ctl->hist_cap) ctl->dt_hist[ctl->step] = dt;
      if (ctl->err && ctl->err_step < 0) ctl->err_step = ctl->step;
      ctl->step += 1;
      if (!(vm > 0.0)) ctl->err |= ERR_NONPHYS;
      __threadfence();
      ctl->ticket = 0u;
    }
  }
}

}  // namespace dgk
