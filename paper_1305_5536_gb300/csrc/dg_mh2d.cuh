// dg_mh2d.cuh -- one MUSCL-Hancock step (Sec. 2.4) of the 2D P1 DG scheme (Euler
// or planar ideal MHD) as a single fused kernel.
//
// The tile is staged as for the Runge-Kutta stages (dg_stage2d.cuh: averages with
// a halo of 2, derivative coefficients with a halo of 1).  Then
//   1. centroid primitives W_c of every staged cell;
//   2. for the tile and its 1-cell ring: primitive gradients by the product rule,
//      the min/max limiter on them (Sec. 2.5; the limited conserved coefficients
//      are kept for the update), the time derivative dW/dt at the centroid from
//      the primitive form of the equations, and the predicted centroid value
//      W_p = W_c + dt/2 dW/dt;
//   3. every face once: the predicted primitive values W_p + grad W . (x - x_c) of
//      both sides at NGF points (1: the face centroid, eq. `GalerkUpdate`; 2: the
//      Gauss pair), the Riemann flux (exact solver, or HLLD with the averaged
//      normal field of Sec. 2.6);
//   4. per cell: the 2x2 Gauss volume integral of the fluxes of the predicted
//      state, the face moments, the diagonal mass matrix, and one update of the
//      limited coefficients, U^{n+1} = U^n + dt L; the Courant speed of U^{n+1} is
//      reduced for the next step as at the end of a Runge-Kutta step.
// The right-hand side is that of dg_stage2d.cuh with, for NGF = 1, S = 2 F and
// D = 0 for every face (one flux at the centroid, weight the face length).
//
// Primitive form (terms proportional to div B dropped: every cell's field is
// divergence free and the limiter keeps it so), W = (rho, vx, vy, p[, Bx, By]):
//   drho/dt = -v.grad rho - rho div v
//   dv/dt   = -(v.grad) v - (grad p + grad(B^2/2) - (B.grad) B) / rho
//   dp/dt   = -v.grad p - gamma p div v
//   dB/dt   = (B.grad) v - (v.grad) B - B div v
// with dBx/dx = a3, dBx/dy = a1, dBy/dx = a2, dBy/dy = -a3.
#pragma once

#include "dg_stage2d.cuh"

namespace dgk {

// Shared-memory layout: the staged averages [NV][R2] and coefficients [NS][R1]
// (limited in place), a region holding the centroid primitives [NP][R2] and then
// the face fluxes [NF][NFX*NGF], [NF][NFY*NGF], the predicted centroid values
// [NP][R1] and the limited primitive gradients [NS][R1].
template <int EQ, int TX, int TY, int NGF>
struct MhTile2D {
  using T = Tile2D<EQ, TX, TY>;
  static constexpr int NV = T::NV, NS = T::NS, NP = T::NP, NF = T::NF;
  static constexpr int R2 = T::R2, R1 = T::R1, NFX = T::NFX, NFY = T::NFY;
  static constexpr int FSZ = NF * NGF * (NFX + NFY);
  static constexpr int WSZ = NP * R2 > FSZ ? NP * R2 : FSZ;
  static constexpr int ELEMS = NV * R2 + NS * R1 + WSZ + NP * R1 + NS * R1;
};

template <int EQ, int TX, int TY, int NGF, class TC>
__host__ __device__ constexpr size_t mh2d_smem_bytes() {
  using T = Tile2D<EQ, TX, TY>;
  return size_t(MhTile2D<EQ, TX, TY, NGF>::ELEMS) * sizeof(TC) + sizeof(int) * (T::R2X + T::R2Y);
}

template <class TC>
struct MhMem2D {
  TileMem<TC> m;  // c0, sl, w, gx, gy as for the Runge-Kutta stages
  TC* wp;         // predicted centroid primitives [NP][R1]
  TC* gw;         // limited primitive gradients [NS][R1]
};

template <int EQ, int TX, int TY, int NGF, class TC>
__device__ __forceinline__ MhMem2D<TC> mh2d_mem(unsigned char* base) {
  using T = Tile2D<EQ, TX, TY>;
  using M = MhTile2D<EQ, TX, TY, NGF>;
  MhMem2D<TC> r;
  r.m.c0 = reinterpret_cast<TC*>(base);
  r.m.sl = r.m.c0 + T::NV * T::R2;
  r.m.w = r.m.sl + T::NS * T::R1;
  r.wp = r.m.w + M::WSZ;
  r.gw = r.wp + T::NP * T::R1;
  r.m.gx = reinterpret_cast<int*>(r.gw + T::NS * T::R1);
  r.m.gy = r.m.gx + T::R2X;
  return r;
}

// Primitive gradients g[] of one cell (slot order of the derivative coefficients:
// (rho, vx, vy, p) x (d/dx, d/dy), then a1, a2, a3) from its conserved
// coefficients s[] at centroid primitives W; with limiter 1 the min/max limiter
// (Sec. 2.5) scales them and s[] receives the limited conserved coefficients
// (the same arithmetic as limit_cell2d), with limiter 2 the WENO-type limiter
// does (dg_weno.cuh).  Wn: the 4 face neighbours' primitives.  WENO selects the
// WENO-type limiter at compile time: as a run-time branch its code, even called
// out of line, raises the register allocation of the min/max kernels by a fifth.
template <int EQ, class TC, bool WENO>
__device__ __forceinline__ void mh_grads2d(const Gas<TC>& G, const TC* hh, const TC* W,
                                           const TC (*Wn)[Tr2<EQ>::NP], int limiter, TC* s,
                                           TC* g) {
  constexpr int NP = Tr2<EQ>::NP;
  if constexpr (WENO) {
    weno_cell2d<EQ, TC>(G, hh, W, Wn, s, g);
    return;
  }
  const bool limit = limiter != 0;
  const TC rho = W[0], vx = W[1], vy = W[2];
  const TC inv = TC(1) / rho;
  TC gr[2], gvx[2], gvy[2], gp[2], gbx[2], gby[2];
  if (EQ == 1) {
    gbx[0] = s[10]; gbx[1] = s[8];
    gby[0] = s[9]; gby[1] = -s[10];
  }
  const TC v2h = TC(0.5) * (vx * vx + vy * vy);
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    gr[d] = s[d];
    gvx[d] = (s[2 + d] - vx * gr[d]) * inv;
    gvy[d] = (s[4 + d] - vy * gr[d]) * inv;
    TC BdB = TC(0);
    if (EQ == 1) BdB = W[4] * gbx[d] + W[5] * gby[d];
    gp[d] = G.gm1 * (s[6 + d] - v2h * gr[d] - rho * (vx * gvx[d] + vy * gvy[d]) - BdB);
  }
  TC ar = TC(1), avx = TC(1), avy = TC(1), ap = TC(1), aB = TC(1);
  if (limit) {
    TC hi[NP], lo[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      TC a = W[q], b = W[q];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        a = Wn[k][q] > a ? Wn[k][q] : a;
        b = Wn[k][q] < b ? Wn[k][q] : b;
      }
      hi[q] = a;
      lo[q] = b;
    }
    ar = limiter_alpha<TC, 2>(W[0], hi[0], lo[0], gr, hh);
    avx = limiter_alpha<TC, 2>(W[1], hi[1], lo[1], gvx, hh);
    avy = limiter_alpha<TC, 2>(W[2], hi[2], lo[2], gvy, hh);
    ap = limiter_alpha<TC, 2>(W[3], hi[3], lo[3], gp, hh);
    if (EQ == 1) {
      TC abx = limiter_alpha<TC, 2>(W[4], hi[4], lo[4], gbx, hh);
      TC aby = limiter_alpha<TC, 2>(W[5], hi[5], lo[5], gby, hh);
      aB = abx < aby ? abx : aby;
    }
  }
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    TC r = ar * gr[d], ux = avx * gvx[d], uy = avy * gvy[d], pp = ap * gp[d];
    g[d] = r;
    g[2 + d] = ux;
    g[4 + d] = uy;
    g[6 + d] = pp;
    if (limit) {
      TC BdB = TC(0);
      if (EQ == 1) BdB = aB * (W[4] * gbx[d] + W[5] * gby[d]);
      s[d] = r;
      s[2 + d] = rho * ux + vx * r;
      s[4 + d] = rho * uy + vy * r;
      s[6 + d] = pp * G.inv_gm1 + v2h * r + rho * (vx * ux + vy * uy) + BdB;
    }
  }
  if (EQ == 1) {
    if (limit) { s[8] *= aB; s[9] *= aB; s[10] *= aB; }
    g[8] = s[8]; g[9] = s[9]; g[10] = s[10];
  }
}

// Time derivative of the centroid primitives W from the primitive form above.
template <int EQ, class TC>
__device__ __forceinline__ void mh_rates2d(const Gas<TC>& G, const TC* W, const TC* g, TC* Wt) {
  const TC rho = W[0], vx = W[1], vy = W[2], p = W[3];
  const TC inv = TC(1) / rho;
  const TC divv = g[2] + g[5];
  Wt[0] = -(vx * g[0] + vy * g[1]) - rho * divv;
  Wt[3] = -(vx * g[6] + vy * g[7]) - G.g * p * divv;
  if (EQ == 0) {
    Wt[1] = -(vx * g[2] + vy * g[3]) - g[6] * inv;
    Wt[2] = -(vx * g[4] + vy * g[5]) - g[7] * inv;
  } else {
    const TC bx = W[4], by = W[5], a1 = g[8], a2 = g[9], a3 = g[10];
    Wt[1] = -(vx * g[2] + vy * g[3]) - (g[6] + by * (a2 - a1)) * inv;
    Wt[2] = -(vx * g[4] + vy * g[5]) - (g[7] + bx * (a1 - a2)) * inv;
    Wt[4] = bx * g[2] + by * g[3] - (vx * a3 + vy * a1) - bx * divv;
    Wt[5] = bx * g[4] + by * g[5] - (vx * a2 - vy * a3) - by * divv;
  }
}

// Predicted primitive state at local point (x, y) of a cell: wp[] its predicted
// centroid values, g[] its limited primitive gradients (both strided by `st`).
template <int EQ, class TC>
__device__ __forceinline__ void mh_eval2d(const TC* wp, const TC* g, int st, TC x, TC y, TC* W) {
#pragma unroll
  for (int q = 0; q < 4; ++q) W[q] = wp[q * st] + g[(2 * q) * st] * x + g[(2 * q + 1) * st] * y;
  if (EQ == 1) {
    const TC a1 = g[8 * st], a2 = g[9 * st], a3 = g[10 * st];
    W[4] = wp[4 * st] + a3 * x + a1 * y;
    W[5] = wp[5 * st] + a2 * x - a3 * y;
  }
}

// Physical fluxes along x and y of a primitive state, in face-flux component
// order (rho, mx, my, E[, transverse field: By for x, Bx for y]).
template <int EQ, class TC>
__device__ __forceinline__ void prim_flux2d(const Gas<TC>& G, const TC* W, TC* Fx, TC* Fy,
                                            unsigned& err) {
  const TC rho = W[0], vx = W[1], vy = W[2], p = W[3];
  if (!(rho > TC(0) && p > TC(0))) err |= ERR_NONPHYS;
  TC bx = TC(0), by = TC(0), b2h = TC(0);
  if (EQ == 1) { bx = W[4]; by = W[5]; b2h = TC(0.5) * (bx * bx + by * by); }
  const TC mx = rho * vx, my = rho * vy;
  const TC pT = p + b2h;
  const TC e = p * G.inv_gm1 + TC(0.5) * (mx * vx + my * vy) + b2h + pT;
  Fx[0] = mx;
  Fy[0] = my;
  if (EQ == 0) {
    Fx[1] = mx * vx + p; Fx[2] = my * vx; Fx[3] = e * vx;
    Fy[1] = mx * vy; Fy[2] = my * vy + p; Fy[3] = e * vy;
  } else {
    const TC vB = vx * bx + vy * by;
    Fx[1] = mx * vx + pT - bx * bx; Fx[2] = my * vx - bx * by; Fx[3] = e * vx - bx * vB;
    Fx[4] = by * vx - vy * bx;
    Fy[1] = mx * vy - bx * by; Fy[2] = my * vy + pT - by * by; Fy[3] = e * vy - by * vB;
    Fy[4] = bx * vy - vx * by;
  }
}

// Riemann flux along axis `dir` between primitive states WL (left/lower) and WR.
template <int EQ, class TC>
__device__ __forceinline__ void face_flux_prim2d(const Gas<TC>& G, int dir, const TC* WL,
                                                 const TC* WR, TC* F, unsigned& err) {
  // normal and transverse components picked with selects: one inlined solver
  const bool xd = dir == 0;
  const TC unl = xd ? WL[1] : WL[2], utl = xd ? WL[2] : WL[1];
  const TC unr = xd ? WR[1] : WR[2], utr = xd ? WR[2] : WR[1];
  TC Ff[5];
  if (EQ == 0) {
    exact_flux<TC, 1>(G, WL[0], unl, WL[3], &utl, WR[0], unr, WR[3], &utr, Ff, err);
  } else {
    const TC bn = TC(0.5) * (xd ? WL[4] + WR[4] : WL[5] + WR[5]);
    hlld_flux<TC>(G, WL[0], unl, utl, WL[3], xd ? WL[5] : WL[4], WR[0], unr, utr, WR[3],
                  xd ? WR[5] : WR[4], bn, Ff, err);
    F[4] = Ff[4];
  }
  F[0] = Ff[0];
  F[3] = Ff[3];
  if (dir == 0) { F[1] = Ff[1]; F[2] = Ff[2]; }
  else { F[1] = Ff[2]; F[2] = Ff[1]; }
}

template <int EQ, class TC, class TS, int TX, int TY, int NGF, bool WENO>
__device__ __forceinline__ void mh2d_compute(const Stage2DArgs<TS>& A, int i0, int j0,
                                             unsigned nblk, const MhMem2D<TC>& MM,
                                             TileScalars<TX * TY>& S) {
  using Tr = Tr2<EQ>;
  constexpr int NV = Tr::NV, NS = Tr::NS, NP = Tr::NP, NF = Tr::NF;
  constexpr int R2X = TX + 4, R2Y = TY + 4, R2 = R2X * R2Y;
  constexpr int R1X = TX + 2, R1Y = TY + 2, R1 = R1X * R1Y;
  constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
  constexpr int NT = TX * TY;
  static_assert(NT % 32 == 0, "tile must be whole warps");
  static_assert(NGF == 1 || NGF == 2, "face rule: 1 or 2 points");
  (void)R2Y;
  (void)R1Y;
  TC* s_c0 = MM.m.c0;
  TC* s_w = MM.m.w;
  TC* s_sl = MM.m.sl;
  TC* s_wp = MM.wp;
  TC* s_g = MM.gw;
  TC* s_fx = MM.m.w;
  TC* s_fy = MM.m.w + NF * NGF * NFX;
  const int* s_gx = MM.m.gx;
  const int* s_gy = MM.m.gy;

  const int tid = threadIdx.x;
  const int nx = A.nx, ny = A.ny;
  const size_t ncell = (size_t)A.ncell;
  const Gas<TC> G = gas_of<TC>(A.gas);
  unsigned err = 0;
  const double dt = S.dt;
  const TC dtc = Cvt<TC>::to_tc(dt);
  const TC hdt = TC(0.5) * dtc;

  // ---- 1. centroid primitives of every staged cell
  for (int r = tid; r < R2; r += NT) {
    TC c[NV], W[NP];
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = s_c0[v * R2 + r];
    prims2d<EQ, TC>(G, c, W, err);
#pragma unroll
    for (int q = 0; q < NP; ++q) s_w[q * R2 + r] = W[q];
  }
  __syncthreads();

  const TC dx = Cvt<TC>::to_tc(A.dx), dy = Cvt<TC>::to_tc(A.dy);
  TC hh[2] = {TC(0.5) * dx, TC(0.5) * dy};

  // ---- 2. gradients, limiter and half-step prediction on the tile and its ring
  for (int r1 = tid; r1 < R1; r1 += NT) {
    int ry = r1 / R1X, rx = r1 - ry * R1X;
    int r2 = (ry + 1) * R2X + (rx + 1);
    TC W[NP], Wn[4][NP], s[NS], g[NS], Wt[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      W[q] = s_w[q * R2 + r2];
      Wn[0][q] = s_w[q * R2 + r2 - 1];
      Wn[1][q] = s_w[q * R2 + r2 + 1];
      Wn[2][q] = s_w[q * R2 + r2 - R2X];
      Wn[3][q] = s_w[q * R2 + r2 + R2X];
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) s[k] = s_sl[k * R1 + r1];
    mh_grads2d<EQ, TC, WENO>(G, hh, W, Wn, A.limiter, s, g);
    mh_rates2d<EQ, TC>(G, W, g, Wt);
#pragma unroll
    for (int k = 0; k < NS; ++k) { s_sl[k * R1 + r1] = s[k]; s_g[k * R1 + r1] = g[k]; }
#pragma unroll
    for (int q = 0; q < NP; ++q) s_wp[q * R1 + r1] = W[q] + hdt * Wt[q];
  }
  __syncthreads();  // the primitives are dead from here: their space takes the fluxes

  // ---- 3. faces: Riemann fluxes of the predicted states, each face once
  const TC ox = dx * TC(0.28867513459481288225), oy = dy * TC(0.28867513459481288225);
  for (int e = tid; e < NGF * (NFX + NFY); e += NT) {
    const bool xf = e < NGF * NFX;
    const int ee = xf ? e : e - NGF * NFX;
    const int f = NGF == 2 ? (ee >> 1) : ee;
    const int gp = NGF == 2 ? (ee & 1) : 0;
    int r1l, r1r;
    TC xl, yl, xr, yr;
    if (xf) {
      int fy = f / (TX + 1), fx = f - fy * (TX + 1);
      r1l = (fy + 1) * R1X + fx;
      r1r = r1l + 1;
      TC t = NGF == 2 ? (gp ? oy : -oy) : TC(0);
      xl = hh[0]; xr = -hh[0]; yl = t; yr = t;
    } else {
      int fy = f / TX, fx = f - fy * TX;
      r1l = fy * R1X + fx + 1;
      r1r = r1l + R1X;
      TC t = NGF == 2 ? (gp ? ox : -ox) : TC(0);
      yl = hh[1]; yr = -hh[1]; xl = t; xr = t;
    }
    TC WL[NP], WR[NP], F[NF];
    mh_eval2d<EQ, TC>(s_wp + r1l, s_g + r1l, R1, xl, yl, WL);
    mh_eval2d<EQ, TC>(s_wp + r1r, s_g + r1r, R1, xr, yr, WR);
    face_flux_prim2d<EQ, TC>(G, xf ? 0 : 1, WL, WR, F, err);
    if (xf) {
#pragma unroll
      for (int q = 0; q < NF; ++q) s_fx[(q * NFX + f) * NGF + gp] = F[q];
    } else {
#pragma unroll
      for (int q = 0; q < NF; ++q) s_fy[(q * NFY + f) * NGF + gp] = F[q];
    }
  }
  __syncthreads();

  // ---- 4. per cell: volume integral, face moments, mass matrix, update
  const int lx = tid % TX, ly = tid / TX;
  const int gi = i0 + lx, gj = j0 + ly;
  const bool owner = gi < nx && gj < ny;
  const int r1 = (ly + 1) * R1X + lx + 1;
  const size_t gc = (size_t)s_gy[ly + 2] + s_gx[lx + 2];

  TC sFx[NF], sFy[NF];
#pragma unroll
  for (int q = 0; q < NF; ++q) { sFx[q] = TC(0); sFy[q] = TC(0); }
#pragma unroll
  for (int qp = 0; qp < 4; ++qp) {
    TC W[NP], Fx[NF], Fy[NF];
    mh_eval2d<EQ, TC>(s_wp + r1, s_g + r1, R1, (qp & 1) ? ox : -ox, (qp & 2) ? oy : -oy, W);
    prim_flux2d<EQ, TC>(G, W, Fx, Fy, err);
#pragma unroll
    for (int q = 0; q < NF; ++q) { sFx[q] += Fx[q]; sFy[q] += Fy[q]; }
  }

  const int fxm = ly * (TX + 1) + lx, fym = ly * TX + lx;
  TC Sxm[NF], Sxp[NF], Dxm[NF], Dxp[NF], Sym[NF], Syp[NF], Dym[NF], Dyp[NF];
#pragma unroll
  for (int q = 0; q < NF; ++q) {
    if (NGF == 2) {
      TC a0 = s_fx[(q * NFX + fxm) * 2], a1 = s_fx[(q * NFX + fxm) * 2 + 1];
      TC b0 = s_fx[(q * NFX + fxm + 1) * 2], b1 = s_fx[(q * NFX + fxm + 1) * 2 + 1];
      Sxm[q] = a0 + a1; Dxm[q] = a1 - a0; Sxp[q] = b0 + b1; Dxp[q] = b1 - b0;
      a0 = s_fy[(q * NFY + fym) * 2]; a1 = s_fy[(q * NFY + fym) * 2 + 1];
      b0 = s_fy[(q * NFY + fym + TX) * 2]; b1 = s_fy[(q * NFY + fym + TX) * 2 + 1];
      Sym[q] = a0 + a1; Dym[q] = a1 - a0; Syp[q] = b0 + b1; Dyp[q] = b1 - b0;
    } else {
      Sxm[q] = TC(2) * s_fx[q * NFX + fxm]; Sxp[q] = TC(2) * s_fx[q * NFX + fxm + 1];
      Sym[q] = TC(2) * s_fy[q * NFY + fym]; Syp[q] = TC(2) * s_fy[q * NFY + fym + TX];
      Dxm[q] = Dxp[q] = Dym[q] = Dyp[q] = TC(0);
    }
  }
  const TC inv2dx = TC(0.5) / dx, inv2dy = TC(0.5) / dy;
  const TC c3x = TC(3) / (dx * dx), c3y = TC(3) / (dy * dy);
  const TC r3 = TC(1.7320508075688772935) / (dx * dy);
  TC rc0[NV], rs[NS];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    rc0[v] = -(Sxp[v] - Sxm[v]) * inv2dx - (Syp[v] - Sym[v]) * inv2dy;
    rs[2 * v] = c3x * (sFx[v] - (Sxp[v] + Sxm[v])) - r3 * (Dyp[v] - Dym[v]);
    rs[2 * v + 1] = c3y * (sFy[v] - (Syp[v] + Sym[v])) - r3 * (Dxp[v] - Dxm[v]);
  }
  if (EQ == 1) {
    rc0[4] = -(Syp[4] - Sym[4]) * inv2dy;
    rc0[5] = -(Sxp[4] - Sxm[4]) * inv2dx;
    rs[8] = c3y * (sFy[4] - (Syp[4] + Sym[4]));
    rs[9] = c3x * (sFx[4] - (Sxp[4] + Sxm[4]));
    const TC ca3 = TC(1.7320508075688772935) / (dx * dx + dy * dy);
    rs[10] = ca3 * ((dy / dx) * (Dxp[4] - Dxm[4]) - (dx / dy) * (Dyp[4] - Dym[4]));
  }

  // U^{n+1} = U^n + dt L, U^n the limited step input
  double o0[NV];
  TC os[NS];
#pragma unroll
  for (int v = 0; v < NV; ++v) o0[v] = fma(dt, Cvt<TC>::to_f64(rc0[v]), A.in.c0[v * ncell + gc]);
#pragma unroll
  for (int k = 0; k < NS; ++k) os[k] = s_sl[k * R1 + r1] + dtc * rs[k];
  if (owner) {
#pragma unroll
    for (int v = 0; v < NV; ++v) A.out.c0[v * ncell + gc] = o0[v];
#pragma unroll
    for (int k = 0; k < NS; ++k) A.out.sl[k * ncell + gc] = (TS)os[k];
  }
  courant_commit2d<EQ, TC, TS, NT>(A, G, owner, o0, dx, dy, dt, nblk, err, S);
}

template <int EQ, class TC, class TS, int TX, int TY, int NGF, bool WENO>
__global__ void __launch_bounds__(TX * TY) mh2d_kernel(const Stage2DArgs<TS> A) {
  griddep_launch_dependents();  // programmatic dependent launch: see griddep_wait()
  griddep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ TileScalars<TX * TY> S;
  const MhMem2D<TC> M = mh2d_mem<EQ, TX, TY, NGF, TC>(smem_raw);
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  stage2d_setup<EQ, TC, TS, TX, TY>(A, i0, j0, M.m, S);
  __syncthreads();
  stage2d_load<EQ, TC, TS, TX, TY>(A, M.m);
  __syncthreads();
  mh2d_compute<EQ, TC, TS, TX, TY, NGF, WENO>(A, i0, j0, gridDim.x * gridDim.y, M, S);
}

}  // namespace dgk
