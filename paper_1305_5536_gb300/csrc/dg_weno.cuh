// dg_weno.cuh -- the WENO-type limiter of Sec. 2.5 for one cell (2D and 3D).
//
// Per primitive phi two candidate gradients: the unlimited DG gradient and the
// stencil gradient of the FV method, i.e. the central difference of the face
// neighbours' centroid values, min/max limited (limiter_alpha).  For each
// candidate the oscillation factor
//   o = sum over the faces f of |Delta phi_f| + |phi_nbr(f) - (phi + Delta phi_f)|,
//   Delta phi_f = grad phi . (f - s),
// and the limited gradient is the mean of the candidates weighted by
// (eps + o)^(-1/2), eps the machine epsilon of double precision.  The magnetic
// field of 2D MHD has one weight pair, so that the blend stays divergence free:
// its stencil candidate (the min/max-limited central differences of Bx and By) is
// projected in L2 over the cell onto the divergence-free basis,
//   a1 = dBx/dy, a2 = dBy/dx, a3 = (dBx/dx dx^2 - dBy/dy dy^2) / (dx^2 + dy^2),
// and its oscillation factor is that of Bx plus that of By.  The limited
// primitive gradients go back to conserved derivative coefficients by the
// product rule, as for the min/max limiter.
#pragma once

#include "dg_physics.cuh"

namespace dgk {

constexpr double kWenoEps = 2.220446049250313e-16;

// Oscillation factor of gradient g[DIM] for centroid value phi; nb[2d] and
// nb[2d+1] are the - and + neighbours along axis d, hh the half cell sizes.
template <class TC, int DIM>
__device__ __forceinline__ TC weno_osc(TC phi, const TC* nb, const TC* g, const TC* hh) {
  TC o = TC(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const TC a = g[d] * hh[d];  // Delta phi at the + face (-a at the - face)
    o += TC(2) * fabs(a) + fabs(nb[2 * d + 1] - (phi + a)) + fabs(nb[2 * d] - (phi - a));
  }
  return o;
}

// Min/max-limited central difference of the neighbour values (the stencil
// candidate of one primitive).
template <class TC, int DIM>
__device__ __forceinline__ void weno_stencil(TC phi, TC hi, TC lo, const TC* nb, const TC* hh,
                                             TC* gs) {
#pragma unroll
  for (int d = 0; d < DIM; ++d) gs[d] = (nb[2 * d + 1] - nb[2 * d]) * (TC(0.25) / hh[d]);
  const TC a = limiter_alpha<TC, DIM>(phi, hi, lo, gs, hh);
#pragma unroll
  for (int d = 0; d < DIM; ++d) gs[d] *= a;
}

// The WENO blend of one primitive's DG gradient g[DIM] (replaced in place).
template <class TC, int DIM>
__device__ __forceinline__ void weno_blend(TC phi, TC hi, TC lo, const TC* nb, const TC* hh,
                                           TC* g) {
  TC gs[DIM];
  weno_stencil<TC, DIM>(phi, hi, lo, nb, hh, gs);
  const TC wd = TC(1) / sqrt(TC(kWenoEps) + weno_osc<TC, DIM>(phi, nb, g, hh));
  const TC ws = TC(1) / sqrt(TC(kWenoEps) + weno_osc<TC, DIM>(phi, nb, gs, hh));
  const TC inv = TC(1) / (wd + ws);
#pragma unroll
  for (int d = 0; d < DIM; ++d) g[d] = (wd * g[d] + ws * gs[d]) * inv;
}

// 2D cell: W its centroid primitives (rho, vx, vy, p[, Bx, By]), Wn the
// neighbours' (-x, +x, -y, +y), s[] the conserved derivative coefficients in the
// slot order (rho, mx, my, E) x (d/dx, d/dy)[, a1, a2, a3], limited in place.
// gout (may be null) receives the limited primitive gradients in the same slots.
template <int EQ, class TC>
__device__ __forceinline__ void weno_cell2d(const Gas<TC>& G, const TC* hh, const TC* W,
                                            const TC (*Wn)[EQ == 1 ? 6 : 4], TC* s, TC* gout) {
  constexpr int NP = EQ == 1 ? 6 : 4;
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
  const TC rho = W[0], vx = W[1], vy = W[2];
  const TC inv = TC(1) / rho;
  const TC v2h = TC(0.5) * (vx * vx + vy * vy);
  TC a1 = TC(0), a2 = TC(0), a3 = TC(0);
  if (EQ == 1) { a1 = s[8]; a2 = s[9]; a3 = s[10]; }
  TC g[4][2];
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    g[0][d] = s[d];
    g[1][d] = (s[2 + d] - vx * g[0][d]) * inv;
    g[2][d] = (s[4 + d] - vy * g[0][d]) * inv;
    TC BdB = TC(0);
    if (EQ == 1) BdB = d == 0 ? W[4] * a3 + W[5] * a2 : W[4] * a1 - W[5] * a3;
    g[3][d] = G.gm1 * (s[6 + d] - v2h * g[0][d] - rho * (vx * g[1][d] + vy * g[2][d]) - BdB);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const TC nb[4] = {Wn[0][q], Wn[1][q], Wn[2][q], Wn[3][q]};
    weno_blend<TC, 2>(W[q], hi[q], lo[q], nb, hh, g[q]);
  }
  TC bx[2] = {TC(0), TC(0)}, by[2] = {TC(0), TC(0)};  // limited field gradients
  if (EQ == 1) {
    const TC nbx[4] = {Wn[0][4], Wn[1][4], Wn[2][4], Wn[3][4]};
    const TC nby[4] = {Wn[0][5], Wn[1][5], Wn[2][5], Wn[3][5]};
    TC gx[2], gy[2];
    weno_stencil<TC, 2>(W[4], hi[4], lo[4], nbx, hh, gx);
    weno_stencil<TC, 2>(W[5], hi[5], lo[5], nby, hh, gy);
    const TC h02 = hh[0] * hh[0], h12 = hh[1] * hh[1];
    const TC st1 = gx[1], st2 = gy[0], st3 = (gx[0] * h02 - gy[1] * h12) / (h02 + h12);
    const TC dbx[2] = {a3, a1}, dby[2] = {a2, -a3};
    const TC sbx[2] = {st3, st1}, sby[2] = {st2, -st3};
    const TC wd = TC(1) / sqrt(TC(kWenoEps) + weno_osc<TC, 2>(W[4], nbx, dbx, hh) +
                               weno_osc<TC, 2>(W[5], nby, dby, hh));
    const TC ws = TC(1) / sqrt(TC(kWenoEps) + weno_osc<TC, 2>(W[4], nbx, sbx, hh) +
                               weno_osc<TC, 2>(W[5], nby, sby, hh));
    const TC iw = TC(1) / (wd + ws);
    a1 = (wd * a1 + ws * st1) * iw;
    a2 = (wd * a2 + ws * st2) * iw;
    a3 = (wd * a3 + ws * st3) * iw;
    bx[0] = a3; bx[1] = a1;
    by[0] = a2; by[1] = -a3;
  }
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const TC r = g[0][d], ux = g[1][d], uy = g[2][d], pp = g[3][d];
    TC BdB = TC(0);
    if (EQ == 1) BdB = W[4] * bx[d] + W[5] * by[d];
    s[d] = r;
    s[2 + d] = rho * ux + vx * r;
    s[4 + d] = rho * uy + vy * r;
    s[6 + d] = pp * G.inv_gm1 + v2h * r + rho * (vx * ux + vy * uy) + BdB;
    if (gout) {
      gout[d] = r;
      gout[2 + d] = ux;
      gout[4 + d] = uy;
      gout[6 + d] = pp;
    }
  }
  if (EQ == 1) {
    s[8] = a1; s[9] = a2; s[10] = a3;
    if (gout) { gout[8] = a1; gout[9] = a2; gout[10] = a3; }
  }
}

// 3D Euler cell: W (rho, vx, vy, vz, p), Wn the neighbours (-x, +x, -y, +y, -z,
// +z), s[v*3+d] the conserved derivative coefficients, limited in place; gout
// (may be null) receives the limited primitive gradients g[v*3+d].
template <class TC>
__device__ __forceinline__ void weno_cell3d(const Gas<TC>& G, const TC* hh, const TC* W,
                                            const TC (*Wn)[5], TC* s, TC* gout) {
  const TC rho = W[0], inv = TC(1) / rho;
  const TC v[3] = {W[1], W[2], W[3]};
  const TC v2h = TC(0.5) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  TC g[5][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    g[0][d] = s[d];
    TC vdv = TC(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      g[1 + i][d] = (s[3 * (1 + i) + d] - v[i] * g[0][d]) * inv;
      vdv += v[i] * g[1 + i][d];
    }
    g[4][d] = G.gm1 * (s[12 + d] - v2h * g[0][d] - rho * vdv);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    TC hi = W[q], lo = W[q];
    TC nb[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      nb[k] = Wn[k][q];
      hi = nb[k] > hi ? nb[k] : hi;
      lo = nb[k] < lo ? nb[k] : lo;
    }
    weno_blend<TC, 3>(W[q], hi, lo, nb, hh, g[q]);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const TC r = g[0][d];
    TC vdv = TC(0);
    s[d] = r;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const TC u = g[1 + i][d];
      s[3 * (1 + i) + d] = rho * u + v[i] * r;
      vdv += v[i] * u;
    }
    s[12 + d] = g[4][d] * G.inv_gm1 + v2h * r + rho * vdv;
  }
  if (gout) {
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
      for (int d = 0; d < 3; ++d) gout[3 * q + d] = g[q][d];
  }
}

}  // namespace dgk
