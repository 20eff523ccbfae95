// dg_stage3m.cuh -- one SSP-RK2 stage of the 3D P1 DG scheme for ideal MHD with
// the 11-function locally divergence-free field basis of Sec. 2.2 as one fused
// kernel (the 3D counterpart of the planar-MHD stage of dg_stage2d.cuh).
//
// State per cell: averages (rho, mx, my, mz, E, b1, b2, b3) and 23 derivative
// coefficients: the Taylor derivatives s[v*3+d] of (rho, mx, my, mz, E), then
// a4..a11 of V4 = (y,0,0), V5 = (z,0,0), V6 = (0,x,0), V7 = (0,z,0), V8 = (0,0,x),
// V9 = (0,0,y), V10 = (x,-y,0), V11 = (x,0,-z) in slots 15..22, i.e.
//   Bx = b1 + (a10 + a11) x + a4 y + a5 z,
//   By = b2 + a6 x - a10 y + a7 z,
//   Bz = b3 + a8 x + a9 y - a11 z.
// The tile is processed as in dg_stage3d.cuh: primitives of the cells the limiter
// reads, the min/max limiter on the tile and its face slabs (one factor for the
// whole field, so every cell stays divergence free), the volume integral at the
// 8 Gauss points, and
// the faces one orientation at a time (HLLD with two transverse components and
// the averaged normal field of Sec. 2.6, at the 2x2 Gauss points), gathered by
// both cells.
//
// Field right-hand side.  V4..V9 are each one field component times one
// coordinate, with their own diagonal mass, so their equations are those of the
// Taylor derivatives of that component: the kernel gathers the three field
// components like Taylor variables into r[i][d] ("d/dx_d of B_i", i, d = x, y, z)
// and takes a4 = r[x][y], a5 = r[x][z], a6 = r[y][x], a7 = r[y][z], a8 = r[z][x],
// a9 = r[z][y].  V10 = x e_x - y e_y and V11 = x e_x - z e_z couple through their
// mass block (V/12) [[hx^2+hy^2, hx^2], [hx^2, hx^2+hz^2]]; their weak right-hand
// sides are (V/12)(hx^2 r[x][x] - hy^2 r[y][y]) and (V/12)(hx^2 r[x][x] - hz^2
// r[z][z]), and the 2x2 system is solved in closed form.
#pragma once

#include "dg_stage3d.cuh"

namespace dgk {

// The primitives (laid out as the halo-2 box [8][R2]) are dead once the limiter
// has run; the face fluxes [8][4][FMAX] then reuse their space.
template <int TX, int TY, int TZ, class TC>
__host__ __device__ constexpr size_t stage3m_wsz() {
  return size_t(8) * (TX + 4) * (TY + 4) * (TZ + 4) > size_t(8) * 4 * stage3d_face_max<TX, TY, TZ, TC>()
             ? size_t(8) * (TX + 4) * (TY + 4) * (TZ + 4)
             : size_t(8) * 4 * stage3d_face_max<TX, TY, TZ, TC>();
}

template <int TX, int TY, int TZ, class TC>
__host__ __device__ constexpr size_t stage3m_smem_bytes() {
  return (stage3m_wsz<TX, TY, TZ, TC>() + size_t(31) * (TX + 2) * (TY + 2) * (TZ + 2)) * sizeof(TC) +
         sizeof(int) * ((TX + 4) + (TY + 4) + (TZ + 4));
}

// Centroid primitives (rho, vx, vy, vz, p, Bx, By, Bz) from averages.
template <class TC>
__device__ __forceinline__ void prims3m(const Gas<TC>& G, const TC* c, TC* W, unsigned& err) {
  TC rho = c[0], inv = TC(1) / rho;
  TC vx = c[1] * inv, vy = c[2] * inv, vz = c[3] * inv;
  TC mag = TC(0.5) * (c[5] * c[5] + c[6] * c[6] + c[7] * c[7]);
  TC p = G.gm1 * (c[4] - TC(0.5) * (c[1] * vx + c[2] * vy + c[3] * vz) - mag);
  if (!(rho > TC(0) && p > TC(0))) err |= ERR_NONPHYS;
  W[0] = rho; W[1] = vx; W[2] = vy; W[3] = vz; W[4] = p;
  W[5] = c[5]; W[6] = c[6]; W[7] = c[7];
}

// Field gradients gB[i][d] = dB_i/dx_d from the coefficients a4..a11 (s[15..22]).
template <class TC>
__device__ __forceinline__ void field_grad3m(const TC* s, TC (*gB)[3]) {
  gB[0][0] = s[21] + s[22]; gB[0][1] = s[15]; gB[0][2] = s[16];
  gB[1][0] = s[17]; gB[1][1] = -s[21]; gB[1][2] = s[18];
  gB[2][0] = s[19]; gB[2][1] = s[20]; gB[2][2] = -s[22];
}

// Min/max limiter of one cell (Sec. 2.5): W its centroid primitives, Wn those of
// its 6 face neighbours (-x, +x, -y, +y, -z, +z), s[23] limited in place.
template <class TC>
__device__ __forceinline__ void limit_cell3m(const Gas<TC>& G, const TC* hh, const TC* W,
                                             const TC (*Wn)[8], TC* s) {
  TC hi[8], lo[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    TC a = W[q], b = W[q];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      a = Wn[k][q] > a ? Wn[k][q] : a;
      b = Wn[k][q] < b ? Wn[k][q] : b;
    }
    hi[q] = a;
    lo[q] = b;
  }
  const TC rho = W[0], inv = TC(1) / rho;
  const TC v[3] = {W[1], W[2], W[3]};
  const TC v2h = TC(0.5) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  TC gB[3][3];
  field_grad3m<TC>(s, gB);
  TC gr[3], gv[3][3], gp[3], BdB[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    gr[d] = s[d];
    TC vdv = TC(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      gv[i][d] = (s[3 * (1 + i) + d] - v[i] * gr[d]) * inv;
      vdv += v[i] * gv[i][d];
    }
    BdB[d] = W[5] * gB[0][d] + W[6] * gB[1][d] + W[7] * gB[2][d];
    gp[d] = G.gm1 * (s[12 + d] - v2h * gr[d] - rho * vdv - BdB[d]);
  }
  const TC ar = limiter_alpha<TC, 3>(W[0], hi[0], lo[0], gr, hh);
  TC av[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) av[i] = limiter_alpha<TC, 3>(W[1 + i], hi[1 + i], lo[1 + i], gv[i], hh);
  const TC ap = limiter_alpha<TC, 3>(W[4], hi[4], lo[4], gp, hh);
  TC aB = TC(1);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    TC a = limiter_alpha<TC, 3>(W[5 + i], hi[5 + i], lo[5 + i], gB[i], hh);
    aB = a < aB ? a : aB;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    TC r = ar * gr[d];
    TC vdv = TC(0);
    s[d] = r;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      TC u = av[i] * gv[i][d];
      s[3 * (1 + i) + d] = rho * u + v[i] * r;
      vdv += v[i] * u;
    }
    s[12 + d] = ap * gp[d] * G.inv_gm1 + v2h * r + rho * vdv + aB * BdB[d];
  }
#pragma unroll
  for (int k = 15; k < 23; ++k) s[k] *= aB;
}

// WENO-type limiter of one cell (Sec. 2.5, dg_weno.cuh): the primitives rho, v, p
// blend their DG gradient with their min/max-limited central difference by the
// oscillation weights.  The field has one weight pair: its stencil candidate is
// the min/max-limited central differences G[i][d] of B_i, projected in L2 over
// the cell onto the divergence-free basis; the cross derivatives are basis
// coefficients themselves (a4 = G_xy, a5 = G_xz, a6 = G_yx, a7 = G_yz,
// a8 = G_zx, a9 = G_zy) and (a10, a11) solve
//   [[hx^2 + hy^2, hx^2], [hx^2, hx^2 + hz^2]] (a10, a11)
//     = (hx^2 G_xx - hy^2 G_yy, hx^2 G_xx - hz^2 G_zz),
// and the oscillation factors of the three components are added.  s[23] is
// limited in place (product rule back as in limit_cell3m).
template <class TC>
__device__ __forceinline__ void weno_cell3m(const Gas<TC>& G, const TC* hh, const TC* W,
                                            const TC (*Wn)[8], TC* s) {
  TC hi[8], lo[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    TC a = W[q], b = W[q];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      a = Wn[k][q] > a ? Wn[k][q] : a;
      b = Wn[k][q] < b ? Wn[k][q] : b;
    }
    hi[q] = a;
    lo[q] = b;
  }
  const TC rho = W[0], inv = TC(1) / rho;
  const TC v[3] = {W[1], W[2], W[3]};
  const TC v2h = TC(0.5) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  TC gB[3][3];
  field_grad3m<TC>(s, gB);
  TC g[5][3];  // primitive gradients of rho, vx, vy, vz, p
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    g[0][d] = s[d];
    TC vdv = TC(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      g[1 + i][d] = (s[3 * (1 + i) + d] - v[i] * g[0][d]) * inv;
      vdv += v[i] * g[1 + i][d];
    }
    const TC BdB = W[5] * gB[0][d] + W[6] * gB[1][d] + W[7] * gB[2][d];
    g[4][d] = G.gm1 * (s[12 + d] - v2h * g[0][d] - rho * vdv - BdB);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    TC nb[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) nb[k] = Wn[k][q];
    weno_blend<TC, 3>(W[q], hi[q], lo[q], nb, hh, g[q]);
  }
  // the field: stencil candidate, its projection, one weight pair
  TC Gs[3][3], od = TC(0), os = TC(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    TC nb[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) nb[k] = Wn[k][5 + i];
    weno_stencil<TC, 3>(W[5 + i], hi[5 + i], lo[5 + i], nb, hh, Gs[i]);
    od += weno_osc<TC, 3>(W[5 + i], nb, gB[i], hh);
  }
  const TC hx2 = hh[0] * hh[0], hy2 = hh[1] * hh[1], hz2 = hh[2] * hh[2];
  const TC P = hx2 * Gs[0][0] - hy2 * Gs[1][1], Q = hx2 * Gs[0][0] - hz2 * Gs[2][2];
  const TC Am = hx2 + hy2, Bm = hx2 + hz2;
  const TC idet = TC(1) / (Am * Bm - hx2 * hx2);
  TC st[23];  // the projected stencil field in slots 15..22
  st[15] = Gs[0][1]; st[16] = Gs[0][2]; st[17] = Gs[1][0];
  st[18] = Gs[1][2]; st[19] = Gs[2][0]; st[20] = Gs[2][1];
  st[21] = (Bm * P - hx2 * Q) * idet;
  st[22] = (Am * Q - hx2 * P) * idet;
  TC sB[3][3];
  field_grad3m<TC>(st, sB);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    TC nb[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) nb[k] = Wn[k][5 + i];
    os += weno_osc<TC, 3>(W[5 + i], nb, sB[i], hh);
  }
  const TC wd = TC(1) / sqrt(TC(kWenoEps) + od);
  const TC ws = TC(1) / sqrt(TC(kWenoEps) + os);
  const TC iw = TC(1) / (wd + ws);
#pragma unroll
  for (int k = 15; k < 23; ++k) s[k] = (wd * s[k] + ws * st[k]) * iw;
  field_grad3m<TC>(s, gB);  // the limited field's gradients
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
    const TC BdB = W[5] * gB[0][d] + W[6] * gB[1][d] + W[7] * gB[2][d];
    s[12 + d] = g[4][d] * G.inv_gm1 + v2h * r + rho * vdv + BdB;
  }
}

// The limiter of the kernels: WENO (compile time) selects the WENO-type one.
template <class TC, bool WENO>
__device__ __forceinline__ void limit3m(const Gas<TC>& G, const TC* hh, const TC* W,
                                        const TC (*Wn)[8], TC* s) {
  if constexpr (WENO) weno_cell3m<TC>(G, hh, W, Wn, s);
  else limit_cell3m<TC>(G, hh, W, Wn, s);
}

// Conserved values (rho, mx, my, mz, E, Bx, By, Bz) of the cell polynomial at
// local point (x, y, z).
template <class TC>
__device__ __forceinline__ void eval3m(const TC* c0, const TC* s, TC x, TC y, TC z, TC* c) {
#pragma unroll
  for (int v = 0; v < 5; ++v) c[v] = c0[v] + s[3 * v] * x + s[3 * v + 1] * y + s[3 * v + 2] * z;
  c[5] = c0[5] + (s[21] + s[22]) * x + s[15] * y + s[16] * z;
  c[6] = c0[6] + s[17] * x - s[21] * y + s[18] * z;
  c[7] = c0[7] + s[19] * x + s[20] * y - s[22] * z;
}

// Physical flux along axis d (uniform across the CTA) of a conserved state, in
// the component order (rho, mx, my, mz, E, Bx, By, Bz).
template <class TC>
__device__ __forceinline__ void phys_flux3m(const Gas<TC>& G, const TC* c, int d, TC* F,
                                            unsigned& err) {
  const TC rho = c[0], inv = TC(1) / rho;
  const TC v[3] = {c[1] * inv, c[2] * inv, c[3] * inv};
  const TC B[3] = {c[5], c[6], c[7]};
  const TC b2h = TC(0.5) * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  const TC p = G.gm1 * (c[4] - TC(0.5) * (c[1] * v[0] + c[2] * v[1] + c[3] * v[2]) - b2h);
  if (!(rho > TC(0) && p > TC(0))) err |= ERR_NONPHYS;
  const TC pT = p + b2h;
  const TC vd = d == 0 ? v[0] : (d == 1 ? v[1] : v[2]);
  const TC Bd = d == 0 ? B[0] : (d == 1 ? B[1] : B[2]);
  const TC vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
  F[0] = rho * vd;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    F[1 + i] = c[1 + i] * vd - B[i] * Bd + (i == d ? pT : TC(0));
    F[5 + i] = B[i] * vd - v[i] * Bd;
  }
  F[4] = (c[4] + pT) * vd - Bd * vB;
}

// HLLD flux through a face along axis d (uniform across the CTA) between the
// primitive states Wl, Wr (rho, v, p, B), with the normal field replaced by the
// average of both sides (Sec. 2.6); lab frame, component order of phys_flux3m.
// The face frame is (n, t1, t2) = (d, d+1, d+2) cyclically, picked with selects.
template <class TC>
__device__ __forceinline__ void face_flux_prim3m(const Gas<TC>& G, int d, const TC* Wl,
                                                 const TC* Wr, TC* F, unsigned& err) {
  auto pick = [&](const TC* W, int o, int k) {  // component k (0 n, 1 t1, 2 t2) of W[o..o+2]
    const int a = d + k >= 3 ? d + k - 3 : d + k;
    return a == 0 ? W[o] : (a == 1 ? W[o + 1] : W[o + 2]);
  };
  const TC bn = TC(0.5) * (pick(Wl, 5, 0) + pick(Wr, 5, 0));
  TC Ff[7];
  hlld_flux3<TC>(G, Wl[0], pick(Wl, 1, 0), pick(Wl, 1, 1), pick(Wl, 1, 2), Wl[4], pick(Wl, 5, 1),
                 pick(Wl, 5, 2), Wr[0], pick(Wr, 1, 0), pick(Wr, 1, 1), pick(Wr, 1, 2), Wr[4],
                 pick(Wr, 5, 1), pick(Wr, 5, 2), bn, Ff, err);
  // lab component a is face component k = a - d (mod 3)
  F[0] = Ff[0];
  F[4] = Ff[4];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int k = a - d < 0 ? a - d + 3 : a - d;
    F[1 + a] = k == 0 ? Ff[1] : (k == 1 ? Ff[2] : Ff[3]);
    F[5 + a] = k == 0 ? TC(0) : (k == 1 ? Ff[5] : Ff[6]);
  }
}

// The same between conserved states cl, cr (the solver checks positivity).
template <class TC>
__device__ __forceinline__ void face_flux3m(const Gas<TC>& G, int d, const TC* cl, const TC* cr,
                                            TC* F, unsigned& err) {
  TC Wl[8], Wr[8];
  unsigned e2 = 0;
  prims3m<TC>(G, cl, Wl, e2);
  prims3m<TC>(G, cr, Wr, e2);
  face_flux_prim3m<TC>(G, d, Wl, Wr, F, err);
}

// Field part of the right-hand side from the Taylor-like gathers r[3*(5+i)+d].
template <class TC>
__device__ __forceinline__ void field_rhs3m(const TC* rs24, const TC* hd, TC* ra) {
  const TC rxx = rs24[15], rxy = rs24[16], rxz = rs24[17];
  const TC ryx = rs24[18], ryy = rs24[19], ryz = rs24[20];
  const TC rzx = rs24[21], rzy = rs24[22], rzz = rs24[23];
  ra[0] = rxy; ra[1] = rxz; ra[2] = ryx; ra[3] = ryz; ra[4] = rzx; ra[5] = rzy;
  const TC hx2 = hd[0] * hd[0], hy2 = hd[1] * hd[1], hz2 = hd[2] * hd[2];
  const TC P = hx2 * rxx - hy2 * ryy, Q = hx2 * rxx - hz2 * rzz;
  const TC A = hx2 + hy2, Bm = hx2 + hz2;
  const TC det = A * Bm - hx2 * hx2;
  ra[6] = (Bm * P - hx2 * Q) / det;
  ra[7] = (A * Q - hx2 * P) / det;
}

// FP32: two resident 256-thread CTAs per SM (128 registers a thread); FP64 keeps
// its registers.
template <int NT, class TC>
struct Stage3mMinBlocks {
  static constexpr int v = sizeof(TC) == 4 && 65536 / (128 * NT) > 0 ? 65536 / (128 * NT) : 1;
};

template <class TC, class TS, int TX, int TY, int TZ, int STAGE, bool WENO>
__global__ void __launch_bounds__(TX * TY * TZ, (Stage3mMinBlocks<TX * TY * TZ, TC>::v))
    stage3m_kernel(const Stage3DArgs<TS> A) {
  griddep_launch_dependents();  // programmatic dependent launch: see griddep_wait()
  griddep_wait();
  constexpr int R2X = TX + 4, R2Y = TY + 4, R2Z = TZ + 4, R2 = R2X * R2Y * R2Z;
  constexpr int R1X = TX + 2, R1Y = TY + 2, R1Z = TZ + 2, R1 = R1X * R1Y * R1Z;
  constexpr int NT = TX * TY * TZ;
  constexpr int FMAX = stage3d_face_max<TX, TY, TZ, TC>();
  static_assert(NT % 32 == 0, "tile must be whole warps");
  (void)R1Z;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int WS = (int)stage3m_wsz<TX, TY, TZ, TC>();
  TC* s_w = reinterpret_cast<TC*>(smem_raw);  // 8 x R2 primitives, then
  TC* s_f = s_w;                              //   8 x 4 x FMAX face fluxes
  TC* s_c0 = s_w + WS;                        // 8 x R1 averages
  TC* s_sl = s_c0 + 8 * R1;                   // 23 x R1 derivative coefficients
  int* s_gx = reinterpret_cast<int*>(s_sl + 23 * R1);
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

  // ---- primitives where the limiter reads them; averages of the halo-1 box
  if (STAGE == 2) stage3d_prefetch_base<8, 23, TX, TY>(A, ncell, s_gx, s_gy, s_gz);
  stage3d_issue<8, 23, TX, TY, TZ, TS, TC, 0, 0, true, true>(A.in, ncell, s_gx, s_gy, s_gz, s_sl);
  // the halo-2 cells the limiter reads: the halo-1 box, then the six outer face
  // layers (e < R1 is the cell's halo-1 index)
#pragma unroll 1
  for (int e = tid; e < halo3d_count<TX, TY, TZ>(); e += NT) {
    int rx, ry, rz;
    halo3d_cell<TX, TY, TZ>(e, rx, ry, rz);
    const int r = (rz * R2Y + ry) * R2X + rx;
    size_t g = (size_t)s_gz[rz] + s_gy[ry] + s_gx[rx];
    TC c[8], W[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) c[v] = Cvt<TC>::to_tc(__ldg(&A.in.c0[v * ncell + g]));
    prims3m<TC>(G, c, W, err);
#pragma unroll
    for (int q = 0; q < 8; ++q) s_w[q * R2 + r] = W[q];
    if (e < R1) {
#pragma unroll
      for (int v = 0; v < 8; ++v) s_c0[v * R1 + e] = c[v];
    }
  }
  cp_async_wait_all();
  __syncthreads();

  const TC dx = Cvt<TC>::to_tc(A.dx), dy = Cvt<TC>::to_tc(A.dy), dz = Cvt<TC>::to_tc(A.dz);
  const TC hh[3] = {TC(0.5) * dx, TC(0.5) * dy, TC(0.5) * dz};
  const TC oo[3] = {dx * TC(0.28867513459481288225), dy * TC(0.28867513459481288225),
                    dz * TC(0.28867513459481288225)};
  const TC hd[3] = {dx, dy, dz};

  // ---- limiter on the tile and its face slabs (the cells the faces read)
  if (A.limiter) {
    for (int e = tid; e < ring3d_count<TX, TY, TZ>(); e += NT) {
      int rx, ry, rz;
      ring3d_cell<TX, TY, TZ>(e, rx, ry, rz);
      const int r1 = (rz * R1Y + ry) * R1X + rx;
      const int r2 = ((rz + 1) * R2Y + (ry + 1)) * R2X + (rx + 1);
      TC W[8], Wn[6][8], s[23];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        W[q] = s_w[q * R2 + r2];
        Wn[0][q] = s_w[q * R2 + r2 - 1];
        Wn[1][q] = s_w[q * R2 + r2 + 1];
        Wn[2][q] = s_w[q * R2 + r2 - R2X];
        Wn[3][q] = s_w[q * R2 + r2 + R2X];
        Wn[4][q] = s_w[q * R2 + r2 - R2X * R2Y];
        Wn[5][q] = s_w[q * R2 + r2 + R2X * R2Y];
      }
#pragma unroll
      for (int k = 0; k < 23; ++k) s[k] = s_sl[k * R1 + r1];
      limit3m<TC, WENO>(G, hh, W, Wn, s);
#pragma unroll
      for (int k = 0; k < 23; ++k) s_sl[k * R1 + r1] = s[k];
    }
    __syncthreads();
  }

  // ---- per-cell volume integral
  const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
  const int r1c = ((lz + 1) * R1Y + (ly + 1)) * R1X + (lx + 1);
  TC rc0[8], rs[24];
#pragma unroll
  for (int v = 0; v < 8; ++v) rc0[v] = TC(0);
  {
    TC c0[8], s[23];
#pragma unroll
    for (int v = 0; v < 8; ++v) c0[v] = s_c0[v * R1 + r1c];
#pragma unroll
    for (int k = 0; k < 23; ++k) s[k] = s_sl[k * R1 + r1c];
#pragma unroll
    for (int k = 0; k < 24; ++k) rs[k] = TC(0);
#pragma unroll 1
    for (int qp = 0; qp < 8; ++qp) {
      TC c[8];
      eval3m<TC>(c0, s, (qp & 1) ? oo[0] : -oo[0], (qp & 2) ? oo[1] : -oo[1],
                 (qp & 4) ? oo[2] : -oo[2], c);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        TC F[8];
        phys_flux3m<TC>(G, c, d, F, err);
        const TC w = TC(1.5) / (hd[d] * hd[d]);
#pragma unroll
        for (int v = 0; v < 8; ++v) rs[3 * v + d] += w * F[v];
      }
    }
  }

  // ---- faces, one orientation at a time
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
    for (int e = tid; e < 4 * NFACE; e += NT) {
      const int f = e >> 2, g = e & 3;
      const int fz = div_by_magic(f, mXY), fr = f - fz * (FX * FY);
      const int fy = div_by_magic(fr, mX), fx = fr - fy * FX;
      const int r1r = ((fz + 1) * R1Y + (fy + 1)) * R1X + (fx + 1);
      const int r1l = r1r - step;
      const TC a = (g & 2) ? o1 : -o1, b = (g & 1) ? o2 : -o2;
      const TC xl = d == 0 ? hn : a, xr = d == 0 ? -hn : a;
      const TC yl = d == 1 ? hn : (d == 0 ? a : b), yr = d == 1 ? -hn : (d == 0 ? a : b);
      const TC zl = d == 2 ? hn : b, zr = d == 2 ? -hn : b;
      TC cl0[8], cr0[8], sl[23], sr[23], cl[8], cr[8], F[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) { cl0[v] = s_c0[v * R1 + r1l]; cr0[v] = s_c0[v * R1 + r1r]; }
#pragma unroll
      for (int k = 0; k < 23; ++k) { sl[k] = s_sl[k * R1 + r1l]; sr[k] = s_sl[k * R1 + r1r]; }
      eval3m<TC>(cl0, sl, xl, yl, zl, cl);
      eval3m<TC>(cr0, sr, xr, yr, zr, cr);
      face_flux3m<TC>(G, d, cl, cr, F, err);
#pragma unroll
      for (int v = 0; v < 8; ++v) s_f[(v * FMAX + f) * 4 + g] = F[v];
    }
    __syncthreads();
    {
      const int fm = (lz * FY + ly) * FX + lx;
      const int fp = fm + (d == 0 ? 1 : (d == 1 ? FX : FX * FY));
      // gather3d for the 5 Taylor variables and the 3 field components
      if (d == 0) {
        gather3d<0, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
        gather3d<0, TC, 3>(s_f + 5 * FMAX * 4, FMAX, fm, fp, hd, rc0 + 5, rs + 15);
      } else if (d == 1) {
        gather3d<1, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
        gather3d<1, TC, 3>(s_f + 5 * FMAX * 4, FMAX, fm, fp, hd, rc0 + 5, rs + 15);
      } else {
        gather3d<2, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
        gather3d<2, TC, 3>(s_f + 5 * FMAX * 4, FMAX, fm, fp, hd, rc0 + 5, rs + 15);
      }
    }
    __syncthreads();
  }
  TC rsl[23];
#pragma unroll
  for (int k = 0; k < 15; ++k) rsl[k] = rs[k];
  field_rhs3m<TC>(rs, hd, rsl + 15);

  // ---- Runge-Kutta combination
  const int gi = i0 + lx, gj = j0 + ly, gk = k0 + lz;
  const bool owner = gi < nx && gj < ny && gk < nz;
  const size_t gc = (size_t)s_gz[lz + 2] + s_gy[ly + 2] + s_gx[lx + 2];
  const double dt = s_dt;
  const TC dtc = Cvt<TC>::to_tc(dt);
  double o0[8];
  TC os[23];
  if (STAGE == 1) {
#pragma unroll
    for (int v = 0; v < 8; ++v) o0[v] = fma(dt, Cvt<TC>::to_f64(rc0[v]), A.in.c0[v * ncell + gc]);
#pragma unroll
    for (int k = 0; k < 23; ++k) os[k] = s_sl[k * R1 + r1c] + dtc * rsl[k];
    if (A.limiter && A.lim_sl && owner) {
#pragma unroll
      for (int k = 0; k < 23; ++k) A.lim_sl[k * ncell + gc] = (TS)s_sl[k * R1 + r1c];
    }
  } else {
    TC sn[23];
    if (A.limiter && A.lim_sl) {
#pragma unroll
      for (int k = 0; k < 23; ++k) sn[k] = (TC)A.lim_sl[k * ncell + gc];
    } else {
#pragma unroll
      for (int k = 0; k < 23; ++k) sn[k] = (TC)A.base.sl[k * ncell + gc];
    }
    if (A.limiter && !A.lim_sl) {
      TC c[8], W[8], Wn[6][8];
#pragma unroll
      for (int v = 0; v < 8; ++v) c[v] = Cvt<TC>::to_tc(A.base.c0[v * ncell + gc]);
      prims3m<TC>(G, c, W, err);
      const size_t nb[6] = {(size_t)s_gz[lz + 2] + s_gy[ly + 2] + s_gx[lx + 1],
                            (size_t)s_gz[lz + 2] + s_gy[ly + 2] + s_gx[lx + 3],
                            (size_t)s_gz[lz + 2] + s_gy[ly + 1] + s_gx[lx + 2],
                            (size_t)s_gz[lz + 2] + s_gy[ly + 3] + s_gx[lx + 2],
                            (size_t)s_gz[lz + 1] + s_gy[ly + 2] + s_gx[lx + 2],
                            (size_t)s_gz[lz + 3] + s_gy[ly + 2] + s_gx[lx + 2]};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int v = 0; v < 8; ++v) c[v] = Cvt<TC>::to_tc(A.base.c0[v * ncell + nb[k]]);
        prims3m<TC>(G, c, Wn[k], err);
      }
      limit3m<TC, WENO>(G, hh, W, Wn, sn);
    }
#pragma unroll
    for (int v = 0; v < 8; ++v)
      o0[v] = half_f64(A.base.c0[v * ncell + gc] +
                       fma(dt, Cvt<TC>::to_f64(rc0[v]), A.in.c0[v * ncell + gc]));
#pragma unroll
    for (int k = 0; k < 23; ++k)
      os[k] = TC(0.5) * sn[k] + TC(0.5) * (s_sl[k * R1 + r1c] + dtc * rsl[k]);
  }
  if (owner) {
#pragma unroll
    for (int v = 0; v < 8; ++v) A.out.c0[v * ncell + gc] = o0[v];
#pragma unroll
    for (int k = 0; k < 23; ++k) A.out.sl[k * ncell + gc] = (TS)os[k];
  }

  if (STAGE == 2) {
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
  } else {
    if (err) atomicOr(&s_err, err);
    __syncthreads();
    if (tid == 0 && s_err) atomicOr(&A.ctl->err, s_err);
  }
}

}  // namespace dgk
