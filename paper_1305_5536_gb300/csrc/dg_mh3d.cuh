// dg_mh3d.cuh -- one MUSCL-Hancock step (Sec. 2.4) of the 3D P1 DG scheme for the
// Euler equations (Taylor basis 1, x, y, z; eqs. `fv3d`, `dgderiv3d` with the
// update of eq. `GalerkUpdate`) as one fused kernel.
//
// One CTA owns a TX x TY x TZ tile.  Shared memory holds the centroid primitives
// of the tile plus a halo of 2 cells (the limiter's neighbour extrema; the space
// then takes the face fluxes), the predicted centroid values of the tile plus a
// halo of 1 cell, and the derivative coefficients of the same box, replaced in
// place by the limited primitive gradients.  Steps:
//   1. primitives of the halo-2 box; coefficients of the halo-1 box;
//   2. on the halo-1 box: primitive gradients by the product rule, the min/max
//      limiter (Sec. 2.5), dW/dt at the centroid from the primitive form
//        drho/dt = -v.grad rho - rho div v,  dv/dt = -(v.grad) v - grad p / rho,
//        dp/dt = -v.grad p - gamma p div v,
//      and the predicted centroid values W_c + dt/2 dW/dt;
//   3. per cell: fluxes of the predicted state at the 8 volume Gauss points;
//   4. faces of one orientation at a time: the Riemann flux (exact solver) of the
//      predicted values of both sides at NGF^2 points (1: the face centroid,
//      eq. `GalerkUpdate`; 4: the 2x2 Gauss points), gathered by both cells;
//   5. the update U^{n+1} = U^n + dt L of the limited coefficients (rebuilt from
//      the limited gradients by the product rule) and the Courant reduction of
//      U^{n+1} for the next step.
// The right-hand side is that of dg_stage3d.cuh; a face-centroid flux F stands for
// four equal Gauss-point fluxes (S = 4F, D = 0).
#pragma once

#include "dg_stage3d.cuh"

namespace dgk {

template <int TX, int TY, int TZ, int NGF, class TC>
__host__ __device__ constexpr size_t mh3d_smem_bytes() {
  constexpr size_t R2 = size_t(TX + 4) * (TY + 4) * (TZ + 4);
  constexpr size_t R1 = size_t(TX + 2) * (TY + 2) * (TZ + 2);
  constexpr size_t FS = size_t(5) * NGF * NGF * stage3d_face_max<TX, TY, TZ, TC>();
  return ((5 * R2 > FS ? 5 * R2 : FS) + 5 * R1 + 15 * R1) * sizeof(TC) +
         sizeof(int) * ((TX + 4) + (TY + 4) + (TZ + 4));
}

// Primitive gradients g[v*3+d] (v = rho, vx, vy, vz, p) of one cell from its
// conserved coefficients s[] at centroid primitives W; limiter 1: the min/max
// limiter scales them, 2: the WENO-type limiter (dg_weno.cuh) replaces them (Wn:
// the 6 face neighbours' primitives).  WENO selects the WENO-type limiter at
// compile time, so that the min/max kernels keep their register allocation.
template <class TC, bool WENO>
__device__ __forceinline__ void mh_grads3d(const Gas<TC>& G, const TC* hh, const TC* W,
                                           const TC (*Wn)[5], int limiter, const TC* s, TC* g) {
  if constexpr (WENO) {
    TC sc[15];
#pragma unroll
    for (int k = 0; k < 15; ++k) sc[k] = s[k];
    weno_cell3d<TC>(G, hh, W, Wn, sc, g);
    return;
  }
  const bool limit = limiter != 0;
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
    g[12 + d] = G.gm1 * (s[12 + d] - v2h * g[d] - rho * vdv);
  }
  if (!limit) return;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    TC hi = W[q], lo = W[q];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      hi = Wn[k][q] > hi ? Wn[k][q] : hi;
      lo = Wn[k][q] < lo ? Wn[k][q] : lo;
    }
    const TC a = limiter_alpha<TC, 3>(W[q], hi, lo, g + 3 * q, hh);
#pragma unroll
    for (int d = 0; d < 3; ++d) g[3 * q + d] *= a;
  }
}

// Limited conserved coefficients from the limited primitive gradients (the
// product rule back, as at the end of limit_cell3d).
template <class TC>
__device__ __forceinline__ void mh_cons3d(const Gas<TC>& G, const TC* W, const TC* g, TC* s) {
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
    s[12 + d] = g[12 + d] * G.inv_gm1 + v2h * r + rho * vdv;
  }
}

template <class TC>
__device__ __forceinline__ void mh_rates3d(const Gas<TC>& G, const TC* W, const TC* g, TC* Wt) {
  const TC rho = W[0], inv = TC(1) / rho, p = W[4];
  const TC v[3] = {W[1], W[2], W[3]};
  const TC divv = g[3] + g[7] + g[11];
  Wt[0] = -(v[0] * g[0] + v[1] * g[1] + v[2] * g[2]) - rho * divv;
#pragma unroll
  for (int i = 0; i < 3; ++i)
    Wt[1 + i] = -(v[0] * g[3 * (1 + i)] + v[1] * g[3 * (1 + i) + 1] + v[2] * g[3 * (1 + i) + 2]) -
                g[12 + i] * inv;
  Wt[4] = -(v[0] * g[12] + v[1] * g[13] + v[2] * g[14]) - G.g * p * divv;
}

// Predicted primitive state of a cell at local point (x, y, z): wp[] its predicted
// centroid values, g[] its limited primitive gradients (strided by `st`).
template <class TC>
__device__ __forceinline__ void mh_eval3d(const TC* wp, const TC* g, int st, TC x, TC y, TC z,
                                          TC* W) {
#pragma unroll
  for (int q = 0; q < 5; ++q)
    W[q] = wp[q * st] + g[(3 * q) * st] * x + g[(3 * q + 1) * st] * y + g[(3 * q + 2) * st] * z;
}

// Physical flux along axis d of a primitive state (rho, v, p).
template <class TC>
__device__ __forceinline__ void prim_flux3d(const Gas<TC>& G, const TC* W, int d, TC* F,
                                            unsigned& err) {
  const TC rho = W[0], p = W[4];
  if (!(rho > TC(0) && p > TC(0))) err |= ERR_NONPHYS;
  const TC m[3] = {rho * W[1], rho * W[2], rho * W[3]};
  const TC vd = W[1 + d];
  const TC E = p * G.inv_gm1 + TC(0.5) * (m[0] * W[1] + m[1] * W[2] + m[2] * W[3]);
  F[0] = m[d];
  F[1] = m[0] * vd;
  F[2] = m[1] * vd;
  F[3] = m[2] * vd;
  F[1 + d] += p;
  F[4] = (E + p) * vd;
}

// Exact-solver flux along axis d between primitive states (selects, as face_flux3d).
template <class TC>
__device__ __forceinline__ void face_flux_prim3d(const Gas<TC>& G, int d, const TC* WL,
                                                 const TC* WR, TC* F, unsigned& err) {
  const TC nl = d == 0 ? WL[1] : (d == 1 ? WL[2] : WL[3]);
  const TC nr = d == 0 ? WR[1] : (d == 1 ? WR[2] : WR[3]);
  TC tl[2] = {d == 0 ? WL[2] : WL[1], d == 2 ? WL[2] : WL[3]};
  TC tr[2] = {d == 0 ? WR[2] : WR[1], d == 2 ? WR[2] : WR[3]};
  TC Ff[5];
  exact_flux<TC, 2>(G, WL[0], nl, WL[4], tl, WR[0], nr, WR[4], tr, Ff, err);
  F[0] = Ff[0];
  F[1] = d == 0 ? Ff[1] : Ff[2];
  F[2] = d == 1 ? Ff[1] : (d == 0 ? Ff[2] : Ff[3]);
  F[3] = d == 2 ? Ff[1] : Ff[3];
  F[4] = Ff[4];
}

// Add the two face-centroid fluxes of orientation D of a cell to its right-hand
// side (gather3d with four equal Gauss-point fluxes) for NV variables.
template <int D, class TC, int NV = 5>
__device__ __forceinline__ void gather3d_centroid(const TC* s_f, int FMAX, int fm, int fp,
                                                  const TC* hd, TC* rc0, TC* rs) {
  const TC c0f = TC(1) / hd[D];
  const TC csf = TC(6) / (hd[D] * hd[D]);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const TC m = s_f[v * FMAX + fm], p = s_f[v * FMAX + fp];
    rc0[v] -= (p - m) * c0f;
    rs[3 * v + D] -= csf * (p + m);
  }
}

template <class TC, class TS, int TX, int TY, int TZ, int NGF, bool WENO>
__global__ void __launch_bounds__(TX * TY * TZ) mh3d_kernel(const Stage3DArgs<TS> A) {
  griddep_launch_dependents();  // programmatic dependent launch: see griddep_wait()
  griddep_wait();
  constexpr int R2X = TX + 4, R2Y = TY + 4, R2Z = TZ + 4, R2 = R2X * R2Y * R2Z;
  constexpr int R1X = TX + 2, R1Y = TY + 2, R1Z = TZ + 2, R1 = R1X * R1Y * R1Z;
  constexpr int NT = TX * TY * TZ;
  constexpr int FMAX = stage3d_face_max<TX, TY, TZ, TC>();
  constexpr int NPT = NGF * NGF;
  constexpr int WS = 5 * R2 > 5 * NPT * FMAX ? 5 * R2 : 5 * NPT * FMAX;
  static_assert(NT % 32 == 0, "tile must be whole warps");
  static_assert(NGF == 1 || NGF == 2, "face rule: 1 or 2 points per face dimension");
  (void)R1Z;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* s_w = reinterpret_cast<TC*>(smem_raw);  // 5 x R2 primitives, then face fluxes
  TC* s_f = s_w;
  TC* s_wp = s_w + WS;                        // 5 x R1 predicted centroid values
  TC* s_g = s_wp + 5 * R1;                    // 15 x R1 coefficients -> limited gradients
  int* s_gx = reinterpret_cast<int*>(s_g + 15 * R1);
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
  stage3d_issue<5, 15, TX, TY, TZ>(A.in, ncell, s_gx, s_gy, s_gz, s_g);
  for (int r = tid; r < R2; r += NT) {
    int rz = r / (R2X * R2Y), rr = r - rz * (R2X * R2Y);
    int ry = rr / R2X, rx = rr - ry * R2X;
    size_t g = (size_t)s_gz[rz] + s_gy[ry] + s_gx[rx];
    TC c[5], W[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) c[v] = Cvt<TC>::to_tc(__ldg(&A.in.c0[v * ncell + g]));
    prims3d<TC>(G, c, W, err);
#pragma unroll
    for (int q = 0; q < 5; ++q) s_w[q * R2 + r] = W[q];
  }
  cp_async_wait_all();
  __syncthreads();

  const TC dx = Cvt<TC>::to_tc(A.dx), dy = Cvt<TC>::to_tc(A.dy), dz = Cvt<TC>::to_tc(A.dz);
  const TC hh[3] = {TC(0.5) * dx, TC(0.5) * dy, TC(0.5) * dz};
  const TC oo[3] = {dx * TC(0.28867513459481288225), dy * TC(0.28867513459481288225),
                    dz * TC(0.28867513459481288225)};
  const TC hd[3] = {dx, dy, dz};

  // ---- 2. gradients, limiter, half-step prediction on the halo-1 box
  for (int r1 = tid; r1 < R1; r1 += NT) {
    int rz = r1 / (R1X * R1Y), rr = r1 - rz * (R1X * R1Y);
    int ry = rr / R1X, rx = rr - ry * R1X;
    int r2 = ((rz + 1) * R2Y + (ry + 1)) * R2X + (rx + 1);
    TC W[5], Wn[6][5], s[15], g[15], Wt[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      W[q] = s_w[q * R2 + r2];
      Wn[0][q] = s_w[q * R2 + r2 - 1];
      Wn[1][q] = s_w[q * R2 + r2 + 1];
      Wn[2][q] = s_w[q * R2 + r2 - R2X];
      Wn[3][q] = s_w[q * R2 + r2 + R2X];
      Wn[4][q] = s_w[q * R2 + r2 - R2X * R2Y];
      Wn[5][q] = s_w[q * R2 + r2 + R2X * R2Y];
    }
#pragma unroll
    for (int k = 0; k < 15; ++k) s[k] = s_g[k * R1 + r1];
    mh_grads3d<TC, WENO>(G, hh, W, Wn, A.limiter, s, g);
    mh_rates3d<TC>(G, W, g, Wt);
#pragma unroll
    for (int k = 0; k < 15; ++k) s_g[k * R1 + r1] = g[k];
#pragma unroll
    for (int q = 0; q < 5; ++q) s_wp[q * R1 + r1] = W[q] + hdt * Wt[q];
  }
  __syncthreads();  // the primitives are dead from here: their space takes the fluxes

  // ---- 3. per cell: volume integral of the predicted state's fluxes
  const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
  const int r1c = ((lz + 1) * R1Y + (ly + 1)) * R1X + (lx + 1);
  TC rc0[5], rs[15];
#pragma unroll
  for (int v = 0; v < 5; ++v) rc0[v] = TC(0);
  {
    TC sF[3][5];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v) sF[d][v] = TC(0);
#pragma unroll
    for (int qp = 0; qp < 8; ++qp) {
      TC W[5];
      mh_eval3d<TC>(s_wp + r1c, s_g + r1c, R1, (qp & 1) ? oo[0] : -oo[0],
                    (qp & 2) ? oo[1] : -oo[1], (qp & 4) ? oo[2] : -oo[2], W);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        TC F[5];
        prim_flux3d<TC>(G, W, d, F, err);
#pragma unroll
        for (int v = 0; v < 5; ++v) sF[d][v] += F[v];
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int d = 0; d < 3; ++d) rs[3 * v + d] = TC(1.5) / (hd[d] * hd[d]) * sF[d][v];
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
      TC WL[5], WR[5], F[5];
      mh_eval3d<TC>(s_wp + r1l, s_g + r1l, R1, xl, yl, zl, WL);
      mh_eval3d<TC>(s_wp + r1r, s_g + r1r, R1, xr, yr, zr, WR);
      face_flux_prim3d<TC>(G, d, WL, WR, F, err);
#pragma unroll
      for (int v = 0; v < 5; ++v) s_f[(v * FMAX + f) * NPT + g] = F[v];
    }
    __syncthreads();
    {
      const int fm = (lz * FY + ly) * FX + lx;
      const int fp = fm + (d == 0 ? 1 : (d == 1 ? FX : FX * FY));
      if (NPT == 4) {
        if (d == 0) gather3d<0, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
        else if (d == 1) gather3d<1, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
        else gather3d<2, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
      } else {
        if (d == 0) gather3d_centroid<0, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
        else if (d == 1) gather3d_centroid<1, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
        else gather3d_centroid<2, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
      }
    }
    __syncthreads();
  }

  // ---- 5. update of the limited coefficients, Courant speed of the new state
  const int gi = i0 + lx, gj = j0 + ly, gk = k0 + lz;
  const bool owner = gi < nx && gj < ny && gk < nz;
  const size_t gc = (size_t)s_gz[lz + 2] + s_gy[ly + 2] + s_gx[lx + 2];
  TC sn[15];
  if (A.limiter) {
    TC c[5], W[5], g[15];
#pragma unroll
    for (int v = 0; v < 5; ++v) c[v] = Cvt<TC>::to_tc(A.in.c0[v * ncell + gc]);
    prims3d<TC>(G, c, W, err);
#pragma unroll
    for (int k = 0; k < 15; ++k) g[k] = s_g[k * R1 + r1c];
    mh_cons3d<TC>(G, W, g, sn);
  } else {
#pragma unroll
    for (int k = 0; k < 15; ++k) sn[k] = (TC)A.in.sl[k * ncell + gc];
  }
  double o0[5];
  TC os[15];
#pragma unroll
  for (int v = 0; v < 5; ++v) o0[v] = fma(dt, Cvt<TC>::to_f64(rc0[v]), A.in.c0[v * ncell + gc]);
#pragma unroll
  for (int k = 0; k < 15; ++k) os[k] = sn[k] + dtc * rs[k];
  if (owner) {
#pragma unroll
    for (int v = 0; v < 5; ++v) A.out.c0[v * ncell + gc] = o0[v];
#pragma unroll
    for (int k = 0; k < 15; ++k) A.out.sl[k * ncell + gc] = (TS)os[k];
  }

  TC sp = TC(0);
  if (owner) {
    TC c[5], W[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) c[v] = Cvt<TC>::to_tc(o0[v]);
    prims3d<TC>(G, c, W, err);
    TC cs = sqrt(G.g * W[4] / W[0]);
    sp = (fabs(W[1]) + cs) / dx + (fabs(W[2]) + cs) / dy + (fabs(W[3]) + cs) / dz;
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
