// dg_stage2d.cuh -- one SSP-RK2 stage of the 2D P1 DG scheme (Euler or planar
// ideal MHD) as a single fused kernel.
//
// One CTA owns a TX x TY tile of cells.  It stages in shared memory the cell
// averages of the tile plus a halo of 2 cells and the derivative coefficients of
// the tile plus a halo of 1 cell (periodic wrap), then
//   1. centroid primitives of every staged cell,
//   2. the min/max limiter (Sec. 2.5) of the tile and its 1-cell ring, in place,
//   3. every face of the tile once: the two one-sided polynomials at the 2 Gauss
//      points, the Riemann flux (exact solver, or HLLD with the averaged normal
//      field of Sec. 2.6), kept in shared memory for both neighbours,
//   4. per cell: 2x2 Gauss volume integral of F . grad W, the face moments, the
//      (diagonal on a Cartesian cell) mass-matrix solve of Sec. 2.2, and the
//      Runge-Kutta combination;
//   stage 2 also reduces the Courant signal speed of the new state (warp shuffles,
//   one atomic per CTA; the last CTA publishes it for the next step).
//
// Right-hand sides, with S = F(g0) + F(g1) and D = F(g1) - F(g0) the sum and the
// difference of a face's two Gauss-point fluxes (g1 at the positive transverse
// coordinate), superscripts +/- the faces at +/- dx/2, dy/2, and sum_q the sum
// over the 4 volume Gauss points (the weak form of Sec. 2.2 on a Cartesian cell):
//   d avg/dt  = -(Sx+ - Sx-)/(2dx) - (Sy+ - Sy-)/(2dy)
//   d Ux/dt   = 3/dx^2 (sum_q Fx - (Sx+ + Sx-)) - sqrt3/(dx dy) (Dy+ - Dy-)
//   d Uy/dt   = 3/dy^2 (sum_q Fy - (Sy+ + Sy-)) - sqrt3/(dx dy) (Dx+ - Dx-)
//   magnetic block (x faces carry the By flux, y faces the Bx flux):
//   d b1/dt = -(Sy+ - Sy-)/(2dy),  d b2/dt = -(Sx+ - Sx-)/(2dx)
//   d a1/dt = 3/dy^2 (sum_q Fy(Bx) - (Sy+ + Sy-)),  d a2/dt = 3/dx^2 (sum_q Fx(By) - (Sx+ + Sx-))
//   d a3/dt = sqrt3/(dx^2+dy^2) ((dy/dx)(Dx+ - Dx-) - (dx/dy)(Dy+ - Dy-))
#pragma once

#include "dg_common.cuh"
#include "dg_physics.cuh"
#include "dg_weno.cuh"

namespace dgk {

template <int EQ> struct Tr2;
template <> struct Tr2<0> {  // Euler: (rho, mx, my, E)
  static constexpr int NV = 4, NS = 8, NP = 4, NF = 4;
};
template <> struct Tr2<1> {  // planar MHD: (rho, mx, my, E, b1, b2) + (.., a1, a2, a3)
  static constexpr int NV = 6, NS = 11, NP = 6, NF = 5;
};

// Shared-memory working set of one tile (element counts of the arithmetic type
// TC): averages [NV][R2], derivative coefficients [NS][R1], and one region that
// first holds the centroid primitives [NP][R2] and, once the limiter is done with
// them, the face fluxes [NF][(TX+1)TY][2] and [NF][TX(TY+1)][2].
template <int EQ, int TX, int TY>
struct Tile2D {
  using Tr = Tr2<EQ>;
  static constexpr int NV = Tr::NV, NS = Tr::NS, NP = Tr::NP, NF = Tr::NF;
  static constexpr int R2X = TX + 4, R2Y = TY + 4, R2 = R2X * R2Y;
  static constexpr int R1X = TX + 2, R1Y = TY + 2, R1 = R1X * R1Y;
  static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
  static constexpr int NT = TX * TY;
  static constexpr int WSZ = NP * R2 > NF * 2 * (NFX + NFY) ? NP * R2 : NF * 2 * (NFX + NFY);
  static constexpr int ELEMS = NV * R2 + NS * R1 + WSZ;
};

template <int EQ, int TX, int TY, class TC>
__host__ __device__ constexpr size_t stage2d_smem_bytes() {
  using T = Tile2D<EQ, TX, TY>;
  return size_t(T::ELEMS) * sizeof(TC) + sizeof(int) * (T::R2X + T::R2Y);
}

template <class TC>
struct TileMem {
  TC* c0;
  TC* sl;
  TC* w;  // primitives, then face fluxes
  int* gx;
  int* gy;
};

template <int EQ, int TX, int TY, class TC>
__device__ __forceinline__ TileMem<TC> tile_mem(unsigned char* base) {
  using T = Tile2D<EQ, TX, TY>;
  TileMem<TC> m;
  m.c0 = reinterpret_cast<TC*>(base);
  m.sl = m.c0 + T::NV * T::R2;
  m.w = m.sl + T::NS * T::R1;
  m.gx = reinterpret_cast<int*>(m.w + T::WSZ);
  m.gy = m.gx + T::R2X;
  return m;
}

// Per-tile scalars shared by the CTA.
template <int NT>
struct TileScalars {
  double dt;
  unsigned err;
  double red[NT / 32];
};

// Centroid primitives (rho, vx, vy, p[, Bx, By]) from averages.
template <int EQ, class TC>
__device__ __forceinline__ void prims2d(const Gas<TC>& G, const TC* c, TC* W, unsigned& err) {
  TC rho = c[0];
  TC inv = TC(1) / rho;
  TC vx = c[1] * inv, vy = c[2] * inv;
  TC kin = TC(0.5) * (c[1] * vx + c[2] * vy);
  TC mag = TC(0);
  if (EQ == 1) mag = TC(0.5) * (c[4] * c[4] + c[5] * c[5]);
  TC p = G.gm1 * (c[3] - kin - mag);
  if (!(rho > TC(0) && p > TC(0))) err |= ERR_NONPHYS;
  W[0] = rho; W[1] = vx; W[2] = vy; W[3] = p;
  if (EQ == 1) { W[4] = c[4]; W[5] = c[5]; }
}

// Limit the derivative coefficients s[] of one cell (Sec. 2.5): W its centroid
// primitives, Wn[k] those of its 4 face neighbours.  Slope order: (rho, mx, my,
// E) x (d/dx, d/dy), then a1, a2, a3 for MHD.
template <int EQ, class TC>
__device__ __forceinline__ void limit_cell2d(const Gas<TC>& G, const TC* hh, const TC* W,
                                             const TC (*Wn)[Tr2<EQ>::NP], TC* s) {
  constexpr int NP = Tr2<EQ>::NP;
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
  TC gr[2], gvx[2], gvy[2], gp[2], gbx[2], gby[2];
  if (EQ == 1) {
    gbx[0] = s[10]; gbx[1] = s[8];   // dBx/dx = a3, dBx/dy = a1
    gby[0] = s[9]; gby[1] = -s[10];  // dBy/dx = a2, dBy/dy = -a3
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
  const TC ar = limiter_alpha<TC, 2>(W[0], hi[0], lo[0], gr, hh);
  const TC avx = limiter_alpha<TC, 2>(W[1], hi[1], lo[1], gvx, hh);
  const TC avy = limiter_alpha<TC, 2>(W[2], hi[2], lo[2], gvy, hh);
  const TC ap = limiter_alpha<TC, 2>(W[3], hi[3], lo[3], gp, hh);
  TC aB = TC(1);
  if (EQ == 1) {
    TC abx = limiter_alpha<TC, 2>(W[4], hi[4], lo[4], gbx, hh);
    TC aby = limiter_alpha<TC, 2>(W[5], hi[5], lo[5], gby, hh);
    aB = abx < aby ? abx : aby;
  }
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    TC r = ar * gr[d], ux = avx * gvx[d], uy = avy * gvy[d], pp = ap * gp[d];
    TC BdB = TC(0);
    if (EQ == 1) BdB = aB * (W[4] * gbx[d] + W[5] * gby[d]);
    s[d] = r;
    s[2 + d] = rho * ux + vx * r;
    s[4 + d] = rho * uy + vy * r;
    s[6 + d] = pp * G.inv_gm1 + v2h * r + rho * (vx * ux + vy * uy) + BdB;
  }
  if (EQ == 1) {
    s[8] *= aB; s[9] *= aB; s[10] *= aB;
  }
}

// Physical fluxes along x and y of a state given by conserved values c[] (rho,
// mx, my, E[, Bx, By]).  Output in face-flux component order: (rho, mx, my, E[,
// transverse field]) where the transverse field is By for x, Bx for y.
template <int EQ, class TC>
__device__ __forceinline__ void phys_flux2d(const Gas<TC>& G, const TC* c, TC* Fx, TC* Fy,
                                            unsigned& err) {
  TC rho = c[0], inv = TC(1) / rho;
  TC vx = c[1] * inv, vy = c[2] * inv;
  TC bx = TC(0), by = TC(0), b2h = TC(0);
  if (EQ == 1) { bx = c[4]; by = c[5]; b2h = TC(0.5) * (bx * bx + by * by); }
  TC p = G.gm1 * (c[3] - TC(0.5) * (c[1] * vx + c[2] * vy) - b2h);
  if (!(rho > TC(0) && p > TC(0))) err |= ERR_NONPHYS;
  TC pT = p + b2h;
  TC e = c[3] + pT;
  Fx[0] = c[1];
  Fy[0] = c[2];
  if (EQ == 0) {
    Fx[1] = c[1] * vx + p; Fx[2] = c[2] * vx; Fx[3] = e * vx;
    Fy[1] = c[1] * vy; Fy[2] = c[2] * vy + p; Fy[3] = e * vy;
  } else {
    TC vB = vx * bx + vy * by;
    Fx[1] = c[1] * vx + pT - bx * bx; Fx[2] = c[2] * vx - bx * by; Fx[3] = e * vx - bx * vB;
    Fx[4] = by * vx - vy * bx;
    Fy[1] = c[1] * vy - bx * by; Fy[2] = c[2] * vy + pT - by * by; Fy[3] = e * vy - by * vB;
    Fy[4] = bx * vy - vx * by;
  }
}

// Conserved values of the cell polynomial at local point (x, y): averages c0[],
// derivative coefficients s[] in the slope order of limit_cell2d.
template <int EQ, class TC>
__device__ __forceinline__ void eval2d(const TC* c0, const TC* s, TC x, TC y, TC* c) {
#pragma unroll
  for (int v = 0; v < 4; ++v) c[v] = c0[v] + s[2 * v] * x + s[2 * v + 1] * y;
  if (EQ == 1) {
    c[4] = c0[4] + s[10] * x + s[8] * y;
    c[5] = c0[5] + s[9] * x - s[10] * y;
  }
}

// Riemann flux at one Gauss point of a face along axis `dir` (0: x, 1: y)
// between conserved states cl (left/lower) and cr; lab-frame output in face-flux
// component order.
template <int EQ, class TC>
__device__ __forceinline__ void face_flux2d(const Gas<TC>& G, int dir, const TC* cl,
                                            const TC* cr, TC* F, unsigned& err) {
  TC rl = cl[0], rr = cr[0];
  TC il = TC(1) / rl, ir = TC(1) / rr;
  TC vxl = cl[1] * il, vyl = cl[2] * il, vxr = cr[1] * ir, vyr = cr[2] * ir;
  TC magl = TC(0), magr = TC(0);
  if (EQ == 1) {
    magl = TC(0.5) * (cl[4] * cl[4] + cl[5] * cl[5]);
    magr = TC(0.5) * (cr[4] * cr[4] + cr[5] * cr[5]);
  }
  TC pl = G.gm1 * (cl[3] - TC(0.5) * (cl[1] * vxl + cl[2] * vyl) - magl);
  TC pr = G.gm1 * (cr[3] - TC(0.5) * (cr[1] * vxr + cr[2] * vyr) - magr);
  // the face frame's normal and transverse components, picked with selects so
  // that the solver is inlined once for both orientations
  const bool xd = dir == 0;
  const TC unl = xd ? vxl : vyl, utl = xd ? vyl : vxl;
  const TC unr = xd ? vxr : vyr, utr = xd ? vyr : vxr;
  TC Ff[5];
  if (EQ == 0) {
    exact_flux<TC, 1>(G, rl, unl, pl, &utl, rr, unr, pr, &utr, Ff, err);
  } else {
    const TC bn = TC(0.5) * (xd ? cl[4] + cr[4] : cl[5] + cr[5]);
    hlld_flux<TC>(G, rl, unl, utl, pl, xd ? cl[5] : cl[4], rr, unr, utr, pr, xd ? cr[5] : cr[4],
                  bn, Ff, err);
    F[4] = Ff[4];
  }
  F[0] = Ff[0];
  F[3] = Ff[3];
  if (dir == 0) { F[1] = Ff[1]; F[2] = Ff[2]; }
  else { F[1] = Ff[2]; F[2] = Ff[1]; }
}

// Start of a tile: the time step, the error word, and the wrapped global row and
// column offsets of the halo-2 region.  The caller synchronises afterwards.
template <int EQ, class TC, class TS, int TX, int TY>
__device__ __forceinline__ void stage2d_setup(const Stage2DArgs<TS>& A, int i0, int j0,
                                              const TileMem<TC>& M, TileScalars<TX * TY>& S) {
  using T = Tile2D<EQ, TX, TY>;
  const int tid = threadIdx.x;
  if (tid == 0) {
    S.err = 0;
    double dt = A.dt_override > 0.0 ? A.dt_override : A.ctl->dt_cur;
    if (!(dt > 0.0) || !(dt < 1e300)) S.err |= ERR_NONPHYS;
    S.dt = dt;
  }
  if (tid < T::R2X) M.gx[tid] = wrap_index(i0 - 2 + tid, A.nx);
  else if (tid < T::R2X + T::R2Y) M.gy[tid - T::R2X] = wrap_index(j0 - 2 + (tid - T::R2X), A.ny) * A.nx;
}

// Stage the tile from global memory (periodic wrap): averages with halo 2,
// derivative coefficients with halo 1.  The staged arrays are walked as rows of
// RX cells: thread t takes column t % RX of every C-th row from row t / RX on
// (C = NT / RX rows per pass), so its column's global offset is looked up once
// and a row costs one lookup of the row offset.  Every load of a thread is in
// flight before the first one is used, so that their DRAM latencies overlap:
// plain copies go through cp.async, and the FP64 averages of the FP32 path are
// loaded into registers in chunks of 8 passes and converted after each chunk.
// The caller synchronises.
template <int EQ, class TC, class TS, int TX, int TY>
__device__ __forceinline__ void stage2d_load(const Stage2DArgs<TS>& A, const TileMem<TC>& M) {
  using T = Tile2D<EQ, TX, TY>;
  static_assert(sizeof(TS) == sizeof(TC), "derivative coefficients are staged as stored");
  constexpr int C1 = T::NT / T::R1X, C0 = T::NT / T::R2X;
  static_assert(C1 >= 1 && C1 <= T::R1Y && C0 >= 1 && C0 <= T::R2Y,
                "a pass of rows advances by at most one variable");
  const size_t ncell = (size_t)A.ncell;
  const int tid = threadIdx.x;
  {  // derivative coefficients: rows (v, ry) of the halo-1 region
    const int rx = tid % T::R1X, row0 = tid / T::R1X;
    if (row0 < C1) {
      const TS* src = A.in.sl + M.gx[rx + 1];
      size_t voff = 0;
      int ry = row0;
      for (int row = row0; row < T::NS * T::R1Y; row += C1) {
        cp_async_elem<sizeof(TS)>(&M.sl[row * T::R1X + rx], src + voff + M.gy[ry + 1]);
        ry += C1;
        if (ry >= T::R1Y) { ry -= T::R1Y; voff += ncell; }
      }
    }
  }
  {  // averages: rows (v, ry) of the halo-2 region
    constexpr int ROWS = T::NV * T::R2Y, P = (ROWS + C0 - 1) / C0, CH = 8;
    const int rx = tid % T::R2X, row0 = tid / T::R2X;
    if (row0 < C0) {
      const double* src = A.in.c0 + M.gx[rx];
      TC* dst = M.c0 + row0 * T::R2X + rx;
      size_t voff = 0;
      int ry = row0;
      if constexpr (sizeof(TC) == 8) {
        for (int p = 0; p < P && row0 + p * C0 < ROWS; ++p) {
          cp_async_elem<8>(dst + p * C0 * T::R2X, src + voff + M.gy[ry]);
          ry += C0;
          if (ry >= T::R2Y) { ry -= T::R2Y; voff += ncell; }
        }
      } else {
#pragma unroll
        for (int p0 = 0; p0 < P; p0 += CH) {
          double a[CH];
#pragma unroll
          for (int i = 0; i < CH; ++i) {
            if (p0 + i < P && row0 + (p0 + i) * C0 < ROWS) {
              a[i] = __ldg(src + voff + M.gy[ry]);
              ry += C0;
              if (ry >= T::R2Y) { ry -= T::R2Y; voff += ncell; }
            }
          }
#pragma unroll
          for (int i = 0; i < CH; ++i)
            if (p0 + i < P && row0 + (p0 + i) * C0 < ROWS)
              dst[(p0 + i) * C0 * T::R2X] = Cvt<TC>::to_tc(a[i]);
        }
      }
    }
  }
  cp_async_wait_all();
}

// Stage 2 reads the step's input state U^n of its own cell only at the end (the
// Runge-Kutta combination): request those lines into L2 while the tile stages.
template <int EQ, class TC, class TS, int TX, int TY>
__device__ __forceinline__ void stage2d_prefetch_base(const Stage2DArgs<TS>& A,
                                                      const TileMem<TC>& M) {
  using T = Tile2D<EQ, TX, TY>;
  const size_t ncell = (size_t)A.ncell;
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  const size_t gc = (size_t)M.gy[ly + 2] + M.gx[lx + 2];
  const TS* sl = A.limiter && A.lim_sl ? A.lim_sl : A.base.sl;
#pragma unroll
  for (int v = 0; v < T::NV; ++v) prefetch_l2(&A.base.c0[v * ncell + gc]);
#pragma unroll
  for (int k = 0; k < T::NS; ++k) prefetch_l2(&sl[k * ncell + gc]);
}

// End of a step on one tile: the Courant signal speed of the new averages o0[]
// of this thread's cell, reduced over the grid (in TC; the CTA maximum is widened
// to FP64 for the grid-wide atomic maximum); the last CTA of the grid to finish
// publishes it for the next step and advances the time.  Also commits the error
// word.
template <int EQ, class TC, class TS, int NT>
__device__ __forceinline__ void courant_commit2d(const Stage2DArgs<TS>& A, const Gas<TC>& G,
                                                 bool owner, const double* o0, TC dx, TC dy,
                                                 double dt, unsigned nblk, unsigned err,
                                                 TileScalars<NT>& S) {
  constexpr int NV = Tr2<EQ>::NV, NP = Tr2<EQ>::NP;
  const int tid = threadIdx.x;
  // Courant signal speed of the new state, reduced over the grid (in TC; the
  // CTA maximum is widened to FP64 for the grid-wide atomic maximum)
  TC sp = TC(0);
  if (owner) {
    TC c[NV], W[NP];
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = Cvt<TC>::to_tc(o0[v]);
    prims2d<EQ, TC>(G, c, W, err);
    TC cx, cy;
    if (EQ == 0) {
      cx = cy = sqrt(G.g * W[3] / W[0]);
    } else {
      TC b2 = W[4] * W[4] + W[5] * W[5];
      cx = fast_speed(G, W[0], W[3], b2, W[4]);
      cy = fast_speed(G, W[0], W[3], b2, W[5]);
    }
    sp = (fabs(W[1]) + cx) / dx + (fabs(W[2]) + cy) / dy;
    if (!courant_ok(sp, W[0], W[3])) { err |= ERR_NONPHYS; sp = TC(0); }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    TC t = __shfl_xor_sync(0xffffffffu, sp, o);
    sp = t > sp ? t : sp;
  }
  if ((tid & 31) == 0) S.red[tid >> 5] = Cvt<TC>::to_f64(sp);
  if (err) atomicOr(&S.err, err);
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < NT / 32; ++w) m = S.red[w] > m ? S.red[w] : m;
    Ctl* ctl = A.ctl;
    atomicMax(&ctl->vmax_next, (unsigned long long)__double_as_longlong(m));
    if (S.err) atomicOr(&ctl->err, S.err);
    __threadfence();
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

// The rest of a tile once it is staged: primitives, limiter, faces, per-cell
// right-hand side and Runge-Kutta combination; `nblk` is the number of tiles of
// the problem (the last of them to finish stage 2 publishes the Courant speed).
// WENO = false compiles the WENO-type limiter out (for launches with limiter 0
// or 1: its code raises the registers and stack of the common path).
// `ph` (profiling build): phases 1 primitives, 2 limiter, 3 faces, 4 per-cell
// right-hand side and combination, 5 Courant reduction and commit.
template <int EQ, class TC, class TS, int TX, int TY, int STAGE, bool WENO = true>
__device__ __forceinline__ void stage2d_compute(const Stage2DArgs<TS>& A, int i0, int j0,
                                                unsigned nblk, const TileMem<TC>& M,
                                                TileScalars<TX * TY>& S,
                                                PhaseStamp* ph = nullptr) {
  using Tr = Tr2<EQ>;
  constexpr int NV = Tr::NV, NS = Tr::NS, NP = Tr::NP, NF = Tr::NF;
  constexpr int R2X = TX + 4, R2Y = TY + 4, R2 = R2X * R2Y;
  constexpr int R1X = TX + 2, R1Y = TY + 2, R1 = R1X * R1Y;
  constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
  constexpr int NT = TX * TY;
  static_assert(NT % 32 == 0, "tile must be whole warps");
  (void)R2Y;
  (void)R1Y;
  TC* s_c0 = M.c0;
  TC* s_w = M.w;
  TC* s_sl = M.sl;
  TC* s_fx = M.w;
  TC* s_fy = M.w + NF * 2 * NFX;
  const int* s_gx = M.gx;
  const int* s_gy = M.gy;

  const int tid = threadIdx.x;
  const int nx = A.nx, ny = A.ny;
  const size_t ncell = (size_t)A.ncell;
  const Gas<TC> G = gas_of<TC>(A.gas);
  unsigned err = 0;

  // ---- centroid primitives of every staged cell
  for (int r = tid; r < R2; r += NT) {
    TC c[NV], W[NP];
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = s_c0[v * R2 + r];
    prims2d<EQ, TC>(G, c, W, err);
#pragma unroll
    for (int q = 0; q < NP; ++q) s_w[q * R2 + r] = W[q];
  }
  __syncthreads();
  if (ph) ph->mark(1);

  const TC dx = Cvt<TC>::to_tc(A.dx), dy = Cvt<TC>::to_tc(A.dy);
  TC hh[2] = {TC(0.5) * dx, TC(0.5) * dy};

  // ---- limiter on the tile and its 1-cell ring, in place
  if (A.limiter) {
    for (int r1 = tid; r1 < R1; r1 += NT) {
      int ry = r1 / R1X, rx = r1 - ry * R1X;
      int r2 = (ry + 1) * R2X + (rx + 1);
      TC W[NP], Wn[4][NP], s[NS];
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
      if (WENO && A.limiter == 2) weno_cell2d<EQ, TC>(G, hh, W, Wn, s, nullptr);
      else limit_cell2d<EQ, TC>(G, hh, W, Wn, s);
#pragma unroll
      for (int k = 0; k < NS; ++k) s_sl[k * R1 + r1] = s[k];
    }
  }
  __syncthreads();  // the primitives are dead from here: their space takes the fluxes
  if (ph) ph->mark(2);

  // ---- faces: Riemann fluxes at the Gauss points, each face once
  const TC ox = dx * TC(0.28867513459481288225), oy = dy * TC(0.28867513459481288225);
  for (int e = tid; e < 2 * (NFX + NFY); e += NT) {
    const bool xf = e < 2 * NFX;
    const int ee = xf ? e : e - 2 * NFX;
    const int f = ee >> 1, g = ee & 1;
    int r1l, r1r;
    TC xl, yl, xr, yr;
    if (xf) {
      int fy = f / (TX + 1), fx = f - fy * (TX + 1);
      r1l = (fy + 1) * R1X + fx;
      r1r = r1l + 1;
      TC t = g ? oy : -oy;
      xl = hh[0]; xr = -hh[0]; yl = t; yr = t;
    } else {
      int fy = f / TX, fx = f - fy * TX;
      r1l = fy * R1X + fx + 1;
      r1r = r1l + R1X;
      TC t = g ? ox : -ox;
      yl = hh[1]; yr = -hh[1]; xl = t; xr = t;
    }
    const int r2l = (r1l / R1X + 1) * R2X + (r1l % R1X) + 1;
    const int r2r = (r1r / R1X + 1) * R2X + (r1r % R1X) + 1;
    TC c0l[NV], c0r[NV], sl[NS], sr[NS], cl[NV], cr[NV], F[NF];
#pragma unroll
    for (int v = 0; v < NV; ++v) { c0l[v] = s_c0[v * R2 + r2l]; c0r[v] = s_c0[v * R2 + r2r]; }
#pragma unroll
    for (int k = 0; k < NS; ++k) { sl[k] = s_sl[k * R1 + r1l]; sr[k] = s_sl[k * R1 + r1r]; }
    eval2d<EQ, TC>(c0l, sl, xl, yl, cl);
    eval2d<EQ, TC>(c0r, sr, xr, yr, cr);
    face_flux2d<EQ, TC>(G, xf ? 0 : 1, cl, cr, F, err);
    if (xf) {
#pragma unroll
      for (int q = 0; q < NF; ++q) s_fx[(q * NFX + f) * 2 + g] = F[q];
    } else {
#pragma unroll
      for (int q = 0; q < NF; ++q) s_fy[(q * NFY + f) * 2 + g] = F[q];
    }
  }
  __syncthreads();
  if (ph) ph->mark(3);

  // ---- per cell: volume integral, face moments, mass matrix, RK combination
  const int lx = tid % TX, ly = tid / TX;
  const int gi = i0 + lx, gj = j0 + ly;
  const bool owner = gi < nx && gj < ny;
  const int r2 = (ly + 2) * R2X + lx + 2, r1 = (ly + 1) * R1X + lx + 1;
  const size_t gc = (size_t)s_gy[ly + 2] + s_gx[lx + 2];
  const double dt = S.dt;
  const TC dtc = Cvt<TC>::to_tc(dt);
  TC c0[NV], s[NS];
#pragma unroll
  for (int v = 0; v < NV; ++v) c0[v] = s_c0[v * R2 + r2];
#pragma unroll
  for (int k = 0; k < NS; ++k) s[k] = s_sl[k * R1 + r1];

  TC sFx[NF], sFy[NF];
#pragma unroll
  for (int q = 0; q < NF; ++q) { sFx[q] = TC(0); sFy[q] = TC(0); }
#pragma unroll
  for (int qp = 0; qp < 4; ++qp) {
    TC c[NV], Fx[NF], Fy[NF];
    eval2d<EQ, TC>(c0, s, (qp & 1) ? ox : -ox, (qp & 2) ? oy : -oy, c);
    phys_flux2d<EQ, TC>(G, c, Fx, Fy, err);
#pragma unroll
    for (int q = 0; q < NF; ++q) { sFx[q] += Fx[q]; sFy[q] += Fy[q]; }
  }

  const int fxm = ly * (TX + 1) + lx, fym = ly * TX + lx;
  TC Sxm[NF], Sxp[NF], Dxm[NF], Dxp[NF], Sym[NF], Syp[NF], Dym[NF], Dyp[NF];
#pragma unroll
  for (int q = 0; q < NF; ++q) {
    TC a0 = s_fx[(q * NFX + fxm) * 2], a1 = s_fx[(q * NFX + fxm) * 2 + 1];
    TC b0 = s_fx[(q * NFX + fxm + 1) * 2], b1 = s_fx[(q * NFX + fxm + 1) * 2 + 1];
    Sxm[q] = a0 + a1; Dxm[q] = a1 - a0; Sxp[q] = b0 + b1; Dxp[q] = b1 - b0;
    a0 = s_fy[(q * NFY + fym) * 2]; a1 = s_fy[(q * NFY + fym) * 2 + 1];
    b0 = s_fy[(q * NFY + fym + TX) * 2]; b1 = s_fy[(q * NFY + fym + TX) * 2 + 1];
    Sym[q] = a0 + a1; Dym[q] = a1 - a0; Syp[q] = b0 + b1; Dyp[q] = b1 - b0;
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

  double o0[NV];
  TC os[NS];
  if (STAGE == 1) {
    // V^1 = U^n + dt L(U^n), U^n = limited V^n
#pragma unroll
    for (int v = 0; v < NV; ++v) o0[v] = fma(dt, Cvt<TC>::to_f64(rc0[v]), A.in.c0[v * ncell + gc]);
#pragma unroll
    for (int k = 0; k < NS; ++k) os[k] = s[k] + dtc * rs[k];
    if (A.limiter && A.lim_sl && owner) {
#pragma unroll
      for (int k = 0; k < NS; ++k) A.lim_sl[k * ncell + gc] = (TS)s[k];
    }
  } else {
    // V^{n+1} = 1/2 U^n + 1/2 (U^1 + dt L(U^1)), U^n = limited V^n of this cell
    TC sn[NS];
    if (A.limiter && A.lim_sl) {
      // limited by stage 1 of this step
#pragma unroll
      for (int k = 0; k < NS; ++k) sn[k] = (TC)A.lim_sl[k * ncell + gc];
    } else {
#pragma unroll
      for (int k = 0; k < NS; ++k) sn[k] = (TC)A.base.sl[k * ncell + gc];
    }
    if (A.limiter && !A.lim_sl) {
      TC cn[NV], W[NP], Wn[4][NP];
#pragma unroll
      for (int v = 0; v < NV; ++v) cn[v] = Cvt<TC>::to_tc(A.base.c0[v * ncell + gc]);
      prims2d<EQ, TC>(G, cn, W, err);
      const size_t nb[4] = {(size_t)s_gy[ly + 2] + s_gx[lx + 1], (size_t)s_gy[ly + 2] + s_gx[lx + 3],
                            (size_t)s_gy[ly + 1] + s_gx[lx + 2], (size_t)s_gy[ly + 3] + s_gx[lx + 2]};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        TC c[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) c[v] = Cvt<TC>::to_tc(A.base.c0[v * ncell + nb[k]]);
        prims2d<EQ, TC>(G, c, Wn[k], err);
      }
      if (WENO && A.limiter == 2) weno_cell2d<EQ, TC>(G, hh, W, Wn, sn, nullptr);
      else limit_cell2d<EQ, TC>(G, hh, W, Wn, sn);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
      o0[v] = half_f64(A.base.c0[v * ncell + gc] +
                       fma(dt, Cvt<TC>::to_f64(rc0[v]), A.in.c0[v * ncell + gc]));
#pragma unroll
    for (int k = 0; k < NS; ++k) os[k] = TC(0.5) * sn[k] + TC(0.5) * (s[k] + dtc * rs[k]);
  }
  if (owner) {
#pragma unroll
    for (int v = 0; v < NV; ++v) A.out.c0[v * ncell + gc] = o0[v];
#pragma unroll
    for (int k = 0; k < NS; ++k) A.out.sl[k * ncell + gc] = (TS)os[k];
  }

  if (ph) ph->mark(4);
  if (STAGE == 2) {
    courant_commit2d<EQ, TC, TS, NT>(A, G, owner, o0, dx, dy, dt, nblk, err, S);
  } else {
    if (err) atomicOr(&S.err, err);
    __syncthreads();
    if (tid == 0 && S.err) atomicOr(&A.ctl->err, S.err);
  }
  if (ph) ph->mark(5);
}



// One tile of one stage (classic staging): the CTA owns cells [i0, i0+TX) x
// [j0, j0+TY) of the problem described by A.
template <int EQ, class TC, class TS, int TX, int TY, int STAGE, bool WENO = true>
__device__ __forceinline__ void stage2d_tile(const Stage2DArgs<TS>& A, int i0, int j0,
                                             unsigned nblk, unsigned char* smem_raw) {
  __shared__ TileScalars<TX * TY> S;
  PhaseStamp ph;  // phase 0: set-up and staging (profiling build)
  ph.begin(A.phase, STAGE);
  const TileMem<TC> M = tile_mem<EQ, TX, TY, TC>(smem_raw);
  stage2d_setup<EQ, TC, TS, TX, TY>(A, i0, j0, M, S);
  __syncthreads();
  if (STAGE == 2) stage2d_prefetch_base<EQ, TC, TS, TX, TY>(A, M);
  stage2d_load<EQ, TC, TS, TX, TY>(A, M);
  __syncthreads();
  ph.mark(0);
  stage2d_compute<EQ, TC, TS, TX, TY, STAGE, WENO>(A, i0, j0, nblk, M, S, &ph);
}

// FP32: as many resident CTAs as 72 registers a thread allow for 128-thread
// tiles (7 CTAs) and 64 for 256-thread tiles (4 CTAs, which their shared memory
// also allows; measured +3 % over 80 registers and 3 CTAs despite 16-80 bytes of
// spills): the stage kernels are issue and latency bound.  FP64 keeps its
// registers (it would spill).
template <int NT, class TC>
struct StageMinBlocks {
  static constexpr int R = NT >= 256 ? 64 : 72;
  static constexpr int v = sizeof(TC) == 4 && 65536 / (R * NT) > 0 ? 65536 / (R * NT) : 1;
};

template <int EQ, class TC, class TS, int TX, int TY, int STAGE, bool WENO>
__global__ void __launch_bounds__(TX * TY, (StageMinBlocks<TX * TY, TC>::v))
    stage2d_kernel(const Stage2DArgs<TS> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // launched as a programmatic dependent of the previous stage: everything of the
  // tile reads that stage's output, so wait for it before anything else
  griddep_launch_dependents();
  griddep_wait();
  stage2d_tile<EQ, TC, TS, TX, TY, STAGE, WENO>(A, blockIdx.x * TX, blockIdx.y * TY,
                                          gridDim.x * gridDim.y, smem_raw);
}

}  // namespace dgk
