// dg_stage3d.cuh -- one SSP-RK2 stage of the 3D P1 DG scheme for the Euler
// equations (Taylor basis 1, x, y, z; Sec. 2.2 eqs. `fv3d`, `dgderiv3d`) as one
// fused kernel.
//
// One CTA owns a TX x TY x TZ tile.  Shared memory holds the centroid primitives
// of the cells the limiter's neighbour extrema read (the tile plus a halo of 1
// cell, and one more layer beyond each face of the tile), the averages and
// derivative coefficients of the tile plus a halo of 1 cell, and one
// face-flux buffer.  After the limiter (Sec. 2.5) has been applied in place to the
// tile and its ring, the faces of each orientation are processed in turn: the
// Riemann flux at the 2x2 Gauss points of every face of that orientation is
// computed once into the buffer, then every cell adds its two faces to the
// right-hand side it keeps in registers.
//
// With S = sum of a face's 4 Gauss-point fluxes and D_e = the difference between
// the points on the + and - side of the transverse axis e, superscripts +/- the
// faces at +/- dx_d/2, and sum_q over the 8 volume Gauss points:
//   d avg/dt     += -(S+ - S-) / (4 dx_d)
//   d U_d/dt     += 3/(2 dx_d^2) (sum_q F_d - (S+ + S-))
//   d U_e/dt     += -sqrt3/(2 dx_e dx_d) (D_e+ - D_e-)       (e != d)
#pragma once

#include "dg_common.cuh"
#include "dg_physics.cuh"
#include "dg_weno.cuh"

namespace dgk {

template <int TX, int TY, int TZ, class TC>
__host__ __device__ constexpr int stage3d_face_max() {
  return ((TX + 1) * TY * TZ > TX * (TY + 1) * TZ)
             ? (((TX + 1) * TY * TZ > TX * TY * (TZ + 1)) ? (TX + 1) * TY * TZ
                                                          : TX * TY * (TZ + 1))
             : ((TX * (TY + 1) * TZ > TX * TY * (TZ + 1)) ? TX * (TY + 1) * TZ
                                                          : TX * TY * (TZ + 1));
}

// The primitives (laid out as the halo-2 box [5][R2], of which the cells of
// halo3d_cell are written) are dead once the limiter has run; the face fluxes [5][4][FMAX] then reuse their space.
template <int TX, int TY, int TZ, class TC>
__host__ __device__ constexpr size_t stage3d_wsz() {
  return (size_t(5) * (TX + 4) * (TY + 4) * (TZ + 4) > size_t(5) * 4 * stage3d_face_max<TX, TY, TZ, TC>()
              ? size_t(5) * (TX + 4) * (TY + 4) * (TZ + 4) + 3
              : size_t(5) * 4 * stage3d_face_max<TX, TY, TZ, TC>() + 3) / 4 * 4;
}

template <int TX, int TY, int TZ, class TC>
__host__ __device__ constexpr size_t stage3d_smem_bytes() {
  return (stage3d_wsz<TX, TY, TZ, TC>() + size_t(20) * (TX + 2) * (TY + 2) * (TZ + 2)) * sizeof(TC) +
         sizeof(int) * ((TX + 4) + (TY + 4) + (TZ + 4));
}

template <class TC>
__device__ __forceinline__ void prims3d(const Gas<TC>& G, const TC* c, TC* W, unsigned& err) {
  TC rho = c[0], inv = TC(1) / rho;
  TC vx = c[1] * inv, vy = c[2] * inv, vz = c[3] * inv;
  TC p = G.gm1 * (c[4] - TC(0.5) * (c[1] * vx + c[2] * vy + c[3] * vz));
  if (!(rho > TC(0) && p > TC(0))) err |= ERR_NONPHYS;
  W[0] = rho; W[1] = vx; W[2] = vy; W[3] = vz; W[4] = p;
}

// Limit the 15 derivative coefficients s[v*3+d] of one cell; W its centroid
// primitives, Wn[k] those of its 6 face neighbours.
template <class TC>
__device__ __forceinline__ void limit_cell3d(const Gas<TC>& G, const TC* hh, const TC* W,
                                             const TC (*Wn)[5], TC* s) {
  TC hi[5], lo[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
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
  TC gr[3], gv[3][3], gp[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    gr[d] = s[d];
    TC vdv = TC(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      gv[i][d] = (s[3 * (1 + i) + d] - v[i] * gr[d]) * inv;
      vdv += v[i] * gv[i][d];
    }
    gp[d] = G.gm1 * (s[12 + d] - v2h * gr[d] - rho * vdv);
  }
  const TC ar = limiter_alpha<TC, 3>(W[0], hi[0], lo[0], gr, hh);
  TC av[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) av[i] = limiter_alpha<TC, 3>(W[1 + i], hi[1 + i], lo[1 + i], gv[i], hh);
  const TC ap = limiter_alpha<TC, 3>(W[4], hi[4], lo[4], gp, hh);
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
    s[12 + d] = ap * gp[d] * G.inv_gm1 + v2h * r + rho * vdv;
  }
}

template <class TC>
__device__ __forceinline__ void eval3d(const TC* c0, const TC* s, TC x, TC y, TC z, TC* c) {
#pragma unroll
  for (int v = 0; v < 5; ++v) c[v] = c0[v] + s[3 * v] * x + s[3 * v + 1] * y + s[3 * v + 2] * z;
}

// A staged cell of the 3D Euler tile as one record of 20 elements (16-byte
// aligned): the 5 averages, then the 15 derivative coefficients in slope order,
// so that a thread reads a cell with 5 (FP32) or 10 (FP64) 16-byte shared loads;
// at a stride of 20 words the 8 threads of each phase of such a load hit
// disjoint banks.
constexpr int kRec3d = 20;
template <class TC>
__device__ __forceinline__ void rec_get(const TC* rec, TC* v) {
  if constexpr (sizeof(TC) == 4) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const float4 q = reinterpret_cast<const float4*>(rec)[i];
      v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
      const double2 q = reinterpret_cast<const double2*>(rec)[i];
      v[2 * i] = q.x; v[2 * i + 1] = q.y;
    }
  }
}
template <class TC>
__device__ __forceinline__ void rec_put(TC* rec, const TC* v) {
  if constexpr (sizeof(TC) == 4) {
#pragma unroll
    for (int i = 0; i < 5; ++i)
      reinterpret_cast<float4*>(rec)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < 10; ++i) reinterpret_cast<double2*>(rec)[i] = make_double2(v[2 * i], v[2 * i + 1]);
  }
}

// Physical flux along axis d of conserved (rho, m, E).
template <class TC>
__device__ __forceinline__ void phys_flux3d(const Gas<TC>& G, const TC* c, int d, TC* F,
                                            unsigned& err) {
  TC rho = c[0], inv = TC(1) / rho;
  TC v[3] = {c[1] * inv, c[2] * inv, c[3] * inv};
  TC p = G.gm1 * (c[4] - TC(0.5) * (c[1] * v[0] + c[2] * v[1] + c[3] * v[2]));
  if (!(rho > TC(0) && p > TC(0))) err |= ERR_NONPHYS;
  TC vd = v[d];
  F[0] = c[1 + d];
  F[1] = c[1] * vd;
  F[2] = c[2] * vd;
  F[3] = c[3] * vd;
  F[1 + d] += p;
  F[4] = (c[4] + p) * vd;
}

// Exact-solver flux through a face along axis d (0, 1, 2; uniform across the
// CTA) between conserved cl, cr; lab frame (rho, mx, my, mz, E).  Normal and
// transverse components are picked with selects, so one inlined copy of the
// solver serves all three orientations.
template <class TC>
__device__ __forceinline__ void face_flux3d(const Gas<TC>& G, int d, const TC* cl, const TC* cr,
                                            TC* F, unsigned& err) {
  TC il = TC(1) / cl[0], ir = TC(1) / cr[0];
  TC lx = cl[1] * il, ly = cl[2] * il, lz = cl[3] * il;
  TC rx = cr[1] * ir, ry = cr[2] * ir, rz = cr[3] * ir;
  TC pl = G.gm1 * (cl[4] - TC(0.5) * (cl[1] * lx + cl[2] * ly + cl[3] * lz));
  TC pr = G.gm1 * (cr[4] - TC(0.5) * (cr[1] * rx + cr[2] * ry + cr[3] * rz));
  // normal n, transverse t1 (x unless d == 0), t2 (z unless d == 2)
  const TC nl = d == 0 ? lx : (d == 1 ? ly : lz), nr = d == 0 ? rx : (d == 1 ? ry : rz);
  TC tl[2] = {d == 0 ? ly : lx, d == 2 ? ly : lz};
  TC tr[2] = {d == 0 ? ry : rx, d == 2 ? ry : rz};
  TC Ff[5];
  exact_flux<TC, 2>(G, cl[0], nl, pl, tl, cr[0], nr, pr, tr, Ff, err);
  F[0] = Ff[0];
  F[1] = d == 0 ? Ff[1] : Ff[2];
  F[2] = d == 1 ? Ff[1] : (d == 0 ? Ff[2] : Ff[3]);
  F[3] = d == 2 ? Ff[1] : Ff[3];
  F[4] = Ff[4];
}

// Add the two faces of orientation D of a cell to its right-hand side for NV
// variables; s_f holds [var][face][gauss point] with the 2x2 points in the order
// (a, b) = (--, -+, +-, ++) of the transverse axes (e1, e2).
template <int D, class TC, int NV = 5>
__device__ __forceinline__ void gather3d(const TC* s_f, int FMAX, int fm, int fp, const TC* hd,
                                         TC* rc0, TC* rs) {
  constexpr int E1 = D == 0 ? 1 : 0, E2 = D == 2 ? 1 : 2;
  const TC c0f = TC(0.25) / hd[D];
  const TC csf = TC(1.5) / (hd[D] * hd[D]);
  const TC ce1 = TC(0.86602540378443864676) / (hd[E1] * hd[D]);
  const TC ce2 = TC(0.86602540378443864676) / (hd[E2] * hd[D]);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const TC* m = s_f + (v * FMAX + fm) * 4;
    const TC* p = s_f + (v * FMAX + fp) * 4;
    TC Sm = (m[0] + m[1]) + (m[2] + m[3]), Sp = (p[0] + p[1]) + (p[2] + p[3]);
    TC Dm1 = (m[2] + m[3]) - (m[0] + m[1]), Dp1 = (p[2] + p[3]) - (p[0] + p[1]);
    TC Dm2 = (m[1] + m[3]) - (m[0] + m[2]), Dp2 = (p[1] + p[3]) - (p[0] + p[2]);
    rc0[v] -= (Sp - Sm) * c0f;
    rs[3 * v + D] -= csf * (Sp + Sm);
    rs[3 * v + E1] -= ce1 * (Dp1 - Dm1);
    rs[3 * v + E2] -= ce2 * (Dp2 - Dm2);
  }
}

// Start of the staging of a 3D tile: the NS derivative coefficients of the
// halo-1 box are copied with cp.async (in flight while the averages are read),
// and every average of the halo-2 box that this thread reads next is requested
// into L2, so that the DRAM latencies of the staging overlap.  The caller then
// reads the averages, calls cp_async_wait_all() and synchronises.
// REC > 0: the coefficients go into per-cell records of REC elements, coefficient
// k of halo-1 cell r1 at s_sl[r1 * REC + OFF + k]; else planes s_sl[k * R1 + r1].
// PREFETCH = false leaves out the L2 requests for the averages (the 3D Euler
// kernel, which reads them two cells at a time, measured 1 % faster without);
// HALO = true requests only the cells of halo3d_cell, the ones a kernel whose
// limiter covers the tile and its face slabs reads.
template <int NV, int NS, int TX, int TY, int TZ, class TS, class TC, int REC = 0, int OFF = 0,
          bool PREFETCH = true, bool HALO = false>
__device__ __forceinline__ void stage3d_issue(const StateBuf<TS>& in, size_t ncell,
                                              const int* s_gx, const int* s_gy, const int* s_gz,
                                              TC* s_sl) {
  constexpr int R2X = TX + 4, R2Y = TY + 4, R2 = R2X * R2Y * (TZ + 4);
  constexpr int R1X = TX + 2, R1Y = TY + 2;
  constexpr int NT = TX * TY * TZ;
  static_assert(sizeof(TS) == sizeof(TC), "derivative coefficients are staged as stored");
  {  // planes (v, rz) of R1X x R1Y cells: thread t keeps position t % PL of every
     // C1-th plane from plane t / PL on, so a copy costs one plane-offset lookup
    constexpr int PL = R1X * R1Y, R1Z = TZ + 2, C1 = NT / PL;
    static_assert(C1 >= 1 && C1 <= R1Z, "a pass of planes advances by at most one variable");
    const int q = threadIdx.x % PL, p0 = threadIdx.x / PL;
    if (p0 < C1) {
      const int ry = q / R1X, rx = q - ry * R1X;
      const TS* src = in.sl + s_gy[ry + 1] + s_gx[rx + 1];
      size_t voff = 0;
      int rz = p0, k = 0;
      for (int p = p0; p < NS * R1Z; p += C1) {
        TC* dst = REC > 0 ? &s_sl[(rz * PL + q) * REC + OFF + k] : &s_sl[p * PL + q];
        cp_async_elem<sizeof(TS)>(dst, src + voff + s_gz[rz + 1]);
        rz += C1;
        if (rz >= R1Z) { rz -= R1Z; voff += ncell; ++k; }
      }
    }
  }
  if (PREFETCH) {
    for (int r = threadIdx.x; r < (HALO ? halo3d_count<TX, TY, TZ>() : R2); r += NT) {
      int rx, ry, rz;
      if (HALO) {
        halo3d_cell<TX, TY, TZ>(r, rx, ry, rz);
      } else {
        rz = r / (R2X * R2Y);
        const int rr = r - rz * (R2X * R2Y);
        ry = rr / R2X;
        rx = rr - ry * R2X;
      }
      const size_t g = (size_t)s_gz[rz] + s_gy[ry] + s_gx[rx];
#pragma unroll
      for (int v = 0; v < NV; ++v) prefetch_l2(&in.c0[v * ncell + g]);
    }
  }
}

// Stage 2 reads the step's input state U^n of its own cell only at the end (the
// Runge-Kutta combination): request those lines into L2 while the tile stages.
template <int NV, int NS, int TX, int TY, class TS>
__device__ __forceinline__ void stage3d_prefetch_base(const Stage3DArgs<TS>& A, size_t ncell,
                                                      const int* s_gx, const int* s_gy,
                                                      const int* s_gz) {
  const int lx = threadIdx.x % TX, ly = (threadIdx.x / TX) % TY, lz = threadIdx.x / (TX * TY);
  const size_t gc = (size_t)s_gz[lz + 2] + s_gy[ly + 2] + s_gx[lx + 2];
  const TS* sl = A.limiter && A.lim_sl ? A.lim_sl : A.base.sl;
#pragma unroll
  for (int v = 0; v < NV; ++v) prefetch_l2(&A.base.c0[v * ncell + gc]);
#pragma unroll
  for (int k = 0; k < NS; ++k) prefetch_l2(&sl[k * ncell + gc]);
}

// FP32: as many resident CTAs as 80 registers a thread allow (the kernel is
// latency bound); FP64 keeps its registers.
template <int NT, class TC>
struct Stage3dMinBlocks {
  static constexpr int v = sizeof(TC) == 4 && 65536 / (80 * NT) > 0 ? 65536 / (80 * NT) : 1;
};

// WENO = false compiles the WENO-type limiter out (launches with limiter 0 or 1).
template <class TC, class TS, int TX, int TY, int TZ, int STAGE, bool WENO>
__global__ void __launch_bounds__(TX * TY * TZ, (Stage3dMinBlocks<TX * TY * TZ, TC>::v))
    stage3d_kernel(const Stage3DArgs<TS> A) {
  griddep_launch_dependents();  // programmatic dependent launch: see griddep_wait()
  griddep_wait();
  constexpr int R2X = TX + 4, R2Y = TY + 4, R2Z = TZ + 4, R2 = R2X * R2Y * R2Z;
  constexpr int R1X = TX + 2, R1Y = TY + 2, R1Z = TZ + 2, R1 = R1X * R1Y * R1Z;
  constexpr int NT = TX * TY * TZ;
  constexpr int FMAX = stage3d_face_max<TX, TY, TZ, TC>();
  static_assert(NT % 32 == 0, "tile must be whole warps");

  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int WS = (int)stage3d_wsz<TX, TY, TZ, TC>();
  TC* s_w = reinterpret_cast<TC*>(smem_raw);  // 5 x R2 primitives, then
  TC* s_f = s_w;                              //   5 x 4 x FMAX face fluxes
  TC* s_rec = s_w + WS;                       // R1 records: 5 averages, 15 derivatives
  int* s_gx = reinterpret_cast<int*>(s_rec + kRec3d * R1);
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
  // profiling build: phases 0 staging and primitives, 1 limiter, 2 volume
  // integral, 3 + 2d faces and 4 + 2d their gather (d = 0, 1, 2), 9 combination
  // and store, 10 Courant reduction and commit
  PhaseStamp ph;
  ph.begin(A.phase, STAGE);
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
  if (STAGE == 2) stage3d_prefetch_base<5, 15, TX, TY>(A, ncell, s_gx, s_gy, s_gz);
  stage3d_issue<5, 15, TX, TY, TZ, TS, TC, kRec3d, 5, false>(A.in, ncell, s_gx, s_gy, s_gz, s_rec);
  // the halo-2 cells the limiter reads (the halo-1 box and the six outer face
  // layers), two per pass, all ten FP64 loads in flight before the first is
  // converted (the second cell of the last pass re-reads the first if it is past
  // the set, so every load stays in the grid)
  constexpr int NH = halo3d_count<TX, TY, TZ>();
  auto cell_of = [&](int e, int& r, int& r1ok) {
    int rx, ry, rz;
    halo3d_cell<TX, TY, TZ>(e, rx, ry, rz);
    r = (rz * R2Y + ry) * R2X + rx;
    r1ok = e < R1;
    return (size_t)s_gz[rz] + s_gy[ry] + s_gx[rx];
  };
  auto put = [&](int e, int r, int r1ok, const double* a) {
    TC c[5], W[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) c[v] = Cvt<TC>::to_tc(a[v]);
    prims3d<TC>(G, c, W, err);
#pragma unroll
    for (int q = 0; q < 5; ++q) s_w[q * R2 + r] = W[q];
    if (r1ok) {  // e is the cell's halo-1 index
#pragma unroll
      for (int v = 0; v < 5; ++v) s_rec[e * kRec3d + v] = c[v];
    }
  };
  for (int e = tid; e < NH; e += 2 * NT) {
    const int eb = e + NT;
    const bool two = eb < NH;
    int ra, rb, oka, okb;
    const size_t ga = cell_of(e, ra, oka);
    const size_t gb = two ? cell_of(eb, rb, okb) : ga;
    double a[5], b[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      a[v] = __ldg(&A.in.c0[v * ncell + ga]);
      b[v] = __ldg(&A.in.c0[v * ncell + gb]);
    }
    put(e, ra, oka, a);
    if (two) put(eb, rb, okb, b);
  }
  cp_async_wait_all();
  __syncthreads();
  ph.mark(0);

  const TC dx = Cvt<TC>::to_tc(A.dx), dy = Cvt<TC>::to_tc(A.dy), dz = Cvt<TC>::to_tc(A.dz);
  const TC hh[3] = {TC(0.5) * dx, TC(0.5) * dy, TC(0.5) * dz};
  const TC oo[3] = {dx * TC(0.28867513459481288225), dy * TC(0.28867513459481288225),
                    dz * TC(0.28867513459481288225)};

  // ---- limiter on the tile and its face slabs (the cells the faces read)
  if (A.limiter) {
    for (int e = tid; e < ring3d_count<TX, TY, TZ>(); e += NT) {
      int rx, ry, rz;
      ring3d_cell<TX, TY, TZ>(e, rx, ry, rz);
      const int r1 = (rz * R1Y + ry) * R1X + rx;
      const int r2 = ((rz + 1) * R2Y + (ry + 1)) * R2X + (rx + 1);
      TC W[5], Wn[6][5], s[15];
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
      TC v[kRec3d];
      rec_get<TC>(s_rec + r1 * kRec3d, v);
      if (WENO && A.limiter == 2) weno_cell3d<TC>(G, hh, W, Wn, v + 5, nullptr);
      else limit_cell3d<TC>(G, hh, W, Wn, v + 5);
      rec_put<TC>(s_rec + r1 * kRec3d, v);
    }
    __syncthreads();
  }
  ph.mark(1);

  // ---- per-cell state, volume integral
  const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
  const int r1c = ((lz + 1) * R1Y + (ly + 1)) * R1X + (lx + 1);
  TC rc0[5], rs[15];
#pragma unroll
  for (int v = 0; v < 5; ++v) rc0[v] = TC(0);
  {
    // the cell's own coefficients are read here and again for the combination
    // (not kept in registers across the face loop)
    TC c0[5], s[15];
    {
      TC v[kRec3d];
      rec_get<TC>(s_rec + r1c * kRec3d, v);
#pragma unroll
      for (int q = 0; q < 5; ++q) c0[q] = v[q];
#pragma unroll
      for (int k = 0; k < 15; ++k) s[k] = v[5 + k];
    }
    TC sF[3][5];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v) sF[d][v] = TC(0);
#pragma unroll
    for (int qp = 0; qp < 8; ++qp) {
      TC c[5];
      eval3d<TC>(c0, s, (qp & 1) ? oo[0] : -oo[0], (qp & 2) ? oo[1] : -oo[1],
                 (qp & 4) ? oo[2] : -oo[2], c);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        TC F[5];
        phys_flux3d<TC>(G, c, d, F, err);
#pragma unroll
        for (int v = 0; v < 5; ++v) sF[d][v] += F[v];
      }
    }
    const TC hd[3] = {dx, dy, dz};
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int d = 0; d < 3; ++d) rs[3 * v + d] = TC(1.5) / (hd[d] * hd[d]) * sF[d][v];
  }

  ph.mark(2);
  // ---- faces, one orientation at a time (rolled loop: one copy of the solver)
  const TC hd[3] = {dx, dy, dz};
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
      // the cell on the + side of the face has tile coordinates (fx, fy, fz),
      // i.e. halo-1 coordinates (fx+1, fy+1, fz+1); the - side is one step back
      // along d
      const int r1r = ((fz + 1) * R1Y + (fy + 1)) * R1X + (fx + 1);
      const int r1l = r1r - step;
      const TC a = (g & 2) ? o1 : -o1, b = (g & 1) ? o2 : -o2;
      // local coordinates of the Gauss point in the - cell (normal +hn) and the
      // + cell (normal -hn)
      const TC xl = d == 0 ? hn : a, xr = d == 0 ? -hn : a;
      const TC yl = d == 1 ? hn : (d == 0 ? a : b), yr = d == 1 ? -hn : (d == 0 ? a : b);
      const TC zl = d == 2 ? hn : b, zr = d == 2 ? -hn : b;
      TC vl[kRec3d], vr[kRec3d], cl[5], cr[5], F[5];
      rec_get<TC>(s_rec + r1l * kRec3d, vl);
      rec_get<TC>(s_rec + r1r * kRec3d, vr);
      eval3d<TC>(vl, vl + 5, xl, yl, zl, cl);
      eval3d<TC>(vr, vr + 5, xr, yr, zr, cr);
      face_flux3d<TC>(G, d, cl, cr, F, err);
#pragma unroll
      for (int v = 0; v < 5; ++v) s_f[(v * FMAX + f) * 4 + g] = F[v];
    }
    __syncthreads();
    ph.mark(3 + 2 * d);
    {
      const int fm = (lz * FY + ly) * FX + lx;
      const int fp = fm + (d == 0 ? 1 : (d == 1 ? FX : FX * FY));
      if (d == 0) gather3d<0, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
      else if (d == 1) gather3d<1, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
      else gather3d<2, TC>(s_f, FMAX, fm, fp, hd, rc0, rs);
    }
    __syncthreads();
    ph.mark(4 + 2 * d);
  }

  // ---- Runge-Kutta combination
  TC s[15];
  {
    TC v[kRec3d];
    rec_get<TC>(s_rec + r1c * kRec3d, v);
#pragma unroll
    for (int k = 0; k < 15; ++k) s[k] = v[5 + k];
  }
  const int gi = i0 + lx, gj = j0 + ly, gk = k0 + lz;
  const bool owner = gi < nx && gj < ny && gk < nz;
  const size_t gc = (size_t)s_gz[lz + 2] + s_gy[ly + 2] + s_gx[lx + 2];
  const double dt = s_dt;
  const TC dtc = Cvt<TC>::to_tc(dt);
  double o0[5];
  TC os[15];
  if (STAGE == 1) {
#pragma unroll
    for (int v = 0; v < 5; ++v) o0[v] = fma(dt, Cvt<TC>::to_f64(rc0[v]), A.in.c0[v * ncell + gc]);
#pragma unroll
    for (int k = 0; k < 15; ++k) os[k] = s[k] + dtc * rs[k];
    if (A.limiter && A.lim_sl && owner) {
#pragma unroll
      for (int k = 0; k < 15; ++k) A.lim_sl[k * ncell + gc] = (TS)s[k];
    }
  } else {
    TC sn[15];
    if (A.limiter && A.lim_sl) {
#pragma unroll
      for (int k = 0; k < 15; ++k) sn[k] = (TC)A.lim_sl[k * ncell + gc];
    } else {
#pragma unroll
      for (int k = 0; k < 15; ++k) sn[k] = (TC)A.base.sl[k * ncell + gc];
    }
    if (A.limiter && !A.lim_sl) {
      TC c[5], W[5], Wn[6][5];
#pragma unroll
      for (int v = 0; v < 5; ++v) c[v] = Cvt<TC>::to_tc(A.base.c0[v * ncell + gc]);
      prims3d<TC>(G, c, W, err);
      const size_t nb[6] = {(size_t)s_gz[lz + 2] + s_gy[ly + 2] + s_gx[lx + 1],
                            (size_t)s_gz[lz + 2] + s_gy[ly + 2] + s_gx[lx + 3],
                            (size_t)s_gz[lz + 2] + s_gy[ly + 1] + s_gx[lx + 2],
                            (size_t)s_gz[lz + 2] + s_gy[ly + 3] + s_gx[lx + 2],
                            (size_t)s_gz[lz + 1] + s_gy[ly + 2] + s_gx[lx + 2],
                            (size_t)s_gz[lz + 3] + s_gy[ly + 2] + s_gx[lx + 2]};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int v = 0; v < 5; ++v) c[v] = Cvt<TC>::to_tc(A.base.c0[v * ncell + nb[k]]);
        prims3d<TC>(G, c, Wn[k], err);
      }
      if (WENO && A.limiter == 2) weno_cell3d<TC>(G, hh, W, Wn, sn, nullptr);
      else limit_cell3d<TC>(G, hh, W, Wn, sn);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v)
      o0[v] = half_f64(A.base.c0[v * ncell + gc] +
                       fma(dt, Cvt<TC>::to_f64(rc0[v]), A.in.c0[v * ncell + gc]));
#pragma unroll
    for (int k = 0; k < 15; ++k) os[k] = TC(0.5) * sn[k] + TC(0.5) * (s[k] + dtc * rs[k]);
  }
  if (owner) {
#pragma unroll
    for (int v = 0; v < 5; ++v) A.out.c0[v * ncell + gc] = o0[v];
#pragma unroll
    for (int k = 0; k < 15; ++k) A.out.sl[k * ncell + gc] = (TS)os[k];
  }
  ph.mark(9);

  if (STAGE == 2) {
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
  } else {
    if (err) atomicOr(&s_err, err);
    __syncthreads();
    if (tid == 0 && s_err) atomicOr(&A.ctl->err, s_err);
  }
  ph.mark(10);
}

}  // namespace dgk
