// dg_dual.cuh -- forward-mode dual numbers for the device and the dual versions
// of the 2D Euler building blocks used by the adjoint kernels: conserved ->
// primitive conversion, physical fluxes, the exact Riemann flux and the min/max
// limiter.  A Dn<T, N> carries a value and N tangents; branches are decided on
// values (the derivative of the active branch).
#pragma once

#include "dg_physics.cuh"

namespace dgk {

template <class T, int N>
struct Dn {
  T v;
  T d[N];
  Dn() = default;
  // a constant (zero tangents), so that code written for a scalar type T (its
  // T(0.5), T(1) ...) also runs on Dn<T, N>
  __host__ __device__ Dn(T a) : v(a) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = T(0);
  }
};

template <class T, int N>
__device__ __forceinline__ Dn<T, N> dconst(T a) {
  Dn<T, N> r;
  r.v = a;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = T(0);
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator+(const Dn<T, N>& a, const Dn<T, N>& b) {
  Dn<T, N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator-(const Dn<T, N>& a, const Dn<T, N>& b) {
  Dn<T, N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator-(const Dn<T, N>& a) {
  Dn<T, N> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator*(const Dn<T, N>& a, const Dn<T, N>& b) {
  Dn<T, N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator/(const Dn<T, N>& a, const Dn<T, N>& b) {
  Dn<T, N> r;
  T ib = T(1) / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator+(const Dn<T, N>& a, T b) {
  Dn<T, N> r = a;
  r.v += b;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator+(T b, const Dn<T, N>& a) { return a + b; }
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator-(const Dn<T, N>& a, T b) {
  Dn<T, N> r = a;
  r.v -= b;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator-(T b, const Dn<T, N>& a) {
  Dn<T, N> r = -a;
  r.v += b;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator*(const Dn<T, N>& a, T b) {
  Dn<T, N> r;
  r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator*(T b, const Dn<T, N>& a) { return a * b; }
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator/(const Dn<T, N>& a, T b) { return a * (T(1) / b); }
template <class T, int N>
__device__ __forceinline__ Dn<T, N> operator/(T a, const Dn<T, N>& b) {
  Dn<T, N> r;
  T ib = T(1) / b.v;
  r.v = a * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -r.v * b.d[i] * ib;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> dsqrt(const Dn<T, N>& a) {
  Dn<T, N> r;
  r.v = rsqrtv(a.v);
  T k = r.v > T(0) ? T(0.5) / r.v : T(0);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * k;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> dpow(const Dn<T, N>& a, T e) {
  Dn<T, N> r;
  r.v = rpow(a.v, e);
  T k = a.v != T(0) ? e * r.v / a.v : T(0);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * k;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> dabs(const Dn<T, N>& a) { return a.v < T(0) ? -a : a; }

// What the scalar device physics needs besides arithmetic, so that its templates
// (hlld_flux, fast_speed, phys_flux2d) instantiate on Dn<T, N>: comparisons of
// the values (branches follow the value: the derivative of the active branch),
// |x|, the square root, and the solver tolerances of the scalar type.
template <class T, int N>
__device__ __forceinline__ bool operator<(const Dn<T, N>& a, const Dn<T, N>& b) { return a.v < b.v; }
template <class T, int N>
__device__ __forceinline__ bool operator>(const Dn<T, N>& a, const Dn<T, N>& b) { return a.v > b.v; }
template <class T, int N>
__device__ __forceinline__ bool operator<=(const Dn<T, N>& a, const Dn<T, N>& b) { return a.v <= b.v; }
template <class T, int N>
__device__ __forceinline__ bool operator>=(const Dn<T, N>& a, const Dn<T, N>& b) { return a.v >= b.v; }
template <class T, int N>
__device__ __forceinline__ Dn<T, N> fabs(const Dn<T, N>& a) { return dabs(a); }
template <class T, int N>
__device__ __forceinline__ Dn<T, N>& operator*=(Dn<T, N>& a, const Dn<T, N>& b) {
  a = a * b;
  return a;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N>& operator+=(Dn<T, N>& a, const Dn<T, N>& b) {
  a = a + b;
  return a;
}
template <class T, int N>
__device__ __forceinline__ Dn<T, N> rsqrtv(const Dn<T, N>& a) { return dsqrt(a); }
template <class T, int N>
struct Prec<Dn<T, N>> {
  static constexpr T newton_tol = Prec<T>::newton_tol;
  static constexpr int newton_max = Prec<T>::newton_max;
  static constexpr T hlld_degenerate = Prec<T>::hlld_degenerate;
};

// Primitive (rho, u, v, p) of conserved (rho, mx, my, E) in 2D, dual.
template <class T, int N>
__device__ __forceinline__ void dprims2d(const Gas<T>& G, const Dn<T, N>* c, Dn<T, N>* W) {
  Dn<T, N> inv = T(1) / c[0];
  Dn<T, N> vx = c[1] * inv, vy = c[2] * inv;
  W[0] = c[0];
  W[1] = vx;
  W[2] = vy;
  W[3] = G.gm1 * (c[3] - T(0.5) * (c[1] * vx + c[2] * vy));
}

// Physical fluxes along x and y of conserved (rho, mx, my, E), dual.
template <class T, int N>
__device__ __forceinline__ void dphys_flux2d(const Gas<T>& G, const Dn<T, N>* c, Dn<T, N>* Fx,
                                             Dn<T, N>* Fy) {
  Dn<T, N> W[4];
  dprims2d<T, N>(G, c, W);
  Dn<T, N> e = c[3] + W[3];
  Fx[0] = c[1]; Fx[1] = c[1] * W[1] + W[3]; Fx[2] = c[2] * W[1]; Fx[3] = e * W[1];
  Fy[0] = c[2]; Fy[1] = c[1] * W[2]; Fy[2] = c[2] * W[2] + W[3]; Fy[3] = e * W[2];
}

template <class T, int N>
__device__ __forceinline__ void dpressure_fn(const Gas<T>& G, const Dn<T, N>& p, const Dn<T, N>& rK,
                                             const Dn<T, N>& pK, const Dn<T, N>& cK, Dn<T, N>& f,
                                             Dn<T, N>& df) {
  if (p.v > pK.v) {
    Dn<T, N> A = G.two_gp1 / rK;
    Dn<T, N> B = G.g6 * pK;
    Dn<T, N> q = dsqrt(A / (p + B));
    f = (p - pK) * q;
    df = q * (T(1) - T(0.5) * (p - pK) / (B + p));
  } else {
    Dn<T, N> pr = p / pK;
    f = (T(2) * G.inv_gm1) * cK * (dpow(pr, G.z) - T(1));
    df = T(1) / (rK * cK) * dpow(pr, G.mzp);
  }
}

// Exact-solver flux in the face frame (mass, normal momentum, transverse
// momentum, energy) of dual primitive states; p* from the value solve, its
// derivative from one Newton step taken in dual arithmetic at the root.
template <class T, int N>
__device__ void dexact_flux(const Gas<T>& G, const Dn<T, N>& rL, const Dn<T, N>& uL,
                            const Dn<T, N>& pL, const Dn<T, N>& vL, const Dn<T, N>& rR,
                            const Dn<T, N>& uR, const Dn<T, N>& pR, const Dn<T, N>& vR,
                            Dn<T, N>* F, unsigned& err) {
  typedef Dn<T, N> D;
  if (!(rL.v > T(0) && pL.v > T(0) && rR.v > T(0) && pR.v > T(0))) {
    err |= ERR_NONPHYS;
    for (int q = 0; q < 4; ++q) F[q] = dconst<T, N>(T(0));
    return;
  }
  D cL = dsqrt(G.g * pL / rL), cR = dsqrt(G.g * pR / rR);
  const T pv = exact_pstar(G, rL.v, uL.v, pL.v, cL.v, rR.v, uR.v, pR.v, cR.v, err);
  D p0 = dconst<T, N>(pv);
  D fL, dfL, fR, dfR;
  dpressure_fn(G, p0, rL, pL, cL, fL, dfL);
  dpressure_fn(G, p0, rR, pR, cR, fR, dfR);
  D p = p0 - (fL + fR + (uR - uL)) / (dfL + dfR);
  p.v = pv;
  dpressure_fn(G, p, rL, pL, cL, fL, dfL);
  dpressure_fn(G, p, rR, pR, cR, fR, dfR);
  D us = T(0.5) * (uL + uR) + T(0.5) * (fR - fL);
  D rho, u, pp, vt;
  if (T(0) <= us.v) {
    vt = vL;
    if (p.v > pL.v) {
      D SL = uL - cL * dsqrt(G.shk1 * p / pL + G.z);
      if (T(0) <= SL.v) { rho = rL; u = uL; pp = pL; }
      else { rho = rL * ((p / pL + G.g6) / (G.g6 * p / pL + T(1))); u = us; pp = p; }
    } else {
      D SHL = uL - cL;
      if (T(0) <= SHL.v) { rho = rL; u = uL; pp = pL; }
      else {
        D cmL = cL * dpow(p / pL, G.z);
        if (T(0) > (us - cmL).v) { rho = rL * dpow(p / pL, G.inv_g); u = us; pp = p; }
        else {
          D c = G.two_gp1 * (cL + T(0.5) * G.gm1 * uL);
          u = c;
          rho = rL * dpow(c / cL, G.two_gm1);
          pp = pL * dpow(c / cL, G.inv_z);
        }
      }
    }
  } else {
    vt = vR;
    if (p.v > pR.v) {
      D SR = uR + cR * dsqrt(G.shk1 * p / pR + G.z);
      if (T(0) >= SR.v) { rho = rR; u = uR; pp = pR; }
      else { rho = rR * ((p / pR + G.g6) / (G.g6 * p / pR + T(1))); u = us; pp = p; }
    } else {
      D SHR = uR + cR;
      if (T(0) >= SHR.v) { rho = rR; u = uR; pp = pR; }
      else {
        D cmR = cR * dpow(p / pR, G.z);
        if (T(0) < (us + cmR).v) { rho = rR * dpow(p / pR, G.inv_g); u = us; pp = p; }
        else {
          D c = G.two_gp1 * (cR - T(0.5) * G.gm1 * uR);
          u = -c;
          rho = rR * dpow(c / cR, G.two_gm1);
          pp = pR * dpow(c / cR, G.inv_z);
        }
      }
    }
  }
  D E = pp * G.inv_gm1 + T(0.5) * rho * (u * u + vt * vt);
  D mu = rho * u;
  F[0] = mu;
  F[1] = mu * u + pp;
  F[2] = mu * vt;
  F[3] = u * (E + pp);
}

// Lab-frame exact flux through a face along `dir` between dual conserved states.
template <class T, int N>
__device__ __forceinline__ void dface_flux2d(const Gas<T>& G, int dir, const Dn<T, N>* cl,
                                             const Dn<T, N>* cr, Dn<T, N>* F, unsigned& err) {
  Dn<T, N> Wl[4], Wr[4], Ff[4];
  dprims2d<T, N>(G, cl, Wl);
  dprims2d<T, N>(G, cr, Wr);
  if (dir == 0) dexact_flux<T, N>(G, Wl[0], Wl[1], Wl[3], Wl[2], Wr[0], Wr[1], Wr[3], Wr[2], Ff, err);
  else dexact_flux<T, N>(G, Wl[0], Wl[2], Wl[3], Wl[1], Wr[0], Wr[2], Wr[3], Wr[1], Ff, err);
  F[0] = Ff[0];
  F[3] = Ff[3];
  if (dir == 0) { F[1] = Ff[1]; F[2] = Ff[2]; }
  else { F[1] = Ff[2]; F[2] = Ff[1]; }
}

// Dual min/max limiter of one 2D Euler cell (Sec. 2.5): c0/s its averages and
// derivative coefficients, cn[k] the averages of its 4 face neighbours; s is
// replaced by the limited coefficients.
template <class T, int N>
__device__ void dlimit_cell2d(const Gas<T>& G, const T* hh, const Dn<T, N>* c0,
                              const Dn<T, N> (*cn)[4], Dn<T, N>* s) {
  typedef Dn<T, N> D;
  D W[4], Wn[4][4];
  dprims2d<T, N>(G, c0, W);
#pragma unroll
  for (int k = 0; k < 4; ++k) dprims2d<T, N>(G, cn[k], Wn[k]);
  const D inv = T(1) / W[0];
  D gr[2], gvx[2], gvy[2], gp[2];
  const D v2h = T(0.5) * (W[1] * W[1] + W[2] * W[2]);
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    gr[d] = s[d];
    gvx[d] = (s[2 + d] - W[1] * gr[d]) * inv;
    gvy[d] = (s[4 + d] - W[2] * gr[d]) * inv;
    gp[d] = G.gm1 * (s[6 + d] - v2h * gr[d] - W[0] * (W[1] * gvx[d] + W[2] * gvy[d]));
  }
  D alpha[4];
  const D* grads[4] = {gr, gvx, gvy, gp};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    D hi = W[q], lo = W[q];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (Wn[k][q].v > hi.v) hi = Wn[k][q];
      if (Wn[k][q].v < lo.v) lo = Wn[k][q];
    }
    D a0 = dabs(grads[q][0] * hh[0]), a1 = dabs(grads[q][1] * hh[1]);
    D amax = a1.v > a0.v ? a1 : a0;
    if (!(amax.v > T(0))) {
      alpha[q] = dconst<T, N>(T(1));
    } else {
      D up = hi - W[q], dn = W[q] - lo;
      D m = up.v < dn.v ? up : dn;
      D psi = m / amax;
      alpha[q] = psi.v < T(1) ? psi : dconst<T, N>(T(1));
    }
  }
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    D r = alpha[0] * gr[d], ux = alpha[1] * gvx[d], uy = alpha[2] * gvy[d], pp = alpha[3] * gp[d];
    s[d] = r;
    s[2 + d] = W[0] * ux + W[1] * r;
    s[4 + d] = W[0] * uy + W[2] * r;
    s[6 + d] = pp * G.inv_gm1 + v2h * r + W[0] * (W[1] * ux + W[2] * uy);
  }
}

}  // namespace dgk
