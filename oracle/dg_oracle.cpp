// dg_oracle.cpp -- TEST INFRASTRUCTURE, not part of the product.
//
// A plain, slow, double-precision CPU statement of one explicit time step of the
// second-order centroidal-Taylor discontinuous Galerkin (DG) scheme of Mocz,
// Vogelsberger, Sijacki, Pakmor & Hernquist (2013), "A discontinuous Galerkin
// method for solving the fluid and MHD equations in astrophysical simulations":
//   * Sec. 2.1  eq. `cons`      conservative ideal-MHD system (Euler when B = 0)
//   * Sec. 2.2  eq. `dg`        weak form, Taylor basis (1, x, y[, z]) about the
//                               centroid, eqs. `fv`, `dgderiv`, `fv3d`,
//                               `dgderiv3d`, mass matrix M, locally
//                               divergence-free magnetic bases V1..V5 (2D)
//                               and V1..V11 (3D)
//   * Sec. 2.3                  exact Riemann solver (Euler), HLLD (MHD; two
//                               transverse components in 3D)
//   * Sec. 2.5                  min/max slope limiter on primitive variables, and
//                               the WENO-type limiter (limiter = 2; the field's
//                               stencil gradient L2-projected onto the basis)
//   * Sec. 2.6                  averaged normal B at faces; Stokes div-B estimate
// The time integrator is the two-stage strong-stability-preserving Runge-Kutta
// method (the "traditional DG" integrator named in Sec. 2.4) and faces are
// integrated with 2-point Gauss rules per face dimension; volumes with 2^dim
// tensor Gauss points.  A second integrator, the MUSCL-Hancock step of Sec. 2.4
// (half-step prediction of primitive values, one update by eq. `GalerkUpdate`),
// integrates faces with one point at the face centroid (the paper's form) or the
// same 2-point Gauss rules.
//
// Everything is written as the generic weak form: for every basis function W the
// face integral of F.n W and the volume integral of F . grad W are evaluated by
// quadrature, the mass matrix  M_kl = int W_k W_l  is evaluated by quadrature, and
// the small system M dc/dt = -face + volume is solved by Gaussian elimination.
// No blocking, fusion or reordering beyond that.  Templated on the scalar type so
// that the same code, instantiated on a forward-mode dual number, gives the
// tangent (Jacobian-vector product) of the step.
//
// Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
// load this library.  Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

namespace oracle {

// ------------------------------------------------------------------------------
// Scalar types.  `double` for the step, `Dual` (value + one tangent) for the JVP.
// Branches are always taken on the value part (the active branch).
// ------------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double a) : v(a), d(0.0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, Dual b) {
  double q = a / b.v;
  return Dual(q, -q * b.d / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }

inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }

inline double r_sqrt(double a) { return std::sqrt(a); }
inline Dual r_sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, s > 0.0 ? a.d / (2.0 * s) : 0.0);
}
inline double r_pow(double a, double e) { return std::pow(a, e); }
inline Dual r_pow(Dual a, double e) {
  double p = std::pow(a.v, e);
  return Dual(p, a.v != 0.0 ? e * p / a.v * a.d : 0.0);
}
inline double r_abs(double a) { return std::fabs(a); }
inline Dual r_abs(Dual a) { return a.v < 0.0 ? -a : a; }
template <class R> inline R r_min(const R& a, const R& b) { return val(b) < val(a) ? b : a; }
template <class R> inline R r_max(const R& a, const R& b) { return val(b) > val(a) ? b : a; }

// ------------------------------------------------------------------------------
// Problem description.
// ------------------------------------------------------------------------------
enum { EQ_EULER = 0, EQ_MHD = 1 };
enum { RS_EXACT = 0, RS_HLLD = 1 };
enum {
  FLAG_NONPHYS = 1,     // rho <= 0 or p <= 0 where a state is evaluated
  FLAG_VACUUM = 2,      // exact Riemann solver: vacuum generated
  FLAG_NEWTON = 4,      // exact Riemann solver: Newton iteration did not converge
  FLAG_UNSUPPORTED = 8, // a combination the oracle does not define (none at present)
};

struct Cfg {
  int eq;       // EQ_EULER | EQ_MHD
  int dim;      // 2 | 3
  int nx, ny, nz;
  int limiter;  // 0 off, 1 min/max limiter, 2 WENO-type limiter (Sec. 2.5)
  int riemann;  // RS_EXACT | RS_HLLD
  int pad;
  double dx, dy, dz;
  double gamma;
};

// The conserved state is always carried as the 8-vector of Sec. 2.1:
//   U = (rho, rho vx, rho vy, rho vz, rho e, Bx, By, Bz).
// Unused components (vz in 2D, B for Euler) are identically zero.
enum { I_RHO = 0, I_MX = 1, I_MY = 2, I_MZ = 3, I_E = 4, I_BX = 5, I_BY = 6, I_BZ = 7 };

// Layout of the DG coefficients of one cell ("interchange layout", one plane per
// coefficient, planes ordered variable-major):
//   Taylor variables v = 0..nT-1, coefficient k = 0 (average), 1..dim (d/dx_k):
//       plane v*(dim+1)+k
//   MHD only, magnetic block after the Taylor planes:
//       (b1, b2, a1, a2, a3) = coefficients of the basis V1..V5 of Sec. 2.2.
struct Layout {
  int nT;          // number of Taylor variables
  int tvar[5];     // U-index of each Taylor variable
  int nK;          // Taylor coefficients per variable = dim+1
  int nB;          // magnetic coefficients (5 in 2D MHD, 11 in 3D MHD, else 0)
  int nBa;         // of which averages (2 in 2D MHD, 3 in 3D MHD)
  int nplanes;
};

inline Layout layout_of(const Cfg& c) {
  Layout L;
  L.nK = c.dim + 1;
  L.nBa = 0;
  if (c.dim == 2) {
    L.nT = 4; L.tvar[0] = I_RHO; L.tvar[1] = I_MX; L.tvar[2] = I_MY; L.tvar[3] = I_E;
  } else {
    L.nT = 5; L.tvar[0] = I_RHO; L.tvar[1] = I_MX; L.tvar[2] = I_MY; L.tvar[3] = I_MZ;
    L.tvar[4] = I_E;
  }
  L.nB = 0;
  if (c.eq == EQ_MHD) {
    L.nB = c.dim == 2 ? 5 : 11;
    L.nBa = c.dim;
  }
  L.nplanes = L.nT * L.nK + L.nB;
  return L;
}

struct Grid {
  Cfg c;
  Layout L;
  long ncell;
  double h[3];
  double vol;
  explicit Grid(const Cfg& cfg) : c(cfg), L(layout_of(cfg)) {
    if (c.dim == 2) c.nz = 1;
    ncell = (long)c.nx * c.ny * c.nz;
    h[0] = c.dx; h[1] = c.dy; h[2] = (c.dim == 3 ? c.dz : 1.0);
    vol = h[0] * h[1] * (c.dim == 3 ? h[2] : 1.0);
  }
  long idx(int i, int j, int k) const {
    i = ((i % c.nx) + c.nx) % c.nx;
    j = ((j % c.ny) + c.ny) % c.ny;
    k = ((k % c.nz) + c.nz) % c.nz;
    return ((long)k * c.ny + j) * c.nx + i;
  }
  void ijk(long cell, int& i, int& j, int& k) const {
    i = (int)(cell % c.nx);
    j = (int)((cell / c.nx) % c.ny);
    k = (int)(cell / ((long)c.nx * c.ny));
  }
  // periodic neighbour of `cell` across its face with outward normal s*e_d (s=+-1)
  long nbr(long cell, int d, int s) const {
    int i, j, k;
    ijk(cell, i, j, k);
    if (d == 0) i += s; else if (d == 1) j += s; else k += s;
    return idx(i, j, k);
  }
};

// ------------------------------------------------------------------------------
// Gauss-Legendre 2-point rule on [-h/2, h/2]: nodes -+h/(2 sqrt 3), weights h/2.
// ------------------------------------------------------------------------------
inline double gauss_node(int g, double h) {
  return (g == 0 ? -1.0 : 1.0) * h / (2.0 * std::sqrt(3.0));
}
inline double gauss_weight(double h) { return 0.5 * h; }

// ------------------------------------------------------------------------------
// Basis functions (Sec. 2.2).  Local coordinates have their origin at the
// centroid.  Scalar Taylor basis: W_0 = 1, W_k = x_k.  Vector magnetic bases,
// locally divergence free:
//   2D: V1 = (1,0), V2 = (0,1), V3 = (y,0), V4 = (0,x), V5 = (x,-y);
//   3D: V1..V3 the unit vectors, V4 = (y,0,0), V5 = (z,0,0), V6 = (0,x,0),
//       V7 = (0,z,0), V8 = (0,0,x), V9 = (0,0,y), V10 = (x,-y,0), V11 = (x,0,-z).
// ------------------------------------------------------------------------------
inline double taylor_w(int k, const double x[3]) { return k == 0 ? 1.0 : x[k - 1]; }
inline double taylor_dw(int k, int d) { return (k >= 1 && k - 1 == d) ? 1.0 : 0.0; }
inline void mag_w(int dim, int k, const double x[3], double w[3]) {
  w[0] = w[1] = w[2] = 0.0;
  if (dim == 2) {
    switch (k) {
      case 0: w[0] = 1.0; break;
      case 1: w[1] = 1.0; break;
      case 2: w[0] = x[1]; break;
      case 3: w[1] = x[0]; break;
      default: w[0] = x[0]; w[1] = -x[1]; break;
    }
    return;
  }
  switch (k) {
    case 0: w[0] = 1.0; break;
    case 1: w[1] = 1.0; break;
    case 2: w[2] = 1.0; break;
    case 3: w[0] = x[1]; break;
    case 4: w[0] = x[2]; break;
    case 5: w[1] = x[0]; break;
    case 6: w[1] = x[2]; break;
    case 7: w[2] = x[0]; break;
    case 8: w[2] = x[1]; break;
    case 9: w[0] = x[0]; w[1] = -x[1]; break;
    default: w[0] = x[0]; w[2] = -x[2]; break;
  }
}
// d(component c of V_k)/d(x_d)
inline double mag_dw(int dim, int k, int c, int d) {
  double x[3] = {0.0, 0.0, 0.0}, w0[3], w1[3];
  mag_w(dim, k, x, w0);
  x[d] = 1.0;
  mag_w(dim, k, x, w1);
  return w1[c] - w0[c];  // the basis is at most linear
}

// Value of the DG polynomial of cell `cell` at local point x: the 8-vector U.
template <class R>
void eval_poly(const Grid& G, const R* u, long cell, const double x[3], R U[8]) {
  for (int q = 0; q < 8; ++q) U[q] = R(0.0);
  const long n = G.ncell;
  for (int v = 0; v < G.L.nT; ++v) {
    R s(0.0);
    for (int k = 0; k < G.L.nK; ++k)
      s = s + u[(long)(v * G.L.nK + k) * n + cell] * taylor_w(k, x);
    U[G.L.tvar[v]] = s;
  }
  if (G.L.nB) {
    const int b0 = G.L.nT * G.L.nK;
    for (int k = 0; k < G.L.nB; ++k) {
      double w[3];
      mag_w(G.c.dim, k, x, w);
      R c = u[(long)(b0 + k) * n + cell];
      for (int q = 0; q < 3; ++q)
        if (w[q] != 0.0) U[I_BX + q] = U[I_BX + q] + c * w[q];
    }
  }
}

// ------------------------------------------------------------------------------
// Sec. 2.1: equation of state and physical flux.
//   p_gas = (gamma-1) rho u,  rho e = rho u + rho v^2/2 + B^2/2,  p_T = p_gas + B^2/2
// ------------------------------------------------------------------------------
template <class R>
void cons_to_prim(const R U[8], double g, R W[8]) {
  // W = (rho, vx, vy, vz, p_gas, Bx, By, Bz)
  R rho = U[I_RHO];
  W[0] = rho;
  W[1] = U[I_MX] / rho;
  W[2] = U[I_MY] / rho;
  W[3] = U[I_MZ] / rho;
  R kin = 0.5 * (U[I_MX] * W[1] + U[I_MY] * W[2] + U[I_MZ] * W[3]);
  R mag = 0.5 * (U[I_BX] * U[I_BX] + U[I_BY] * U[I_BY] + U[I_BZ] * U[I_BZ]);
  W[4] = (g - 1.0) * (U[I_E] - kin - mag);
  W[5] = U[I_BX];
  W[6] = U[I_BY];
  W[7] = U[I_BZ];
}

template <class R>
void prim_to_cons(const R W[8], double g, R U[8]) {
  R rho = W[0];
  U[I_RHO] = rho;
  U[I_MX] = rho * W[1];
  U[I_MY] = rho * W[2];
  U[I_MZ] = rho * W[3];
  U[I_BX] = W[5];
  U[I_BY] = W[6];
  U[I_BZ] = W[7];
  U[I_E] = W[4] / (g - 1.0) + 0.5 * rho * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) +
           0.5 * (W[5] * W[5] + W[6] * W[6] + W[7] * W[7]);
}

// Flux along axis d of eq. `cons`:
//   rho v_d,  rho v v_d + p_T e_d - B B_d,  (rho e + p_T) v_d - B_d (v.B),  B v_d - v B_d
template <class R>
void phys_flux(const R U[8], int d, double g, R F[8]) {
  R W[8];
  cons_to_prim(U, g, W);
  const R* v = W + 1;
  const R* B = W + 5;
  R pT = W[4] + 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  R vd = v[d], Bd = B[d];
  R vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
  F[I_RHO] = U[I_RHO] * vd;
  for (int i = 0; i < 3; ++i) {
    F[1 + i] = U[1 + i] * vd - B[i] * Bd;
    F[5 + i] = B[i] * vd - v[i] * Bd;
  }
  F[1 + d] = F[1 + d] + pT;
  F[I_E] = (U[I_E] + pT) * vd - Bd * vB;
}

// ------------------------------------------------------------------------------
// Exact Riemann solver for the Euler equations (Sec. 2.3; the textbook solver of
// Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4):
// Newton iteration on the pressure function f_L(p) + f_R(p) + (u_R - u_L) = 0,
// then sampling of the self-similar solution.  Transverse velocities are passive
// scalars carried from the side of the contact the sample lies on.
// ------------------------------------------------------------------------------
struct ExactParams {
  double newton_tol = 1e-12;  // relative pressure change that stops the iteration
  int newton_max = 50;        // iterations before FLAG_NEWTON is raised
};

template <class R>
void pressure_fn(const R& p, const R& rhoK, const R& pK, const R& cK, double g, R& f, R& df) {
  if (val(p) > val(pK)) {  // shock branch
    R A = 2.0 / ((g + 1.0) * rhoK);
    R B = (g - 1.0) / (g + 1.0) * pK;
    R q = r_sqrt(A / (p + B));
    f = (p - pK) * q;
    df = q * (1.0 - 0.5 * (p - pK) / (B + p));
  } else {  // rarefaction branch
    R pr = p / pK;
    f = 2.0 * cK / (g - 1.0) * (r_pow(pr, (g - 1.0) / (2.0 * g)) - 1.0);
    df = 1.0 / (rhoK * cK) * r_pow(pr, -(g + 1.0) / (2.0 * g));
  }
}

// Solution of the 1D Riemann problem (rho, u, p)_L | (rho, u, p)_R.
template <class R>
struct StarState {
  R pstar, ustar;
  int flags;
};

template <class R>
StarState<R> exact_star(const R& rL, const R& uL, const R& pL, const R& rR, const R& uR,
                        const R& pR, double g, const ExactParams& P) {
  StarState<R> S;
  S.flags = 0;
  R cL = r_sqrt(g * pL / rL), cR = r_sqrt(g * pR / rR);
  // pressure positivity condition (vacuum is not generated)
  if (2.0 / (g - 1.0) * (val(cL) + val(cR)) <= val(uR) - val(uL)) S.flags |= FLAG_VACUUM;
  // Initial guess: the adaptive choice between the primitive-variable, two-
  // rarefaction and two-shock approximations (Toro, Sec. 9.5).
  const double z = (g - 1.0) / (2.0 * g);
  double pv = 0.5 * (val(pL) + val(pR)) -
              0.125 * (val(uR) - val(uL)) * (val(rL) + val(rR)) * (val(cL) + val(cR));
  pv = std::max(0.0, pv);
  double pmin = std::min(val(pL), val(pR)), pmax = std::max(val(pL), val(pR));
  double p0;
  if (pmax / pmin <= 2.0 && pmin <= pv && pv <= pmax) {
    p0 = pv;
  } else if (pv < pmin) {
    double num = val(cL) + val(cR) - 0.5 * (g - 1.0) * (val(uR) - val(uL));
    double den = val(cL) / std::pow(val(pL), z) + val(cR) / std::pow(val(pR), z);
    p0 = std::pow(std::max(num, 0.0) / den, 1.0 / z);
  } else {
    double gL = std::sqrt(2.0 / ((g + 1.0) * val(rL)) / ((g - 1.0) / (g + 1.0) * val(pL) + pv));
    double gR = std::sqrt(2.0 / ((g + 1.0) * val(rR)) / ((g - 1.0) / (g + 1.0) * val(pR) + pv));
    p0 = (gL * val(pL) + gR * val(pR) - (val(uR) - val(uL))) / (gL + gR);
  }
  const double pfloor = 1e-10 * pmin;
  if (!(p0 > pfloor)) p0 = pfloor;

  // Newton iteration on the values ...
  double p = p0;
  bool conv = false;
  for (int it = 0; it < P.newton_max; ++it) {
    double fL, dfL, fR, dfR;
    pressure_fn<double>(p, val(rL), val(pL), val(cL), g, fL, dfL);
    pressure_fn<double>(p, val(rR), val(pR), val(cR), g, fR, dfR);
    double pn = p - (fL + fR + (val(uR) - val(uL))) / (dfL + dfR);
    if (!(pn > pfloor)) pn = pfloor;
    double change = 2.0 * std::fabs(pn - p) / (pn + p);
    p = pn;
    if (change < P.newton_tol) { conv = true; break; }
  }
  if (!conv) S.flags |= FLAG_NEWTON;
  // ... then one Newton step in the full scalar type from the converged root,
  // which carries the implicit-function derivative of p* for dual numbers and
  // leaves the value unchanged to rounding.
  R pr(p);
  {
    R fL, dfL, fR, dfR;
    pressure_fn<R>(pr, rL, pL, cL, g, fL, dfL);
    pressure_fn<R>(pr, rR, pR, cR, g, fR, dfR);
    R f = fL + fR + (uR - uL);
    // value part kept at the converged p; the tangent is -(df/dW dW)/(df/dp)
    R step = f / (dfL + dfR);
    pr = pr - step;
    if constexpr (!std::is_same<R, double>::value) pr.v = p;
    else pr = p;
  }
  S.pstar = pr;
  R fL, dfL, fR, dfR;
  pressure_fn<R>(pr, rL, pL, cL, g, fL, dfL);
  pressure_fn<R>(pr, rR, pR, cR, g, fR, dfR);
  S.ustar = 0.5 * (uL + uR) + 0.5 * (fR - fL);
  return S;
}

// Sample the exact solution at speed xi = x/t.  Returns (rho, u, p) and whether
// the sample lies left of the contact (transverse data taken from that side).
template <class R>
bool exact_sample(const R& rL, const R& uL, const R& pL, const R& rR, const R& uR,
                  const R& pR, double g, const StarState<R>& S, double xi, R& rho, R& u,
                  R& p) {
  const R& ps = S.pstar;
  const R& us = S.ustar;
  const double g1 = (g - 1.0) / (g + 1.0);
  if (xi <= val(us)) {  // left of the contact
    R cL = r_sqrt(g * pL / rL);
    if (val(ps) > val(pL)) {  // left shock
      R SL = uL - cL * r_sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g));
      if (xi <= val(SL)) { rho = rL; u = uL; p = pL; }
      else { rho = rL * ((ps / pL + g1) / (g1 * ps / pL + 1.0)); u = us; p = ps; }
    } else {  // left rarefaction
      R SHL = uL - cL;
      if (xi <= val(SHL)) { rho = rL; u = uL; p = pL; }
      else {
        R cmL = cL * r_pow(ps / pL, (g - 1.0) / (2.0 * g));
        R STL = us - cmL;
        if (xi > val(STL)) { rho = rL * r_pow(ps / pL, 1.0 / g); u = us; p = ps; }
        else {  // inside the fan
          R c = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (uL - xi));
          u = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + xi);
          rho = rL * r_pow(c / cL, 2.0 / (g - 1.0));
          p = pL * r_pow(c / cL, 2.0 * g / (g - 1.0));
        }
      }
    }
    return true;
  } else {  // right of the contact
    R cR = r_sqrt(g * pR / rR);
    if (val(ps) > val(pR)) {  // right shock
      R SR = uR + cR * r_sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g));
      if (xi >= val(SR)) { rho = rR; u = uR; p = pR; }
      else { rho = rR * ((ps / pR + g1) / (g1 * ps / pR + 1.0)); u = us; p = ps; }
    } else {  // right rarefaction
      R SHR = uR + cR;
      if (xi >= val(SHR)) { rho = rR; u = uR; p = pR; }
      else {
        R cmR = cR * r_pow(ps / pR, (g - 1.0) / (2.0 * g));
        R STR = us + cmR;
        if (xi < val(STR)) { rho = rR * r_pow(ps / pR, 1.0 / g); u = us; p = ps; }
        else {
          R c = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (uR - xi));
          u = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + xi);
          rho = rR * r_pow(c / cR, 2.0 / (g - 1.0));
          p = pR * r_pow(c / cR, 2.0 * g / (g - 1.0));
        }
      }
    }
    return false;
  }
}

// Godunov flux of the exact solver along axis d, in the lab frame.
template <class R>
int riemann_exact(const R UL[8], const R UR[8], int d, double g, R F[8],
                  const ExactParams& P = ExactParams()) {
  R WL[8], WR[8];
  cons_to_prim(UL, g, WL);
  cons_to_prim(UR, g, WR);
  int flags = 0;
  if (!(val(WL[0]) > 0.0 && val(WL[4]) > 0.0 && val(WR[0]) > 0.0 && val(WR[4]) > 0.0))
    flags |= FLAG_NONPHYS;
  if (flags) {  // no meaningful solution; return the average physical flux
    R FL[8], FR[8];
    phys_flux(UL, d, g, FL);
    phys_flux(UR, d, g, FR);
    for (int q = 0; q < 8; ++q) F[q] = 0.5 * (FL[q] + FR[q]);
    return flags;
  }
  StarState<R> S = exact_star(WL[0], WL[1 + d], WL[4], WR[0], WR[1 + d], WR[4], g, P);
  flags |= S.flags;
  R rho, un, p;
  bool left = exact_sample(WL[0], WL[1 + d], WL[4], WR[0], WR[1 + d], WR[4], g, S, 0.0, rho,
                           un, p);
  R W[8];
  const R* side = left ? WL : WR;
  for (int q = 0; q < 8; ++q) W[q] = side[q];
  W[0] = rho;
  W[1 + d] = un;
  W[4] = p;
  R U[8];
  prim_to_cons(W, g, U);
  phys_flux(U, d, g, F);
  return flags;
}

// ------------------------------------------------------------------------------
// HLLD approximate Riemann solver for ideal MHD (Sec. 2.3; Miyoshi & Kusano 2005,
// J. Comput. Phys. 208, 315).  Works in the frame (n, t1, t2) of the face normal;
// the normal field Bn must be the same on both sides.
// ------------------------------------------------------------------------------
struct HlldParams {
  double degenerate = 1e-8;  // relative size of the denominator treated as zero
};

template <class R>
R fast_speed(const R W[8], int d, double g) {
  // fast magnetosonic speed along axis d
  R a2 = g * W[4] / W[0];
  R b2 = (W[5] * W[5] + W[6] * W[6] + W[7] * W[7]) / W[0];
  R bn2 = W[5 + d] * W[5 + d] / W[0];
  R s = a2 + b2;
  R disc = s * s - 4.0 * a2 * bn2;
  if (val(disc) < 0.0) disc = R(0.0);
  return r_sqrt(0.5 * (s + r_sqrt(disc)));
}

template <class R>
int riemann_hlld(const R UL[8], const R UR[8], int d, double g, R F[8],
                 const HlldParams& P = HlldParams()) {
  const int n = d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  R WLl[8], WRl[8];
  cons_to_prim(UL, g, WLl);
  cons_to_prim(UR, g, WRl);
  int flags = 0;
  if (!(val(WLl[0]) > 0.0 && val(WLl[4]) > 0.0 && val(WRl[0]) > 0.0 && val(WRl[4]) > 0.0))
    flags |= FLAG_NONPHYS;
  if (flags) {
    R FL[8], FR[8];
    phys_flux(UL, d, g, FL);
    phys_flux(UR, d, g, FR);
    for (int q = 0; q < 8; ++q) F[q] = 0.5 * (FL[q] + FR[q]);
    return flags;
  }
  // rotate into the face frame: (rho, u, v, w, p, Bx, By, Bz) with x along n
  auto rot = [&](const R* W, R* Q) {
    Q[0] = W[0]; Q[1] = W[1 + n]; Q[2] = W[1 + t1]; Q[3] = W[1 + t2]; Q[4] = W[4];
    Q[5] = W[5 + n]; Q[6] = W[5 + t1]; Q[7] = W[5 + t2];
  };
  R L[8], Rr[8];
  rot(WLl, L);
  rot(WRl, Rr);
  const R Bx = 0.5 * (L[5] + Rr[5]);  // equal on entry; averaged for safety
  L[5] = Bx; Rr[5] = Bx;

  auto energy = [&](const R* Q) {
    return Q[4] / (g - 1.0) + 0.5 * Q[0] * (Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]) +
           0.5 * (Q[5] * Q[5] + Q[6] * Q[6] + Q[7] * Q[7]);
  };
  auto ptot = [&](const R* Q) { return Q[4] + 0.5 * (Q[5] * Q[5] + Q[6] * Q[6] + Q[7] * Q[7]); };
  // conserved vector and flux in the face frame: (rho, mx, my, mz, E, Bx, By, Bz)
  auto consv = [&](const R* Q, R E, R* U) {
    U[0] = Q[0]; U[1] = Q[0] * Q[1]; U[2] = Q[0] * Q[2]; U[3] = Q[0] * Q[3]; U[4] = E;
    U[5] = Q[5]; U[6] = Q[6]; U[7] = Q[7];
  };
  auto fluxv = [&](const R* Q, R E, R* Fq) {
    R pT = ptot(Q);
    R vB = Q[1] * Q[5] + Q[2] * Q[6] + Q[3] * Q[7];
    Fq[0] = Q[0] * Q[1];
    Fq[1] = Q[0] * Q[1] * Q[1] + pT - Q[5] * Q[5];
    Fq[2] = Q[0] * Q[1] * Q[2] - Q[5] * Q[6];
    Fq[3] = Q[0] * Q[1] * Q[3] - Q[5] * Q[7];
    Fq[4] = (E + pT) * Q[1] - Q[5] * vB;
    Fq[5] = R(0.0);
    Fq[6] = Q[6] * Q[1] - Q[2] * Q[5];
    Fq[7] = Q[7] * Q[1] - Q[3] * Q[5];
  };

  R EL = energy(L), ER = energy(Rr);
  R pTL = ptot(L), pTR = ptot(Rr);
  R cfL = fast_speed(L, 0, g), cfR = fast_speed(Rr, 0, g);
  // outer wave-speed estimates from the fast speeds of both sides
  R cmax = r_max(cfL, cfR);
  R SL = r_min(L[1], Rr[1]) - cmax;
  R SR = r_max(L[1], Rr[1]) + cmax;
  R FLv[8], FRv[8], ULv[8], URv[8];
  fluxv(L, EL, FLv);
  fluxv(Rr, ER, FRv);
  consv(L, EL, ULv);
  consv(Rr, ER, URv);

  R Fo[8];
  if (val(SL) > 0.0) {
    for (int q = 0; q < 8; ++q) Fo[q] = FLv[q];
  } else if (val(SR) < 0.0) {
    for (int q = 0; q < 8; ++q) Fo[q] = FRv[q];
  } else {
    R dL = SL - L[1], dR = SR - Rr[1];
    R den = dR * Rr[0] - dL * L[0];
    R SM = (dR * Rr[0] * Rr[1] - dL * L[0] * L[1] - pTR + pTL) / den;  // contact speed
    R pTs = (dR * Rr[0] * pTL - dL * L[0] * pTR + L[0] * Rr[0] * dR * dL * (Rr[1] - L[1])) /
            den;  // total pressure in the Riemann fan
    // single-star states
    auto star = [&](const R* Q, R E, R S, R pT, R* Qs, R& Es) {
      R dS = S - Q[1];
      R rs = Q[0] * dS / (S - SM);
      R dd = Q[0] * dS * (S - SM) - Bx * Bx;
      Qs[0] = rs;
      Qs[1] = SM;
      Qs[5] = Bx;
      if (val(r_abs(dd)) < P.degenerate * val(Q[0] * dS * dS + Bx * Bx)) {
        Qs[2] = Q[2]; Qs[3] = Q[3]; Qs[6] = Q[6]; Qs[7] = Q[7];
      } else {
        R tv = Bx * (SM - Q[1]) / dd;
        R tb = (Q[0] * dS * dS - Bx * Bx) / dd;
        Qs[2] = Q[2] - Q[6] * tv;
        Qs[3] = Q[3] - Q[7] * tv;
        Qs[6] = Q[6] * tb;
        Qs[7] = Q[7] * tb;
      }
      Qs[4] = R(0.0);  // unused: star states are used through E, not p
      R vB = Q[1] * Q[5] + Q[2] * Q[6] + Q[3] * Q[7];
      R vBs = Qs[1] * Qs[5] + Qs[2] * Qs[6] + Qs[3] * Qs[7];
      Es = ((S - Q[1]) * E - pT * Q[1] + pTs * SM + Bx * (vB - vBs)) / (S - SM);
    };
    R QsL[8], QsR[8], EsL, EsR;
    star(L, EL, SL, pTL, QsL, EsL);
    star(Rr, ER, SR, pTR, QsR, EsR);
    R UsL[8], UsR[8];
    consv(QsL, EsL, UsL);
    consv(QsR, EsR, UsR);
    R sqL = r_sqrt(QsL[0]), sqR = r_sqrt(QsR[0]);
    R SsL = SM - r_abs(Bx) / sqL, SsR = SM + r_abs(Bx) / sqR;  // Alfven waves
    double sg = val(Bx) > 0.0 ? 1.0 : (val(Bx) < 0.0 ? -1.0 : 0.0);
    R FsL[8], FsR[8];
    for (int q = 0; q < 8; ++q) {
      FsL[q] = FLv[q] + SL * (UsL[q] - ULv[q]);
      FsR[q] = FRv[q] + SR * (UsR[q] - URv[q]);
    }
    if (val(SsL) >= 0.0) {
      for (int q = 0; q < 8; ++q) Fo[q] = FsL[q];
    } else if (val(SsR) <= 0.0) {
      for (int q = 0; q < 8; ++q) Fo[q] = FsR[q];
    } else {
      // double-star states
      R inv = 1.0 / (sqL + sqR);
      R Qss[8];
      Qss[0] = R(0.0);
      Qss[1] = SM;
      Qss[2] = (sqL * QsL[2] + sqR * QsR[2] + (QsR[6] - QsL[6]) * sg) * inv;
      Qss[3] = (sqL * QsL[3] + sqR * QsR[3] + (QsR[7] - QsL[7]) * sg) * inv;
      Qss[5] = Bx;
      Qss[6] = (sqL * QsR[6] + sqR * QsL[6] + sqL * sqR * (QsR[2] - QsL[2]) * sg) * inv;
      Qss[7] = (sqL * QsR[7] + sqR * QsL[7] + sqL * sqR * (QsR[3] - QsL[3]) * sg) * inv;
      Qss[4] = R(0.0);
      R vBss = Qss[1] * Qss[5] + Qss[2] * Qss[6] + Qss[3] * Qss[7];
      R vBsL = QsL[1] * QsL[5] + QsL[2] * QsL[6] + QsL[3] * QsL[7];
      R vBsR = QsR[1] * QsR[5] + QsR[2] * QsR[6] + QsR[3] * QsR[7];
      if (val(SM) >= 0.0) {
        R Q2[8];
        for (int q = 0; q < 8; ++q) Q2[q] = Qss[q];
        Q2[0] = QsL[0];
        R E2 = EsL - sqL * (vBsL - vBss) * sg;
        R U2[8];
        consv(Q2, E2, U2);
        for (int q = 0; q < 8; ++q) Fo[q] = FsL[q] + SsL * (U2[q] - UsL[q]);
      } else {
        R Q2[8];
        for (int q = 0; q < 8; ++q) Q2[q] = Qss[q];
        Q2[0] = QsR[0];
        R E2 = EsR + sqR * (vBsR - vBss) * sg;
        R U2[8];
        consv(Q2, E2, U2);
        for (int q = 0; q < 8; ++q) Fo[q] = FsR[q] + SsR * (U2[q] - UsR[q]);
      }
    }
  }
  // rotate back to the lab frame
  F[I_RHO] = Fo[0];
  F[1 + n] = Fo[1]; F[1 + t1] = Fo[2]; F[1 + t2] = Fo[3];
  F[I_E] = Fo[4];
  F[5 + n] = Fo[5]; F[5 + t1] = Fo[6]; F[5 + t2] = Fo[7];
  return flags;
}

template <class R>
int numerical_flux(const Cfg& c, const R UL[8], const R UR[8], int d, R F[8]) {
  if (c.riemann == RS_HLLD) return riemann_hlld(UL, UR, d, c.gamma, F);
  return riemann_exact(UL, UR, d, c.gamma, F);
}

// ------------------------------------------------------------------------------
// Sec. 2.5: min/max slope limiter, applied to primitive variables
// phi in {rho, v, p[, Bx, By]}.  Gradients of primitives from the conserved
// Taylor coefficients by the product rule (Sec. 2.2, eq. after `GalerkUpdate`),
// limited by alpha = min(1, min_faces psi), converted back by the product rule.
// The magnetic field shares one alpha = min(alpha_Bx, alpha_By) for (a1, a2, a3),
// which keeps each cell's field divergence free.
// ------------------------------------------------------------------------------
// Gradients dU[q][d] of the conserved variables of one cell's polynomial: its
// Taylor derivative coefficients and, for MHD, the derivatives of the magnetic
// basis expansion (2D: dBx = (a3, a1), dBy = (a2, -a3)).
template <class R>
void conserved_gradients(const Grid& G, const R* u, long c, R dU[8][3]) {
  const long n = G.ncell;
  const int b0 = G.L.nT * G.L.nK;
  for (int q = 0; q < 8; ++q) for (int d = 0; d < 3; ++d) dU[q][d] = R(0.0);
  for (int v = 0; v < G.L.nT; ++v)
    for (int d = 0; d < G.c.dim; ++d) dU[G.L.tvar[v]][d] = u[(long)(v * G.L.nK + 1 + d) * n + c];
  for (int k = G.L.nBa; k < G.L.nB; ++k)
    for (int q = 0; q < 3; ++q)
      for (int d = 0; d < G.c.dim; ++d) {
        const double w = mag_dw(G.c.dim, k, q, d);
        if (w != 0.0) dU[I_BX + q][d] = dU[I_BX + q][d] + w * u[(long)(b0 + k) * n + c];
      }
}

// Primitive gradients dW[q][d] at centroid primitives W by the product rule
// (Sec. 2.2, the expansion below eq. `GalerkUpdate`):
//   dv = (dm - v drho)/rho,  dp = (gamma-1)(dE - v^2/2 drho - rho v.dv - B.dB).
template <class R>
void primitive_gradients(const R W[8], const R dU[8][3], double g, R dW[8][3]) {
  for (int d = 0; d < 3; ++d) {
    dW[0][d] = dU[I_RHO][d];
    R vdv(0.0), BdB(0.0);
    for (int i = 0; i < 3; ++i) {
      dW[1 + i][d] = (dU[1 + i][d] - W[1 + i] * dU[I_RHO][d]) / W[0];
      vdv = vdv + W[1 + i] * dW[1 + i][d];
      dW[5 + i][d] = dU[5 + i][d];
      BdB = BdB + W[5 + i] * dU[5 + i][d];
    }
    R v2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
    dW[4][d] = (g - 1.0) * (dU[I_E][d] - 0.5 * v2 * dU[I_RHO][d] - W[0] * vdv - BdB);
  }
}

static void invert_small(int m, const double* A, double* Ainv);

template <class R>
void limit_state(const Grid& G, const R* u, R* out, int& flags) {
  const long n = G.ncell;
  const int dim = G.c.dim;
  const double g = G.c.gamma;
  const int np = G.L.nplanes;
  std::copy(u, u + (long)np * n, out);
  if (!G.c.limiter) return;
  const bool mhd = G.L.nB > 0;
  const int b0 = G.L.nT * G.L.nK;

  // centroid primitives of every cell: (rho, vx, vy, vz, p, Bx, By, Bz)
  std::vector<R> prim((size_t)8 * n);
  for (long c = 0; c < n; ++c) {
    const double x0[3] = {0.0, 0.0, 0.0};
    R U[8], W[8];
    eval_poly(G, u, c, x0, U);
    cons_to_prim(U, g, W);
    if (!(val(W[0]) > 0.0 && val(W[4]) > 0.0)) flags |= FLAG_NONPHYS;
    for (int q = 0; q < 8; ++q) prim[(size_t)q * n + c] = W[q];
  }

  for (long c = 0; c < n; ++c) {
    R W[8];
    for (int q = 0; q < 8; ++q) W[q] = prim[(size_t)q * n + c];
    R dU[8][3], dW[8][3];
    conserved_gradients(G, u, c, dU);
    primitive_gradients(W, dU, g, dW);
    // min/max limiter coefficient of primitive q for the gradient grad
    auto alpha_of = [&](int q, const R* grad) {
      R phimax = W[q], phimin = W[q];
      for (int d = 0; d < dim; ++d)
        for (int s = -1; s <= 1; s += 2) {
          R pn = prim[(size_t)q * n + G.nbr(c, d, s)];
          phimax = r_max(phimax, pn);
          phimin = r_min(phimin, pn);
        }
      R alpha(1.0);
      for (int d = 0; d < dim; ++d)
        for (int s = -1; s <= 1; s += 2) {
          // Delta phi = grad phi . (face centroid - cell centroid)
          R dphi = grad[d] * (0.5 * s * G.h[d]);
          R psi(1.0);
          if (val(dphi) > 0.0) psi = (phimax - W[q]) / dphi;
          else if (val(dphi) < 0.0) psi = (phimin - W[q]) / dphi;
          alpha = r_min(alpha, psi);
        }
      return alpha;
    };
    R dWl[8][3];
    for (int q = 0; q < 8; ++q) for (int d = 0; d < 3; ++d) dWl[q][d] = dW[q][d];
    int hydro_vars[5] = {0, 1, 2, 3, 4};
    R aB(1.0);
    R aBk[8];  // the limited magnetic derivative coefficients
    const int nBd = G.L.nB - G.L.nBa;
    if (G.c.limiter == 2) {
      // Sec. 2.5, the WENO-type limiter.  Per primitive, two candidate gradients:
      // the unlimited DG gradient and the stencil gradient of the FV method (the
      // central difference of the face neighbours' centroid values, min/max
      // limited); their weights are (eps + o_k)^(-1/2) with the oscillation factor
      // o_k = sum_faces |Delta phi_f| + |phi_nbr - (phi + Delta phi_f)|.
      const double eps = 2.220446049250313e-16;  // machine epsilon (double)
      auto stencil = [&](int q, R gs[3]) {
        for (int d = 0; d < 3; ++d) gs[d] = R(0.0);
        for (int d = 0; d < dim; ++d)
          gs[d] = (prim[(size_t)q * n + G.nbr(c, d, +1)] - prim[(size_t)q * n + G.nbr(c, d, -1)]) /
                  (2.0 * G.h[d]);
      };
      auto osc = [&](int q, const R* gr) {
        R o(0.0);
        for (int d = 0; d < dim; ++d)
          for (int s = -1; s <= 1; s += 2) {
            R dphi = gr[d] * (0.5 * s * G.h[d]);
            R pn = prim[(size_t)q * n + G.nbr(c, d, s)];
            o = o + r_abs(dphi) + r_abs(pn - (W[q] + dphi));
          }
        return o;
      };
      for (int h = 0; h < 5; ++h) {
        int q = hydro_vars[h];
        if (q == 3 && dim == 2) continue;
        R gs[3];
        stencil(q, gs);
        R a = alpha_of(q, gs);
        for (int d = 0; d < dim; ++d) gs[d] = a * gs[d];
        R wd = 1.0 / r_sqrt(eps + osc(q, dW[q]));
        R ws = 1.0 / r_sqrt(eps + osc(q, gs));
        for (int d = 0; d < dim; ++d) dWl[q][d] = (wd * dW[q][d] + ws * gs[d]) / (wd + ws);
      }
      if (mhd && dim == 3) {
        // 3D: the stencil gradients G[i] of B_i, each min/max limited as in the FV
        // method, projected in L2 over the cell onto the span of the basis
        // functions' gradients: the coefficients c minimise
        //   int |sum_k c_k (grad V_k) x - G x|^2 dOmega
        //     = (V/12) sum_{i,d} h_d^2 (sum_k c_k dV_k,i/dx_d - G[i][d])^2,
        // i.e. the normal equations N c = r with N_kl = sum_{i,d} h_d^2 dV_k,i/dx_d
        // dV_l,i/dx_d and r_k = sum_{i,d} h_d^2 dV_k,i/dx_d G[i][d]
        R Gs[3][3];
        for (int i = 0; i < 3; ++i) {
          stencil(5 + i, Gs[i]);
          R a = alpha_of(5 + i, Gs[i]);
          for (int e = 0; e < 3; ++e) Gs[i][e] = a * Gs[i][e];
        }
        double N[64], Ninv[64];
        for (int k = 0; k < nBd; ++k)
          for (int l = 0; l < nBd; ++l) {
            double s = 0.0;
            for (int i = 0; i < 3; ++i)
              for (int e = 0; e < 3; ++e)
                s += G.h[e] * G.h[e] * mag_dw(3, G.L.nBa + k, i, e) * mag_dw(3, G.L.nBa + l, i, e);
            N[k * nBd + l] = s;
          }
        invert_small(nBd, N, Ninv);
        R rr[8], st[8];
        for (int k = 0; k < nBd; ++k) {
          rr[k] = R(0.0);
          for (int i = 0; i < 3; ++i)
            for (int e = 0; e < 3; ++e)
              rr[k] = rr[k] + G.h[e] * G.h[e] * mag_dw(3, G.L.nBa + k, i, e) * Gs[i][e];
        }
        for (int k = 0; k < nBd; ++k) {
          st[k] = R(0.0);
          for (int l = 0; l < nBd; ++l) st[k] = st[k] + Ninv[k * nBd + l] * rr[l];
        }
        // the projected stencil field's gradients, for its oscillation factor
        R sB[3][3];
        for (int i = 0; i < 3; ++i)
          for (int e = 0; e < 3; ++e) {
            sB[i][e] = R(0.0);
            for (int k = 0; k < nBd; ++k) sB[i][e] = sB[i][e] + st[k] * mag_dw(3, G.L.nBa + k, i, e);
          }
        // one weight pair for the field (oscillation factors of its three
        // components added), so that the blend stays divergence free
        R od(0.0), os(0.0);
        for (int i = 0; i < 3; ++i) {
          od = od + osc(5 + i, dW[5 + i]);
          os = os + osc(5 + i, sB[i]);
        }
        R wd = 1.0 / r_sqrt(eps + od);
        R ws = 1.0 / r_sqrt(eps + os);
        for (int k = 0; k < nBd; ++k)
          aBk[k] = (wd * u[(long)(b0 + G.L.nBa + k) * n + c] + ws * st[k]) / (wd + ws);
        for (int i = 0; i < 3; ++i)
          for (int e = 0; e < 3; ++e) {
            dWl[5 + i][e] = R(0.0);
            for (int k = 0; k < nBd; ++k)
              dWl[5 + i][e] = dWl[5 + i][e] + aBk[k] * mag_dw(3, G.L.nBa + k, i, e);
          }
      } else if (mhd) {
        // stencil gradients of Bx and By, each min/max limited as in the FV
        // method, then projected in L2 over the cell onto the divergence-free
        // basis: a1 = dBx/dy, a2 = dBy/dx, a3 = (dBx/dx dx^2 - dBy/dy dy^2)/(dx^2 + dy^2)
        R gx[3], gy[3];
        stencil(5, gx);
        stencil(6, gy);
        R ax = alpha_of(5, gx), ay = alpha_of(6, gy);
        for (int d = 0; d < dim; ++d) { gx[d] = ax * gx[d]; gy[d] = ay * gy[d]; }
        const double hx2 = G.h[0] * G.h[0], hy2 = G.h[1] * G.h[1];
        R st[3] = {gx[1], gy[0], (gx[0] * hx2 - gy[1] * hy2) / (hx2 + hy2)};
        R dg[3] = {u[(long)(b0 + 2) * n + c], u[(long)(b0 + 3) * n + c],
                   u[(long)(b0 + 4) * n + c]};
        // one weight pair for the field (oscillation factors of Bx and By added),
        // so that the blend stays divergence free
        R sbx[3] = {st[2], st[0], R(0.0)}, sby[3] = {st[1], -st[2], R(0.0)};
        R wd = 1.0 / r_sqrt(eps + osc(5, dW[5]) + osc(6, dW[6]));
        R ws = 1.0 / r_sqrt(eps + osc(5, sbx) + osc(6, sby));
        for (int k = 0; k < 3; ++k) aBk[k] = (wd * dg[k] + ws * st[k]) / (wd + ws);
        dWl[5][0] = aBk[2]; dWl[5][1] = aBk[0];
        dWl[6][0] = aBk[1]; dWl[6][1] = -aBk[2];
      }
    } else {
      for (int h = 0; h < 5; ++h) {
        int q = hydro_vars[h];
        if (q == 3 && dim == 2) continue;  // vz carries no gradient in 2D
        R a = alpha_of(q, dW[q]);
        for (int d = 0; d < dim; ++d) dWl[q][d] = a * dW[q][d];
      }
      if (mhd) {
        // one factor for the whole field: min over its components (2D: Bx, By)
        aB = alpha_of(5, dW[5]);
        for (int q = 1; q < G.L.nBa; ++q) aB = r_min(aB, alpha_of(5 + q, dW[5 + q]));
        for (int q = 0; q < G.L.nBa; ++q)
          for (int d = 0; d < dim; ++d) dWl[5 + q][d] = aB * dW[5 + q][d];
        for (int k = 0; k < nBd; ++k) aBk[k] = aB * u[(long)(b0 + G.L.nBa + k) * n + c];
      }
    }
    // back to conserved gradients by the product rule
    R dUl[8][3];
    for (int d = 0; d < dim; ++d) {
      dUl[I_RHO][d] = dWl[0][d];
      R vdv(0.0), BdB(0.0);
      for (int i = 0; i < 3; ++i) {
        dUl[1 + i][d] = W[0] * dWl[1 + i][d] + W[1 + i] * dWl[0][d];
        vdv = vdv + W[1 + i] * dWl[1 + i][d];
        BdB = BdB + W[5 + i] * dWl[5 + i][d];
      }
      R v2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
      dUl[I_E][d] = dWl[4][d] / (g - 1.0) + 0.5 * v2 * dWl[0][d] + W[0] * vdv + BdB;
    }
    for (int v = 0; v < G.L.nT; ++v)
      for (int d = 0; d < dim; ++d) out[(long)(v * G.L.nK + 1 + d) * n + c] = dUl[G.L.tvar[v]][d];
    if (mhd)
      for (int k = 0; k < nBd; ++k) out[(long)(b0 + G.L.nBa + k) * n + c] = aBk[k];
  }
}

// ------------------------------------------------------------------------------
// Sec. 2.2: right-hand side of the semi-discrete weak form (eq. `dg`) for every
// basis function, divided by the mass matrix:
//   M dc/dt = - sum_faces int F_hat.n W dGamma + int F . grad W dOmega
// Face states for the Riemann problem are the two cells' polynomials at the face
// Gauss points; MHD replaces the normal field by the average of both sides
// (Sec. 2.6).
// ------------------------------------------------------------------------------

// Gaussian elimination with partial pivoting on a small dense system (double).
static void invert_small(int m, const double* A, double* Ainv) {
  double a[16][32];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < 2 * m; ++j) a[i][j] = j < m ? A[i * m + j] : (j - m == i ? 1.0 : 0.0);
  for (int col = 0; col < m; ++col) {
    int piv = col;
    for (int r = col + 1; r < m; ++r)
      if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
    for (int j = 0; j < 2 * m; ++j) std::swap(a[col][j], a[piv][j]);
    double p = a[col][col];
    for (int j = 0; j < 2 * m; ++j) a[col][j] /= p;
    for (int r = 0; r < m; ++r) {
      if (r == col) continue;
      double f = a[r][col];
      for (int j = 0; j < 2 * m; ++j) a[r][j] -= f * a[col][j];
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Ainv[i * m + j] = a[i][j + m];
}

// Volume quadrature points of a cell: 2^dim tensor Gauss points and weights.
struct VolQuad {
  int nq;
  double x[8][3];
  double w[8];
};
inline VolQuad vol_quad(const Grid& G) {
  VolQuad Q;
  Q.nq = 0;
  const int dim = G.c.dim;
  const int nz = dim == 3 ? 2 : 1;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int e = 0; e < nz; ++e) {
        Q.x[Q.nq][0] = gauss_node(a, G.h[0]);
        Q.x[Q.nq][1] = gauss_node(b, G.h[1]);
        Q.x[Q.nq][2] = dim == 3 ? gauss_node(e, G.h[2]) : 0.0;
        Q.w[Q.nq] = gauss_weight(G.h[0]) * gauss_weight(G.h[1]) *
                    (dim == 3 ? gauss_weight(G.h[2]) : 1.0);
        Q.nq++;
      }
  return Q;
}

// Mass matrices by quadrature (exact: the integrands are quadratic).
struct Mass {
  double MT[4 * 4], MTinv[4 * 4];
  double MB[11 * 11], MBinv[11 * 11];
};
inline Mass mass_matrices(const Grid& G) {
  Mass M;
  VolQuad Q = vol_quad(G);
  const int nK = G.L.nK;
  for (int k = 0; k < nK; ++k)
    for (int l = 0; l < nK; ++l) {
      double s = 0.0;
      for (int q = 0; q < Q.nq; ++q) s += Q.w[q] * taylor_w(k, Q.x[q]) * taylor_w(l, Q.x[q]);
      M.MT[k * nK + l] = s;
    }
  invert_small(nK, M.MT, M.MTinv);
  const int nB = G.L.nB ? G.L.nB : 5;  // (the 2D basis when there is no field)
  const int dimB = G.L.nB ? G.c.dim : 2;
  for (int k = 0; k < nB; ++k)
    for (int l = 0; l < nB; ++l) {
      double s = 0.0;
      for (int q = 0; q < Q.nq; ++q) {
        double wk[3], wl[3];
        mag_w(dimB, k, Q.x[q], wk);
        mag_w(dimB, l, Q.x[q], wl);
        s += Q.w[q] * (wk[0] * wl[0] + wk[1] * wl[1] + wk[2] * wl[2]);
      }
      M.MB[k * nB + l] = s;
    }
  invert_small(nB, M.MB, M.MBinv);
  return M;
}

// Face quadrature: the points of the face with outward normal s*e_d of a cell, in
// that cell's local coordinates, and their weights.
struct FaceQuad {
  int ng;
  double x[4][3];
  double w[4];
};
inline FaceQuad face_quad(const Grid& G, int d, int s) {
  FaceQuad F;
  F.ng = 0;
  const int dim = G.c.dim;
  int t[2], nt = 0;
  for (int e = 0; e < dim; ++e) if (e != d) t[nt++] = e;
  const int n1 = 2, n2 = nt == 2 ? 2 : 1;
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n2; ++b) {
      double* x = F.x[F.ng];
      x[0] = x[1] = x[2] = 0.0;
      x[d] = 0.5 * s * G.h[d];
      x[t[0]] = gauss_node(a, G.h[t[0]]);
      double w = gauss_weight(G.h[t[0]]);
      if (nt == 2) { x[t[1]] = gauss_node(b, G.h[t[1]]); w *= gauss_weight(G.h[t[1]]); }
      F.w[F.ng] = w;
      F.ng++;
    }
  return F;
}

template <class R>
void dg_rhs(const Grid& G, const R* u, R* rhs, int& flags) {
  const long n = G.ncell;
  const int dim = G.c.dim;
  const double g = G.c.gamma;
  const bool mhd = G.L.nB > 0;
  const int nT = G.L.nT, nK = G.L.nK, b0 = nT * nK;
  const Mass M = mass_matrices(G);
  const VolQuad VQ = vol_quad(G);

  // 1. numerical fluxes at the Gauss points of every face, computed once per
  //    face: Fh[d][cell][gp][8] is the flux along +e_d through the face between
  //    `cell` (left) and its +e_d neighbour (right).
  std::vector<R> Fh[3];
  FaceQuad FQp[3], FQm[3];
  for (int d = 0; d < dim; ++d) {
    FQp[d] = face_quad(G, d, +1);
    FQm[d] = face_quad(G, d, -1);
    Fh[d].assign((size_t)n * FQp[d].ng * 8, R(0.0));
    for (long c = 0; c < n; ++c) {
      long r = G.nbr(c, d, +1);
      for (int gp = 0; gp < FQp[d].ng; ++gp) {
        R UL[8], UR[8], F[8];
        eval_poly(G, u, c, FQp[d].x[gp], UL);  // left cell at its +d face
        eval_poly(G, u, r, FQm[d].x[gp], UR);  // right cell at its -d face
        if (mhd) {
          // Sec. 2.6: one normal field for the Riemann problem, the average of
          // the two one-sided values; the gas pressure of each side is kept.
          R WL[8], WR[8];
          cons_to_prim(UL, g, WL);
          cons_to_prim(UR, g, WR);
          R bn = 0.5 * (WL[5 + d] + WR[5 + d]);
          WL[5 + d] = bn;
          WR[5 + d] = bn;
          prim_to_cons(WL, g, UL);
          prim_to_cons(WR, g, UR);
        }
        flags |= numerical_flux(G.c, UL, UR, d, F);
        for (int q = 0; q < 8; ++q) Fh[d][((size_t)c * FQp[d].ng + gp) * 8 + q] = F[q];
      }
    }
  }

  // 2. per cell: assemble face and volume integrals for every basis function
  for (long c = 0; c < n; ++c) {
    R bT[5][4], bB[11];
    for (int v = 0; v < 5; ++v) for (int k = 0; k < 4; ++k) bT[v][k] = R(0.0);
    for (int k = 0; k < 11; ++k) bB[k] = R(0.0);
    // face terms: - int F_hat . n W dGamma
    for (int d = 0; d < dim; ++d)
      for (int s = -1; s <= 1; s += 2) {
        const FaceQuad& FQ = s > 0 ? FQp[d] : FQm[d];
        long owner = s > 0 ? c : G.nbr(c, d, -1);  // face stored with its left cell
        for (int gp = 0; gp < FQ.ng; ++gp) {
          const R* F = &Fh[d][((size_t)owner * FQ.ng + gp) * 8];
          const double w = FQ.w[gp] * s;  // F_hat . n = s * F_hat_d
          for (int v = 0; v < nT; ++v)
            for (int k = 0; k < nK; ++k)
              bT[v][k] = bT[v][k] - w * taylor_w(k, FQ.x[gp]) * F[G.L.tvar[v]];
          if (mhd)
            for (int k = 0; k < G.L.nB; ++k) {
              double wk[3];
              mag_w(dim, k, FQ.x[gp], wk);
              bB[k] = bB[k] - w * (wk[0] * F[I_BX] + wk[1] * F[I_BY] + wk[2] * F[I_BZ]);
            }
        }
      }
    // volume terms: + int F . grad W dOmega
    for (int q = 0; q < VQ.nq; ++q) {
      R U[8], W[8];
      eval_poly(G, u, c, VQ.x[q], U);
      cons_to_prim(U, g, W);
      if (!(val(W[0]) > 0.0 && val(W[4]) > 0.0)) flags |= FLAG_NONPHYS;
      for (int d = 0; d < dim; ++d) {
        R F[8];
        phys_flux(U, d, g, F);
        for (int v = 0; v < nT; ++v)
          for (int k = 0; k < nK; ++k)
            bT[v][k] = bT[v][k] + VQ.w[q] * taylor_dw(k, d) * F[G.L.tvar[v]];
        if (mhd)
          for (int k = 0; k < G.L.nB; ++k)
            bB[k] = bB[k] + VQ.w[q] * (mag_dw(dim, k, 0, d) * F[I_BX] +
                                       mag_dw(dim, k, 1, d) * F[I_BY] +
                                       mag_dw(dim, k, 2, d) * F[I_BZ]);
      }
    }
    // solve with the mass matrices
    for (int v = 0; v < nT; ++v)
      for (int k = 0; k < nK; ++k) {
        R s(0.0);
        for (int l = 0; l < nK; ++l) s = s + M.MTinv[k * nK + l] * bT[v][l];
        rhs[(long)(v * nK + k) * n + c] = s;
      }
    if (mhd)
      for (int k = 0; k < G.L.nB; ++k) {
        R s(0.0);
        for (int l = 0; l < G.L.nB; ++l) s = s + M.MBinv[k * G.L.nB + l] * bB[l];
        rhs[(long)(b0 + k) * n + c] = s;
      }
  }
}

// ------------------------------------------------------------------------------
// Two-stage SSP Runge-Kutta step.  The stored state between stages is the stage
// output before limiting; the limiter Lambda acts on every stage input, i.e. at
// the beginning of each step and of each stage (Sec. 2.5):
//   U^n = Lambda(V^n),  V^1 = U^n + dt L(U^n),  U^1 = Lambda(V^1),
//   V^{n+1} = 1/2 U^n + 1/2 (U^1 + dt L(U^1)).
// ------------------------------------------------------------------------------
template <class R>
int rk2_step(const Grid& G, const R* vn, R* vout, double dt) {
  const long tot = (long)G.L.nplanes * G.ncell;
  std::vector<R> un(tot), l(tot), v1(tot), u1(tot);
  int flags = 0;
  limit_state(G, vn, un.data(), flags);
  dg_rhs(G, un.data(), l.data(), flags);
  for (long i = 0; i < tot; ++i) v1[i] = un[i] + dt * l[i];
  limit_state(G, v1.data(), u1.data(), flags);
  dg_rhs(G, u1.data(), l.data(), flags);
  for (long i = 0; i < tot; ++i) vout[i] = 0.5 * un[i] + 0.5 * (u1[i] + dt * l[i]);
  return flags;
}

// Time step from the Courant condition on the cell averages:
//   dt = CFL / max_cells sum_d (|v_d| + c_d) / dx_d,
// c_d the sound speed (Euler) or the fast magnetosonic speed along d (MHD).
inline double cfl_dt(const Grid& G, const double* u, double cfl, int& flags) {
  double smax = 0.0;
  const double x0[3] = {0.0, 0.0, 0.0};
  for (long c = 0; c < G.ncell; ++c) {
    double U[8], W[8];
    eval_poly(G, u, c, x0, U);
    cons_to_prim(U, G.c.gamma, W);
    if (!(W[0] > 0.0 && W[4] > 0.0)) { flags |= FLAG_NONPHYS; continue; }
    double s = 0.0;
    for (int d = 0; d < G.c.dim; ++d) {
      double cd = G.L.nB ? fast_speed(W, d, G.c.gamma) : std::sqrt(G.c.gamma * W[4] / W[0]);
      s += (std::fabs(W[1 + d]) + cd) / G.h[d];
    }
    smax = std::max(smax, s);
  }
  return smax > 0.0 ? cfl / smax : 0.0;
}

// ------------------------------------------------------------------------------
// MUSCL-Hancock step (Sec. 2.4, "Time stepping"), the paper's own integrator.
//   1. Limit at the beginning of the step (Sec. 2.5) and recompute the conserved
//      derivative coefficients from the limited primitive gradients.
//   2. Predict primitive values half a step ahead from the centroid values and
//      their gradients, W(x, t + dt/2) = W_c + grad W . x + dt/2 dW/dt, with the
//      time derivative from the primitive form of eq. `cons` at the centroid.
//   3. Riemann fluxes between the predicted face values of both sides (Sec. 2.3;
//      MHD with the averaged normal field of Sec. 2.6), and volume fluxes of the
//      predicted state at the volume Gauss points ("the same prediction
//      equations" in the volume integral of eq. `GalerkUpdate`).
//   4. One update of the moments Q = int U and R = M grad U (eq. `GalerkUpdate`):
//      Q^{n+1} = Q^n - dt sum_f A_f F_f,
//      R^{n+1} = R^n - dt sum_f A_f F_f c_f + dt int F dOmega,
//      written, as in dg_rhs, as the weak form of every basis function with the
//      face integral taken by a face quadrature rule: one point at the face
//      centroid c_f with weight A_f (eq. `GalerkUpdate`), or the 2-point Gauss
//      rule per face dimension.
// ------------------------------------------------------------------------------

// Primitive form of eq. `cons` along axis d: dW/dt = - sum_d A_d(W) dW/dx_d for
// W = (rho, v, p, B), i.e.
//   drho/dt = -v.grad rho - rho div v
//   dv/dt   = -(v.grad) v - grad p / rho - (grad(B^2/2) - (B.grad) B) / rho
//   dp/dt   = -v.grad p - gamma p div v
//   dB/dt   = (B.grad) v - (v.grad) B - B div v
// (terms proportional to div B are left out: every cell's field is divergence
// free, Sec. 2.2, and the limiter keeps it so).  Row r, column k of A_d.
inline void prim_matrix(const double W[8], int d, double g, double A[8][8]) {
  for (int r = 0; r < 8; ++r) for (int k = 0; k < 8; ++k) A[r][k] = 0.0;
  const double rho = W[0], p = W[4];
  const double* v = W + 1;
  const double* B = W + 5;
  A[0][0] = v[d];
  A[0][1 + d] = rho;
  for (int i = 0; i < 3; ++i) {
    A[1 + i][1 + i] = v[d];
    if (i == d) {
      A[1 + i][4] = 1.0 / rho;
      for (int j = 0; j < 3; ++j) A[1 + i][5 + j] += B[j] / rho;  // grad_d (B^2/2)
    }
    A[1 + i][5 + i] -= B[d] / rho;  // -(B_d d/dx_d) B_i
  }
  A[4][4] = v[d];
  A[4][1 + d] = g * p;
  for (int i = 0; i < 3; ++i) {
    A[5 + i][1 + i] -= B[d];  // (B_d d/dx_d) v_i
    A[5 + i][5 + i] += v[d];  // (v_d d/dx_d) B_i
    A[5 + i][1 + d] += B[i];  // B_i dv_d/dx_d
  }
}

inline void prim_rates(const double W[8], const double dW[8][3], int dim, double g,
                       double Wt[8]) {
  for (int r = 0; r < 8; ++r) Wt[r] = 0.0;
  for (int d = 0; d < dim; ++d) {
    double A[8][8];
    prim_matrix(W, d, g, A);
    for (int r = 0; r < 8; ++r)
      for (int k = 0; k < 8; ++k) Wt[r] -= A[r][k] * dW[k][d];
  }
}

// Face rule with `npts` points: 1 = the face centroid with weight A_f, else the
// 2-point Gauss rule per face dimension (face_quad).
inline FaceQuad face_quad_n(const Grid& G, int d, int s, int npts) {
  if (npts != 1) return face_quad(G, d, s);
  FaceQuad F;
  F.ng = 1;
  F.x[0][0] = F.x[0][1] = F.x[0][2] = 0.0;
  F.x[0][d] = 0.5 * s * G.h[d];
  F.w[0] = G.vol / G.h[d];
  return F;
}

int mh_step(const Grid& G, const double* vn, double* vout, double dt, int face_points) {
  const long n = G.ncell;
  const int dim = G.c.dim;
  const double g = G.c.gamma;
  const bool mhd = G.L.nB > 0;
  const int nT = G.L.nT, nK = G.L.nK, b0 = nT * nK;
  const long tot = (long)G.L.nplanes * n;
  const Mass M = mass_matrices(G);
  const VolQuad VQ = vol_quad(G);
  int flags = 0;

  // 1. limited state U^n
  std::vector<double> un(tot);
  limit_state<double>(G, vn, un.data(), flags);

  // 2. predicted centroid primitives Wp = W_c + dt/2 dW/dt and the primitive
  //    gradients dW of every cell
  std::vector<double> Wp((size_t)8 * n), dW((size_t)24 * n);
  for (long c = 0; c < n; ++c) {
    const double x0[3] = {0.0, 0.0, 0.0};
    double U[8], W[8], dUc[8][3], dWc[8][3], Wt[8];
    eval_poly<double>(G, un.data(), c, x0, U);
    cons_to_prim(U, g, W);
    if (!(W[0] > 0.0 && W[4] > 0.0)) flags |= FLAG_NONPHYS;
    conserved_gradients<double>(G, un.data(), c, dUc);
    primitive_gradients<double>(W, dUc, g, dWc);
    prim_rates(W, dWc, dim, g, Wt);
    for (int q = 0; q < 8; ++q) {
      Wp[(size_t)q * n + c] = W[q] + 0.5 * dt * Wt[q];
      for (int e = 0; e < 3; ++e) dW[((size_t)q * 3 + e) * n + c] = dWc[q][e];
    }
  }
  // predicted primitive state of cell c at local point x
  auto predict = [&](long c, const double x[3], double W[8]) {
    for (int q = 0; q < 8; ++q) {
      double s = Wp[(size_t)q * n + c];
      for (int e = 0; e < dim; ++e) s += dW[((size_t)q * 3 + e) * n + c] * x[e];
      W[q] = s;
    }
    if (!(W[0] > 0.0 && W[4] > 0.0)) flags |= FLAG_NONPHYS;
  };

  // 3a. Riemann fluxes at the face points, each face once (stored with its
  //     left cell, as in dg_rhs)
  std::vector<double> Fh[3];
  FaceQuad FQp[3], FQm[3];
  for (int d = 0; d < dim; ++d) {
    FQp[d] = face_quad_n(G, d, +1, face_points);
    FQm[d] = face_quad_n(G, d, -1, face_points);
    Fh[d].assign((size_t)n * FQp[d].ng * 8, 0.0);
    for (long c = 0; c < n; ++c) {
      long r = G.nbr(c, d, +1);
      for (int gp = 0; gp < FQp[d].ng; ++gp) {
        double WL[8], WR[8], UL[8], UR[8], F[8];
        predict(c, FQp[d].x[gp], WL);
        predict(r, FQm[d].x[gp], WR);
        if (mhd) {
          double bn = 0.5 * (WL[5 + d] + WR[5 + d]);
          WL[5 + d] = bn;
          WR[5 + d] = bn;
        }
        prim_to_cons(WL, g, UL);
        prim_to_cons(WR, g, UR);
        flags |= numerical_flux(G.c, UL, UR, d, F);
        for (int q = 0; q < 8; ++q) Fh[d][((size_t)c * FQp[d].ng + gp) * 8 + q] = F[q];
      }
    }
  }

  // 3b, 4. per cell: face and volume integrals of every basis function, mass
  //        matrix solve, update of the limited coefficients
  for (long c = 0; c < n; ++c) {
    double bT[5][4], bB[11];
    for (int v = 0; v < 5; ++v) for (int k = 0; k < 4; ++k) bT[v][k] = 0.0;
    for (int k = 0; k < 11; ++k) bB[k] = 0.0;
    for (int d = 0; d < dim; ++d)
      for (int s = -1; s <= 1; s += 2) {
        const FaceQuad& FQ = s > 0 ? FQp[d] : FQm[d];
        long owner = s > 0 ? c : G.nbr(c, d, -1);
        for (int gp = 0; gp < FQ.ng; ++gp) {
          const double* F = &Fh[d][((size_t)owner * FQ.ng + gp) * 8];
          const double w = FQ.w[gp] * s;
          for (int v = 0; v < nT; ++v)
            for (int k = 0; k < nK; ++k)
              bT[v][k] -= w * taylor_w(k, FQ.x[gp]) * F[G.L.tvar[v]];
          if (mhd)
            for (int k = 0; k < G.L.nB; ++k) {
              double wk[3];
              mag_w(dim, k, FQ.x[gp], wk);
              bB[k] -= w * (wk[0] * F[I_BX] + wk[1] * F[I_BY] + wk[2] * F[I_BZ]);
            }
        }
      }
    for (int q = 0; q < VQ.nq; ++q) {
      double W[8], U[8];
      predict(c, VQ.x[q], W);
      prim_to_cons(W, g, U);
      for (int d = 0; d < dim; ++d) {
        double F[8];
        phys_flux(U, d, g, F);
        for (int v = 0; v < nT; ++v)
          for (int k = 0; k < nK; ++k) bT[v][k] += VQ.w[q] * taylor_dw(k, d) * F[G.L.tvar[v]];
        if (mhd)
          for (int k = 0; k < G.L.nB; ++k)
            bB[k] += VQ.w[q] * (mag_dw(dim, k, 0, d) * F[I_BX] + mag_dw(dim, k, 1, d) * F[I_BY] +
                                mag_dw(dim, k, 2, d) * F[I_BZ]);
      }
    }
    for (int v = 0; v < nT; ++v)
      for (int k = 0; k < nK; ++k) {
        double s = 0.0;
        for (int l = 0; l < nK; ++l) s += M.MTinv[k * nK + l] * bT[v][l];
        const long i = (long)(v * nK + k) * n + c;
        vout[i] = un[i] + dt * s;
      }
    if (mhd)
      for (int k = 0; k < G.L.nB; ++k) {
        double s = 0.0;
        for (int l = 0; l < G.L.nB; ++l) s += M.MBinv[k * G.L.nB + l] * bB[l];
        const long i = (long)(b0 + k) * n + c;
        vout[i] = un[i] + dt * s;
      }
  }
  return flags;
}

}  // namespace oracle

// ==============================================================================
// C interface (ctypes).  All arrays are float64 in the interchange layout
// [plane][nz][ny][nx].  Return values: OR of the FLAG_* bits.
// ==============================================================================
using namespace oracle;

extern "C" {

int oracle_nplanes(const Cfg* c) { return layout_of(*c).nplanes; }

int oracle_limit(const Cfg* c, const double* u, double* out) {
  Grid G(*c);
  int flags = 0;
  limit_state<double>(G, u, out, flags);
  return flags;
}

int oracle_rhs(const Cfg* c, const double* u, double* out) {
  Grid G(*c);
  int flags = 0;
  dg_rhs<double>(G, u, out, flags);
  return flags;
}

int oracle_step(const Cfg* c, const double* u, double* out, double dt) {
  Grid G(*c);
  return rk2_step<double>(G, u, out, dt);
}

double oracle_cfl_dt(const Cfg* c, const double* u, double cfl, int* flags) {
  Grid G(*c);
  int f = 0;
  double dt = cfl_dt(G, u, cfl, f);
  if (flags) *flags = f;
  return dt;
}

// nsteps steps; dt from the Courant condition before every step unless
// dt_fixed > 0.  dts (may be null) receives the nsteps time steps used.
int oracle_run(const Cfg* c, const double* u, double* out, int nsteps, double cfl,
               double dt_fixed, double* dts) {
  Grid G(*c);
  const long tot = (long)G.L.nplanes * G.ncell;
  std::vector<double> a(u, u + tot), b(tot);
  int flags = 0;
  for (int s = 0; s < nsteps; ++s) {
    double dt = dt_fixed > 0.0 ? dt_fixed : cfl_dt(G, a.data(), cfl, flags);
    if (dts) dts[s] = dt;
    flags |= rk2_step<double>(G, a.data(), b.data(), dt);
    std::swap(a, b);
  }
  std::copy(a.begin(), a.end(), out);
  return flags;
}

// One MUSCL-Hancock step (face_points 1: face centroid, 2: Gauss rule).
int oracle_mh_step(const Cfg* c, const double* u, double* out, double dt, int face_points) {
  Grid G(*c);
  return mh_step(G, u, out, dt, face_points);
}

// nsteps MUSCL-Hancock steps, as oracle_run.
int oracle_mh_run(const Cfg* c, const double* u, double* out, int nsteps, double cfl,
                  double dt_fixed, int face_points, double* dts) {
  Grid G(*c);
  const long tot = (long)G.L.nplanes * G.ncell;
  std::vector<double> a(u, u + tot), b(tot);
  int flags = 0;
  for (int s = 0; s < nsteps; ++s) {
    double dt = dt_fixed > 0.0 ? dt_fixed : cfl_dt(G, a.data(), cfl, flags);
    if (dts) dts[s] = dt;
    flags |= mh_step(G, a.data(), b.data(), dt, face_points);
    std::swap(a, b);
  }
  std::copy(a.begin(), a.end(), out);
  return flags;
}

// Time derivative of the primitives W (8) with gradients dW ([8][3], row-major)
// from the primitive form used by the MUSCL-Hancock prediction.
void oracle_prim_rates(const double* W, const double* dW, int dim, double gamma, double* Wt) {
  double G3[8][3];
  for (int q = 0; q < 8; ++q) for (int e = 0; e < 3; ++e) G3[q][e] = dW[q * 3 + e];
  prim_rates(W, G3, dim, gamma, Wt);
}

// Tangent of one step with the time step held fixed: out = step(u),
// dout = d step(u)/du . du.
int oracle_tangent_step(const Cfg* c, const double* u, const double* du, double* out,
                        double* dout, double dt) {
  Grid G(*c);
  const long tot = (long)G.L.nplanes * G.ncell;
  std::vector<Dual> a(tot), b(tot);
  for (long i = 0; i < tot; ++i) a[i] = Dual(u[i], du[i]);
  int flags = rk2_step<Dual>(G, a.data(), b.data(), dt);
  for (long i = 0; i < tot; ++i) { out[i] = b[i].v; dout[i] = b[i].d; }
  return flags;
}

// Tangent of the right-hand side L(u) (no limiting) in direction du.
int oracle_tangent_rhs(const Cfg* c, const double* u, const double* du, double* out,
                       double* dout) {
  Grid G(*c);
  const long tot = (long)G.L.nplanes * G.ncell;
  std::vector<Dual> a(tot), b(tot);
  for (long i = 0; i < tot; ++i) a[i] = Dual(u[i], du[i]);
  int flags = 0;
  dg_rhs<Dual>(G, a.data(), b.data(), flags);
  for (long i = 0; i < tot; ++i) { out[i] = b[i].v; dout[i] = b[i].d; }
  return flags;
}

// Tangent of the limiter in direction du.
int oracle_tangent_limit(const Cfg* c, const double* u, const double* du, double* out,
                         double* dout) {
  Grid G(*c);
  const long tot = (long)G.L.nplanes * G.ncell;
  std::vector<Dual> a(tot), b(tot);
  for (long i = 0; i < tot; ++i) a[i] = Dual(u[i], du[i]);
  int flags = 0;
  limit_state<Dual>(G, a.data(), b.data(), flags);
  for (long i = 0; i < tot; ++i) { out[i] = b[i].v; dout[i] = b[i].d; }
  return flags;
}

// Single-interface numerical flux along axis d (kind 0 exact, 1 HLLD), for the
// unit tests of the Riemann solvers.  U are conserved 8-vectors.
int oracle_riemann(int kind, const double* UL, const double* UR, int d, double gamma,
                   double* F) {
  if (kind == RS_HLLD) return riemann_hlld<double>(UL, UR, d, gamma, F);
  return riemann_exact<double>(UL, UR, d, gamma, F);
}

// Exact solution of the 1D Euler Riemann problem sampled at speeds xi[0..m-1];
// W = (rho, u, p) per sample; star = (p*, u*).
int oracle_exact_sample(const double* WL, const double* WR, double gamma, int m,
                        const double* xi, double* W, double* star) {
  ExactParams P;
  StarState<double> S = exact_star<double>(WL[0], WL[1], WL[2], WR[0], WR[1], WR[2], gamma, P);
  for (int i = 0; i < m; ++i)
    exact_sample<double>(WL[0], WL[1], WL[2], WR[0], WR[1], WR[2], gamma, S, xi[i], W[3 * i],
                         W[3 * i + 1], W[3 * i + 2]);
  star[0] = S.pstar;
  star[1] = S.ustar;
  return S.flags;
}

void oracle_phys_flux(const double* U, int d, double gamma, double* F) {
  phys_flux<double>(U, d, gamma, F);
}

// Value of the DG polynomial of one cell at a local point x (3 entries).
void oracle_eval(const Cfg* c, const double* u, long cell, const double* x, double* U) {
  Grid G(*c);
  eval_poly<double>(G, u, cell, x, U);
}

void oracle_mass_matrices(const Cfg* c, double* MT, double* MB) {
  Grid G(*c);
  Mass M = mass_matrices(G);
  std::memcpy(MT, M.MT, sizeof(M.MT));
  std::memcpy(MB, M.MB, sizeof(M.MB));
}

// Totals V * sum_cells(average) of every conserved variable (Taylor variables
// then the field averages b1, b2[, b3]), Neumaier-compensated.
void oracle_totals(const Cfg* c, const double* u, double* out) {
  Grid G(*c);
  int nv = G.L.nT + G.L.nBa;
  for (int v = 0; v < nv; ++v) {
    int plane = v < G.L.nT ? v * G.L.nK : G.L.nT * G.L.nK + (v - G.L.nT);
    double s = 0.0, comp = 0.0;
    for (long i = 0; i < G.ncell; ++i) {
      double x = u[(long)plane * G.ncell + i];
      double t = s + x;
      if (std::fabs(s) >= std::fabs(x)) comp += (s - t) + x; else comp += (x - t) + s;
      s = t;
    }
    out[v] = (s + comp) * G.vol;
  }
}

// Sec. 2.6: Stokes estimate of div B per cell, (1/V) sum_faces B.n A, with the
// face-normal field averaged between the two sides and integrated with the face
// Gauss rule.
void oracle_divb(const Cfg* c, const double* u, double* out) {
  Grid G(*c);
  for (long cell = 0; cell < G.ncell; ++cell) {
    double s = 0.0;
    for (int d = 0; d < G.c.dim; ++d)
      for (int sg = -1; sg <= 1; sg += 2) {
        FaceQuad FQ = face_quad(G, d, sg);
        FaceQuad FN = face_quad(G, d, -sg);
        long nb = G.nbr(cell, d, sg);
        for (int gp = 0; gp < FQ.ng; ++gp) {
          double U1[8], U2[8];
          eval_poly<double>(G, u, cell, FQ.x[gp], U1);
          eval_poly<double>(G, u, nb, FN.x[gp], U2);
          s += sg * FQ.w[gp] * 0.5 * (U1[5 + d] + U2[5 + d]);
        }
      }
    out[cell] = s / G.vol;
  }
}

}  // extern "C"
